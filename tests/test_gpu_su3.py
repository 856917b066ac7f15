"""Full su(3) spin-one Hamiltonians on the GPU (quadrupole drives on the
symmetric products of the spin matrices, FP64): every sample against the
oracle for all methods and both frames, the CPU backend's identical
arithmetic, batch independence, and the precision and spin checks."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2204_05586_gb300 import cpu_backend as C, spinsim as S, workloads as W  # noqa: E402

THREADS = os.cpu_count() or 4


def su3_request(t_end=2e-3, seed=4, qdrives=((1.2e3, 0.7e3, 700.3e3, 0.4), (0.9e3, 0.9e3, 1400.2e3, -0.8))):
    f = W.field(bias_hz=700e3, drive_x_hz=2e3, drive_hz=700e3, quad_hz=300.0, pulses=[(60.0, 0.5e-3, 0.2e-3)],
                qdrives=list(qdrives), tones=[(0.5e3, 0.2e3, 699.7e3, 1.0)])
    return W.request(2, f, 0.0, t_end, 1e-8, 1e-6, psi0=W.random_state(3, np.random.default_rng(seed)))


def oracle_run(O, req, frame=True, method=0):
    return O.simulate(2, req["field"], req["t_start"], req["t_end"], req["dt"], req["dt_out"], req["psi0"],
                      rotating_frame=frame, method=method, threads=THREADS)


def run(reqs, **cfg):
    with S.Simulator(**cfg) as sim:
        return sim.simulate(reqs)


@pytest.mark.parametrize("frame", [True, False])
@pytest.mark.parametrize("method", [S.METHOD_CF4, S.METHOD_MIDPOINT, S.METHOD_HEUN])
def test_su3_against_oracle(oracle_mod, frame, method):
    req = su3_request()
    (out,) = run([req], precision=S.PREC_FP64, rotating_frame=frame, method=method)
    assert out["status"] == S.OK
    ref = oracle_run(oracle_mod, req, frame=frame, method=method)
    err = np.abs(out["states"].cpu().numpy() - ref["states"]).max()
    assert err < 1e-10, err
    assert np.abs(out["spin"].cpu().numpy() - ref["spin"]).max() < 2e-10


def test_su3_equals_cpu_backend():
    req = su3_request()
    (g,) = run([req], precision=S.PREC_FP64)
    (c,) = C.simulate([req], precision=S.PREC_FP64)
    assert np.abs(g["states"].cpu().numpy() - c["states"]).max() < 1e-12


def test_su3_in_mixed_batches_equals_alone(oracle_mod):
    """su(3) requests beside ordinary and tone requests (FP64): each runs its
    own launch group and equals its run alone bit for bit."""
    reqs = [su3_request(1e-3, seed=1), W.spin_one_sensing(t_end=1e-3), su3_request(7e-4, seed=2, qdrives=[(0.0, 2e3, 5e3, 0.1)]),
            W.multitone_sensing(t_end=5e-4), W.spin_half_rabi(t_end=1e-3)]
    outs = run(reqs, precision=S.PREC_FP64)
    for q, o in zip(reqs, outs):
        assert o["status"] == S.OK
        (alone,) = run([q], precision=S.PREC_FP64)
        assert np.array_equal(alone["states"].cpu().numpy(), o["states"].cpu().numpy())
    ref = oracle_run(oracle_mod, reqs[2])
    assert np.abs(outs[2]["states"].cpu().numpy() - ref["states"]).max() < 1e-10


def test_su3_needs_fp64_and_spin_one():
    with S.Simulator(precision=S.PREC_FP32_BULK) as sim:
        req = su3_request(1e-4)
        outs = sim.allocate([req])
        res = sim.results_struct(outs)
        assert S.spinsim_simulate(sim.handle, [S.make_request(req)], res, 0) == S.E_UNSUPPORTED
        assert res[0].status == S.E_UNSUPPORTED
    half = W.spin_half_rabi(t_end=1e-4)
    half["field"]["qdrives"] = [(1.0, 1.0, 1.0, 0.0)]
    with S.Simulator(precision=S.PREC_FP64) as sim:
        outs = sim.allocate([half])
        res = sim.results_struct(outs)
        assert S.spinsim_simulate(sim.handle, [S.make_request(half)], res, 0) == S.E_ARG


def test_su3_through_the_static_entry_point():
    req = su3_request(1e-3, seed=6)
    cfg = S.make_config(precision=S.PREC_FP64)
    K = S.spinsim_counts(S.make_request(req))[1]
    states = torch.full((K, 3, 2), float("nan"), dtype=torch.float64, device="cuda")
    res = S.spinsim_result()
    res.states, res.capacity = states.data_ptr(), K
    st = S.spinsim_simulate_static(cfg, S.make_request(req), res, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == S.OK and res.status == S.OK
    (ref,) = run([req], precision=S.PREC_FP64)
    assert np.array_equal(torch.view_as_complex(states).cpu().numpy(), ref["states"].cpu().numpy())


def test_su3_served_mix_equals_alone():
    """su(3) requests and plain ones through the serving queue (FP64): each
    result is bit-identical to the request run alone."""
    reqs = [su3_request(4e-4, seed=s) if s % 2 else W.spin_one_sensing(t_end=4e-4) for s in range(6)]
    alone = [run([q], precision=S.PREC_FP64)[0]["states"].cpu().numpy() for q in reqs]
    with S.Simulator(precision=S.PREC_FP64) as sim:
        outs = sim.allocate(reqs)
        res = sim.results_struct(outs)
        tickets = []
        for q, r in zip([S.make_request(q) for q in reqs], res):
            st, t = S.spinsim_submit(sim.handle, q, r)
            assert st == S.OK
            tickets.append(t)
        for t in tickets:
            assert S.spinsim_poll(sim.handle, t, 10_000_000) == S.OK
    for o, r, a in zip(outs, res, alone):
        assert r.status == S.OK
        assert np.array_equal(torch.view_as_complex(o["states"][:o["K"]]).cpu().numpy(), a)


def test_su3_split_into_ranges(oracle_mod):
    """One su(3) simulation (2e3 samples x 100 steps) in three ranges through
    spinsim_range_begin / spinsim_range_finish: equal to the unsplit run and
    to the oracle."""
    from paper_2204_05586_gb300 import sharded as SH
    req = su3_request(2e-3, seed=9)
    (full,) = run([req], precision=S.PREC_FP64)
    full = full["states"].cpu().numpy()
    K = S.spinsim_counts(S.make_request(req))[1]
    rs = SH.ranges(K, 3)
    backends = [SH.CudaRange(precision=S.PREC_FP64) for _ in rs]
    try:
        aggs = [b.begin(SH.range_request(req, k0, k1, r == len(rs) - 1)) for r, (b, (k0, k1)) in
                enumerate(zip(backends, rs))]
        psis = SH.entering_states(aggs, req["psi0"])
        got = np.concatenate([b.finish(p)[: k1 - k0] for b, p, (k0, k1) in zip(backends, psis, rs)])
    finally:
        for b in backends:
            b.close()
    assert np.abs(got - full).max() < 1e-10
    assert np.abs(got - oracle_run(oracle_mod, req)["states"]).max() < 1e-10


def test_su3_scaled_and_squared_steps(oracle_mod):
    """Lab frame with a 0.5 us step: every exponent's norm is above 1, so the
    general exponential halves it three times and squares back three times."""
    f = W.field(bias_hz=700e3, drive_x_hz=40e3, drive_hz=700e3, quad_hz=3e3,
                qdrives=[(30e3, 20e3, 700e3, 0.4), (25e3, 25e3, 1400e3, -0.8)])
    req = W.request(2, f, 0.0, 2e-4, 5e-7, 2e-6, psi0=W.random_state(3, np.random.default_rng(8)))
    (out,) = run([req], precision=S.PREC_FP64, rotating_frame=False)
    ref = oracle_run(oracle_mod, req, frame=False)
    assert np.abs(out["states"].cpu().numpy() - ref["states"]).max() < 1e-10
