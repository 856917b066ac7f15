"""The library's range entry points (spinsim_range_begin / spinsim_range_finish)
on the GPU: one long simulation split into ranges, each on its own handle as a
separate process would hold it, the range products exchanged in process
(paper_2204_05586_gb300.sharded), the states compared with the unsplit run and
with the oracle.  One GPU runs every range, one after another."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2204_05586_gb300 import sharded as SH, spinsim as S, workloads as W  # noqa: E402

TOL = {S.PREC_FP64: 1e-10, S.PREC_FP32_BULK: 1e-5}


def split_run(req, world, prec):
    K = S.spinsim_counts(S.make_request(req))[1]
    rs = SH.ranges(K, world)
    backends = [SH.CudaRange(precision=prec) for _ in range(world)]
    try:
        aggs = [b.begin(SH.range_request(req, k0, k1, r == world - 1)) for r, (b, (k0, k1)) in
                enumerate(zip(backends, rs))]
        psis = SH.entering_states(aggs, req["psi0"])
        parts = [b.finish(p)[: k1 - k0] for b, p, (k0, k1) in zip(backends, psis, rs)]
    finally:
        for b in backends:
            b.close()
    return np.concatenate(parts), aggs


@pytest.mark.parametrize("prec", [S.PREC_FP64, S.PREC_FP32_BULK])
@pytest.mark.parametrize("spin_x2", [2, 1])
def test_split_equals_unsplit(oracle_mod, prec, spin_x2):
    """A 20 ms sensing-like run (2e4 samples x 100 steps) in 1, 2 and 3 ranges:
    equal to the unsplit library run and to the oracle."""
    req = W.spin_one_sensing(t_end=2e-2) if spin_x2 == 2 else W.spin_half_rabi(t_end=2e-2, dt=1e-8, dt_out=1e-6)
    with S.Simulator(precision=prec) as sim:
        (full,) = sim.simulate([req])
    full = full["states"].cpu().numpy()
    ref = oracle_mod.simulate(req["spin_x2"], req["field"], req["t_start"], req["t_end"], req["dt"], req["dt_out"],
                              req["psi0"], threads=16)["states"]
    for world in (1, 2, 3):
        got, aggs = split_run(req, world, prec)
        assert got.shape == full.shape
        # the same operators up to the rounding of each range's start time, which
        # moves a 700 kHz drive phase by ~1e-12 rad, and FP64 products
        assert np.abs(got - full).max() < (1e-10 if prec == S.PREC_FP64 else 1e-6), world
        assert np.abs(got - ref).max() < TOL[prec], world
        # every range product is unitary: to FP64 rounding, or for FP32-bulk to the
        # operators' departure from unitarity (~1e-11 per sample; the apply
        # renormalises each written state)
        for A in aggs:
            assert np.abs(A.conj().T @ A - np.eye(A.shape[0])).max() < (1e-10 if prec == S.PREC_FP64 else 1e-6)


def test_range_errors():
    req = W.spin_one_sensing(t_end=1e-3)
    with S.Simulator(precision=S.PREC_FP64) as sim:
        h = sim.handle
        assert S.spinsim_range_finish(h, req["psi0"]) == S.E_ARG          # nothing begun
        outs = sim.allocate([req])
        res = S.Simulator.results_struct(outs)
        st, _ = S.spinsim_range_begin(h, S.make_request(req), res[0])
        assert st == S.OK
        assert S.spinsim_range_finish(h, [1.0, 0.5, 0.0]) == S.E_NORM    # not normalised
        assert S.spinsim_range_finish(h, req["psi0"]) == S.E_ARG          # the range was closed by the error
        st, _ = S.spinsim_range_begin(h, S.make_request(req), res[0])
        sim.simulate([req])                                              # another call discards the range
        assert S.spinsim_range_finish(h, req["psi0"]) == S.E_ARG
        short = S.Simulator.results_struct(sim.allocate([W.spin_one_sensing(t_end=5e-4)]))
        st, _ = S.spinsim_range_begin(h, S.make_request(req), short[0])
        assert st == S.E_CAPACITY
