"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (max |psi_gpu - psi_oracle| over every sample and component):
  FP64 path       1e-10   (both sides are FP64; differences are rounding order)
  FP32-bulk path  1e-5    (against the oracle at its default tau = 24)
Spin projections are compared at 2x the state tolerance (|<J>| error <=
2 |dpsi| for normalised states).  Operators are compared entrywise.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2204_05586_gb300 import spinsim as S, workloads as W  # noqa: E402

THREADS = os.cpu_count() or 4
TOL = {S.PREC_FP64: 1e-10, S.PREC_FP32_BULK: 1e-5}


def oracle_run(O, req, tau=24, frame=True, method=0, want_ops=False, threads=THREADS):
    return O.simulate(req["spin_x2"], req["field"], req["t_start"], req["t_end"], req["dt"], req["dt_out"],
                      req["psi0"], rotating_frame=frame, tau=tau, method=method, want_ops=want_ops, threads=threads)


def gpu_run(reqs, want_ops=False, **cfg):
    with S.Simulator(**cfg) as sim:
        outs = sim.simulate(reqs, want_ops=want_ops)
        info = sim.last_launch()
    return outs, info


def assert_parity(out, ref, tol, what=""):
    assert out["status"] == S.OK, (what, out["status"])
    st = out["states"].cpu().numpy()
    assert st.shape == ref["states"].shape, (what, st.shape, ref["states"].shape)
    err = np.abs(st - ref["states"]).max() if st.size else 0.0
    assert err <= tol, f"{what}: max |dpsi| = {err:.3e} > {tol:.0e}"
    if out["spin"] is not None and st.size:
        serr = np.abs(out["spin"].cpu().numpy() - ref["spin"]).max()
        assert serr <= 2 * tol, f"{what}: max |d<J>| = {serr:.3e}"
    return err


# --------------------------------------------------------- full-size configs
@pytest.mark.parametrize("prec", [S.PREC_FP64, S.PREC_FP32_BULK])
def test_spin_half_rabi_full(oracle_mod, prec):
    """Spin-half, 20 kHz bias, 2 x 1 kHz drive, 5 ms, 500 samples x 100 steps."""
    req = W.spin_half_rabi()
    (out,), _ = gpu_run([req], precision=prec)
    assert_parity(out, oracle_run(oracle_mod, req), TOL[prec], "spin-half rabi")


@pytest.mark.parametrize("prec", [S.PREC_FP64, S.PREC_FP32_BULK])
def test_spin_one_sensing_full(oracle_mod, prec):
    """Spin-one sensing workload at full size: 100 ms, 1e5 samples x 100 steps
    (1e7 CF4 steps), compared on every sample."""
    req = W.spin_one_sensing()
    (out,), info = gpu_run([req], precision=prec)
    ref = oracle_run(oracle_mod, req)
    err = assert_parity(out, ref, TOL[prec], "spin-one sensing")
    norms = np.linalg.norm(out["states"].cpu().numpy(), axis=1)
    # FP64: no renormalisation, drift of 1e7 FP64 steps; FP32-bulk: states renormalised in FP64
    assert np.abs(norms - 1).max() < (1e-10 if prec == S.PREC_FP64 else 1e-14)
    print(f"spin-one sensing prec={prec}: max|dpsi| = {err:.3e}, launch {info}")


@pytest.mark.parametrize("prec", [S.PREC_FP64, S.PREC_FP32_BULK])
def test_spin_one_operators(oracle_mod, prec):
    req = W.spin_one_sensing(t_end=3e-4)
    (out,), _ = gpu_run([req], want_ops=True, precision=prec)
    ref = oracle_run(oracle_mod, req, want_ops=True)
    dU = np.abs(out["ops"].cpu().numpy() - ref["ops"]).max()
    assert dU <= (1e-12 if prec == S.PREC_FP64 else 1e-7), dU
    U = out["ops"].cpu().numpy()
    gram = np.einsum("kji,kjl->kil", U.conj(), U)
    tol = 1e-13 if prec == S.PREC_FP64 else 1e-10   # FP32-bulk: defect of the FP32 second-order rest
    assert np.abs(gram - np.eye(3)).max() < tol
    assert np.abs(np.linalg.det(U) - 1).max() < tol


@pytest.mark.parametrize("tau", [-1, 0, 4])
def test_fp32_matches_oracle_at_same_tau(oracle_mod, tau):
    """FP32-bulk against the oracle run with the same number of squarings
    (-1: the per-request choice the library reports)."""
    req = W.spin_one_sensing(t_end=2e-3)
    (out,), info = gpu_run([req], precision=S.PREC_FP32_BULK, tau=tau)
    used = info["trotter_squares"]
    assert tau < 0 or used == tau
    assert_parity(out, oracle_run(oracle_mod, req, tau=used), 1e-5, f"fp32 vs oracle tau={used}")


def test_automatic_tau_choice():
    """FP32-bulk default: the fewest squarings whose splitting-error bound,
    summed over the run, is <= 1e-6 -- none in the rotating frame of the
    sensing field, 9 in the lab frame for the full 100 ms run (step angle
    ~0.04 rad), fewer for a shorter run; FP64 keeps the paper's 24."""
    full, short = W.spin_one_sensing(), W.spin_one_sensing(t_end=2e-4)
    assert gpu_run([full], precision=S.PREC_FP32_BULK)[1]["trotter_squares"] == 0
    assert gpu_run([full], precision=S.PREC_FP32_BULK, rotating_frame=False)[1]["trotter_squares"] == 9
    (out,), info = gpu_run([short], precision=S.PREC_FP32_BULK, rotating_frame=False)
    assert info["trotter_squares"] == 4 and out["trotter_squares"] == 4
    assert gpu_run([short], precision=S.PREC_FP64)[1]["trotter_squares"] == 24
    # per request within one batch; the launch reports the largest
    outs, info = gpu_run([short, full, W.spin_half_rabi()], precision=S.PREC_FP32_BULK, rotating_frame=False)
    assert [o["trotter_squares"] for o in outs] == [4, 9, 0] and info["trotter_squares"] == 9


def test_fp32_lab_frame_is_flagged(oracle_mod):
    """FP32-bulk without the rotating frame: each 1 us sample of the 700 kHz
    field turns by 4.4 rad, the FP32 rounding of that rotation is the same in
    every sample and adds up, so the request is flagged (the run still
    completes and stays normalised); in the rotating frame, and in FP64, it is
    not flagged and meets the accuracy targets."""
    req = W.spin_one_sensing(t_end=2e-4)
    ref = oracle_run(oracle_mod, req, frame=False)
    (lab,), _ = gpu_run([req], precision=S.PREC_FP32_BULK, rotating_frame=False)
    assert lab["status"] == S.OK and lab["flags"] & S.WARN_FP32_LAB
    st = lab["states"].cpu().numpy()
    assert np.abs(np.linalg.norm(st, axis=1) - 1).max() < 1e-8
    err = np.abs(st - ref["states"]).max()
    print(f"\nFP32-bulk, lab frame, 0.2 ms sensing field: max |dpsi| = {err:.2e}")
    assert err < 1e-2
    (fr,), _ = gpu_run([req], precision=S.PREC_FP32_BULK)
    assert fr["flags"] == 0
    assert_parity(fr, oracle_run(oracle_mod, req), 1e-5, "rotating frame")
    (f64,), _ = gpu_run([req], precision=S.PREC_FP64, rotating_frame=False)
    assert f64["flags"] == 0
    assert_parity(f64, ref, 1e-10, "FP64 lab frame")


# ------------------------------------------------- methods, frames, fields
@pytest.mark.parametrize("spin", [1, 2])
@pytest.mark.parametrize("frame", [True, False])
@pytest.mark.parametrize("method", [S.METHOD_CF4, S.METHOD_MIDPOINT, S.METHOD_HEUN])
def test_methods_and_frames_fp64(oracle_mod, spin, frame, method):
    f = W.field(bias_hz=300e3, drive_x_hz=3e3, drive_y_hz=1e3, drive_hz=300.2e3, drive_phase=0.7,
                quad_hz=450.0 if spin == 2 else 0.0, pulses=[(120.0, 4e-4, 1e-4), (-60.0, 6e-4, 2e-4)])
    rng = np.random.default_rng(3)
    req = W.request(spin, f, 1e-4, 9e-4, 2e-8, 1e-6, psi0=W.random_state(spin + 1, rng))
    (out,), _ = gpu_run([req], precision=S.PREC_FP64, method=method, rotating_frame=frame)
    ref = oracle_run(oracle_mod, req, frame=frame, method=method)
    assert_parity(out, ref, 1e-10, f"spin={spin} frame={frame} method={method}")


@pytest.mark.parametrize("spin", [1, 2])
@pytest.mark.parametrize("method", [S.METHOD_MIDPOINT, S.METHOD_HEUN])
@pytest.mark.parametrize("tones", [(), ((1e3, 0.5e3, 300.5e3, 0.3),)])
def test_methods_fp32_bulk(oracle_mod, spin, method, tones):
    """FP32-bulk at the midpoint and Heun methods (rotating frame, small
    angles): the paired kernels, and with a further tone the tones kernel with
    the small-angle series, against the oracle at the same method."""
    f = W.field(bias_hz=300e3, drive_x_hz=3e3, drive_y_hz=1e3, drive_hz=300.2e3, drive_phase=0.7,
                quad_hz=450.0 if spin == 2 else 0.0, pulses=[(120.0, 4e-4, 1e-4), (-60.0, 6e-4, 2e-4)],
                tones=list(tones))
    rng = np.random.default_rng(5)
    req = W.request(spin, f, 1e-4, 2.1e-3, 2e-8, 1e-6, psi0=W.random_state(spin + 1, rng))
    (out,), _ = gpu_run([req], precision=S.PREC_FP32_BULK, method=method)
    ref = oracle_run(oracle_mod, req, method=method)
    assert_parity(out, ref, TOL[S.PREC_FP32_BULK], f"spin={spin} method={method} tones={len(tones)}")


@pytest.mark.parametrize("tau", [0, 3, 8])
def test_trotter_squares_parameter(oracle_mod, tau):
    req = W.spin_one_sensing(t_end=5e-4, dt=1e-7)
    (out,), info = gpu_run([req], precision=S.PREC_FP64, tau=tau)
    assert info["trotter_squares"] == tau
    assert_parity(out, oracle_run(oracle_mod, req, tau=tau), 1e-10, f"tau={tau}")


def test_large_angle_fallbacks(oracle_mod):
    """Lab frame with few squarings: step angles beyond the series range."""
    f = W.field(bias_hz=2e5, drive_x_hz=8e4, drive_hz=1.9e5, quad_hz=3e4)
    req = W.request(2, f, 0.0, 2e-4, 5e-7, 1e-5)
    (out,), _ = gpu_run([req], precision=S.PREC_FP64, rotating_frame=False, tau=2)
    assert_parity(out, oracle_run(oracle_mod, req, tau=2, frame=False), 1e-10, "large angles")
    req = W.request(1, f, 0.0, 2e-4, 5e-7, 1e-5)
    (out,), _ = gpu_run([req], precision=S.PREC_FP64, rotating_frame=False)
    assert_parity(out, oracle_run(oracle_mod, req, frame=False), 1e-10, "large angles half")


# --------------------------------------------------------------- edge cases
def test_edge_cases_in_one_batch(oracle_mod):
    """K = 0, K = 1, L = 1, ragged chunk and run tails, K < 16, mixed spins,
    and invalid requests that must not stop the valid ones."""
    base = W.field(bias_hz=150e3, drive_x_hz=4e3, drive_hz=150.5e3, quad_hz=300.0, pulses=[(90.0, 3e-4, 1e-4)])
    reqs = [
        W.request(2, base, 0.0, 0.0, 1e-8, 1e-6),          # K = 0
        W.request(2, base, 0.0, 1e-6, 1e-8, 1e-6),         # K = 1: only psi_0
        W.request(1, base, 0.0, 7e-6, 1e-6, 1e-6),         # L = 1, K = 7
        W.request(2, base, 2e-5, 2e-5 + 529e-6, 1e-7, 1e-6),   # K = 529: ragged chunk + run tail
        W.request(1, base, 0.0, 1037e-6, 2.5e-7, 1e-6),    # K = 1037, L = 4
        W.request(2, base, 0.0, 3e-6, 1e-6 / 3, 1e-6),     # L = 3: segments of 0, 1, 1, 1 steps
        W.request(2, base, 0.0, 1e-5, 3e-7, 1e-6),         # invalid ratio
        W.request(2, base, 0.0, 1e-5, 1e-8, 1e-6, psi0=[1.0, 0.5, 0.0]),  # not normalised
    ]
    with S.Simulator(precision=S.PREC_FP64) as sim:
        outs = sim.allocate(reqs[:6] + [W.request(2, base, 0.0, 1e-5, 1e-7, 1e-6)] * 2)
        res = sim.results_struct(outs)
        arr = (S.spinsim_request * len(reqs))(*[S.make_request(q) for q in reqs])
        st = S.spinsim_simulate(sim.handle, arr, res, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
    assert st == S.E_STEP_RATIO
    assert res[6].status == S.E_STEP_RATIO and res[7].status == S.E_NORM
    assert [r.n_samples for r in res[:6]] == [0, 1, 7, 529, 1037, 3]
    for i in range(6):
        r = reqs[i]
        ref = oracle_run(oracle_mod, r)
        view = S.Simulator._view(outs[i], res[i])
        assert_parity(view, ref, 1e-10, f"edge case {i}")


def test_chain_tree_heights_in_one_batch(oracle_mod):
    """One FP64 batch whose chain trees have 0, 1, 2 and 3 levels above the lane
    runs (K = 1 ... 300,000 at one step per sample), spin-one and spin-half:
    the level-0 apply, the fused top, and the down-sweeps at levels 1 and 2 all
    run, for simulations of different heights side by side.  Every sample of
    every simulation against the oracle."""
    base = W.field(bias_hz=120e3, drive_x_hz=3e3, drive_hz=120.4e3, quad_hz=250.0, pulses=[(60.0, 0.1, 0.03)])
    Ks = [1, 128, 129, 4097, 140000, 300000]
    reqs = [W.request(2, base, 0.0, K * 1e-6, 1e-6, 1e-6) for K in Ks]
    reqs += [W.request(1, base, 1e-4, 1e-4 + K * 1e-6, 1e-6, 1e-6) for K in (4097, 300000)]
    outs, _ = gpu_run(reqs, precision=S.PREC_FP64)
    for req, out in zip(reqs, outs):
        ref = oracle_run(oracle_mod, req)
        assert_parity(out, ref, TOL[S.PREC_FP64], f"spin_x2 {req['spin_x2']} K {out['K']}")


@pytest.mark.parametrize("prec", [S.PREC_FP64, S.PREC_FP32_BULK])
def test_neural_pulse_field(oracle_mod, prec):
    """The paper's benchmark field (Eq. neural_pulse: 700 kHz bias, 2 x 1 kHz drive,
    a 70 Hz single sine cycle of 1 ms on J_z), the cycle inside a 3 ms run, at
    the paper's 100 ns step: spin-one and spin-half, every sample against the
    oracle."""
    for spin_x2 in (2, 1):
        req = W.neural_pulse(t_end=3e-3, t_p=1.2e-3, spin_x2=spin_x2)
        (out,), _ = gpu_run([req], precision=prec)
        assert_parity(out, oracle_run(oracle_mod, req), TOL[prec], f"neural pulse spin_x2 {spin_x2}")


@pytest.mark.parametrize("prec", [S.PREC_FP64, S.PREC_FP32_BULK])
def test_neural_workload_full_size(oracle_mod, prec):
    """The paper's benchmark field exactly as the bench times it (100 ms at the
    100 ns step, 1e5 samples x 10 steps, graph replay): every sample."""
    req = W.neural_pulse()
    (out,), _ = gpu_run([req], precision=prec, use_graphs=True)
    assert_parity(out, oracle_run(oracle_mod, req), TOL[prec], "neural workload, full size")


@pytest.mark.parametrize("frame", [True, False])
def test_mixed_pulse_kinds_fp64(oracle_mod, frame):
    """Gaussian and sine-cycle pulses in one field, both frames, FP64, with the
    cycle's edges between steps."""
    f = W.field(bias_hz=90e3, drive_x_hz=3e3, drive_y_hz=1e3, drive_hz=90.2e3, quad_hz=200.0,
                pulses=[(150.0, 0.4e-3, 0.1e-3), (400.0, 0.13e-3, 0.37e-3, "sine"), (-90.0, 0.7e-3, 0.2e-3, "sine")])
    req = W.request(2, f, 0.0, 1.2e-3, 4e-8, 2e-6)
    (out,), _ = gpu_run([req], precision=S.PREC_FP64, rotating_frame=frame)
    assert_parity(out, oracle_run(oracle_mod, req, frame=frame), TOL[S.PREC_FP64], f"mixed pulses frame {frame}")


def test_capacity_error_and_spin_only_outputs(oracle_mod):
    req = W.spin_half_rabi(t_end=1e-4)
    with S.Simulator(precision=S.PREC_FP64) as sim:
        outs = sim.allocate([req], want_spin=False)
        outs[0]["K"] = 5        # too small
        res = sim.results_struct(outs)
        st = S.spinsim_simulate(sim.handle, [S.make_request(req)], res, 0)
        torch.cuda.synchronize()
    assert st == S.E_CAPACITY and res[0].status == S.E_CAPACITY


# ------------------------------------------------------------- invariance
def test_launch_shape_does_not_change_results():
    req = W.spin_one_sensing(t_end=3e-3)
    got = []
    for lanes in (1, 2, 4):
        for block in (64, 256):
            (out,), info = gpu_run([req], precision=S.PREC_FP32_BULK, lanes=lanes, block=block)
            assert info["lanes_per_sample"] == lanes and info["threads_per_block"] == block
            got.append(out["states"].cpu().numpy())
    for g in got[1:]:
        assert np.array_equal(g, got[0])
    # the full sensing run: one round of bulk tiles and a tail whose split
    # (lanes per pair) follows from the shape, every shape bit for bit alike
    req = W.spin_one_sensing()
    got = []
    for lanes, block in ((1, 256), (1, 64), (2, 128), (4, 64)):
        (out,), _ = gpu_run([req], precision=S.PREC_FP32_BULK, lanes=lanes, block=block)
        got.append(out["states"].cpu().numpy())
    for g in got[1:]:
        assert np.array_equal(g, got[0])


def test_alone_equals_in_batch():
    reqs = W.sweep(24, t_min=1e-4, t_max=3e-3)
    alone = []
    for q in reqs[:4]:
        (o,), _ = gpu_run([q], precision=S.PREC_FP32_BULK, lanes=4, block=128)
        alone.append(o["states"].cpu().numpy())
    outs, _ = gpu_run(reqs[::-1], precision=S.PREC_FP32_BULK, lanes=1, block=256)
    for i in range(4):
        assert np.array_equal(outs[len(reqs) - 1 - i]["states"].cpu().numpy(), alone[i])


def test_paired_kernel_odd_sample_counts(oracle_mod):
    """Spin-one FP32-bulk small-angle requests run two samples per thread;
    the host places every simulation of the launch at an even operator index
    (an odd K takes one unused slot).  Simulations of odd and even K (1 to 129,
    both tau = 0 and tau at run time) in one batch equal their runs alone bit
    for bit, whatever their place in the batch, and match the oracle."""
    base = W.field(bias_hz=700e3, drive_x_hz=2e3, drive_hz=700.3e3, quad_hz=300.0, pulses=[(40.0, 1e-5, 3e-5)])
    reqs = [W.request(2, base, 0.0, K * 1e-6, 1e-8 if K % 2 else 2e-8, 1e-6) for K in (1, 2, 3, 5, 64, 65, 128, 129)]
    strong = W.field(bias_hz=700e3, drive_x_hz=20e3, drive_hz=700.3e3, quad_hz=300.0, pulses=[(2e3, 3e-5, 2e-5)])
    reqs.append(W.request(2, strong, 0.0, 77e-6, 1e-7, 1e-6))        # a strong drive: tau > 0 at run time
    outs, _ = gpu_run(reqs, precision=S.PREC_FP32_BULK)
    outs_rev, _ = gpu_run(reqs[::-1], precision=S.PREC_FP32_BULK)
    for i, q in enumerate(reqs):
        (alone,), _ = gpu_run([q], precision=S.PREC_FP32_BULK)
        a = alone["states"].cpu().numpy()
        assert np.array_equal(outs[i]["states"].cpu().numpy(), a), i
        assert np.array_equal(outs_rev[len(reqs) - 1 - i]["states"].cpu().numpy(), a), i
        assert_parity(outs[i], oracle_run(oracle_mod, q), TOL[S.PREC_FP32_BULK], f"K={a.shape[0]}")


def test_paired_tail_tiles_mix_segment_splits(oracle_mod):
    """One batch of more than a wave of paired samples whose simulations take
    5, 20 and 150 steps per sample (segment splits 2, 4 and 8): its tail tiles
    use as many lanes per pair as the smallest split allows, so they hold pairs
    whose lanes each run several segments, and two lanes per pair share the
    FP64 epilogue.  Every simulation equals its run alone bit for bit, in
    either order, and matches the oracle."""
    base = W.field(bias_hz=700e3, drive_x_hz=1e3, drive_hz=700.2e3, quad_hz=300.0, pulses=[(30.0, 6e-3, 2e-3)])
    reqs = [W.request(2, base, 0.0, K * 1e-6, 1e-6 / L, 1e-6) for K, L in ((26001, 5), (31000, 20), (27003, 150))]
    outs, _ = gpu_run(reqs, precision=S.PREC_FP32_BULK, lanes=1, block=256)
    outs_rev, _ = gpu_run(reqs[::-1], precision=S.PREC_FP32_BULK, lanes=1, block=256)
    for i, q in enumerate(reqs):
        (alone,), _ = gpu_run([q], precision=S.PREC_FP32_BULK, lanes=1, block=256)
        a = alone["states"].cpu().numpy()
        assert np.array_equal(outs[i]["states"].cpu().numpy(), a), i
        assert np.array_equal(outs_rev[len(reqs) - 1 - i]["states"].cpu().numpy(), a), i
        assert_parity(outs[i], oracle_run(oracle_mod, q), TOL[S.PREC_FP32_BULK], f"L={round(q['dt_out'] / q['dt'])}")


def test_host_buffers_match_device_buffers():
    req = W.spin_one_sensing(t_end=2e-3)
    (dev,), _ = gpu_run([req], precision=S.PREC_FP32_BULK)
    with S.Simulator(precision=S.PREC_FP32_BULK) as sim:
        outs = sim.allocate([req], want_ops=True, device="cpu", pin_memory=False)
        res = sim.results_struct(outs)
        st = S.spinsim_simulate(sim.handle, [S.make_request(req)], res, 0)
        torch.cuda.synchronize()
    assert st == S.OK
    host = torch.view_as_complex(outs[0]["states"]).numpy()
    assert np.array_equal(host, dev["states"].cpu().numpy())


@pytest.mark.parametrize("direct", [False, True])
def test_pinned_host_outputs_written_directly_or_staged(direct):
    """Pinned host result buffers (one block, as a large batch allocates them),
    written by the kernels directly (direct_host_outputs = 1) or staged and
    copied back: states, <J> and operators equal the device-buffer run bit for
    bit, for a mixed batch (both spins, uneven lengths, graph replay on the
    second call), and the launch info counts the bytes that reached the host."""
    reqs = W.sweep(5, t_min=1e-4, t_max=3e-3) + [W.spin_half_rabi(t_end=2e-3), W.spin_one_sensing(t_end=1e-3)]
    dev, _ = gpu_run(reqs, want_ops=True, precision=S.PREC_FP32_BULK)
    with S.Simulator(precision=S.PREC_FP32_BULK, use_graphs=True, direct_host_outputs=direct) as sim:
        outs = sim.allocate(reqs, want_ops=True, device="cpu", pin_memory=True, one_buffer=True)
        res = sim.results_struct(outs)
        arr = (S.spinsim_request * len(reqs))(*[S.make_request(q) for q in reqs])
        for call in range(2):
            for o in outs:
                o["states"].fill_(float("nan"))
            assert S.spinsim_simulate(sim.handle, arr, res, 0) == S.OK
            torch.cuda.synchronize()
            info = sim.last_launch()
            want = sum(o["K"] * (16 * (q["spin_x2"] + 1) + 24 + 16 * (q["spin_x2"] + 1) ** 2) for o, q in zip(outs, reqs))
            assert info["d2h_bytes"] == want
            for o, d in zip(outs, dev):
                K = o["K"]
                assert np.array_equal(torch.view_as_complex(o["states"][:K]).numpy(), d["states"].cpu().numpy())
                assert np.array_equal(o["spin"][:K].numpy(), d["spin"].cpu().numpy())
                assert np.array_equal(torch.view_as_complex(o["ops"][:K]).numpy(), d["ops"].cpu().numpy())


def test_graph_replay_matches_eager():
    reqs = W.sweep(16, t_min=1e-4, t_max=2e-3)
    eager, _ = gpu_run(reqs, precision=S.PREC_FP32_BULK, lanes=2, block=128)
    with S.Simulator(precision=S.PREC_FP32_BULK, lanes=2, block=128, use_graphs=True, profile=True) as sim:
        outs = sim.allocate(reqs)
        first = sim.simulate(reqs, outs=outs)
        a = [o["states"].cpu().numpy().copy() for o in first]
        for o in outs:
            o["states"].zero_()
        second = sim.simulate(reqs, outs=outs)
        info = sim.last_launch()
        assert info["graph_replayed"] == 1
        # the replay records the profiling events as graph nodes: live kernel times
        assert info["integrate_ms"] > 0.0 and info["chain_ms"] > 0.0
        b = [o["states"].cpu().numpy() for o in second]
    for x, y, e in zip(a, b, eager):
        assert np.array_equal(x, y) and np.array_equal(x, e["states"].cpu().numpy())


# ------------------------------------------------------- batched sweep
def test_sweep_full_size_sampled(oracle_mod):
    """4096-simulation sweep at full size (FP32-bulk) in one launch: every
    state stays normalised, and a stratified subset of simulations (shortest,
    median, longest, and some between) matches the oracle on every sample."""
    reqs = W.sweep(4096)
    outs, info = gpu_run(reqs, precision=S.PREC_FP32_BULK)
    assert all(o["status"] == S.OK for o in outs)
    worst = 0.0
    for o in outs[::97]:
        worst = max(worst, float((o["states"].abs().pow(2).sum(1) - 1).abs().max()))
    assert worst < 1e-9
    T = np.array([q["t_end"] for q in reqs])
    order = np.argsort(T)
    pick = [order[0], order[1], order[len(order) // 4], order[len(order) // 2], order[-1]]
    for i in pick:
        ref = oracle_run(oracle_mod, reqs[i])
        assert_parity(outs[i], ref, 1e-5, f"sweep sim {i} (T={T[i]:.4f})")


# ------------------------------------------------------------------ serving
def test_served_results_equal_alone():
    arrivals, reqs = W.serving_stream(60, t_max=3e-3)
    alone = []
    for q in reqs:
        (o,), _ = gpu_run([q], precision=S.PREC_FP32_BULK)
        alone.append(o["states"].cpu().numpy())
    with S.Simulator(precision=S.PREC_FP32_BULK) as sim:
        outs = sim.allocate(reqs)
        res = sim.results_struct(outs)
        reqs_c = [S.make_request(q) for q in reqs]
        tickets = []
        for q, r in zip(reqs_c, res):
            st, t = S.spinsim_submit(sim.handle, q, r)
            assert st == S.OK
            tickets.append(t)
        for t in tickets:
            assert S.spinsim_poll(sim.handle, t, 10_000_000) == S.OK
        assert S.spinsim_poll(sim.handle, tickets[0], 0) == S.E_ARG   # forgotten once reported
    for o, r, a in zip(outs, res, alone):
        assert r.status == S.OK
        assert np.array_equal(torch.view_as_complex(o["states"][:o["K"]]).cpu().numpy(), a)
