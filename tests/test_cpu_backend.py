"""The multicore CPU backend (include/spinsim_cpu.h, libspinsim_cpu.so): the
integrator's per-sample arithmetic compiled for the host and run over worker
threads, then the chain in order.  Checked on the CPU against the oracle
(same tolerances as the GPU path), for determinism across thread counts, for
batch independence and for its separation from the GPU library."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2204_05586_gb300 import cpu_backend as C, spinsim as S, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = {S.PREC_FP64: 1e-10, S.PREC_FP32_BULK: 1e-5}
THREADS = os.cpu_count() or 2


def oracle_run(O, req, frame=True, method=0, tau=24, want_ops=False):
    return O.simulate(req["spin_x2"], req["field"], req["t_start"], req["t_end"], req["dt"], req["dt_out"],
                      req["psi0"], rotating_frame=frame, tau=tau, method=method, want_ops=want_ops, threads=THREADS)


def check(out, ref, tol, what):
    assert out["status"] == S.OK, (what, out["status"])
    assert out["states"].shape == ref["states"].shape, what
    if out["states"].size:
        err = np.abs(out["states"] - ref["states"]).max()
        assert err <= tol, f"{what}: {err:.3e}"
        assert np.abs(out["spin"] - ref["spin"]).max() <= 2 * tol, what
    return out


def test_header_symbol_is_exported_by_the_cpu_library_only():
    src = open(os.path.join(ROOT, "include", "spinsim_cpu.h")).read()
    decl = set(re.findall(r"^\s*int\s+(spinsim_[a-z_]+)\s*\(", src, re.M))
    assert decl == {"spinsim_cpu_simulate"}
    lib = C.load()
    assert hasattr(lib, "spinsim_cpu_simulate")
    # the GPU library and its binding neither contain nor load the CPU backend
    assert not hasattr(S.load(), "spinsim_cpu_simulate")
    assert "cpu_backend" not in open(os.path.join(ROOT, "paper_2204_05586_gb300", "spinsim.py")).read()


@pytest.mark.parametrize("prec", [S.PREC_FP32_BULK, S.PREC_FP64])
def test_sensing_and_rabi_against_oracle(oracle_mod, prec):
    """Spin-one sensing field (2 ms, 2e5 steps) and the spin-half Rabi run
    (5e4 steps): states, <J> and every operator."""
    for req in (W.spin_one_sensing(t_end=2e-3), W.spin_half_rabi()):
        (out,) = C.simulate([req], precision=prec, want_ops=True)
        ref = oracle_run(oracle_mod, req, want_ops=True)
        check(out, ref, TOL[prec], f"spin_x2={req['spin_x2']} prec={prec}")
        assert np.abs(out["ops"] - ref["ops"]).max() <= TOL[prec]
        if prec == S.PREC_FP32_BULK:
            assert np.abs(np.linalg.norm(out["states"], axis=1) - 1).max() < 1e-14


@pytest.mark.parametrize("spin", [1, 2])
@pytest.mark.parametrize("frame", [True, False])
@pytest.mark.parametrize("method", [S.METHOD_CF4, S.METHOD_MIDPOINT, S.METHOD_HEUN])
def test_methods_and_frames_fp64(oracle_mod, spin, frame, method):
    f = W.field(bias_hz=300e3, drive_x_hz=3e3, drive_y_hz=1e3, drive_hz=300.2e3, drive_phase=0.7,
                quad_hz=450.0 if spin == 2 else 0.0, pulses=[(120.0, 4e-4, 1e-4), (-60.0, 6e-4, 2e-4)])
    rng = np.random.default_rng(3)
    req = W.request(spin, f, 1e-4, 4e-4, 2e-8, 1e-6, psi0=W.random_state(spin + 1, rng))
    (out,) = C.simulate([req], precision=S.PREC_FP64, method=method, rotating_frame=frame)
    check(out, oracle_run(oracle_mod, req, frame=frame, method=method), 1e-10, f"{spin} {frame} {method}")


@pytest.mark.parametrize("prec", [S.PREC_FP32_BULK, S.PREC_FP64])
def test_tones_and_pulse_kinds(oracle_mod, prec):
    """Further tones, a Gaussian and a single-sine-cycle pulse together."""
    f = W.field(bias_hz=700e3, drive_x_hz=2e3, drive_hz=700e3, quad_hz=300.0,
                pulses=[(60.0, 0.2e-3, 0.5e-3, "sine"), (40.0, 0.6e-3, 0.1e-3)],
                tones=[(1.2e3, 0.9e3, 700.4e3, 0.8), (0.0, 1.5e3, 740e3, -1.3), (0.7e3, 0.0, 7e3, 2.2)])
    req = W.request(2, f, 0.0, 1e-3, 1e-8, 1e-6, psi0=W.random_state(3, np.random.default_rng(5)))
    (out,) = C.simulate([req], precision=prec)
    check(out, oracle_run(oracle_mod, req), TOL[prec], "tones")


@pytest.mark.parametrize("spin", [2, 1])
def test_small_angle_sine_cycle_variant(oracle_mod, spin):
    """The paper's benchmark field (a single sine cycle on J_z) in FP32-bulk takes
    the small-angle kernel's twin with sine cycles; with a Gaussian beside the
    cycle both pulse kinds meet in one step loop.  Against the oracle at the
    FP32-bulk tolerance, both spins."""
    for req in (W.neural_pulse(t_end=3e-3, t_p=1.2e-3, spin_x2=spin),
                W.request(spin, W.field(bias_hz=700e3, drive_x_hz=2e3, drive_hz=700.1e3,
                                        quad_hz=250.0 if spin == 2 else 0.0,
                                        pulses=[(40.0, 0.6e-3, 0.2e-3), (70.0, 1.0e-3, 1e-3, "sine")]),
                          0.0, 2.5e-3, 1e-7, 1e-6)):
        (out,) = C.simulate([req], precision=S.PREC_FP32_BULK)
        check(out, oracle_run(oracle_mod, req), 1e-5, f"small-angle sine cycles, spin_x2 {spin}")


def test_batch_edge_cases_and_determinism(oracle_mod):
    """A batch with K = 0, K = 1, L = 1, L = 3, both spins, an invalid request
    and a short capacity: statuses as documented, every valid request equal
    (bitwise) to its run alone, and bitwise independent of the thread count."""
    good = [W.spin_one_sensing(t_end=0.0), W.spin_one_sensing(t_end=1e-6), W.spin_one_sensing(t_end=3e-4, dt=1e-6),
            W.spin_one_sensing(t_end=3e-4, dt=1e-6 / 3), W.spin_half_rabi(t_end=2e-3), W.spin_one_sensing(t_end=1e-3)]
    bad = W.spin_one_sensing(t_end=1e-4)
    bad["psi0"] = np.array([1.0, 0.5, 0.0], dtype=np.complex128)      # not normalised
    reqs = good[:3] + [bad] + good[3:]
    outs = C.simulate(reqs, threads=3)
    assert outs[3]["status"] == S.E_NORM
    alone = [C.simulate([q], threads=1)[0] for q in good]
    for o, a, q in zip(outs[:3] + outs[4:], alone, good):
        assert o["status"] == S.OK and np.array_equal(o["states"], a["states"])
        ref = oracle_run(oracle_mod, q)
        check(o, ref, 1e-5, "edge case")
    # capacity below K
    res = (S.spinsim_result * 1)()
    st = np.zeros((5, 3), np.complex128)
    res[0].states, res[0].capacity = st.ctypes.data, 5
    reqs_c = (S.spinsim_request * 1)(S.make_request(W.spin_one_sensing(t_end=1e-5)))
    assert C.spinsim_cpu_simulate(C.make_cpu_config(), reqs_c, res, 2) == S.E_CAPACITY
    assert res[0].status == S.E_CAPACITY


def test_variants_agree():
    """The small-angle variant (sensing, FP32) and the tones variant (the same
    request with a zero-amplitude tone) agree up to FP32 rounding."""
    a = W.spin_one_sensing(t_end=2e-3)
    b = W.spin_one_sensing(t_end=2e-3)
    b["field"]["tones"] = [(0.0, 0.0, 701e3, 0.3)]
    (oa,), (ob,) = C.simulate([a]), C.simulate([b])
    assert np.abs(oa["states"] - ob["states"]).max() < 2e-6


def test_call_errors():
    cfg = C.make_cpu_config()
    reqs = (S.spinsim_request * 1)(S.make_request(W.spin_one_sensing(t_end=1e-5)))
    res = (S.spinsim_result * 1)()
    lib = C.load()
    assert lib.spinsim_cpu_simulate(ctypes.byref(cfg), reqs, res, -1, 0) == S.E_ARG
    assert lib.spinsim_cpu_simulate(ctypes.byref(cfg), reqs, res, 1, -2) == S.E_ARG
    bad = C.make_cpu_config(method=7)
    assert lib.spinsim_cpu_simulate(ctypes.byref(bad), reqs, res, 1, 0) == S.E_ARG
    assert lib.spinsim_cpu_simulate(ctypes.byref(cfg), reqs, res, 1, 0) == S.E_ARG   # states NULL
    assert res[0].status == S.E_ARG


def su3_request(t_end=1e-3):
    f = W.field(bias_hz=700e3, drive_x_hz=2e3, drive_hz=700e3, quad_hz=300.0, pulses=[(60.0, 0.5e-3, 0.2e-3)],
                qdrives=[(1.2e3, 0.7e3, 700.3e3, 0.4), (0.9e3, 0.9e3, 1400.2e3, -0.8)],
                tones=[(0.5e3, 0.2e3, 699.7e3, 1.0)])
    return W.request(2, f, 0.0, t_end, 1e-8, 1e-6, psi0=W.random_state(3, np.random.default_rng(4)))


@pytest.mark.parametrize("frame", [True, False])
def test_full_su3_fp64_against_oracle(oracle_mod, frame):
    """Both quadrupole drives (near the one- and two-quantum resonances), a
    tone and a pulse: FP64, every sample."""
    req = su3_request()
    (out,) = C.simulate([req], precision=S.PREC_FP64, rotating_frame=frame)
    check(out, oracle_run(oracle_mod, req, frame=frame), 1e-10, f"su3 frame={frame}")


def test_full_su3_needs_fp64_and_spin_one():
    (o32,) = C.simulate([su3_request(1e-4)])
    assert o32["status"] == S.E_UNSUPPORTED
    half = W.spin_half_rabi(t_end=1e-4)
    half["field"]["qdrives"] = [(1.0, 1.0, 1.0, 0.0)]
    (oh,) = C.simulate([half], precision=S.PREC_FP64)
    assert oh["status"] == S.E_ARG


@pytest.mark.parametrize("method", [S.METHOD_MIDPOINT, S.METHOD_HEUN])
def test_full_su3_other_methods(oracle_mod, method):
    req = su3_request(5e-4)
    (out,) = C.simulate([req], precision=S.PREC_FP64, method=method)
    check(out, oracle_run(oracle_mod, req, method=method), 1e-10, f"su3 method={method}")


def test_full_su3_scaled_and_squared_steps(oracle_mod):
    """Lab frame with a 0.5 us step: every exponent's norm is above 1, so the
    general exponential halves it three times and squares back three times."""
    f = W.field(bias_hz=700e3, drive_x_hz=40e3, drive_hz=700e3, quad_hz=3e3,
                qdrives=[(30e3, 20e3, 700e3, 0.4), (25e3, 25e3, 1400e3, -0.8)])
    req = W.request(2, f, 0.0, 2e-4, 5e-7, 2e-6, psi0=W.random_state(3, np.random.default_rng(8)))
    (out,) = C.simulate([req], precision=S.PREC_FP64, rotating_frame=False)
    check(out, oracle_run(oracle_mod, req, frame=False), 1e-10, "su3 squared")
