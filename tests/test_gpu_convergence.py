"""Precision and convergence study (spin-half Rabi field and spin-one sensing
field) at integration steps 1e-6, 1e-7, 1e-8 and 1e-9 s, FP64 and FP32-bulk.

For every case it records the error against the oracle at the same step
(implementation precision), against the oracle at the finest step
(truncation error, from which the observed order follows), the norm drift,
and -- to show why the cross-sample product is kept in FP64 -- the error of
chaining the same GPU operators in float32 instead of float64 (host-side
control arm).  Run with -s to see the table."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2204_05586_gb300 import spinsim as S, workloads as W  # noqa: E402

THREADS = os.cpu_count() or 4
STEPS = (1e-6, 1e-7, 1e-8, 1e-9)


def chain(ops, psi0, dtype):
    psi = psi0.astype(dtype)
    out = np.empty((ops.shape[0], ops.shape[1]), dtype=dtype)
    U = ops.astype(dtype)
    for k in range(U.shape[0]):
        psi = U[k] @ psi
        out[k] = psi
    return out


def study(oracle_mod, base):
    refs = {}
    for dt in STEPS:
        r = dict(base, dt=dt)
        refs[dt] = oracle_mod.simulate(r["spin_x2"], r["field"], r["t_start"], r["t_end"], dt, r["dt_out"],
                                       r["psi0"], threads=THREADS)["states"]
    finest = refs[STEPS[-1]]
    rows = []
    for prec in (S.PREC_FP64, S.PREC_FP32_BULK):
        for dt in STEPS:
            r = dict(base, dt=dt)
            with S.Simulator(precision=prec) as sim:
                out = sim.simulate([r], want_ops=True)[0]
                tau = sim.last_launch()["trotter_squares"]
            st = out["states"].cpu().numpy()
            ops = out["ops"].cpu().numpy()
            rows.append(dict(prec="fp64" if prec == S.PREC_FP64 else "fp32-bulk", dt=dt, tau=tau,
                             err_same=np.abs(st - refs[dt]).max(), err_conv=np.abs(st - finest).max(),
                             drift=np.abs(np.linalg.norm(st, axis=1) - 1).max(),
                             err_chain32=np.abs(chain(ops, r["psi0"], np.complex64) - refs[dt]).max()))
    return rows


def report(name, rows):
    print(f"\n{name}")
    print(f"{'precision':10s} {'dt':>8s} {'tau':>4s} {'|dpsi| same dt':>15s} {'|dpsi| vs 1e-9':>15s} "
          f"{'norm drift':>11s} {'fp32 chain':>11s}")
    for r in rows:
        print(f"{r['prec']:10s} {r['dt']:8.0e} {r['tau']:4d} {r['err_same']:15.3e} {r['err_conv']:15.3e} "
              f"{r['drift']:11.2e} {r['err_chain32']:11.2e}")


def orders(rows, prec):
    e = [r["err_conv"] for r in rows if r["prec"] == prec][:-1]
    return [np.log10(a / b) for a, b in zip(e[:-1], e[1:])]


def test_spin_half_rabi_field(oracle_mod):
    rows = study(oracle_mod, W.spin_half_rabi())
    report("spin-half: 20 kHz bias, 2x1 kHz drive, 5 ms, dt_out 1e-5", rows)
    for r in rows:
        assert r["err_same"] <= (1e-10 if r["prec"] == "fp64" else 1e-5), r
    o = orders(rows, "fp64")
    assert o[0] > 3.6, o      # CF4: fourth order while truncation dominates


def test_spin_one_sensing_field(oracle_mod):
    rows = study(oracle_mod, W.spin_one_sensing(t_end=2e-3))
    report("spin-one: 700 kHz bias, 2x1 kHz drive, q 400 Hz, pulse; first 2 ms, dt_out 1e-6", rows)
    for r in rows:
        assert r["err_same"] <= (1e-10 if r["prec"] == "fp64" else 1e-5), r
        assert r["drift"] <= (1e-11 if r["prec"] == "fp64" else 1e-14), r


def host_norm_drift(ops, psi0):
    """max_k | ||U_k ... U_1 psi0|| - 1 | chained in FP64 without renormalisation."""
    psi = np.asarray(psi0, dtype=np.complex128)
    worst = 0.0
    for U in ops[1:]:
        psi = U @ psi
        worst = max(worst, abs(np.linalg.norm(psi) - 1.0))
    return worst


def test_sensing_field_full_duration(oracle_mod):
    """The spin-one sensing field (700 kHz bias, 2x1 kHz drive, q = 400 Hz,
    Gaussian pulse) over its whole 100 ms at delta_t = 1e-6, 1e-7, 1e-8 s,
    every sample against the oracle at the same step; delta_t = 1e-9 over the
    first 10 ms (1e7 steps).  FP64 and FP32-bulk, the FP32-bulk norm drift
    before the chain's renormalisation, and the control arm whose
    cross-sample product runs in FP32 on the device (chain_precision = 1).
    The observed order comes from the 10 ms prefix against delta_t = 1e-9."""
    full = W.spin_one_sensing()
    prefix_end = 1e-2
    rows = []
    ref_prefix = {}
    for dt in STEPS:
        r = dict(full, dt=dt, t_end=prefix_end if dt == 1e-9 else full["t_end"])
        ref = oracle_mod.simulate(r["spin_x2"], r["field"], r["t_start"], r["t_end"], dt, r["dt_out"], r["psi0"],
                                  threads=THREADS)["states"]
        ref_prefix[dt] = ref[: int(round(prefix_end / r["dt_out"]))]
        for prec in (S.PREC_FP64, S.PREC_FP32_BULK):
            with S.Simulator(precision=prec) as sim:
                out = sim.simulate([r], want_ops=prec == S.PREC_FP32_BULK)[0]
                tau = sim.last_launch()["trotter_squares"]
            st = out["states"].cpu().numpy()
            row = dict(prec="fp64" if prec == S.PREC_FP64 else "fp32-bulk", dt=dt, tau=tau,
                       span_ms=1e3 * (r["t_end"] - r["t_start"]), err_same=np.abs(st - ref).max(),
                       drift=np.abs(np.linalg.norm(st, axis=1) - 1).max(), prefix=st[: len(ref_prefix[dt])])
            if prec == S.PREC_FP32_BULK:
                row["drift_raw"] = host_norm_drift(out["ops"].cpu().numpy(), r["psi0"])
                with S.Simulator(precision=prec, chain_fp32=True) as sim32:
                    o32 = sim32.simulate([r])[0]
                row["err_chain32"] = np.abs(o32["states"].cpu().numpy() - ref).max()
            rows.append(row)
    finest = ref_prefix[1e-9]
    for row in rows:
        row["err_conv"] = np.abs(row["prefix"] - finest).max()
    print("\nspin-one sensing field, 100 ms (1e-9: first 10 ms); |dpsi| vs the oracle")
    print(f"{'precision':10s} {'dt':>8s} {'span ms':>8s} {'tau':>4s} {'same dt':>10s} {'vs 1e-9':>10s} "
          f"{'drift':>9s} {'raw drift':>10s} {'fp32 chain':>11s}")
    for r in rows:
        print(f"{r['prec']:10s} {r['dt']:8.0e} {r['span_ms']:8.1f} {r['tau']:4d} {r['err_same']:10.2e} "
              f"{r['err_conv']:10.2e} {r['drift']:9.1e} {r.get('drift_raw', float('nan')):10.1e} "
              f"{r.get('err_chain32', float('nan')):11.2e}")
    # FP64 bound of this study: 3e-10.  Over 100 ms the drive phase 2 pi f t
    # reaches 4.4e5 rad, whose FP64 rounding (about 6e-11 rad) the oracle (the
    # argument formed at each node) and the library (reduced once per sample)
    # take differently; the per-sample errors of the drive axis add up as a
    # random walk (1.6e-10 at delta_t = 1e-6, 1e5 samples).  At delta_t = 1e-9
    # (1000 steps per sample) the oracle's full-matrix accumulation of each
    # sample adds its rounding (2.1e-10 over 10 ms).  The configured step
    # (1e-8) stays within 1e-10, as the full-size parity test requires.
    for r in rows:
        assert r["err_same"] <= (3e-10 if r["prec"] == "fp64" else 1e-5), (r["prec"], r["dt"], r["err_same"])
        if r["prec"] == "fp64" and r["dt"] == 1e-8:
            assert r["err_same"] <= 1e-10
        assert r["drift"] <= (1e-9 if r["prec"] == "fp64" else 1e-14), (r["prec"], r["dt"], r["drift"])
        if r["prec"] == "fp32-bulk":
            assert r["drift_raw"] < 1e-5 and r["err_chain32"] > r["err_same"]
    e = [r["err_conv"] for r in rows if r["prec"] == "fp64"]
    assert np.log10(e[0] / e[1]) > 3.6, e     # CF4: fourth order while truncation dominates
