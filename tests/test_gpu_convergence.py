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
