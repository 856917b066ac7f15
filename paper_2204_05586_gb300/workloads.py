"""Seeded synthetic workloads shaped like the paper's sensing benchmark.

This module only draws parameters; it holds none of the integration method's
arithmetic, and it is the one module that both the CUDA path's callers and
the oracle's callers import.  A request is a plain ``dict``:

    spin_x2        1 = spin-half, 2 = spin-one
    field          dict(bias_hz, drive_x_hz, drive_y_hz, drive_hz, drive_phase,
                        quad_hz, pulses=[(amp_hz, centre_s, width_s[, kind]), ...])
                   w_x = 2 pi drive_x_hz cos(2 pi drive_hz t + drive_phase)
                   w_y = 2 pi drive_y_hz sin(2 pi drive_hz t + drive_phase)
                   w_z = 2 pi (bias_hz + sum_p amp_p shape_p(t))
                   w_q = 2 pi quad_hz
                   shape_p: kind "gauss" (default) exp(-(t-c_p)^2 / (2 w_p^2));
                   kind "sine" a single cycle sin(2 pi (t-c_p)/w_p) for
                   c_p <= t < c_p + w_p, else 0 (the paper's sinp pulse)
                   tones=[(x_hz, y_hz, hz, phase), ...]: up to 3 further drive
                   tones, each added to w_x, w_y like the first
                   qdrives=[(x_hz, y_hz, hz, phase), (x_hz, y_hz, hz, phase)]: up to
                   two quadrupole drives (spin-one), of the same form, on
                   (D_xz, D_yz) and (D_x2y2, D_xy), completing su(3)
    t_start, t_end, dt, dt_out   seconds
    psi0           complex initial state, basis m = +j ... -j

The paper's benchmark field (Eq. neural_pulse: 700 kHz bias, a 2 x 1 kHz
linearly polarised drive, a ms-scale signal pulse, 100 ms) is reached through
the ``neural-sense`` package, which is not available here; these generators
stand in for it with the same scales (MHz-scale bias, kHz drive, ms pulses).
"""
from __future__ import annotations

import math

import numpy as np

SEED = 20220411

UP_HALF = np.array([1.0, 0.0], dtype=np.complex128)
UP_ONE = np.array([1.0, 0.0, 0.0], dtype=np.complex128)


def field(bias_hz=0.0, drive_x_hz=0.0, drive_y_hz=0.0, drive_hz=0.0, drive_phase=0.0, quad_hz=0.0,
          pulses=(), tones=(), qdrives=()):
    def pulse(p):
        kind = p[3] if len(p) > 3 else "gauss"
        if kind not in ("gauss", "sine"):
            raise ValueError(f"unknown pulse kind {kind!r}")
        return (float(p[0]), float(p[1]), float(p[2]), kind)
    return dict(bias_hz=float(bias_hz), drive_x_hz=float(drive_x_hz), drive_y_hz=float(drive_y_hz),
                drive_hz=float(drive_hz), drive_phase=float(drive_phase), quad_hz=float(quad_hz),
                pulses=[pulse(p) for p in pulses], tones=[tuple(map(float, t)) for t in tones],
                qdrives=[tuple(map(float, q)) for q in qdrives])


def request(spin_x2, fld, t_start, t_end, dt, dt_out, psi0=None):
    if psi0 is None:
        psi0 = UP_HALF if spin_x2 == 1 else UP_ONE
    return dict(spin_x2=int(spin_x2), field=fld, t_start=float(t_start), t_end=float(t_end), dt=float(dt),
                dt_out=float(dt_out), psi0=np.asarray(psi0, dtype=np.complex128).copy())


def spin_half_rabi(t_end=5e-3, dt=1e-7, dt_out=1e-5):
    """Spin-half, B_z = 20 kHz, B_x = 2 x 1 kHz cos(2 pi 20 kHz t), [0, 5 ms], |up>."""
    return request(1, field(bias_hz=20e3, drive_x_hz=2e3, drive_hz=20e3), 0.0, t_end, dt, dt_out)


def spin_one_sensing(t_end=0.1, dt=1e-8, dt_out=1e-6):
    """Spin-one, B_z = 700 kHz, B_x = 2 x 1 kHz cos(2 pi 700 kHz t), q = 400 Hz,
    Gaussian z pulse 50 Hz x exp(-(t - 50 ms)^2 / (2 (1 ms)^2)), [0, 100 ms], |m=+1>."""
    return request(2, field(bias_hz=700e3, drive_x_hz=2e3, drive_hz=700e3, quad_hz=400.0,
                            pulses=[(50.0, 50e-3, 1e-3)]), 0.0, t_end, dt, dt_out)


MULTITONE = [(1e3, 1e3, 700.5e3, 0.4), (0.5e3, 0.0, 698e3, 1.1), (0.0, 0.8e3, 705e3, -0.6)]


def multitone_sensing(t_end=0.1, dt=1e-8, dt_out=1e-6):
    """The spin-one sensing field with three further drive tones (Sec. 3.1:
    drives of several tones and polarisations): a circularly polarised tone
    500 Hz above resonance, a linearly polarised one 2 kHz below, and a
    y-polarised one 5 kHz above (amplitudes 1, 0.5, 0.8 kHz)."""
    r = spin_one_sensing(t_end, dt, dt_out)
    r["field"]["tones"] = list(MULTITONE)
    return r


QDRIVES = [(1e3, 1e3, 700.3e3, 0.4), (0.5e3, 0.5e3, 1400.2e3, -0.8)]


def su3_sensing(t_end=0.1, dt=1e-8, dt_out=1e-6):
    """The spin-one sensing field with both quadrupole drives (Sec. 1.2.1: an
    arbitrary point in su(3)): a circular 1 kHz drive on (D_xz, D_yz) 300 Hz
    above the one-quantum resonance and a circular 0.5 kHz drive on
    (D_x2y2, D_xy) 200 Hz above the two-quantum resonance.  FP64 only."""
    r = spin_one_sensing(t_end, dt, dt_out)
    r["field"]["qdrives"] = list(QDRIVES)
    return r


def neural_pulse(t_end=0.1, t_p=0.05, dt=1e-7, dt_out=1e-6, spin_x2=2):
    """The paper's benchmark field, Eq. neural_pulse:
    H = w J_z + 2 W cos(w t) J_x + W_p sinp(W (t - t_p)) J_z with w = 2 pi 700 kHz,
    W = 2 pi 1 kHz, W_p = 2 pi 70 Hz and sinp one cycle of a sine wave (1 ms), over
    100 ms at the 100 ns integration step of the paper's speed benchmark, from
    |m = +1> (|up> for spin-half).  The printed t_p = 233 ms lies outside the 100 ms
    run; the pulse is placed at t_p = 50 ms so that the run contains it."""
    return request(spin_x2, field(bias_hz=700e3, drive_x_hz=2e3, drive_hz=700e3,
                                  pulses=[(70.0, t_p, 1e-3, "sine")]), 0.0, t_end, dt, dt_out)


def sweep(n=4096, seed=SEED, t_min=1e-3, t_max=0.1, dt=1e-8, dt_out=1e-6, spin_x2=2):
    """Batched spin-one sweep over an array of atom clouds.

    Per simulation (numpy PCG64, fixed draw order): bias ~ U(600, 800) kHz,
    Rabi R ~ U(0.5, 2) kHz (drive amplitude 2R), detuning ~ U(-500, 500) Hz,
    q ~ U(0, 600) Hz, pulse amplitude ~ U(0, 100) Hz, pulse centre ~ U(0, T),
    duration T log-uniform on [t_min, t_max]; pulse width 1 ms.  T is rounded
    to a whole number of output steps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    bias = rng.uniform(600e3, 800e3, n)
    rabi = rng.uniform(0.5e3, 2e3, n)
    det = rng.uniform(-500.0, 500.0, n)
    q = rng.uniform(0.0, 600.0, n)
    amp = rng.uniform(0.0, 100.0, n)
    cfrac = rng.uniform(0.0, 1.0, n)
    T = np.exp(rng.uniform(math.log(t_min), math.log(t_max), n))
    reqs = []
    for i in range(n):
        K = max(1, int(round(T[i] / dt_out)))
        Ti = K * dt_out
        f = field(bias_hz=bias[i], drive_x_hz=2.0 * rabi[i], drive_hz=bias[i] + det[i], quad_hz=q[i],
                  pulses=[(amp[i], cfrac[i] * Ti, 1e-3)])
        reqs.append(request(spin_x2, f, 0.0, Ti, dt, dt_out))
    return reqs


def serving_stream(n=20000, rate_hz=2000.0, seed=SEED + 1, frac_spin_one=0.7, t_min=1e-4, t_max=0.1,
                   dt=1e-8, dt_out=1e-6):
    """Poisson arrivals of mixed spin-one / spin-half requests (fields as in
    :func:`sweep`, durations log-uniform on [t_min, t_max]).  Returns
    (arrival_times_s [n], requests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, n)
    arrivals = np.cumsum(gaps) - gaps[0]
    spins = np.where(rng.uniform(0.0, 1.0, n) < frac_spin_one, 2, 1)
    bias = rng.uniform(600e3, 800e3, n)
    rabi = rng.uniform(0.5e3, 2e3, n)
    det = rng.uniform(-500.0, 500.0, n)
    q = rng.uniform(0.0, 600.0, n)
    amp = rng.uniform(0.0, 100.0, n)
    cfrac = rng.uniform(0.0, 1.0, n)
    T = np.exp(rng.uniform(math.log(t_min), math.log(t_max), n))
    reqs = []
    for i in range(n):
        K = max(1, int(round(T[i] / dt_out)))
        Ti = K * dt_out
        f = field(bias_hz=bias[i], drive_x_hz=2.0 * rabi[i], drive_hz=bias[i] + det[i],
                  quad_hz=q[i] if spins[i] == 2 else 0.0, pulses=[(amp[i], cfrac[i] * Ti, 1e-3)])
        reqs.append(request(int(spins[i]), f, 0.0, Ti, dt, dt_out))
    return arrivals, reqs


def random_state(n, rng):
    v = rng.normal(size=n) + 1j * rng.normal(size=n)
    return v / np.linalg.norm(v)


def total_steps(reqs):
    """Number of CF4 integration steps in a list of requests."""
    tot = 0
    for r in reqs:
        K = int(round((r["t_end"] - r["t_start"]) / r["dt_out"]))
        L = int(round(r["dt_out"] / r["dt"]))
        tot += max(K - 1, 0) * L
    return tot
