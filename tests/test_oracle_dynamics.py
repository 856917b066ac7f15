"""Pins of the oracle's whole-run dynamics (Secs. 1.2.2, 1.2.4, 1.2.5) against
closed-form solutions, an independent adaptive ODE solver (the paper's own
check was a SciPy ivp baseline, Sec. 1.3.1), convergence orders and
invariants.  Sizes are small so the suite runs in seconds."""
import numpy as np
import pytest
import scipy.linalg as sl
from scipy.integrate import solve_ivp
from scipy.special import erf

from paper_2204_05586_gb300 import workloads as W
from test_oracle_expm import JX1, JY1, JZ1, Q1, SX, SY, SZ, majorana

TWO_PI = 2 * np.pi


def ops_of(spin_x2):
    if spin_x2 == 1:
        return SX / 2, SY / 2, SZ / 2, np.zeros((2, 2))
    return JX1, JY1, JZ1, Q1


def hamiltonian(spin_x2, w):
    jx, jy, jz, q = ops_of(spin_x2)
    return w[0] * jx + w[1] * jy + w[2] * jz + w[3] * q


def times(t_start, t_end, dt_out):
    K = int(round((t_end - t_start) / dt_out))
    return t_start + dt_out * np.arange(K)


# ---------------------------------------------------------------- field model
def test_field_sample_formula(oracle_mod):
    f = W.field(bias_hz=700e3, drive_x_hz=2e3, drive_y_hz=0.5e3, drive_hz=701e3, drive_phase=0.3,
                quad_hz=400, pulses=[(50, 0.05, 1e-3), (-20, 0.051, 2e-3)])
    for t in (0.0, 0.0493, 0.05, 0.0999):
        w = oracle_mod.field_sample(f, t)
        ph = TWO_PI * 701e3 * t + 0.3
        gz = 700e3 + 50 * np.exp(-((t - 0.05) / 1e-3) ** 2 / 2) - 20 * np.exp(-((t - 0.051) / 2e-3) ** 2 / 2)
        assert np.allclose(w, [TWO_PI * 2e3 * np.cos(ph), TWO_PI * 0.5e3 * np.sin(ph), TWO_PI * gz,
                               TWO_PI * 400], rtol=1e-13, atol=1e-9)


def test_field_sample_formula_extra_tones(oracle_mod):
    """Further drive tones add to w_x and w_y like the first (Sec. 3.1: drives of
    any number of tones and polarisations)."""
    tones = [(1.5e3, -0.4e3, 703e3, 1.1), (0.0, 0.8e3, 698.5e3, -0.7), (-0.3e3, 0.3e3, 1.2e3, 2.9)]
    f = W.field(bias_hz=700e3, drive_x_hz=2e3, drive_y_hz=0.5e3, drive_hz=701e3, drive_phase=0.3, tones=tones)
    for t in (0.0, 0.0493, 0.0999):
        w = oracle_mod.field_sample(f, t)
        ph = TWO_PI * 701e3 * t + 0.3
        wx = TWO_PI * 2e3 * np.cos(ph) + sum(TWO_PI * x * np.cos(TWO_PI * hz * t + p) for x, _, hz, p in tones)
        wy = TWO_PI * 0.5e3 * np.sin(ph) + sum(TWO_PI * y * np.sin(TWO_PI * hz * t + p) for _, y, hz, p in tones)
        assert np.allclose(w[:3], [wx, wy, TWO_PI * 700e3], rtol=1e-13, atol=1e-8)
    with pytest.raises(ValueError):
        oracle_mod.field_sample(W.field(tones=tones + [(1.0, 1.0, 1.0, 0.0)]), 0.0)


def test_counts(oracle_mod):
    assert oracle_mod.counts(0.0, 5e-3, 1e-7, 1e-5) == (500, 100)
    assert oracle_mod.counts(0.0, 0.1, 1e-8, 1e-6) == (100000, 100)
    assert oracle_mod.counts(0.0, 0.0, 1e-8, 1e-6) == (0, 100)
    with pytest.raises(ValueError):
        oracle_mod.counts(0.0, 5e-3, 3e-7, 1e-5)
    with pytest.raises(ValueError):
        oracle_mod.counts(0.0, 5.5e-6, 1e-7, 1e-5)


# ------------------------------------------------------ P1: constant field
@pytest.mark.parametrize("spin_x2", [1, 2])
def test_constant_field_is_exact(oracle_mod, spin_x2):
    """Constant H: the two CF4 exponentials commute and multiply to exp(-iH dt)."""
    f = W.field(bias_hz=3e3, drive_x_hz=1.1e3, drive_y_hz=0.7e3, drive_hz=0.0, drive_phase=0.4, quad_hz=900)
    rng = np.random.default_rng(7)
    psi0 = W.random_state(2 if spin_x2 == 1 else 3, rng)
    out = oracle_mod.simulate(spin_x2, f, 0.0, 2e-3, 1e-6, 1e-4, psi0, rotating_frame=False)
    H = hamiltonian(spin_x2, oracle_mod.field_sample(f, 0.0))
    ts = times(0.0, 2e-3, 1e-4)
    ref = np.stack([sl.expm(-1j * H * t) @ psi0 for t in ts])
    assert np.abs(out["states"] - ref).max() < 1e-12


# ------------------------------------------ P2: circular drive, exact solution
def circular_exact(spin_x2, w0, wd, Om, wq, psi0, ts):
    jx, jy, jz, q = ops_of(spin_x2)
    Hr = (w0 - wd) * jz + Om * jx + wq * q
    return np.stack([sl.expm(-1j * wd * t * jz) @ sl.expm(-1j * Hr * t) @ psi0 for t in ts])


def circular_case(spin_x2, frame, dt, t_end=1e-3, dt_out=1e-4):
    f0, fd, om, q = 50e3, 49.2e3, 4e3, (700.0 if spin_x2 == 2 else 0.0)
    f = W.field(bias_hz=f0, drive_x_hz=om, drive_y_hz=om, drive_hz=fd, quad_hz=q)
    rng = np.random.default_rng(11)
    psi0 = W.random_state(2 if spin_x2 == 1 else 3, rng)
    ts = times(0.0, t_end, dt_out)
    ref = circular_exact(spin_x2, TWO_PI * f0, TWO_PI * fd, TWO_PI * om, TWO_PI * q, psi0, ts)
    return f, psi0, ref


@pytest.mark.parametrize("spin_x2", [1, 2])
@pytest.mark.parametrize("frame", [False, True])
def test_circular_drive_exact_solution(oracle_mod, spin_x2, frame):
    f, psi0, ref = circular_case(spin_x2, frame, None)
    out = oracle_mod.simulate(spin_x2, f, 0.0, 1e-3, 2.5e-8, 1e-4, psi0, rotating_frame=frame)
    assert np.abs(out["states"] - ref).max() < 5e-11


@pytest.mark.parametrize("spin_x2", [1, 2])
def test_cf4_is_fourth_order(oracle_mod, spin_x2):
    """P3: global error against the exact circular-drive solution falls by ~16
    per halving of delta_t (Eq. cf4_implementation has an O(dt^5) local error)."""
    f, psi0, ref = circular_case(spin_x2, False, None)
    errs = []
    for dt in (2e-6, 1e-6, 5e-7):
        out = oracle_mod.simulate(spin_x2, f, 0.0, 1e-3, dt, 1e-4, psi0, rotating_frame=False)
        errs.append(np.abs(out["states"] - ref).max())
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((r > 14) & (r < 18)), (errs, r)


@pytest.mark.parametrize("method", [1, 2])
def test_euler_sampling_methods_are_second_order(oracle_mod, method):
    """Midpoint and Heun sampling (Sec. 1.3.1) are second-order methods."""
    f, psi0, ref = circular_case(2, False, None)
    errs = []
    for dt in (1e-6, 5e-7, 2.5e-7):
        out = oracle_mod.simulate(2, f, 0.0, 1e-3, dt, 1e-4, psi0, rotating_frame=False, method=method)
        errs.append(np.abs(out["states"] - ref).max())
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((r > 3.5) & (r < 4.5)), (errs, r)


# ------------------------------------- P4: diagonal H with a Gaussian pulse
@pytest.mark.parametrize("frame", [False, True])
def test_gaussian_pulse_phase_closed_form(oracle_mod, frame):
    """With no transverse field psi_m(t) = psi_m(0) exp(-i int (m w_z + Q_mm w_q)),
    and the Gaussian integrates to erf (Sec. 1.2.1 field functions)."""
    B, A, c, w, q = 2e3, 300.0, 1.2e-3, 0.4e-3, 250.0
    f = W.field(bias_hz=B, quad_hz=q, pulses=[(A, c, w)])
    rng = np.random.default_rng(13)
    psi0 = W.random_state(3, rng)
    out = oracle_mod.simulate(2, f, 0.0, 3e-3, 1e-6, 5e-5, psi0, rotating_frame=frame)
    ts = times(0.0, 3e-3, 5e-5)
    iz = TWO_PI * (B * ts + A * w * np.sqrt(np.pi / 2) * (erf((ts - c) / (np.sqrt(2) * w))
                                                          - erf((0 - c) / (np.sqrt(2) * w))))
    iq = TWO_PI * q * ts
    m = np.array([1.0, 0.0, -1.0])
    qd = np.array([1.0, -2.0, 1.0]) / 3
    ref = psi0[None, :] * np.exp(-1j * (m[None, :] * iz[:, None] + qd[None, :] * iq[:, None]))
    assert np.abs(out["states"] - ref).max() < 1e-11


# ------------------------------- P4': diagonal H with a single-cycle sine pulse
def sine_cycle_integral(ts, A, tp, T):
    """int_0^t 2 pi A sinp(2 pi (t' - tp) / T) dt' with sinp one cycle of a sine:
    A T (1 - cos(2 pi (t - tp) / T)) inside the cycle, 0 before it and after it."""
    x = np.clip((ts - tp) / T, 0.0, 1.0)
    return A * T * (1.0 - np.cos(TWO_PI * x))


@pytest.mark.parametrize("frame", [False, True])
def test_sine_cycle_pulse_phase_closed_form(oracle_mod, frame):
    """The paper's signal pulse (Eq. neural_pulse: Omega_p sinp(Omega (t - t_p)) J_z,
    sinp a single cycle of a sine wave).  With no transverse field
    psi_m(t) = psi_m(0) exp(-i int (m w_z + Q_mm w_q)) and the cycle integrates in
    closed form; the pulse starts and ends on step boundaries, where CF4's
    two-node quadrature of the phase is fourth order."""
    B, A, tp, T, q = 2e3, 700.0, 0.8e-3, 1.0e-3, 250.0
    f = W.field(bias_hz=B, quad_hz=q, pulses=[(A, tp, T, "sine")])
    rng = np.random.default_rng(29)
    psi0 = W.random_state(3, rng)
    out = oracle_mod.simulate(2, f, 0.0, 3e-3, 1e-6, 5e-5, psi0, rotating_frame=frame)
    ts = times(0.0, 3e-3, 5e-5)
    iz = TWO_PI * B * ts + sine_cycle_integral(ts, A, tp, T)
    iq = TWO_PI * q * ts
    m = np.array([1.0, 0.0, -1.0])
    qd = np.array([1.0, -2.0, 1.0]) / 3
    ref = psi0[None, :] * np.exp(-1j * (m[None, :] * iz[:, None] + qd[None, :] * iq[:, None]))
    assert np.abs(out["states"] - ref).max() < 1e-11
    # the pulse is really there: without it the phase differs by A T (1 - cos) ~ 1.4 rad at mid-cycle
    assert np.abs(sine_cycle_integral(ts, A, tp, T)).max() > 1.0


def test_sine_cycle_pulse_spin_half_before_during_after(oracle_mod):
    """Spin-half relative phase through the cycle: zero pulse contribution
    before t_p, A T (1 - cos) during, and none after the full cycle."""
    B, A, tp, T = 5e3, -300.0, 1.0e-3, 0.5e-3
    f = W.field(bias_hz=B, pulses=[(A, tp, T, "sine")])
    psi0 = np.array([1.0, 1.0], dtype=np.complex128) / np.sqrt(2)
    out = oracle_mod.simulate(1, f, 0.0, 2.5e-3, 1e-7, 1e-5, psi0)
    ts = times(0.0, 2.5e-3, 1e-5)
    rel = np.angle(out["states"][:, 1] / out["states"][:, 0])     # = int w_z (spin-half: m = -+1/2)
    ref = np.angle(np.exp(1j * (TWO_PI * B * ts + sine_cycle_integral(ts, A, tp, T))))
    assert np.abs(np.angle(np.exp(1j * (rel - ref)))).max() < 1e-10


# ------------------------------------ brute force: independent ODE solver
def ivp_reference(spin_x2, f, psi0, ts, oracle_mod):
    n = len(psi0)

    def rhs(t, y):
        psi = y[:n] + 1j * y[n:]
        d = -1j * hamiltonian(spin_x2, oracle_mod.field_sample(f, t)) @ psi
        return np.concatenate([d.real, d.imag])

    sol = solve_ivp(rhs, (ts[0], ts[-1]), np.concatenate([psi0.real, psi0.imag]), method="DOP853",
                    t_eval=ts, rtol=1e-13, atol=1e-13)
    return (sol.y[:n] + 1j * sol.y[n:]).T


@pytest.mark.parametrize("spin_x2", [1, 2])
@pytest.mark.parametrize("frame", [False, True])
def test_against_adaptive_ode_solver(oracle_mod, spin_x2, frame):
    """Sensing-like field (bias, linear drive, quadratic shift, a Gaussian pulse
    and a single-cycle sine pulse) vs scipy DOP853 at tight tolerance: the
    paper's own validation route."""
    f = W.field(bias_hz=20e3, drive_x_hz=2e3, drive_hz=20.3e3, quad_hz=300.0 if spin_x2 == 2 else 0.0,
                pulses=[(400.0, 0.3e-3, 0.1e-3), (250.0, 0.1e-3, 0.2e-3, "sine")])
    rng = np.random.default_rng(17)
    psi0 = W.random_state(2 if spin_x2 == 1 else 3, rng)
    out = oracle_mod.simulate(spin_x2, f, 0.0, 6e-4, 2e-7, 2e-5, psi0, rotating_frame=frame)
    ts = times(0.0, 6e-4, 2e-5)
    ref = ivp_reference(spin_x2, f, psi0, ts, oracle_mod)
    assert np.abs(out["states"] - ref).max() < 1e-9


@pytest.mark.parametrize("spin_x2", [1, 2])
def test_circular_drive_split_over_tones(oracle_mod, spin_x2):
    """The circular drive of the exact-solution case carried by the first tone
    and two further tones at the same frequency and phase (amplitudes summing
    to the drive's), plus a zero-amplitude tone elsewhere: the exact solution."""
    f0, fd, om, q = 50e3, 49.2e3, 4e3, (700.0 if spin_x2 == 2 else 0.0)
    f = W.field(bias_hz=f0, drive_x_hz=0.5 * om, drive_y_hz=0.25 * om, drive_hz=fd, quad_hz=q,
                tones=[(0.25 * om, 0.5 * om, fd, 0.0), (0.25 * om, 0.25 * om, fd, 0.0), (0.0, 0.0, 3e3, 1.0)])
    rng = np.random.default_rng(11)
    psi0 = W.random_state(2 if spin_x2 == 1 else 3, rng)
    out = oracle_mod.simulate(spin_x2, f, 0.0, 1e-3, 5e-8, 1e-4, psi0, rotating_frame=True)
    ts = times(0.0, 1e-3, 1e-4)
    ref = circular_exact(spin_x2, TWO_PI * f0, TWO_PI * fd, TWO_PI * om, TWO_PI * q, psi0, ts)
    assert np.abs(out["states"] - ref).max() < 1e-10


@pytest.mark.parametrize("spin_x2", [1, 2])
def test_extra_tones_against_adaptive_ode_solver(oracle_mod, spin_x2):
    """Four tones of different frequencies, phases and polarisations (two near
    resonance, one detuned by 40 kHz, one at 7 kHz) with a Gaussian pulse vs
    scipy DOP853."""
    f = W.field(bias_hz=20e3, drive_x_hz=2e3, drive_hz=20.3e3, quad_hz=300.0 if spin_x2 == 2 else 0.0,
                pulses=[(400.0, 0.3e-3, 0.1e-3)],
                tones=[(1.2e3, 0.9e3, 19.6e3, 0.8), (0.0, 1.5e3, 60e3, -1.3), (0.7e3, 0.0, 7e3, 2.2)])
    rng = np.random.default_rng(23)
    psi0 = W.random_state(2 if spin_x2 == 1 else 3, rng)
    out = oracle_mod.simulate(spin_x2, f, 0.0, 6e-4, 1e-7, 2e-5, psi0, rotating_frame=True)
    ts = times(0.0, 6e-4, 2e-5)
    ref = ivp_reference(spin_x2, f, psi0, ts, oracle_mod)
    assert np.abs(out["states"] - ref).max() < 1e-9


# ------------------------------------------------- P5, P6, P9, P10 and <J>
def test_majorana_whole_run(oracle_mod):
    """q = 0: spin-one U_k equal the symmetric representation of spin-half U_k."""
    f = W.field(bias_hz=30e3, drive_x_hz=3e3, drive_hz=30.5e3, pulses=[(200.0, 2e-4, 1e-4)])
    o1 = oracle_mod.simulate(2, f, 0.0, 4e-4, 1e-7, 2e-5, W.UP_ONE, want_ops=True)
    oh = oracle_mod.simulate(1, f, 0.0, 4e-4, 1e-7, 2e-5, W.UP_HALF, want_ops=True)
    for k in range(o1["ops"].shape[0]):
        assert np.abs(o1["ops"][k] - majorana(oh["ops"][k])).max() < 1e-12
    # spin-one |+1> is the product |uu>, so <J> doubles (Sec. 1.2.1 spin projection)
    assert np.abs(o1["spin"] - 2 * oh["spin"]).max() < 1e-12


@pytest.mark.parametrize("spin_x2", [1, 2])
def test_unitarity_and_norm(oracle_mod, spin_x2):
    req = W.spin_half_rabi(t_end=1e-3) if spin_x2 == 1 else W.spin_one_sensing(t_end=2e-5)
    out = oracle_mod.simulate(spin_x2, req["field"], req["t_start"], req["t_end"], req["dt"], req["dt_out"],
                              req["psi0"], want_ops=True)
    U = out["ops"]
    n = U.shape[1]
    gram = np.einsum("kji,kjl->kil", U.conj(), U)
    assert np.abs(gram - np.eye(n)).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13
    assert np.abs(np.linalg.norm(out["states"], axis=1) - 1).max() < 1e-12


@pytest.mark.parametrize("spin_x2", [1, 2])
def test_frame_is_exact_change_of_variables(oracle_mod, spin_x2):
    """P9: with the frame on and off the results converge to the same solution."""
    f = W.field(bias_hz=200e3, drive_x_hz=2e3, drive_hz=200e3, quad_hz=500 if spin_x2 == 2 else 0,
                pulses=[(80.0, 1e-4, 5e-5)])
    psi0 = W.UP_HALF if spin_x2 == 1 else W.UP_ONE
    on = oracle_mod.simulate(spin_x2, f, 0.0, 2e-4, 1e-8, 1e-5, psi0, rotating_frame=True)
    off = oracle_mod.simulate(spin_x2, f, 0.0, 2e-4, 1e-8, 1e-5, psi0, rotating_frame=False)
    assert np.abs(on["states"] - off["states"]).max() < 1e-10


def test_frame_rate_is_interval_midpoint_z_field(oracle_mod):
    """Sec. 1.2.5: w_r = w_z(t_{k-1} + Delta_t / 2) for interval [t_{k-1}, t_k];
    any constant w_r is an exact change of variables, so only this check (not
    the dynamics) pins the choice."""
    req = W.spin_one_sensing()
    f = req["field"]
    for k in (1, 2, 50000, 99999):
        t_mid = (k - 1) * 1e-6 + 0.5e-6
        wz = 2 * np.pi * (700e3 + 50 * np.exp(-((t_mid - 0.05) / 1e-3) ** 2 / 2))
        got = oracle_mod.frame_rate(2, f, 0.0, 0.1, 1e-8, 1e-6, k)
        assert abs(got - wz) <= 1e-12 * wz
    assert oracle_mod.frame_rate(2, f, 0.0, 0.1, 1e-8, 1e-6, 5, rotating_frame=False) == 0.0


def test_composition_checkpoint(oracle_mod):
    """P10: [t0, T] equals [t0, T/2] followed by [T/2, T] seeded with psi(T/2)."""
    req = W.spin_one_sensing(t_end=4e-5)
    f = req["field"]
    full = oracle_mod.simulate(2, f, 0.0, 4e-5, 1e-8, 1e-6, req["psi0"])
    a = oracle_mod.simulate(2, f, 0.0, 2e-5, 1e-8, 1e-6, req["psi0"])
    # psi at t = 2e-5 is sample 20 of the full run
    b = oracle_mod.simulate(2, f, 2e-5, 4e-5, 1e-8, 1e-6, full["states"][20])
    assert np.abs(a["states"] - full["states"][:20]).max() == 0
    assert np.abs(b["states"] - full["states"][20:]).max() < 1e-14


def test_chain_matches_simulate(oracle_mod):
    req = W.spin_half_rabi(t_end=2e-4)
    f = req["field"]
    out = oracle_mod.simulate(1, f, 0.0, 2e-4, 1e-7, 1e-5, req["psi0"], want_ops=True)
    ops = oracle_mod.sample_operators(1, f, 0.0, 2e-4, 1e-7, 1e-5, threads=3)
    assert np.array_equal(ops, out["ops"])
    st, sp = oracle_mod.chain(ops, req["psi0"])
    assert np.array_equal(st, out["states"]) and np.array_equal(sp, out["spin"])


def test_spin_projection_known_states(oracle_mod):
    """<J> of basis states and of the |+x> eigenstates."""
    eye3 = np.eye(3, dtype=complex)[None]
    _, sp = oracle_mod.chain(eye3, np.array([0, 0, 1], dtype=complex))
    assert np.allclose(sp[0], [0, 0, -1])
    px = np.array([0.5, R2 := 1 / np.sqrt(2), 0.5], dtype=complex)   # J_x eigenvalue +1
    _, sp = oracle_mod.chain(eye3, px)
    assert np.allclose(sp[0], [1, 0, 0], atol=1e-15)
    py = np.array([0.5, 1j * R2, -0.5])   # J_y eigenvalue +1
    _, sp = oracle_mod.chain(eye3, py)
    assert np.allclose(sp[0], [0, 1, 0], atol=1e-15)
    _, sp = oracle_mod.chain(np.eye(2, dtype=complex)[None], np.array([1, 1j]) / np.sqrt(2))
    assert np.allclose(sp[0], [0, 0.5, 0], atol=1e-15)


def test_error_metric_definition(oracle_mod):
    """Eq. error with the 1/K outside the square root, as printed."""
    a = np.zeros((4, 3), dtype=complex)
    b = a.copy()
    b[1, 2] = 3.0
    b[3, 0] = 4j
    assert abs(oracle_mod.error_metric(a, b) - 5.0 / 4) < 1e-15
