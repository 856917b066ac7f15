"""Pins of the oracle's full su(3) spin-one Hamiltonians (Sec. 1.2.1: an
arbitrary point in su(3)): the basis, the general exponential against scipy,
the quadrupole-drive field formula, exact solutions of a quadrupole drive of
either pair, and an independent adaptive ODE solver in both frames.  The four
operators that complete su(3) are built here from the spin matrices, not taken
from the oracle."""
import numpy as np
import pytest
import scipy.linalg as sl
from scipy.integrate import solve_ivp

from paper_2204_05586_gb300 import workloads as W
from test_oracle_expm import JX1, JY1, JZ1, Q1

TWO_PI = 2 * np.pi
G = [JX1, JY1, JZ1, Q1, JX1 @ JZ1 + JZ1 @ JX1, JY1 @ JZ1 + JZ1 @ JY1, JX1 @ JX1 - JY1 @ JY1,
     JX1 @ JY1 + JY1 @ JX1]


def hamiltonian8(w):
    return sum(a * g for a, g in zip(w, G))


def test_basis_spans_su3():
    """Eight traceless Hermitian operators, linearly independent over the reals."""
    for g in G:
        assert abs(np.trace(g)) < 1e-15
        assert np.abs(g - g.conj().T).max() < 1e-15
    M = np.array([np.concatenate([g.real.ravel(), g.imag.ravel()]) for g in G])
    assert np.linalg.matrix_rank(M, tol=1e-12) == 8


@pytest.mark.parametrize("scale", [1e-5, 1e-2, 0.4, 6.0])
def test_general_exponential_matches_scipy(oracle_mod, scale):
    rng = np.random.default_rng(int(scale * 1e5) + 3)
    for _ in range(20):
        w = rng.normal(size=8) * scale
        dt = rng.uniform(0.5, 2.0)
        E = oracle_mod.expm_general(w, dt)
        ref = sl.expm(-1j * dt * hamiltonian8(w))
        assert np.abs(E - ref).max() < 2e-15 * max(1.0, scale * 8)
        assert np.abs(E.conj().T @ E - np.eye(3)).max() < 1e-13


def test_general_exponential_without_quadrupole_terms_equals_lie_trotter(oracle_mod):
    rng = np.random.default_rng(8)
    for _ in range(10):
        w = np.concatenate([rng.normal(size=4) * 0.2, np.zeros(4)])
        assert np.abs(oracle_mod.expm_general(w, 1.0) - oracle_mod.expm_spin_one(*w[:4], 1.0, tau=24)).max() < 1e-13


def test_quadrupole_drive_formula(oracle_mod):
    qd = [(1.5e3, -0.7e3, 30.1e3, 0.4), (0.6e3, 2.2e3, 61e3, -1.9)]
    f = W.field(bias_hz=30e3, qdrives=qd)
    for t in (0.0, 1.3e-4, 7.77e-3):
        u = oracle_mod.field_sample_quad(f, t)
        exp = []
        for x, y, hz, ph in qd:
            a = TWO_PI * hz * t + ph
            exp += [TWO_PI * x * np.cos(a), TWO_PI * y * np.sin(a)]
        assert np.allclose(u, exp, rtol=1e-13, atol=1e-9)
    assert np.all(oracle_mod.field_sample_quad(W.field(bias_hz=1.0), 0.3) == 0.0)


@pytest.mark.parametrize("pair", [0, 1])
def test_quadrupole_drive_exact_solution(oracle_mod, pair):
    """A circularly polarised quadrupole drive at w on the pair (D_xz, D_yz)
    (k = 1) or (D_x2y2, D_xy) (k = 2) with a bias w0: in the frame turning at
    w / k about z the Hamiltonian is constant, so
    psi(t) = exp(-i (w/k) t J_z) exp(-i t ((w0 - w/k) J_z + u D)) psi0."""
    w0, w, u = TWO_PI * 50e3, TWO_PI * 49.2e3, TWO_PI * 3e3
    qd = [(0.0, 0.0, 0.0, 0.0), (0.0, 0.0, 0.0, 0.0)]
    qd[pair] = (3e3, 3e3, 49.2e3, 0.0)
    f = W.field(bias_hz=50e3, quad_hz=0.0, qdrives=qd)
    psi0 = W.random_state(3, np.random.default_rng(12 + pair))
    k = 1 + pair
    D = G[4] if pair == 0 else G[6]
    ts = np.arange(10) * 1e-4
    ref = np.stack([sl.expm(-1j * (w / k) * t * JZ1) @ sl.expm(-1j * t * ((w0 - w / k) * JZ1 + u * D)) @ psi0
                    for t in ts])
    for frame in (True, False):
        out = oracle_mod.simulate(2, f, 0.0, 1e-3, 2.5e-8, 1e-4, psi0, rotating_frame=frame)
        assert np.abs(out["states"] - ref).max() < 1e-10, (frame, np.abs(out["states"] - ref).max())


@pytest.mark.parametrize("frame", [True, False])
def test_full_su3_against_adaptive_ode_solver(oracle_mod, frame):
    """Drive, quadratic shift, a Gaussian pulse and both quadrupole drives
    (off resonance, elliptical) vs scipy DOP853 at tight tolerance."""
    f = W.field(bias_hz=20e3, drive_x_hz=2e3, drive_hz=20.3e3, quad_hz=300.0, pulses=[(400.0, 0.3e-3, 0.1e-3)],
                qdrives=[(1.1e3, 0.6e3, 19.7e3, 0.5), (0.8e3, 1.4e3, 40.9e3, -0.3)])
    psi0 = W.random_state(3, np.random.default_rng(31))
    out = oracle_mod.simulate(2, f, 0.0, 6e-4, 1e-7, 2e-5, psi0, rotating_frame=frame)
    ts = 2e-5 * np.arange(30)

    def rhs(t, y):
        w = np.concatenate([oracle_mod.field_sample(f, t), oracle_mod.field_sample_quad(f, t)])
        psi = y[:3] + 1j * y[3:]
        d = -1j * hamiltonian8(w) @ psi
        return np.concatenate([d.real, d.imag])

    sol = solve_ivp(rhs, (ts[0], ts[-1]), np.concatenate([psi0.real, psi0.imag]), method="DOP853", t_eval=ts,
                    rtol=1e-13, atol=1e-13)
    ref = (sol.y[:3] + 1j * sol.y[3:]).T
    assert np.abs(out["states"] - ref).max() < 1e-9


def test_quadrupole_drives_need_spin_one(oracle_mod):
    f = W.field(bias_hz=1e3, qdrives=[(1.0, 1.0, 1.0, 0.0)])
    with pytest.raises(ValueError):
        oracle_mod.simulate(1, f, 0.0, 1e-4, 1e-6, 1e-5, W.UP_HALF)
