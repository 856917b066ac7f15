"""Pins of the oracle's exponentials (Sec. 1.2.3) against things other than itself:
scipy's dense expm, products of library exponentials, high-precision mpmath
arithmetic, group invariants and the Majorana (symmetric) representation."""
import numpy as np
import pytest
import scipy.linalg as sl

R2 = 1 / np.sqrt(2)
JX1 = np.array([[0, R2, 0], [R2, 0, R2], [0, R2, 0]], dtype=complex)
JY1 = np.array([[0, -1j * R2, 0], [1j * R2, 0, -1j * R2], [0, 1j * R2, 0]])
JZ1 = np.diag([1.0, 0.0, -1.0]).astype(complex)
Q1 = np.diag([1.0, -2.0, 1.0]).astype(complex) / 3
SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]])
SZ = np.diag([1.0, -1.0]).astype(complex)


def h_one(wx, wy, wz, wq):
    return wx * JX1 + wy * JY1 + wz * JZ1 + wq * Q1


def h_half(wx, wy, wz):
    return (wx * SX + wy * SY + wz * SZ) / 2


def random_fields(rng, n, scale):
    return rng.normal(size=(n, 4)) * scale


def majorana(U):
    """Spin-one (symmetric) representation P^dagger (U x U) P of a 2x2 U, with
    |+1> = |uu>, |0> = (|ud> + |du>)/sqrt2, |-1> = |dd>."""
    P = np.zeros((4, 3))
    P[0, 0] = 1
    P[1, 1] = P[2, 1] = R2
    P[3, 2] = 1
    return P.T @ np.kron(U, U) @ P


def test_spin_half_matches_dense_expm(oracle_mod):
    rng = np.random.default_rng(1)
    for wx, wy, wz, _ in random_fields(rng, 50, 3.0):
        dt = rng.uniform(0.01, 1.5)
        ref = sl.expm(-1j * h_half(wx, wy, wz) * dt)
        assert np.abs(oracle_mod.expm_spin_half(wx, wy, wz, dt) - ref).max() < 1e-14


def test_spin_half_small_and_zero_angle(oracle_mod):
    assert np.abs(oracle_mod.expm_spin_half(0, 0, 0, 1.0) - np.eye(2)).max() == 0
    for theta in (1e-12, 1e-9, 3e-7, 1e-6, 2e-6):
        w = np.array([0.3, -0.4, 1.2])
        w = w / np.linalg.norm(w) * theta
        ref = sl.expm(-1j * h_half(*w) * 1.0)
        assert np.abs(oracle_mod.expm_spin_half(*w, 1.0) - ref).max() < 1e-17


def test_trotter_T_is_product_of_library_exponentials(oracle_mod):
    """Eq. lie_trotter_4 element by element vs exp(-iD/2) exp(-i Phi J_phi) exp(-iD/2).
    This catches the two misprinted entries (centre, and m=+1,m'=-1)."""
    rng = np.random.default_rng(2)
    for (wx, wy, wz, wq) in random_fields(rng, 40, 2.0):
        for tau in (0, 3, 7):
            dt = rng.uniform(0.1, 1.0)
            n = 2.0 ** tau
            z, q = wz * dt / n, wq * dt / n
            Phi = np.hypot(wx, wy) * dt / n
            phi = np.arctan2(wy, wx)
            D = z * JZ1 + q * Q1
            Jphi = np.cos(phi) * JX1 + np.sin(phi) * JY1
            ref = sl.expm(-0.5j * D) @ sl.expm(-1j * Phi * Jphi) @ sl.expm(-0.5j * D)
            assert np.abs(oracle_mod.trotter_T(wx, wy, wz, wq, dt, tau) - ref).max() < 1e-14


def test_trotter_T_zero_transverse_field(oracle_mod):
    T = oracle_mod.trotter_T(0.0, 0.0, 0.7, -1.3, 1.0, 0)
    ref = sl.expm(-1j * (0.7 * JZ1 - 1.3 * Q1))
    assert np.abs(T - ref).max() < 1e-15


@pytest.mark.parametrize("scale", [0.05, 0.5, 1.0])
def test_spin_one_matches_dense_expm_at_default_tau(oracle_mod, scale):
    rng = np.random.default_rng(3)
    for wx, wy, wz, wq in random_fields(rng, 40, scale):
        ref = sl.expm(-1j * h_one(wx, wy, wz, wq))
        E = oracle_mod.expm_spin_one(wx, wy, wz, wq, 1.0, 24)
        assert np.abs(E - ref).max() < 5e-14


def test_lie_trotter_error_falls_as_n_squared(oracle_mod):
    """Symmetric splitting: error of T^n is O(theta^3 / n^2), so each extra
    squaring divides it by ~4 until rounding takes over (E5 of the paper)."""
    wx, wy, wz, wq, dt = 0.3, -0.7, 0.5, 0.9, 0.8
    ref = sl.expm(-1j * h_one(wx, wy, wz, wq) * dt)
    errs = [np.abs(oracle_mod.expm_spin_one(wx, wy, wz, wq, dt, t) - ref).max() for t in range(0, 12)]
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios[2:] > 3.8) & (ratios[2:] < 4.2)), ratios
    assert errs[0] > 1e-2  # a single leapfrog factor is visibly inexact


def test_residual_squaring_avoids_cancellation(oracle_mod):
    """For tiny angles the residual a = T^n - I must carry full relative
    precision (Sec. 1.2.3); checked against 50-digit mpmath."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    wx, wy, wz, wq = 1.3e-9, -0.6e-9, 2.1e-9, 0.8e-9
    a = oracle_mod.expm_spin_one_residual(wx, wy, wz, wq, 1.0, 24)
    H = mp.matrix(h_one(mp.mpf(wx), mp.mpf(wy), mp.mpf(wz), mp.mpf(wq)).tolist())
    ref = mp.expm(-1j * H) - mp.eye(3)
    ref = np.array([[complex(ref[i, j]) for j in range(3)] for i in range(3)])
    rel = np.abs(a - ref).max() / np.abs(ref).max()
    assert rel < 1e-12
    # Without the residual form the diagonal would be lost to rounding:
    naive = oracle_mod.expm_spin_one(wx, wy, wz, wq, 1.0, 24) - np.eye(3)
    assert np.abs(naive - ref).max() / np.abs(ref).max() > 1e-9


def test_unitarity_and_unit_determinant(oracle_mod):
    rng = np.random.default_rng(4)
    for wx, wy, wz, wq in random_fields(rng, 30, 1.0):
        E = oracle_mod.expm_spin_one(wx, wy, wz, wq, 0.9, 24)
        assert np.abs(E.conj().T @ E - np.eye(3)).max() < 1e-13
        assert abs(np.linalg.det(E) - 1) < 1e-13   # traceless H (Sec. 1.2.1)
        U = oracle_mod.expm_spin_half(wx, wy, wz, 0.9)
        assert np.abs(U.conj().T @ U - np.eye(2)).max() < 1e-15
        assert abs(np.linalg.det(U) - 1) < 1e-15


def test_majorana_representation(oracle_mod):
    """With w_q = 0 the spin-one exponential is the symmetric representation
    of the spin-half one (independent of the Lie-Trotter machinery)."""
    rng = np.random.default_rng(5)
    for wx, wy, wz, _ in random_fields(rng, 30, 1.0):
        U = oracle_mod.expm_spin_half(wx, wy, wz, 0.7)
        E = oracle_mod.expm_spin_one(wx, wy, wz, 0.0, 0.7, 24)
        assert np.abs(E - majorana(U)).max() < 1e-13
