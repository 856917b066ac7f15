"""The kernels' per-thread arithmetic (csrc/device_math.cuh), compiled for the
host by nvcc, against the oracle and scipy on the CPU: the split-residual
Lie-Trotter exponential, the SU(2) closed form, residual products and the
closed-form node-phasor sums used for the exact first-order part."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg as sl

from test_oracle_expm import JX1, JY1, JZ1, Q1, SX, SY, SZ

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
DP = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def hh(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("hh") / "libhh.so")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "host_harness.cu"),
                           os.path.join(ROOT, "paper_2204_05586_gb300", "csrc", "params.cu"), "-o", out])
    L = ctypes.CDLL(out)
    L.hh_expm_one.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int, ctypes.c_int, DP]
    L.hh_expm_one_rest.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int, DP]
    L.hh_expm_half.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int, DP]
    L.hh_product_one.argtypes = [DP, DP, ctypes.c_int, DP]
    L.hh_product_half.argtypes = [DP, DP, DP]
    L.hh_node_phasor_sum.argtypes = [ctypes.c_double, ctypes.c_int64] + [ctypes.c_double] * 4 + [DP]
    L.hh_small_sincos_m.argtypes = [ctypes.c_double, ctypes.c_int, DP]
    L.hh_choose_tau.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] * 8
    L.hh_choose_tau.restype = ctypes.c_int
    L.hh_expm_one_small.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int, DP]
    L.hh_expm_one_general32.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int, DP]
    L.hh_expm_one_tau0.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int, DP, DP]
    L.hh_tiny_sincos.argtypes = [ctypes.c_double, DP]
    L.hh_small_angle_request.restype = ctypes.c_int
    L.hh_small_angle_request.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
    L.hh_tiny_angle_bound.restype = ctypes.c_double
    L.hh_request_variant.restype = ctypes.c_int
    L.hh_request_variant.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.POINTER(ctypes.c_int)]
    L.hh_first_order.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, DP]
    L.hh_widen_bits.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
    L.hh_chain_geom.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.hh_drive_cycles_frac.restype = ctypes.c_double
    L.hh_drive_cycles_frac.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int64]
    L.hh_phasor.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                            ctypes.c_int, ctypes.c_int, DP]
    L.hh_series_match.argtypes = [ctypes.c_double, ctypes.c_int]
    L.hh_expm_general.argtypes = [DP, DP]
    L.hh_expm_general_rest.argtypes = [DP, DP]
    L.hh_series_match.restype = ctypes.c_int
    return L


def P(a):
    return a.ctypes.data_as(DP)


def H1(v):
    return v[0] * JX1 + v[1] * JY1 + v[2] * JZ1 + v[3] * Q1


@pytest.mark.parametrize("scale", [1e-4, 1e-2, 0.3, 1.0])
def test_expm_one_matches_oracle_and_scipy(hh, oracle_mod, scale):
    rng = np.random.default_rng(1)
    for _ in range(20):
        v = rng.normal(size=4) * scale
        for tau in (0, 3, 8, 24):
            out = np.zeros(18)
            hh.hh_expm_one(*v, tau, 0, P(out))
            E = out.view(np.complex128).reshape(3, 3)
            ref = oracle_mod.expm_spin_one(*v, 1.0, tau)   # same tau: same Lie-Trotter approximant
            assert np.abs(E - ref).max() < 1e-14 * max(1.0, scale * 10), (scale, tau)
        assert np.abs(E - sl.expm(-1j * H1(v))).max() < 3e-15


def test_expm_one_rest_is_higher_order(hh):
    """The rest of exp(-i v.A) - I after removing -i v.A is O(|v|^2) and is
    carried with full relative precision (50-digit mpmath reference)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    v = np.array([0.3, -0.2, 0.5, 0.4])
    for s in (1e-2, 1e-3, 1e-4):
        out = np.zeros(18)
        hh.hh_expm_one_rest(*(v * s), 24, P(out))
        rest = out.view(np.complex128).reshape(3, 3)
        Hm = mp.matrix(H1(v * s).tolist())
        refm = mp.expm(-1j * Hm) - mp.eye(3) + 1j * Hm
        ref = np.array([[complex(refm[i, j]) for j in range(3)] for i in range(3)])
        assert np.abs(rest - ref).max() < 1e-13 * s * s
        assert np.abs(rest).max() < s * s


def test_expm_one_fp32(hh):
    rng = np.random.default_rng(2)
    for _ in range(20):
        v = rng.normal(size=4) * 1e-3
        out = np.zeros(18)
        hh.hh_expm_one(*v, 4, 1, P(out))
        E = out.view(np.complex128).reshape(3, 3)
        ref = sl.expm(-1j * H1(v))
        assert np.abs(E - ref).max() < 1e-9


@pytest.mark.parametrize("scale", [1e-5, 1e-2, 0.5, 2.0])
def test_expm_half(hh, scale):
    rng = np.random.default_rng(3)
    for _ in range(20):
        v = rng.normal(size=3) * scale
        ref = sl.expm(-1j * (v[0] * SX + v[1] * SY + v[2] * SZ) / 2)
        for fp32, tol in ((0, 1e-15), (1, 3e-7)):
            out = np.zeros(8)
            hh.hh_expm_half(*v, fp32, P(out))
            assert np.abs(out.view(np.complex128).reshape(2, 2) - ref).max() < tol * max(1.0, scale * scale)


def test_residual_products(hh):
    rng = np.random.default_rng(4)
    for _ in range(10):
        vA = rng.normal(size=4) * 0.1
        vB = rng.normal(size=4) * 0.1
        out = np.zeros(18)
        hh.hh_product_one(P(vA), P(vB), 24, P(out))
        ref = sl.expm(-1j * H1(vB)) @ sl.expm(-1j * H1(vA))   # later operator on the left
        assert np.abs(out.view(np.complex128).reshape(3, 3) - ref).max() < 1e-15
        out = np.zeros(8)
        hh.hh_product_half(P(vA), P(vB), P(out))
        ref = sl.expm(-0.5j * (vB[0] * SX + vB[1] * SY + vB[2] * SZ)) @ sl.expm(-0.5j * (vA[0] * SX + vA[1] * SY + vA[2] * SZ))
        assert np.abs(out.view(np.complex128).reshape(2, 2) - ref).max() < 1e-15


@pytest.mark.parametrize("th,L", [(0.0, 100), (3e-5, 100), (0.088, 100), (2 * np.pi + 1e-7, 37),
                                  (6 * np.pi - 0.2, 50), (2 * np.pi, 10), (4 * np.pi, 11), (1.3, 1), (0.5, 2),
                                  (-0.7, 1000)])
def test_node_phasor_sum_closed_form(hh, th, L):
    for (W1, c1, W2, c2) in ((0.5, 0.2113248654051871, 0.5, 0.7886751345948129), (1.0, 0.5, 0.0, 0.5),
                             (0.5, 0.0, 0.5, 1.0)):
        out = np.zeros(2)
        hh.hh_node_phasor_sum(th, L, W1, c1, W2, c2, P(out))
        l = np.arange(L)
        ref = np.sum(W1 * np.exp(1j * th * (l + c1)) + W2 * np.exp(1j * th * (l + c2)))
        assert abs(out[0] + 1j * out[1] - ref) < 1e-12 * max(1, L)


def test_small_angle_functions(hh):
    """sin x - x and cos x - 1 to full relative precision (50-digit mpmath)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for x in (1e-9, -3e-5, 0.01, 0.0625, -0.2, 1.5):
        out = np.zeros(2)
        hh.hh_small_sincos_m(x, 0, P(out))
        sm = float(mp.sin(mp.mpf(x)) - mp.mpf(x))
        cm = float(mp.cos(mp.mpf(x)) - 1)
        if abs(x) <= 0.0625:   # series branch: full relative precision
            assert abs(out[0] - sm) <= 4e-16 * abs(sm)
            assert abs(out[1] - cm) <= 4e-16 * abs(cm)
        else:                  # libdevice branch: absolute precision of sin x
            assert abs(out[0] - sm) <= 2e-16 * abs(x)
            assert abs(out[1] - cm) <= 4e-16 * abs(cm)
    out = np.zeros(2)
    hh.hh_small_sincos_m(0.0, 0, P(out))
    assert out[0] == 0.0 and out[1] == 0.0


# ------------------------------------------------ automatic squarings (tau)
CF4_A, CF4_B = (3 + 2 * np.sqrt(3)) / 12, (3 - 2 * np.sqrt(3)) / 12


def splitting_bound(phi, vz, vq):
    """|E3| bound of the symmetric splitting for exponent (Phi, v_z, v_q)."""
    s = 2 * abs(vz) + abs(vq)
    return phi * phi * s / 6 + s * s * phi / 24


@pytest.mark.parametrize("seed", range(6))
def test_splitting_error_bound_holds(seed):
    """|T^n - exp(-i H)| <= |E3| / 4^tau (to leading order) for the leapfrog
    T = e^{-iD/2} e^{-i Phi J_phi} e^{-iD/2}, D = v_z J_z + v_q Q; exact
    exponentials from scipy, so this pins the bound, not the code using it."""
    rng = np.random.default_rng(seed)
    for _ in range(20):
        phi, ang = rng.uniform(1e-3, 0.05), rng.uniform(0, 2 * np.pi)
        vz, vq = rng.uniform(-0.05, 0.05), rng.uniform(-0.05, 0.05)
        D = vz * JZ1 + vq * Q1
        Jp = np.cos(ang) * JX1 + np.sin(ang) * JY1
        exact = sl.expm(-1j * (phi * Jp + D))
        for tau in (0, 1, 3):
            n = 2 ** tau
            Th = sl.expm(-0.5j * D / n) @ sl.expm(-1j * phi * Jp / n) @ sl.expm(-0.5j * D / n)
            err = np.abs(np.linalg.matrix_power(Th, n) - exact).max()
            assert err <= splitting_bound(phi, vz, vq) / 4 ** tau * 1.05 + 1e-15, (phi, vz, vq, tau, err)


def tau_rule(frame, n_exp, wa, wb, dt, om_perp, bias_w, pulse_w, q_w, steps, budget=1e-6):
    wabs, wsum = abs(wa) + abs(wb), abs(wa + wb)
    phi = wabs * dt * om_perp
    vz = wabs * dt * pulse_w + (0 if frame else wsum * dt * bias_w)
    err = steps * n_exp * splitting_bound(phi, vz, wsum * dt * q_w)
    return next(t for t in range(25) if err / 4 ** t <= budget or t == 24)


def test_choose_tau_rule(hh):
    tp = 2 * np.pi
    # the 100 ms spin-one sensing run: 2 x 1 kHz drive, 50 Hz pulse, q = 400 Hz, dt 10 ns
    sensing = dict(dt=1e-8, om_perp=tp * 2e3, bias_w=tp * 700e3, pulse_w=tp * 50, q_w=tp * 400, steps=9999900)
    cases = [(1, 2, CF4_A, CF4_B), (0, 2, CF4_A, CF4_B), (1, 1, 1.0, 0.0), (1, 1, 0.5, 0.5)]
    got = []
    for frame, n_exp, wa, wb in cases:
        for steps in (9999900, 19900, 1e12):
            kw = dict(sensing, steps=steps)
            t = hh.hh_choose_tau(-1, 1, frame, n_exp, wa, wb, kw["dt"], kw["om_perp"], kw["bias_w"],
                                 kw["pulse_w"], kw["q_w"], kw["steps"])
            assert t == tau_rule(frame, n_exp, wa, wb, **kw)
            got.append(t)
    assert got[0] == 0 and got[3] == 9          # rotating frame vs lab frame, full run
    assert got[4] < got[3] and got[5] > got[3]  # shorter runs need fewer squarings
    assert hh.hh_choose_tau(-1, 0, 1, 2, CF4_A, CF4_B, 1e-8, 1e4, 1e6, 0, 0, 1e7) == 24   # FP64 default
    assert hh.hh_choose_tau(5, 1, 1, 2, CF4_A, CF4_B, 1e-8, 1e4, 1e6, 0, 0, 1e7) == 5     # explicit tau


# ------------------------------------------------ small-angle FP32 variant
def test_tiny_series_within_bound(hh):
    """The two-term series the FP32 kernels use below kTinyAngleBound = 2^-6:
    sin, cos to FP32 rounding and sin x - x, cos x - 1 to full FP32 relative
    precision against 50-digit mpmath."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    b = hh.hh_tiny_angle_bound()
    assert b == 2.0 ** -6
    for x in np.concatenate([np.linspace(-b, b, 41), [1e-7, -3e-5, 2e-3]]):
        x = float(np.float32(x))
        out = np.zeros(4)
        hh.hh_tiny_sincos(x, P(out))
        X = mp.mpf(x)
        assert abs(out[0] - float(mp.sin(X))) <= 1.2e-7 * max(abs(x), 1e-30)
        assert abs(out[1] - float(mp.cos(X))) <= 1.2e-7
        if x != 0.0:
            assert abs(out[2] - float(mp.sin(X) - X)) <= 3e-7 * abs(float(mp.sin(X) - X))
            assert abs(out[3] - float(mp.cos(X) - 1)) <= 3e-7 * abs(float(mp.cos(X) - 1))


def test_small_angle_exponential_matches_general(hh):
    """Inside the bound the small-angle exponential equals the general FP32
    one to FP32 rounding and the exact exponential (scipy) to the FP32
    accuracy of the split residual."""
    rng = np.random.default_rng(7)
    for scale in (1e-6, 1e-4, 5e-3):
        for _ in range(20):
            v = rng.normal(size=4) * scale
            for tau in (0, 1, 4):
                a, g = np.zeros(18), np.zeros(18)
                hh.hh_expm_one_small(*v, tau, P(a))
                hh.hh_expm_one_general32(*v, tau, P(g))
                A = a.view(np.complex128).reshape(3, 3)
                G = g.view(np.complex128).reshape(3, 3)
                assert np.abs(A - G).max() <= 2e-7 * max(scale * scale, 1e-12) + 1e-13
                if tau == 4:
                    assert np.abs(A - sl.expm(-1j * H1(v))).max() < 1e-8


def test_tau0_closed_form_exponential(hh):
    """The tau = 0 small-angle exponential with the W conjugation folded in:
    in FP64 equal to the squaring path at tau = 0, its rest beyond first
    order equal to the single factor T computed in 50 digits up to rounding
    and the series' truncation; in FP32 equal to the squaring
    path's FP32 result (same approximant) to FP32 rounding.  Includes a zero
    transverse field and pure transverse fields."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(11)
    vs = [rng.normal(size=4) * s for s in (1e-6, 1e-4, 5e-3) for _ in range(12)]
    vs += [np.array([0.0, 0.0, 3e-3, 1e-3]), np.array([4e-3, 0.0, 0.0, 0.0]), np.array([0.0, -4e-3, 0.0, 2e-3])]
    for v in vs:
        out, rest = np.zeros(18), np.zeros(18)
        hh.hh_expm_one_tau0(*v, 0, P(out), P(rest))
        E = out.view(np.complex128).reshape(3, 3)
        ref = np.zeros(18)
        hh.hh_expm_one(*v, 0, 0, P(ref))                  # the squaring path at tau = 0, FP64
        R0 = ref.view(np.complex128).reshape(3, 3)
        assert np.abs(E - R0).max() < 4e-15 * np.abs(v).max() + 1e-18   # ~20 ulp of the entries
        # T itself: e^{-iD/2} e^{-i Phi J_phi} e^{-iD/2}, D = v_z J_z + v_q Q, in 50 digits
        Dm = mp.matrix((v[2] * JZ1 + v[3] * Q1).tolist())
        Pm = mp.matrix((v[0] * JX1 + v[1] * JY1).tolist())
        half = mp.expm(-0.5j * Dm)
        T = half * mp.expm(-1j * Pm) * half
        Hm = mp.matrix(H1(v).tolist())
        refm = T - mp.eye(3) + 1j * Hm
        want = np.array([[complex(refm[i, j]) for j in range(3)] for i in range(3)])
        got = rest.view(np.complex128).reshape(3, 3)
        # FP64 rounding of a second-order quantity, plus the series' truncation
        # (kappa drops y^3 / 5040: at most |v|^7 / 5040 in the transverse entries)
        s_ = np.abs(v).max()
        assert np.abs(got - want).max() <= 1e-15 * s_ ** 2 + s_ ** 7 / 1000 + 1e-30
        o32, r32, s32 = np.zeros(18), np.zeros(18), np.zeros(18)
        hh.hh_expm_one_tau0(*v, 1, P(o32), P(r32))
        hh.hh_expm_one_small(*v, 0, P(s32))
        A = o32.view(np.complex128).reshape(3, 3)
        B = s32.view(np.complex128).reshape(3, 3)
        assert np.abs(A - B).max() <= 2e-7 * max(np.abs(v).max() ** 2, 1e-12) + 1e-13


def test_tau0_variants_follow_the_squarings(hh):
    """Small-angle spin-one requests whose squarings come out as tau = 0 run
    the tau = 0 kernels (no runtime tau branch), exactly when fill_devsim gives
    them tau = 0; others keep the small-angle kernels with tau at run time;
    spin-half never takes them (no squarings); FP64 never takes a small-angle
    kernel."""
    from paper_2204_05586_gb300 import spinsim as S, workloads as W
    GEN, SMALL, TONES, SINE, T0, SINE_T0, SMALL_TONES = 0, 1, 2, 4, 5, 6, 7

    def pick(req, **cfg):
        c = S.make_config(**cfg)
        r = S.make_request(req)
        st, K, L = S.spinsim_counts(r)
        assert st == 0
        tau = ctypes.c_int()
        v = hh.hh_request_variant(ctypes.addressof(c), ctypes.addressof(r), K, L, ctypes.byref(tau))
        return v, tau.value
    assert pick(W.spin_one_sensing()) == (T0, 0)
    assert pick(W.spin_one_sensing(), precision=S.PREC_FP64)[0] == GEN
    v, tau = pick(W.neural_pulse())
    assert (v, tau) == (SINE, 2)                # 100 ns steps: two squarings
    short = W.neural_pulse()
    short["dt"] = 1e-8                          # 10 ns steps: tau = 0
    assert pick(short) == (SINE_T0, 0)
    assert pick(W.spin_half_rabi())[0] == SMALL
    for req in W.sweep(64, seed=W.SEED):
        v, tau = pick(req)
        assert v == (T0 if tau == 0 else SMALL), (v, tau)
    # further tones: the small-angle tones kernel inside the bounds (tau at run
    # time), the general one outside them, with a sine-cycle pulse, or in FP64
    v, tau = pick(W.multitone_sensing())
    assert v == SMALL_TONES and tau == 1, (v, tau)
    assert pick(W.multitone_sensing(), precision=S.PREC_FP64)[0] == TONES
    strong = W.multitone_sensing()
    strong["field"]["tones"] = [(1e6, 0.0, 700e3, 0.0)]        # a 1 MHz tone: Phi/2 > 2^-6
    assert pick(strong)[0] == TONES
    sine = W.multitone_sensing()
    sine["field"]["pulses"] = [(50.0, 0.05, 1e-3, "sine")]
    assert pick(sine)[0] == TONES


def test_small_angle_rule_on_workloads(hh):
    """The host picks the small-angle kernels for the rotating-frame FP32 runs
    of every workload shape, the paper's benchmark field with its
    single-sine-cycle pulse included (the sine-cycle twin of the kernel), and
    refuses them for FP64, for the lab frame and for a request whose step
    angles exceed the bound."""
    from paper_2204_05586_gb300 import spinsim as S, workloads as W
    def rule(req, **cfg):
        c = S.make_config(**cfg)
        r = S.make_request(req)
        L = int(round(req["dt_out"] / req["dt"]))
        return hh.hh_small_angle_request(ctypes.addressof(c), ctypes.addressof(r), L)
    sweep = W.sweep(64, seed=W.SEED)
    _, served = W.serving_stream(64, seed=W.SEED + 1)
    for req in [W.spin_one_sensing(), W.spin_half_rabi()] + sweep + served:
        assert rule(req) == 1
        assert rule(req, precision=S.PREC_FP64) == 0
    assert rule(W.spin_one_sensing(), rotating_frame=False) == 0
    assert rule(W.multitone_sensing()) == 1     # further tones count in the transverse bound
    assert rule(W.multitone_sensing(), precision=S.PREC_FP64) == 0
    assert rule(W.neural_pulse()) == 1          # sine-cycle pulse: the small-angle twin with sine cycles
    assert rule(W.neural_pulse(), precision=S.PREC_FP64) == 0
    big = W.spin_one_sensing(dt=1e-7)           # 10x larger steps: still inside the bound
    assert rule(big) == 1
    far = W.spin_one_sensing()
    far["field"]["drive_hz"] = far["field"]["bias_hz"] + 3e3   # 3 kHz detuning: (w_d - w_r) dt_out > 2^-6
    assert rule(far) == 0


def quadrature_first_order(req, k, L, frame, gsum):
    """g_x + i g_y of sample k written out: the CF4 quadrature (both
    exponentials: node weights a + b at each of the two nodes of every step) of
    the in-frame transverse field (w_x + i w_y) e^{-i w_r tau}, w_r = 2 pi B +
    gsum, tau measured from t_{k-1} (Sec. 1.2.5), from the field formula with
    every tone (numpy, FP64)."""
    f = req["field"]
    dt = req["dt_out"] / L
    t0 = req["t_start"] + (k - 1) * req["dt_out"]
    c1, c2 = 0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)
    tau = np.concatenate([(np.arange(L) + c1) * dt, (np.arange(L) + c2) * dt])
    t = t0 + tau
    tones = [(f["drive_x_hz"], f["drive_y_hz"], f["drive_hz"], f["drive_phase"])] + list(f.get("tones", ()))
    w = np.zeros_like(t, dtype=np.complex128)
    for x, y, hz, ph in tones:
        a = 2 * np.pi * hz * t + ph
        w += 2 * np.pi * (x * np.cos(a) + 1j * y * np.sin(a))
    if frame:
        w *= np.exp(-1j * (2 * np.pi * f["bias_hz"] + gsum) * tau)
    g = 0.5 * dt * w.sum()          # a + b = 1/2 per node, two exponentials
    return g.real, g.imag


@pytest.mark.parametrize("L", [7, 100, 70000])
@pytest.mark.parametrize("frame", [True, False])
def test_first_order_with_tones_is_the_quadrature(hh, L, frame):
    """The epilogue's exact first-order coefficients of a three-tone drive
    (Taylor tables for L <= 65536, else the closed form; with a strong pulse
    the closed form too) equal the quadrature sum written out."""
    from paper_2204_05586_gb300 import spinsim as S, workloads as W
    tones = [(1.2e3, 0.9e3, 19.6e3, 0.8), (0.0, 1.5e3, 60e3, -1.3), (0.7e3, 0.0, 7e3, 2.2)]
    for pulses in ([], [(3e3, 2.5e-4, 1e-4)]):
        f = W.field(bias_hz=20e3, drive_x_hz=2e3, drive_y_hz=0.4e3, drive_hz=20.3e3, drive_phase=0.2,
                    pulses=pulses, tones=tones)
        req = W.request(2, f, 1e-4, 1e-4 + 40 * 1e-5, 1e-5 / L, 1e-5)
        cfg = S.make_config(precision=S.PREC_FP64, rotating_frame=frame)
        r = S.make_request(req)
        for k in (1, 17, 40):
            out = np.zeros(3)
            hh.hh_first_order(ctypes.addressof(cfg), ctypes.addressof(r), 41, L, k, P(out))
            gx, gy = quadrature_first_order(req, k, L, frame, out[2] if frame else 0.0)
            scale = np.hypot(gx, gy) + 1e-3
            assert abs(out[0] - gx) < 1e-11 * scale and abs(out[1] - gy) < 1e-11 * scale, (k, out, gx, gy)


def test_branch_free_series_match_the_branching_ones(hh):
    """The CPU backend's four-sample type takes the series without the branch
    when every lane is small: the same bits as the one-sample functions."""
    rng = np.random.default_rng(9)
    for x in np.concatenate([rng.uniform(-0.0625, 0.0625, 2000), [0.0, 0.0625, -0.0625, 1e-30, -3e-8]]):
        assert hh.hh_series_match(float(x), 1) == 1, x
        assert hh.hh_series_match(float(x), 0) == 1, x


@pytest.mark.parametrize("scale", [1e-5, 3e-2, 0.7, 9.0])
def test_general_su3_exponential(hh, oracle_mod, scale):
    """The kernels' split-residual exponential of a full su(3) spin-one
    Hamiltonian (quadrupole drives) against the oracle's series and scipy."""
    from test_oracle_su3 import hamiltonian8
    rng = np.random.default_rng(int(scale * 1e5) + 11)
    for _ in range(10):
        w = rng.normal(size=8) * scale
        out = np.zeros(18)
        hh.hh_expm_general(P(w), P(out))
        E = out.view(np.complex128).reshape(3, 3)
        ref = sl.expm(-1j * hamiltonian8(w))
        tol = 3e-15 * max(1.0, 8 * scale)
        assert np.abs(E - ref).max() < tol
        assert np.abs(E - oracle_mod.expm_general(w, 1.0)).max() < tol


def test_general_exponential_degree_choice(hh):
    """The Taylor degree is chosen from the scaled norm: just below each
    switch point (and at norms that need scaling) the carried rest of
    exp(-i H) - I still has the accuracy of the first-order term, against a
    50-digit mpmath exponential.  One degree less would miss by 1e-13 and
    more relative to the norm."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    from test_oracle_su3 import hamiltonian8
    rng = np.random.default_rng(21)
    for theta in (1e-9, 6.8e-6, 1.99e-4, 1.57e-3, 6.3e-3, 1.76e-2, 3.8e-2, 7.0e-2, 0.116, 0.176, 0.25, 0.9, 3.0):
        for _ in range(3):
            w = rng.normal(size=8)
            H = hamiltonian8(w)
            w *= theta / np.max(np.sum(np.abs(H.real) + np.abs(H.imag), axis=1))
            out = np.zeros(18)
            hh.hh_expm_general_rest(P(w), P(out))
            rest = out.view(np.complex128).reshape(3, 3)
            Hm = mp.matrix(hamiltonian8(w).tolist())
            HJ = mp.matrix(H1(w[:4]).tolist())
            refm = mp.expm(-1j * Hm) - mp.eye(3) + 1j * HJ
            ref = np.array([[complex(refm[i, j]) for j in range(3)] for i in range(3)])
            assert np.abs(rest - ref).max() < 1e-15 * max(theta, theta ** 2), theta



def exact_cycles(f, t0, dt, m):
    """frac(f (t0 + m dt)) of the binary values f, t0, dt, in exact rational
    arithmetic."""
    from fractions import Fraction as Fr
    x = Fr(f) * (Fr(t0) + m * Fr(dt))
    return x - (x.numerator // x.denominator)


def cyc_dist(a, b):
    d = abs(float(a) - float(b)) % 1.0
    return min(d, 1.0 - d)


def test_drive_cycles_are_exact_to_rounding(hh):
    """The drive phase's fractional cycles at t0 + m dt, split by Dekker
    products, equal the exact rational value to a few 1e-16 cycles at every
    size of f t, where the plain product f t loses about 2^-53 f t."""
    rng = np.random.default_rng(17)
    worst, worst_plain = 0.0, 0.0
    for _ in range(400):
        f = float(rng.uniform(1e5, 3e6))
        t0 = float(rng.choice([0.0, rng.uniform(-1e-2, 0.2)]))
        dt = float(rng.choice([1e-6, 1e-7, 2.5e-7, rng.uniform(1e-8, 1e-5)]))
        m = int(rng.integers(0, 10**7))
        ex = exact_cycles(f, t0, dt, m)
        got = hh.hh_drive_cycles_frac(f, t0, dt, m)
        assert 0.0 <= got < 1.0
        worst = max(worst, cyc_dist(got, ex))
        ft = f * (t0 + m * dt)
        worst_plain = max(worst_plain, cyc_dist(ft - np.floor(ft), ex))
    assert worst < 5e-16, worst
    assert worst_plain > 1e-13   # what the split avoids
    # special cases: no drive, m = 0, t0 = 0
    assert hh.hh_drive_cycles_frac(0.0, 0.3, 1e-6, 12345) == 0.0
    assert cyc_dist(hh.hh_drive_cycles_frac(7e5, 0.0, 1e-6, 0), 0) == 0.0
    assert cyc_dist(hh.hh_drive_cycles_frac(7e5 + 0.25, 0.0, 1.0, 3), exact_cycles(7e5 + 0.25, 0.0, 1.0, 3)) == 0.0


@pytest.mark.parametrize("K", [2, 129, 100001])
def test_drive_phasor_tables_match_the_exact_phasor(hh, K):
    """e^{i beta_k} from the two-level tables (every interval, both table
    edges, the last) against the exact phase and 30-digit sin/cos: within
    1.5e-15 (the roundings of 2 pi cyc + phase and of its reduction, the
    sine and cosine, the product: a few 2^-53 each), where the sine and
    cosine of the FP64 drive phase err by the phase's rounding, which grows
    with f t."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    from paper_2204_05586_gb300 import spinsim as S, workloads as W
    f = W.field(bias_hz=700e3, drive_x_hz=2e3, drive_hz=700.7e3, drive_phase=1.1, quad_hz=400.0)
    dt_out = 1e-6
    req = W.request(2, f, 3e-3, 3e-3 + K * dt_out, 1e-8, dt_out)
    cfg = S.make_config(precision=S.PREC_FP64)
    r = S.make_request(req)
    assert S.spinsim_counts(r)[1] == K
    ks = sorted({1, 2, min(128, K - 1), min(129, K - 1), min(130, K - 1), K - 1, K // 2 + 1})
    rng = np.random.default_rng(3)
    ks += [int(x) for x in rng.integers(1, K, 20)]
    worst_tab, worst_sin = 0.0, 0.0
    for k in ks:
        out = np.zeros(4)
        hh.hh_phasor(ctypes.addressof(cfg), ctypes.addressof(r), K, 100, k, -1, 1, P(out))
        cyc = exact_cycles(f["drive_hz"], req["t_start"], dt_out, k - 1)
        b = 2 * mpmath.pi * mpmath.mpf(cyc.numerator) / cyc.denominator + f["drive_phase"]
        ex = complex(mpmath.cos(b), mpmath.sin(b))
        worst_tab = max(worst_tab, abs(complex(out[0], out[1]) - ex))
        old = np.zeros(4)
        hh.hh_phasor(ctypes.addressof(cfg), ctypes.addressof(r), K, 100, k, -1, 0, P(old))
        worst_sin = max(worst_sin, abs(complex(old[0], old[1]) - ex))
    assert worst_tab < 1.5e-15, worst_tab
    assert worst_sin < 1e-10, worst_sin


@pytest.mark.parametrize("K", [2, 130, 100001])
def test_tone_phasor_tables_match_the_exact_phasor(hh, K):
    """Each further tone's table (after the drive's in the same block) gives
    e^{i beta_j,k} within 1.5e-15 of the exact phase's 30-digit sin/cos, for
    every tone, both table edges and the last interval; the drive's entries
    are unchanged by the tones' tables behind them."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    from paper_2204_05586_gb300 import spinsim as S, workloads as W
    tones = [(1e3, 1e3, 700.5e3, 0.4), (0.5e3, 0.0, 698e3, 1.1), (0.0, 0.8e3, 705.3e3, -0.6)]
    f = W.field(bias_hz=700e3, drive_x_hz=2e3, drive_hz=700.7e3, drive_phase=1.1, quad_hz=400.0, tones=tones)
    dt_out = 1e-6
    req = W.request(2, f, 3e-3, 3e-3 + K * dt_out, 1e-8, dt_out)
    cfg = S.make_config(precision=S.PREC_FP64)
    r = S.make_request(req)
    assert S.spinsim_counts(r)[1] == K
    ks = sorted({1, min(128, K - 1), min(129, K - 1), K - 1, K // 2 + 1})
    worst = 0.0
    for j in range(-1, len(tones)):
        hz, ph = (f["drive_hz"], f["drive_phase"]) if j < 0 else (tones[j][2], tones[j][3])
        for k in ks:
            out = np.zeros(2)
            hh.hh_phasor(ctypes.addressof(cfg), ctypes.addressof(r), K, 100, k, j, 1, P(out))
            cyc = exact_cycles(hz, req["t_start"], dt_out, k - 1)
            b = 2 * mpmath.pi * mpmath.mpf(cyc.numerator) / cyc.denominator + ph
            worst = max(worst, abs(complex(out[0], out[1]) - complex(mpmath.cos(b), mpmath.sin(b))))
    assert worst < 1.5e-15, worst


def test_integer_widening_is_the_ieee_conversion(hh):
    """widen_bits (the epilogue's FP32 -> FP64 in integer instructions)
    against the exact conversion numpy performs, bit for bit: both zeros,
    every subnormal exponent (each mantissa bit alone, plus the smallest and
    the largest subnormal), the normal range's edges, the infinities, and 2^21
    random bit patterns; NaN inputs give NaN of the same sign."""
    pats = [0x00000000, 0x80000000, 0x00000001, 0x80000001, 0x007fffff, 0x807fffff, 0x00800000,
            0x7f7fffff, 0xff7fffff, 0x3f800000, 0xbf800000, 0x7f800000, 0xff800000]
    pats += [1 << b for b in range(23)] + [(1 << b) | 0x80000000 for b in range(23)]
    pats += [(1 << b) | 1 for b in range(1, 23)]
    rng = np.random.default_rng(11)
    bits = np.concatenate([np.array(pats, dtype=np.uint32), rng.integers(0, 2**32, 1 << 21, dtype=np.uint32)])
    out = np.zeros(bits.size, dtype=np.uint64)
    hh.hh_widen_bits(bits.ctypes.data, out.ctypes.data, bits.size)
    f = bits.view(np.float32)
    got = out.view(np.float64)
    nan = np.isnan(f)
    assert nan.sum() > 1000 and (~nan).sum() > 1_000_000
    want = f[~nan].astype(np.float64)
    assert np.array_equal(got[~nan].view(np.uint64), want.view(np.uint64))
    assert np.isnan(got[nan]).all()
    assert np.array_equal(np.signbit(got[nan]), np.signbit(f[nan]))


def test_chain_run_rule(hh):
    """The chain's lane runs depend on K alone: 4 below 16384 samples, at least
    6 from there, one more per 19456 samples beyond 6 x 19456, at most 8; the
    bench's flop model uses the same rule."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    want = {1: 4, 16383: 4, 16384: 6, 100000: 6, 116736: 6, 116737: 7, 136192: 7, 136193: 8, 10**7: 8}
    run, top = ctypes.c_int(), ctypes.c_int()
    for K, r in want.items():
        hh.hh_chain_geom(K, ctypes.byref(run), ctypes.byref(top))
        assert run.value == r, (K, run.value)
        assert bench.chain_run(K) == r, K
    for K in range(1, 300000, 997):
        hh.hh_chain_geom(K, ctypes.byref(run), ctypes.byref(top))
        assert bench.chain_run(K) == run.value, K
