"""ctypes binding of the plain-C FP64 oracle (test infrastructure only).

Every function here is argument marshalling around ``spinsim_oracle.c``; the
method's arithmetic is all in that file.  Field parameters are given as a
plain ``dict`` with the keys of :data:`FIELD_KEYS` (frequencies in Hz, times
in seconds), the same description the seeded workload generators produce.

Parity status: every exported function is pinned by ``tests/test_oracle_*.py``
against closed forms, library exponentials (scipy), an independent ODE solver
and invariants; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spinsim_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libspinsim_oracle.so")

MAX_PULSES = 4
MAX_TONES = 3
FIELD_KEYS = ("bias_hz", "drive_x_hz", "drive_y_hz", "drive_hz", "drive_phase",
              "quad_hz", "pulses")

METHOD_CF4, METHOD_MIDPOINT, METHOD_HEUN = 0, 1, 2
DEFAULT_TAU = 24  # Sec. 1.2.3: n = 2^24 by default


class _Field(ctypes.Structure):
    _fields_ = [
        ("bias_hz", ctypes.c_double),
        ("drive_x_hz", ctypes.c_double),
        ("drive_y_hz", ctypes.c_double),
        ("drive_hz", ctypes.c_double),
        ("drive_phase", ctypes.c_double),
        ("quad_hz", ctypes.c_double),
        ("n_pulses", ctypes.c_int32),
        ("pulse_sine_mask", ctypes.c_int32),
        ("pulse_amp_hz", ctypes.c_double * MAX_PULSES),
        ("pulse_centre_s", ctypes.c_double * MAX_PULSES),
        ("pulse_width_s", ctypes.c_double * MAX_PULSES),
        ("n_tones", ctypes.c_int32),
        ("pad2_", ctypes.c_int32),
        ("tone_x_hz", ctypes.c_double * MAX_TONES),
        ("tone_y_hz", ctypes.c_double * MAX_TONES),
        ("tone_hz", ctypes.c_double * MAX_TONES),
        ("tone_phase", ctypes.c_double * MAX_TONES),
        ("qd_on", ctypes.c_int32),
        ("pad3_", ctypes.c_int32),
        ("qd_x_hz", ctypes.c_double * 2),
        ("qd_y_hz", ctypes.c_double * 2),
        ("qd_hz", ctypes.c_double * 2),
        ("qd_phase", ctypes.c_double * 2),
    ]


class _Plan(ctypes.Structure):
    _fields_ = [
        ("spin_x2", ctypes.c_int32),
        ("method", ctypes.c_int32),
        ("rotating_frame", ctypes.c_int32),
        ("tau", ctypes.c_int32),
        ("t_start", ctypes.c_double),
        ("dt_out", ctypes.c_double),
        ("K", ctypes.c_int64),
        ("L", ctypes.c_int64),
    ]


_lib = None
_lib_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math) into ``oracle/_build``."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lib_lock:
        if _lib is None:
            # SPINSIM_ORACLE_LIB lets the mutation test load a deliberately
            # broken copy of the oracle in a subprocess.
            lib = ctypes.CDLL(os.environ.get("SPINSIM_ORACLE_LIB") or build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_field_sample.argtypes = [ctypes.POINTER(_Field), ctypes.c_double, dp]
            lib.oracle_field_sample_quad.argtypes = [ctypes.POINTER(_Field), ctypes.c_double, dp]
            lib.oracle_expm_general.argtypes = [dp, ctypes.c_double, dp]
            lib.oracle_expm_spin_half.argtypes = [ctypes.c_double] * 4 + [dp]
            for name in ("oracle_trotter_T", "oracle_expm_spin_one", "oracle_expm_spin_one_residual"):
                getattr(lib, name).argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, dp]
            lib.oracle_counts.argtypes = [ctypes.c_double] * 4 + [ctypes.POINTER(ctypes.c_int64)] * 2
            lib.oracle_counts.restype = ctypes.c_int
            lib.oracle_sample_operators.argtypes = [ctypes.POINTER(_Plan), ctypes.POINTER(_Field),
                                                    ctypes.c_int64, ctypes.c_int64, dp]
            lib.oracle_chain.argtypes = [ctypes.c_int32, ctypes.c_int64, dp, dp, dp, dp]
            lib.oracle_simulate.argtypes = [ctypes.POINTER(_Plan), ctypes.POINTER(_Field), dp, dp, dp, dp]
            lib.oracle_frame_rate.argtypes = [ctypes.POINTER(_Plan), ctypes.POINTER(_Field), ctypes.c_int64]
            lib.oracle_frame_rate.restype = ctypes.c_double
            lib.oracle_error_metric.argtypes = [ctypes.c_int32, ctypes.c_int64, dp, dp]
            lib.oracle_error_metric.restype = ctypes.c_double
            _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _field(f: dict) -> _Field:
    s = _Field()
    for k in ("bias_hz", "drive_x_hz", "drive_y_hz", "drive_hz", "drive_phase", "quad_hz"):
        setattr(s, k, float(f.get(k, 0.0)))
    pulses = list(f.get("pulses", ()))
    if len(pulses) > MAX_PULSES:
        raise ValueError("at most 4 pulses")
    s.n_pulses = len(pulses)
    s.pulse_sine_mask = 0
    for i, p in enumerate(pulses):
        amp, centre, width = p[:3]
        kind = p[3] if len(p) > 3 else "gauss"
        if kind not in ("gauss", "sine"):
            raise ValueError(f"unknown pulse kind {kind!r}")
        s.pulse_amp_hz[i] = amp
        s.pulse_centre_s[i] = centre
        s.pulse_width_s[i] = width
        if kind == "sine":
            s.pulse_sine_mask |= 1 << i
    tones = list(f.get("tones", ()))
    if len(tones) > MAX_TONES:
        raise ValueError("at most 3 further tones")
    s.n_tones = len(tones)
    for j, (x, y, hz, ph) in enumerate(tones):
        s.tone_x_hz[j], s.tone_y_hz[j], s.tone_hz[j], s.tone_phase[j] = x, y, hz, ph
    qdrives = list(f.get("qdrives", ()))
    if len(qdrives) > 2:
        raise ValueError("two quadrupole drives at most")
    s.qd_on = 1 if qdrives else 0
    for p, (x, y, hz, ph) in enumerate(qdrives):
        s.qd_x_hz[p], s.qd_y_hz[p], s.qd_hz[p], s.qd_phase[p] = x, y, hz, ph
    return s


def counts(t_start, t_end, dt, dt_out):
    """(K, L): output samples and integration steps per sample (Sec. 1.2.4)."""
    K, L = ctypes.c_int64(), ctypes.c_int64()
    if _load().oracle_counts(t_start, t_end, dt, dt_out, ctypes.byref(K), ctypes.byref(L)) != 0:
        raise ValueError("time span / output step / integration step are not integer ratios")
    return K.value, L.value


def _plan(spin_x2, t_start, t_end, dt, dt_out, rotating_frame, tau, method):
    K, L = counts(t_start, t_end, dt, dt_out)
    p = _Plan()
    p.spin_x2, p.method, p.rotating_frame, p.tau = spin_x2, method, int(bool(rotating_frame)), tau
    p.t_start, p.dt_out, p.K, p.L = t_start, dt_out, K, L
    return p


def field_sample(field: dict, t: float) -> np.ndarray:
    """(w_x, w_y, w_z, w_q) at time t in rad/s."""
    out = np.zeros(4)
    _load().oracle_field_sample(ctypes.byref(_field(field)), t, _dp(out))
    return out


def field_sample_quad(field: dict, t: float) -> np.ndarray:
    """(w_xz, w_yz, w_x2y2, w_xy) of the quadrupole drives at time t in rad/s."""
    out = np.zeros(4)
    _load().oracle_field_sample_quad(ctypes.byref(_field(field)), t, _dp(out))
    return out


def expm_general(w, dt) -> np.ndarray:
    """exp(-i dt sum_j w_j G_j) over the spin-one su(3) basis (J_x, J_y, J_z, Q,
    D_xz, D_yz, D_x2y2, D_xy)."""
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    out = np.zeros(18)
    _load().oracle_expm_general(_dp(w), dt, _dp(out))
    return out.view(np.complex128).reshape(3, 3)


def expm_spin_half(wx, wy, wz, dt) -> np.ndarray:
    out = np.zeros(8)
    _load().oracle_expm_spin_half(wx, wy, wz, dt, _dp(out))
    return out.view(np.complex128).reshape(2, 2)


def trotter_T(wx, wy, wz, wq, dt, tau) -> np.ndarray:
    out = np.zeros(18)
    _load().oracle_trotter_T(wx, wy, wz, wq, dt, tau, _dp(out))
    return out.view(np.complex128).reshape(3, 3)


def expm_spin_one(wx, wy, wz, wq, dt, tau=DEFAULT_TAU) -> np.ndarray:
    out = np.zeros(18)
    _load().oracle_expm_spin_one(wx, wy, wz, wq, dt, tau, _dp(out))
    return out.view(np.complex128).reshape(3, 3)


def expm_spin_one_residual(wx, wy, wz, wq, dt, tau=DEFAULT_TAU) -> np.ndarray:
    out = np.zeros(18)
    _load().oracle_expm_spin_one_residual(wx, wy, wz, wq, dt, tau, _dp(out))
    return out.view(np.complex128).reshape(3, 3)


def sample_operators(spin_x2, field, t_start, t_end, dt, dt_out, k0=0, k1=None, *,
                     rotating_frame=True, tau=DEFAULT_TAU, method=METHOD_CF4, threads=1):
    """U_k for k in [k0, k1) as complex128 [k1-k0, N, N]; U_0 is the identity.

    ``threads`` > 1 splits the k range over Python threads (the C call releases
    the GIL); each U_k is computed exactly as in the single-thread case."""
    p = _plan(spin_x2, t_start, t_end, dt, dt_out, rotating_frame, tau, method)
    if k1 is None:
        k1 = p.K
    n = 2 if spin_x2 == 1 else 3
    out = np.zeros((max(k1 - k0, 0), n, n, 2))
    f = _field(field)
    lib = _load()
    if k1 <= k0:
        return out.view(np.complex128).reshape(-1, n, n)

    def run(a, b):
        lib.oracle_sample_operators(ctypes.byref(p), ctypes.byref(f), a, b, _dp(out[a - k0:b - k0]))

    if threads <= 1:
        run(k0, k1)
    else:
        edges = np.linspace(k0, k1, min(threads * 4, k1 - k0) + 1).astype(np.int64)
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda ab: run(int(ab[0]), int(ab[1])), zip(edges[:-1], edges[1:])))
    return out.view(np.complex128).reshape(-1, n, n)


def frame_rate(spin_x2, field, t_start, t_end, dt, dt_out, k, *, rotating_frame=True):
    """w_r the oracle uses for sample interval k (rad/s)."""
    p = _plan(spin_x2, t_start, t_end, dt, dt_out, rotating_frame, DEFAULT_TAU, METHOD_CF4)
    return _load().oracle_frame_rate(ctypes.byref(p), ctypes.byref(_field(field)), k)


def chain(ops: np.ndarray, psi0) -> tuple[np.ndarray, np.ndarray]:
    """psi_k = U_k psi_{k-1} sequentially; returns (states [K,N], spin [K,3])."""
    ops = np.ascontiguousarray(ops, dtype=np.complex128)
    K, n, _ = ops.shape
    spin_x2 = 1 if n == 2 else 2
    psi0 = np.ascontiguousarray(np.asarray(psi0, dtype=np.complex128))
    states = np.zeros((K, n), dtype=np.complex128)
    spin = np.zeros((K, 3))
    _load().oracle_chain(spin_x2, K, _dp(ops.view(np.float64)), _dp(psi0.view(np.float64)),
                         _dp(states.view(np.float64)), _dp(spin))
    return states, spin


def simulate(spin_x2, field, t_start, t_end, dt, dt_out, psi0, *, rotating_frame=True,
             tau=DEFAULT_TAU, method=METHOD_CF4, want_ops=False, threads=1):
    """Whole simulation. Returns dict(states [K,N] c128, spin [K,3], ops [K,N,N] or None).

    With threads > 1 the sample operators are computed in parallel threads and
    then chained sequentially (same arithmetic per U_k as threads == 1)."""
    n = 2 if spin_x2 == 1 else 3
    psi0 = np.ascontiguousarray(np.asarray(psi0, dtype=np.complex128))
    if psi0.shape != (n,):
        raise ValueError("psi0 has the wrong length")
    if spin_x2 == 1 and field.get("qdrives"):
        raise ValueError("quadrupole drives need spin one")
    if threads > 1:
        ops = sample_operators(spin_x2, field, t_start, t_end, dt, dt_out, rotating_frame=rotating_frame,
                               tau=tau, method=method, threads=threads)
        states, spin = chain(ops, psi0)
        return {"states": states, "spin": spin, "ops": ops if want_ops else None}
    p = _plan(spin_x2, t_start, t_end, dt, dt_out, rotating_frame, tau, method)
    states = np.zeros((p.K, n), dtype=np.complex128)
    spin = np.zeros((p.K, 3))
    ops = np.zeros((p.K, n, n), dtype=np.complex128) if want_ops else None
    rc = _load().oracle_simulate(ctypes.byref(p), ctypes.byref(_field(field)), _dp(psi0.view(np.float64)),
                                 _dp(states.view(np.float64)), _dp(spin),
                                 _dp(ops.view(np.float64)) if want_ops else None)
    if rc != 0:
        raise ValueError("bad spin")
    return {"states": states, "spin": spin, "ops": ops}


def error_metric(states: np.ndarray, base: np.ndarray) -> float:
    """Eq. error of the paper (RMS-type error with 1/K outside the root)."""
    states = np.ascontiguousarray(states, dtype=np.complex128)
    base = np.ascontiguousarray(base, dtype=np.complex128)
    K, n = states.shape
    return _load().oracle_error_metric(1 if n == 2 else 2, K, _dp(states.view(np.float64)),
                                       _dp(base.view(np.float64)))
