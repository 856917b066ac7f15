"""Thin ctypes binding of the C ABI in ``include/spinsim.h``.

Functions named ``spinsim_*`` are one-to-one wrappers of the C entry points
(argument marshalling only).  :class:`Simulator` adds the convenience of
allocating the output buffers as torch tensors; torch is used only for device
memory and streams.  Every step of the integration runs in the CUDA library;
if it cannot be loaded, the functions here raise instead of falling back.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

MAX_PULSES = 4
MAX_TONES = 3

OK, PENDING = 0, 1
E_ARG, E_STEP_RATIO, E_NORM, E_NOMEM, E_CUDA, E_TIMEOUT, E_CAPACITY, E_UNSUPPORTED = -1, -2, -3, -4, -5, -6, -7, -8
WARN_MAGNUS = 1
WARN_FP32_LAB = 2
METHOD_CF4, METHOD_MIDPOINT, METHOD_HEUN = 0, 1, 2
PREC_FP64, PREC_FP32_BULK = 0, 1


class SpinsimError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})" if what else status_string(status))


class spinsim_config(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("precision", ctypes.c_int32), ("rotating_frame", ctypes.c_int32),
                ("trotter_squares", ctypes.c_int32), ("lanes_per_sample", ctypes.c_int32),
                ("threads_per_block", ctypes.c_int32), ("use_graphs", ctypes.c_int32), ("device", ctypes.c_int32),
                ("mem_budget", ctypes.c_int64), ("profile", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("chain_precision", ctypes.c_int32), ("direct_host_outputs", ctypes.c_int32)]


class spinsim_field(ctypes.Structure):
    _fields_ = [("bias_hz", ctypes.c_double), ("drive_x_hz", ctypes.c_double), ("drive_y_hz", ctypes.c_double),
                ("drive_hz", ctypes.c_double), ("drive_phase", ctypes.c_double), ("quad_hz", ctypes.c_double),
                ("n_pulses", ctypes.c_int32), ("pulse_sine_mask", ctypes.c_int32),
                ("pulse_amp_hz", ctypes.c_double * MAX_PULSES), ("pulse_centre_s", ctypes.c_double * MAX_PULSES),
                ("pulse_width_s", ctypes.c_double * MAX_PULSES),
                ("n_tones", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("tone_x_hz", ctypes.c_double * MAX_TONES), ("tone_y_hz", ctypes.c_double * MAX_TONES),
                ("tone_hz", ctypes.c_double * MAX_TONES), ("tone_phase", ctypes.c_double * MAX_TONES),
                ("qd_on", ctypes.c_int32), ("reserved2", ctypes.c_int32),
                ("qd_x_hz", ctypes.c_double * 2), ("qd_y_hz", ctypes.c_double * 2),
                ("qd_hz", ctypes.c_double * 2), ("qd_phase", ctypes.c_double * 2)]


class spinsim_request(ctypes.Structure):
    _fields_ = [("spin_x2", ctypes.c_int32), ("reserved", ctypes.c_int32), ("field", spinsim_field),
                ("t_start", ctypes.c_double), ("t_end", ctypes.c_double), ("dt", ctypes.c_double),
                ("dt_out", ctypes.c_double), ("psi0", ctypes.c_double * 6)]


class spinsim_result(ctypes.Structure):
    _fields_ = [("states", ctypes.c_void_p), ("spin", ctypes.c_void_p), ("ops", ctypes.c_void_p),
                ("capacity", ctypes.c_int64), ("n_samples", ctypes.c_int64), ("status", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("trotter_squares", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class spinsim_launch_info(ctypes.Structure):
    _fields_ = [("lanes_per_sample", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("kernels_launched", ctypes.c_int32),
                ("trotter_squares", ctypes.c_int32), ("graph_replayed", ctypes.c_int32),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64), ("integrate_ms", ctypes.c_double),
                ("chain_ms", ctypes.c_double)]


class spinsim_memory_info(ctypes.Structure):
    _fields_ = [("budget", ctypes.c_int64), ("held", ctypes.c_int64), ("peak_held", ctypes.c_int64),
                ("arena", ctypes.c_int64), ("pool", ctypes.c_int64), ("pool_in_use", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("in_flight", ctypes.c_int64)]


EXPORTED = ("spinsim_config_default", "spinsim_create", "spinsim_destroy", "spinsim_counts", "spinsim_footprint",
            "spinsim_simulate", "spinsim_submit", "spinsim_poll", "spinsim_poll_any", "spinsim_memory",
            "spinsim_last_launch", "spinsim_status_string",
            "spinsim_simulate_static", "spinsim_range_begin", "spinsim_range_finish",
            "spinsim_range_entering_state", "spinsim_debug_bounds")

_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libspinsim.so (building it first if needed); raises if impossible.
    With SPINSIM_BOUNDS=1 in the environment the process loads the debug
    library with range-checked kernels instead (libspinsim_bounds.so)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        bounds = os.environ.get("SPINSIM_BOUNDS") == "1"
        path = _build.BOUNDS_LIB if bounds else _build.LIB
        if build_if_missing:
            path = _build.build_bounds() if bounds else _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run paper_2204_05586_gb300.build.build()")
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        L.spinsim_config_default.argtypes = [P(spinsim_config)]
        L.spinsim_create.argtypes = [P(spinsim_config), P(ctypes.c_void_p)]
        L.spinsim_destroy.argtypes = [ctypes.c_void_p]
        L.spinsim_destroy.restype = None
        L.spinsim_counts.argtypes = [P(spinsim_request), P(ctypes.c_int64), P(ctypes.c_int64)]
        L.spinsim_footprint.argtypes = [ctypes.c_void_p, P(spinsim_request), ctypes.c_int64]
        L.spinsim_footprint.restype = ctypes.c_int64
        L.spinsim_simulate.argtypes = [ctypes.c_void_p, P(spinsim_request), P(spinsim_result), ctypes.c_int64,
                                       ctypes.c_void_p]
        L.spinsim_submit.argtypes = [ctypes.c_void_p, P(spinsim_request), P(spinsim_result), P(ctypes.c_int64)]
        L.spinsim_poll.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32]
        L.spinsim_poll_any.argtypes = [ctypes.c_void_p, P(ctypes.c_int64), ctypes.c_int64, ctypes.c_int32,
                                       P(ctypes.c_int64)]
        L.spinsim_memory.argtypes = [ctypes.c_void_p, P(spinsim_memory_info)]
        L.spinsim_last_launch.argtypes = [ctypes.c_void_p, P(spinsim_launch_info)]
        L.spinsim_simulate_static.argtypes = [P(spinsim_config), P(spinsim_request), P(spinsim_result),
                                              ctypes.c_void_p]
        L.spinsim_range_begin.argtypes = [ctypes.c_void_p, P(spinsim_request), P(spinsim_result),
                                          P(ctypes.c_double), ctypes.c_void_p]
        L.spinsim_range_finish.argtypes = [ctypes.c_void_p, P(ctypes.c_double), ctypes.c_void_p]
        L.spinsim_range_entering_state.argtypes = [ctypes.c_int32, P(ctypes.c_double), ctypes.c_int32,
                                                   P(ctypes.c_double), P(ctypes.c_double)]
        L.spinsim_debug_bounds.argtypes = [ctypes.c_int32, P(ctypes.c_uint64)]
        L.spinsim_status_string.argtypes = [ctypes.c_int]
        L.spinsim_status_string.restype = ctypes.c_char_p
        _lib = L
        return L


# ---------------------------------------------------------------- raw C ABI
def spinsim_config_default(cfg: spinsim_config) -> int:
    return load().spinsim_config_default(ctypes.byref(cfg))


def spinsim_create(cfg: spinsim_config) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    st = load().spinsim_create(ctypes.byref(cfg), ctypes.byref(h))
    if st != OK:
        raise SpinsimError(st, "spinsim_create")
    return h


def spinsim_destroy(h) -> None:
    load().spinsim_destroy(h)


def spinsim_counts(req: spinsim_request):
    K, L = ctypes.c_int64(), ctypes.c_int64()
    st = load().spinsim_counts(ctypes.byref(req), ctypes.byref(K), ctypes.byref(L))
    return st, K.value, L.value


def spinsim_footprint(h, reqs) -> int:
    arr = (spinsim_request * len(reqs))(*reqs)
    return load().spinsim_footprint(h, arr, len(reqs))


def spinsim_simulate(h, reqs, results, stream: int = 0) -> int:
    """reqs, results: ctypes arrays (or lists) of spinsim_request / spinsim_result."""
    n = len(reqs)
    ra = reqs if isinstance(reqs, ctypes.Array) else (spinsim_request * n)(*reqs)
    rs = results if isinstance(results, ctypes.Array) else (spinsim_result * n)(*results)
    return load().spinsim_simulate(h, ra, rs, n, ctypes.c_void_p(stream))


def spinsim_simulate_static(cfg: spinsim_config, req: spinsim_request, res: spinsim_result, stream: int = 0) -> int:
    """One request with no allocation by the library (scratch in a fixed
    device array); the outputs must be device buffers."""
    return load().spinsim_simulate_static(ctypes.byref(cfg), ctypes.byref(req), ctypes.byref(res),
                                          ctypes.c_void_p(stream))


def spinsim_range_begin(h, req: spinsim_request, res: spinsim_result, stream: int = 0):
    """Returns (status, agg) with agg the range's ordered product as a
    complex128 [N, N] numpy array."""
    import numpy as np
    n = req.spin_x2 + 1
    agg = (ctypes.c_double * (2 * n * n))()
    st = load().spinsim_range_begin(h, ctypes.byref(req), ctypes.byref(res), agg, stream)
    a = np.frombuffer(agg, dtype=np.float64).copy().view(np.complex128).reshape(n, n)
    return st, a


def spinsim_range_finish(h, psi_in, stream: int = 0) -> int:
    import numpy as np
    psi = np.ascontiguousarray(np.asarray(psi_in, dtype=np.complex128)).view(np.float64)
    buf = (ctypes.c_double * 6)(*([float(x) for x in psi] + [0.0] * (6 - len(psi))))
    return load().spinsim_range_finish(h, buf, stream)


def spinsim_range_entering_state(spin_x2: int, aggs, rank: int, psi_init):
    """Returns (status, psi) with psi the complex128 [N] state entering range
    `rank` from the ranges' propagators aggs[0 .. rank-1] (complex [N, N])."""
    n = spin_x2 + 1
    a = np.ascontiguousarray(np.asarray(aggs[:rank], dtype=np.complex128).reshape(-1)).view(np.float64) \
        if rank > 0 else np.zeros(2, np.float64)
    p = np.ascontiguousarray(np.asarray(psi_init, dtype=np.complex128)).view(np.float64)
    if p.size != 2 * n:
        return E_ARG, None
    out = np.zeros(2 * n, np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    st = load().spinsim_range_entering_state(spin_x2, a.ctypes.data_as(dp), rank, p.ctypes.data_as(dp),
                                             out.ctypes.data_as(dp))
    return st, out.view(np.complex128)


def spinsim_submit(h, req: spinsim_request, res: spinsim_result):
    t = ctypes.c_int64()
    st = load().spinsim_submit(h, ctypes.byref(req), ctypes.byref(res), ctypes.byref(t))
    return st, t.value


def spinsim_poll(h, ticket: int, wait_us: int = 0) -> int:
    return load().spinsim_poll(h, ticket, wait_us)


def spinsim_poll_any(h, buf, wait_us: int = 0):
    """buf: a ctypes c_int64 array receiving completed tickets.
    Returns (status, number written)."""
    n = ctypes.c_int64()
    st = load().spinsim_poll_any(h, buf, len(buf), wait_us, ctypes.byref(n))
    return st, n.value


def spinsim_memory(h) -> dict:
    info = spinsim_memory_info()
    st = load().spinsim_memory(h, ctypes.byref(info))
    if st != OK:
        raise SpinsimError(st, "spinsim_memory")
    return {f: getattr(info, f) for f, _ in spinsim_memory_info._fields_}


def spinsim_debug_bounds(device: int = 0):
    """Returns (status, word): the debug build's error word of `device`
    (0 = every checked index in range), read and cleared."""
    w = ctypes.c_uint64()
    st = load().spinsim_debug_bounds(device, ctypes.byref(w))
    return st, w.value


def spinsim_last_launch(h) -> spinsim_launch_info:
    info = spinsim_launch_info()
    load().spinsim_last_launch(h, ctypes.byref(info))
    return info


def spinsim_status_string(status: int) -> str:
    return load().spinsim_status_string(status).decode()


status_string = spinsim_status_string


# ------------------------------------------------------------- marshalling
def make_request(req: dict) -> spinsim_request:
    """spinsim_request from a workload dict (see ``workloads``)."""
    r = spinsim_request()
    r.spin_x2 = int(req["spin_x2"])
    f = req["field"]
    for k in ("bias_hz", "drive_x_hz", "drive_y_hz", "drive_hz", "drive_phase", "quad_hz"):
        setattr(r.field, k, float(f.get(k, 0.0)))
    pulses = list(f.get("pulses", ()))
    r.field.n_pulses = len(pulses)
    r.field.pulse_sine_mask = 0
    for i, p in enumerate(pulses):
        a, c, w = p[:3]
        kind = p[3] if len(p) > 3 else "gauss"
        if kind not in ("gauss", "sine"):
            raise SpinsimError(E_ARG, f"unknown pulse kind {kind!r}")
        r.field.pulse_amp_hz[i], r.field.pulse_centre_s[i], r.field.pulse_width_s[i] = a, c, w
        if kind == "sine":
            r.field.pulse_sine_mask |= 1 << i
    tones = list(f.get("tones", ()))
    if len(tones) > MAX_TONES:
        raise SpinsimError(E_ARG, f"at most {MAX_TONES} further tones")
    r.field.n_tones = len(tones)
    for j, (x, y, hz, ph) in enumerate(tones):
        r.field.tone_x_hz[j], r.field.tone_y_hz[j], r.field.tone_hz[j], r.field.tone_phase[j] = x, y, hz, ph
    qdrives = list(f.get("qdrives", ()))
    if len(qdrives) > 2:
        raise SpinsimError(E_ARG, "two quadrupole drives at most")
    r.field.qd_on = 1 if qdrives else 0
    for p, (x, y, hz, ph) in enumerate(qdrives):
        r.field.qd_x_hz[p], r.field.qd_y_hz[p], r.field.qd_hz[p], r.field.qd_phase[p] = x, y, hz, ph
    r.t_start, r.t_end, r.dt, r.dt_out = req["t_start"], req["t_end"], req["dt"], req["dt_out"]
    psi = np.asarray(req["psi0"], dtype=np.complex128)
    for i, z in enumerate(psi):
        r.psi0[2 * i], r.psi0[2 * i + 1] = z.real, z.imag
    return r


def make_config(precision=PREC_FP32_BULK, method=METHOD_CF4, rotating_frame=True, tau=-1, lanes=0, block=0,
                use_graphs=False, device=0, mem_budget=0, profile=False, blocks_per_sm=0,
                chain_fp32=False, direct_host_outputs=True) -> spinsim_config:
    c = spinsim_config()
    spinsim_config_default(c)
    c.precision, c.method, c.rotating_frame, c.trotter_squares = precision, method, int(bool(rotating_frame)), tau
    c.lanes_per_sample, c.threads_per_block, c.use_graphs, c.device = lanes, block, int(bool(use_graphs)), device
    c.mem_budget = mem_budget
    c.profile = int(bool(profile))
    c.blocks_per_sm = blocks_per_sm
    c.chain_precision = 1 if chain_fp32 else 0
    c.direct_host_outputs = 1 if direct_host_outputs else 0
    return c


class Simulator:
    """One handle of the library plus torch-allocated outputs.

    ``simulate(requests)`` runs a batch and returns, per request, a dict with
    ``states`` (complex128 [K, N] torch tensor), ``spin`` (float64 [K, 3]),
    optionally ``ops`` (complex128 [K, N, N]), ``status`` and ``flags``.
    """

    def __init__(self, **cfg):
        import torch  # noqa: F401  (device memory and streams only)
        self.config = make_config(**cfg)
        self.handle = spinsim_create(self.config)

    def close(self):
        if self.handle:
            spinsim_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def counts(self, req: dict):
        st, K, L = spinsim_counts(make_request(req))
        if st != OK:
            raise SpinsimError(st, "spinsim_counts")
        return K, L

    def allocate(self, reqs, want_spin=True, want_ops=False, device="cuda", pin_memory=False, one_buffer=False):
        """Output buffers per request.  With one_buffer, every buffer is a view
        of one allocation (each piece 256-byte aligned), e.g. one pinned host
        block for a large batch instead of thousands of small ones."""
        import torch
        shapes = []
        for q in reqs:
            st, K, _ = spinsim_counts(make_request(q))
            K = max(K, 0)
            n = 2 if q["spin_x2"] == 1 else 3
            shapes.append((K, n))
        kw = dict(dtype=torch.float64, device=device)
        if device == "cpu":
            kw["pin_memory"] = pin_memory
        if one_buffer:
            def pad(x):
                return -(-x // 32) * 32
            sizes = [pad(max(K, 1) * n * 2) + (pad(max(K, 1) * 3) if want_spin else 0) +
                     (pad(max(K, 1) * n * n * 2) if want_ops else 0) for K, n in shapes]
            flat = torch.empty(sum(sizes), **kw)
            at = [0]

            def take(shape):
                numel = 1
                for d in shape:
                    numel *= d
                v = flat[at[0]:at[0] + numel].view(shape)
                at[0] += pad(numel)
                return v
        else:
            def take(shape):
                return torch.empty(shape, **kw)
        outs = []
        for K, n in shapes:
            o = {"states": take((max(K, 1), n, 2))}
            o["spin"] = take((max(K, 1), 3)) if want_spin else None
            o["ops"] = take((max(K, 1), n, n, 2)) if want_ops else None
            o["K"] = K
            outs.append(o)
        return outs

    @staticmethod
    def results_struct(outs):
        res = (spinsim_result * len(outs))()
        for r, o in zip(res, outs):
            r.states = o["states"].data_ptr()
            r.spin = o["spin"].data_ptr() if o["spin"] is not None else None
            r.ops = o["ops"].data_ptr() if o["ops"] is not None else None
            r.capacity = o["K"]
        return res

    def simulate(self, reqs, want_spin=True, want_ops=False, stream=None, outs=None, sync=True, check=True):
        import torch
        if outs is None:
            outs = self.allocate(reqs, want_spin, want_ops)
        req_arr = (spinsim_request * len(reqs))(*[make_request(q) for q in reqs])
        res = self.results_struct(outs)
        if stream is None:
            stream = torch.cuda.current_stream()
        st = spinsim_simulate(self.handle, req_arr, res, stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
        if check and st != OK:
            raise SpinsimError(st, "spinsim_simulate")
        if sync:
            torch.cuda.synchronize()
        return [self._view(o, r) for o, r in zip(outs, res)]

    @staticmethod
    def _view(o, r):
        import torch
        K = o["K"]
        out = {"status": r.status, "flags": r.flags, "trotter_squares": r.trotter_squares, "K": K,
               "states": torch.view_as_complex(o["states"][:K]) if K else o["states"][:0, :, 0].to(torch.complex128)}
        out["spin"] = o["spin"][:K] if o["spin"] is not None else None
        out["ops"] = torch.view_as_complex(o["ops"][:K]) if o["ops"] is not None and K else None
        return out

    def last_launch(self):
        i = spinsim_last_launch(self.handle)
        return {f: getattr(i, f) for f, _ in spinsim_launch_info._fields_}
