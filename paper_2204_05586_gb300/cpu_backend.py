"""ctypes binding of the multicore CPU backend (``include/spinsim_cpu.h``).

The same method on the host's cores (the paper's multicore CPU target): a
separate library, ``libspinsim_cpu.so``, with one entry point that the caller
selects explicitly.  The GPU binding (``spinsim``) never loads or calls it.
Argument marshalling only: every step runs in the library.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build
from .spinsim import (METHOD_CF4, PREC_FP32_BULK, SpinsimError, make_request, spinsim_config, spinsim_request,
                      spinsim_result)

_lib = None
_lock = threading.Lock()


def load(build_if_missing: bool = True):
    """Load libspinsim_cpu.so (building both libraries if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.CPU_LIB):
            if not build_if_missing:
                raise SpinsimError(-5, f"{_build.CPU_LIB} is not built")
            _build.build()
        lib = ctypes.CDLL(_build.CPU_LIB)
        lib.spinsim_cpu_simulate.restype = ctypes.c_int
        lib.spinsim_cpu_simulate.argtypes = [ctypes.POINTER(spinsim_config), ctypes.POINTER(spinsim_request),
                                             ctypes.POINTER(spinsim_result), ctypes.c_int64, ctypes.c_int32]
        _lib = lib
        return lib


def spinsim_cpu_simulate(cfg, reqs, results, threads: int = 0) -> int:
    """The C entry point: cfg a spinsim_config or None, reqs / results ctypes
    arrays (or sequences) of spinsim_request / spinsim_result with host buffers."""
    lib = load()
    n = len(reqs)
    req_arr = reqs if isinstance(reqs, ctypes.Array) else (spinsim_request * n)(*reqs)
    res_arr = results if isinstance(results, ctypes.Array) else (spinsim_result * n)(*results)
    st = lib.spinsim_cpu_simulate(ctypes.byref(cfg) if cfg is not None else None, req_arr, res_arr, n, threads)
    if not isinstance(results, ctypes.Array):
        for i in range(n):
            results[i] = res_arr[i]
    return st


def make_cpu_config(precision=PREC_FP32_BULK, method=METHOD_CF4, rotating_frame=True, tau=-1) -> spinsim_config:
    c = spinsim_config()
    c.precision, c.method, c.rotating_frame, c.trotter_squares = precision, method, int(bool(rotating_frame)), tau
    return c


def _samples(req: dict) -> int:
    k = np.floor((req["t_end"] - req["t_start"]) / req["dt_out"] + 0.5)
    return int(max(k, 0)) if np.isfinite(k) else 0


def simulate(requests, precision=PREC_FP32_BULK, method=METHOD_CF4, rotating_frame=True, tau=-1, threads=0,
             want_spin=True, want_ops=False):
    """Run workload dicts (see ``workloads``) on the host's cores.  Returns per
    request a dict with ``states`` (complex128 [K, N] numpy), ``spin``
    (float64 [K, 3] or None), ``ops`` (complex128 [K, N, N] or None),
    ``status``, ``flags`` and ``trotter_squares``; raises on a call error."""
    n = len(requests)
    outs, res = [], (spinsim_result * n)()
    for i, q in enumerate(requests):
        K, N = _samples(q), int(q["spin_x2"]) + 1
        o = {"K": K, "states": np.zeros((K, N), np.complex128),
             "spin": np.zeros((K, 3)) if want_spin else None,
             "ops": np.zeros((K, N, N), np.complex128) if want_ops else None}
        res[i].states = o["states"].ctypes.data
        res[i].spin = o["spin"].ctypes.data if want_spin else None
        res[i].ops = o["ops"].ctypes.data if want_ops else None
        res[i].capacity = K
        outs.append(o)
    reqs = (spinsim_request * n)(*[make_request(q) for q in requests])
    st = spinsim_cpu_simulate(make_cpu_config(precision, method, rotating_frame, tau), reqs, res, threads)
    if st < 0 and all(res[i].status == 0 for i in range(n)):
        raise SpinsimError(st, "spinsim_cpu_simulate")
    for i, o in enumerate(outs):
        o.update(status=res[i].status, flags=res[i].flags, trotter_squares=res[i].trotter_squares)
    return outs
