"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point that include/spinsim.h declares, the struct layouts of the ctypes
binding match the header, and the host-only validation behaves as documented.
No call here launches GPU work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2204_05586_gb300 import spinsim as S, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spinsim.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(spinsim_[a-z_]+)\s*\(", src, re.M)))


def test_header_declarations_are_exported():
    lib = S.load()
    decl = declared_functions()
    assert "spinsim_simulate" in decl and "spinsim_create" in decl and "spinsim_destroy" in decl
    for name in decl:
        assert hasattr(lib, name), f"{name} declared in spinsim.h but not exported"
    assert sorted(S.EXPORTED) == sorted(decl)


def test_struct_sizes_match_header():
    """Compile a probe against the header and compare sizeof/offsetof."""
    import subprocess
    import tempfile
    probe = r'''
#include <stdio.h>
#include <stddef.h>
#include "spinsim.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(spinsim_config), sizeof(spinsim_field), sizeof(spinsim_request),
         sizeof(spinsim_result), sizeof(spinsim_launch_info), sizeof(spinsim_memory_info));
  printf("%zu %zu %zu %zu\n", offsetof(spinsim_request, field), offsetof(spinsim_request, t_start),
         offsetof(spinsim_request, psi0), offsetof(spinsim_result, status));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        open(c, "w").write(probe)
        exe = os.path.join(d, "probe")
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    sizes = list(map(int, out))
    assert sizes[:6] == [ctypes.sizeof(S.spinsim_config), ctypes.sizeof(S.spinsim_field),
                         ctypes.sizeof(S.spinsim_request), ctypes.sizeof(S.spinsim_result),
                         ctypes.sizeof(S.spinsim_launch_info), ctypes.sizeof(S.spinsim_memory_info)]
    assert sizes[6:] == [S.spinsim_request.field.offset, S.spinsim_request.t_start.offset,
                         S.spinsim_request.psi0.offset, S.spinsim_result.status.offset]


def test_config_default():
    c = S.spinsim_config()
    assert S.spinsim_config_default(c) == S.OK
    assert (c.method, c.precision, c.rotating_frame, c.trotter_squares) == (S.METHOD_CF4, S.PREC_FP32_BULK, 1, -1)


def test_counts_and_validation(oracle_mod):
    r = S.make_request(W.spin_half_rabi())
    assert S.spinsim_counts(r) == (S.OK, 500, 100)
    r = S.make_request(W.spin_one_sensing())
    assert S.spinsim_counts(r) == (S.OK, 100000, 100)
    # same (K, L) as the oracle's reading of the sample convention
    for t_end, dt, dt_out in [(5e-3, 1e-7, 1e-5), (1e-3, 2.5e-8, 1e-4), (0.0, 1e-8, 1e-6), (3e-6, 1e-6, 1e-6)]:
        q = W.request(1, W.field(bias_hz=1.0), 0.0, t_end, dt, dt_out)
        assert S.spinsim_counts(S.make_request(q))[1:] == oracle_mod.counts(0.0, t_end, dt, dt_out)
    bad = S.make_request(W.request(1, W.field(), 0.0, 5e-3, 3e-7, 1e-5))
    assert S.spinsim_counts(bad)[0] == S.E_STEP_RATIO
    bad = S.make_request(W.request(1, W.field(), 0.0, 5e-3, 1e-7, 1e-5, psi0=[1.0, 0.1]))
    assert S.spinsim_counts(bad)[0] == S.E_NORM
    bad = S.make_request(W.request(3, W.field(), 0.0, 5e-3, 1e-7, 1e-5, psi0=[1.0, 0.0]))
    assert S.spinsim_counts(bad)[0] == S.E_ARG
    bad = S.make_request(W.request(1, W.field(pulses=[(1.0, 0.0, 0.0)]), 0.0, 5e-3, 1e-7, 1e-5))
    assert S.spinsim_counts(bad)[0] == S.E_ARG
    bad = S.make_request(W.request(1, W.field(), 0.0, 5e-3, -1e-7, 1e-5))
    assert S.spinsim_counts(bad)[0] == S.E_ARG


def test_status_strings():
    for st in (S.OK, S.PENDING, S.E_ARG, S.E_STEP_RATIO, S.E_NORM, S.E_NOMEM, S.E_CUDA, S.E_TIMEOUT,
               S.E_CAPACITY, S.E_UNSUPPORTED):
        assert S.spinsim_status_string(st) != "unknown status"
    assert S.spinsim_status_string(12345) == "unknown status"


def test_create_rejects_bad_config():
    c = S.make_config()
    c.lanes_per_sample = 3
    h = ctypes.c_void_p()
    assert S.load().spinsim_create(ctypes.byref(c), ctypes.byref(h)) == S.E_ARG
    c = S.make_config(tau=41)
    assert S.load().spinsim_create(ctypes.byref(c), ctypes.byref(h)) == S.E_ARG


def test_workload_generators_are_seeded():
    a = W.sweep(8)
    b = W.sweep(8)
    assert [x["field"] for x in a] == [x["field"] for x in b]
    T = np.array([x["t_end"] for x in W.sweep(4096)])
    assert T.min() >= 1e-3 - 1e-12 and T.max() <= 0.1 + 1e-12
    arr, reqs = W.serving_stream(2000)
    assert np.all(np.diff(arr) >= 0) and abs(len(reqs) / arr[-1] - 2000) < 200
    spins = np.array([r["spin_x2"] for r in reqs])
    assert abs((spins == 2).mean() - 0.7) < 0.05


def test_warning_bits_match_header():
    src = open(HEADER).read()
    bits = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define SPINSIM_WARN_([A-Z0-9_]+)\s+(\d+)", src)}
    assert bits == {"MAGNUS": S.WARN_MAGNUS, "FP32_LAB": S.WARN_FP32_LAB}
    assert all(v & (v - 1) == 0 for v in bits.values()) and len(set(bits.values())) == len(bits)


def test_debug_bounds_entry_point():
    """The normal library carries no range checks: spinsim_debug_bounds says
    so without touching the GPU.  The debug library (-DSPINSIM_BOUNDS) builds
    and exports the same entry points."""
    assert S.spinsim_debug_bounds(0) == (S.E_UNSUPPORTED, 0)
    from paper_2204_05586_gb300 import build as B
    lib = ctypes.CDLL(B.build_bounds())
    for name in declared_functions():
        assert hasattr(lib, name), name
