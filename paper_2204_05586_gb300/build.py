"""Build the shared libraries in-tree.

``_build/libspinsim.so``: nvcc compiles every ``csrc/*.cu`` for sm_103a in
parallel and links them into one shared object with the static CUDA runtime
(the C ABI of ``include/spinsim.h``).

``_build/libspinsim_cpu.so``: the multicore CPU backend
(``include/spinsim_cpu.h``): ``csrc/cpu/*.cu`` and the shared host logic of
``csrc/params.cu``, compiled as C++ by the host compiler (the device-math
headers compile as plain C++), no CUDA runtime.

No cmake, no torch extension machinery; both are loaded with ctypes.
"""
from __future__ import annotations

import fcntl
import glob
import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libspinsim.so")
CPU_LIB = os.path.join(BUILD, "libspinsim_cpu.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr"]


# -ffp-contract=off: no multiply-add is fused unless the source says fma(), so
# the host backend gives the same results on every host architecture
CXX_FLAGS = ["-x", "c++", "-O3", "-std=c++17", "-ffp-contract=off", "-fPIC", "-pthread"]


def cxx() -> str:
    for cand in (os.environ.get("CXX"), shutil.which("g++"), shutil.which("c++")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("no C++ compiler found for libspinsim_cpu")


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libspinsim")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _cpu_sources():
    return sorted(glob.glob(os.path.join(CSRC, "cpu", "*.cu")))


def _fingerprint() -> str:
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(CSRC, "*.*")) + glob.glob(os.path.join(CSRC, "cpu", "*.*")) +
                    [os.path.join(INCLUDE, "spinsim.h"), os.path.join(INCLUDE, "spinsim_cpu.h")]):
        with open(p, "rb") as f:
            h.update(os.path.basename(p).encode())
            h.update(f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + CXX_FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if sources changed) and return the path of libspinsim.so.
    Concurrent callers (e.g. parallel test workers) are serialised by a file lock."""
    os.makedirs(BUILD, exist_ok=True)
    with open(os.path.join(BUILD, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            return _build_locked(force, verbose)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build_locked(force: bool, verbose: bool) -> str:
    stamp = os.path.join(BUILD, "libspinsim.sha256")
    fp = _fingerprint()
    if (not force and os.path.exists(LIB) and os.path.exists(CPU_LIB) and os.path.exists(stamp)
            and open(stamp).read() == fp):
        return LIB
    exe = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [exe, *ARCH, *NVCC_FLAGS, "-I", INCLUDE, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    cuda_include = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(exe))), "include")

    def compile_host(src):
        obj = os.path.join(BUILD, "host_" + os.path.basename(src)[:-3] + ".o")
        cmd = [cxx(), *CXX_FLAGS, "-I", INCLUDE, "-I", cuda_include, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"host compile failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    srcs = _sources()
    host_srcs = _cpu_sources() + [os.path.join(CSRC, "params.cu")]
    with ThreadPoolExecutor(max(1, min(len(srcs) + len(host_srcs), os.cpu_count() or 1))) as ex:
        gpu_jobs = [ex.submit(compile_one, s) for s in srcs]
        host_jobs = [ex.submit(compile_host, s) for s in host_srcs]
        gpu_objs = [j.result() for j in gpu_jobs]
        host_objs, host_error = None, None
        try:
            host_objs = [j.result() for j in host_jobs]
        except (RuntimeError, OSError) as e:   # the GPU library does not depend on it
            host_error = e

    def link(out, cmd):
        tmp = out + f".tmp{os.getpid()}"
        r = subprocess.run(cmd + ["-o", tmp], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of {os.path.basename(out)} failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, out)

    link(LIB, [exe, *ARCH, "-shared", "-cudart", "static", *gpu_objs])
    if host_error is not None:
        # the CPU backend library is left unbuilt (its binding raises when it is
        # loaded); no stamp, so the next build tries again
        print(f"libspinsim_cpu not built: {host_error}", file=sys.stderr)
        return LIB
    link(CPU_LIB, [cxx(), "-shared", "-pthread", *host_objs])
    with open(stamp, "w") as f:
        f.write(fp)
    return LIB


BOUNDS_LIB = os.path.join(BUILD, "libspinsim_bounds.so")


def build_bounds(force: bool = False) -> str:
    """The debug library with range checks of the kernels' indices
    (-DSPINSIM_BOUNDS; bounds.cuh), _build/libspinsim_bounds.so.  Built on
    demand only (the tests that use it call this), not by build()."""
    os.makedirs(os.path.join(BUILD, "bounds"), exist_ok=True)
    with open(os.path.join(BUILD, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            stamp = os.path.join(BUILD, "libspinsim_bounds.sha256")
            fp = _fingerprint()
            if not force and os.path.exists(BOUNDS_LIB) and os.path.exists(stamp) and open(stamp).read() == fp:
                return BOUNDS_LIB
            exe = nvcc()

            def compile_one(src):
                obj = os.path.join(BUILD, "bounds", os.path.basename(src)[:-3] + ".o")
                cmd = [exe, *ARCH, *NVCC_FLAGS, "-DSPINSIM_BOUNDS", "-I", INCLUDE, "-c", src, "-o", obj]
                r = subprocess.run(cmd, capture_output=True, text=True)
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
                return obj

            srcs = _sources()
            with ThreadPoolExecutor(max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
                objs = list(ex.map(compile_one, srcs))
            tmp = BOUNDS_LIB + f".tmp{os.getpid()}"
            r = subprocess.run([exe, *ARCH, "-shared", "-cudart", "static", *objs, "-o", tmp], capture_output=True,
                               text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link of libspinsim_bounds.so failed:\n{r.stdout}\n{r.stderr}")
            os.replace(tmp, BOUNDS_LIB)
            with open(stamp, "w") as f:
                f.write(fp)
            return BOUNDS_LIB
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
