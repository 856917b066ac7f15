#!/usr/bin/env python3
"""Throughput benchmark of the CF4 spin integrator on GB300.

Default workload (one "step" = one pass of the whole hot path over one batch):
the batched spin-one sweep -- 4096 simulations of the seeded parameter sweep
(bias 600-800 kHz, Rabi 0.5-2 kHz, detuning, quadratic shift, a Gaussian z
pulse; durations log-uniform over 1-100 ms; delta_t = 10 ns, Delta_t = 1 us;
about 9e9 CF4 steps) -- run in FP32-bulk precision with the FP64 chain as one
CUDA graph replay, inputs resident on the device.  The same line carries the
served stream (p50/p99 latency at three offered loads) and the single 100 ms
sensing simulation as extra keys, and, on rank 0, the FP64 oracle's errors
and CPU time on a stratified subset.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload sweep|sensing|serve|neural|multitone|su3] [--precision fp32|fp64]

Prints one JSON line (rank 0).  Under torchrun (N > 1) the sweep grows to
4096 N simulations split over the ranks by estimated steps (weak scaling, no
data-path collective); the timing is the maximum over ranks.  `--impl
reference` times the FP64 CPU oracle on the host cores instead, on bounded
windows of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spin-one CF4 steps/s at ≤1e-5 state err vs FP64 oracle; p50/p99 served latency"
UNIT = "steps/s"
# Peak of the dominant kernel's bound: FP32 FMA throughput derived from the
# unit counts and the maximum SM clock (152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz).
N_SM, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = N_SM * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
# FP64 peak from the unit counts: 152 SMs x 2 FP64 FMA lanes per cycle (the dfma
# peak_sustained ncu reports) x 2 flop x 2070 MHz; an FMA-chain probe of dependent
# chains reached 0.98 TFLOP/s of it, the su(3) integrate kernel keeps the pipe 91 % busy
FP64_DERIVED_TFLOPS = N_SM * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP64_PEAK_SOURCE = "derived: 152 SMs x 2 FP64 FMA lanes x 2 flop x 2070 MHz"


def chain_flops_per_sample(spin_x2: int, run: int) -> float:
    """Algorithmic FP64 flops of the chain per sample (FMA = 2): the lane runs'
    products ((run - 1) / run 3x3 complex products of 216 flops, spin-one; SU(2)
    products of 32 for spin-half), one matrix-vector product (72 / 16), the
    renormalisation and <J> (~60 / ~30); the trees add under 2 %."""
    if spin_x2 == 2:
        return (run - 1) / run * 216.0 + 72.0 + 60.0
    return (run - 1) / run * 32.0 + 16.0 + 30.0
L2_FLUSH_BYTES = 256 << 20
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one integrate launch
# (profiles/integrate_kernel_spin_one_sensing.md, integrate_kernel_neural.md,
# integrate_tones_kernel_multitone.md, integrate_su3_kernel_su3.md: the operators stay
# in L2; profiles/launches_sweep512.md: the 512-simulation sweep's tau = 0 launch scaled
# by samples to the 4096-simulation sweep's, whose 12.8 GB of operators go to HBM)
INTEGRATE_TRAFFIC_BYTES = {("sensing", "fp32"): 87808, ("neural", "fp32"): 98304, ("multitone", "fp32"): 183552,
                           ("su3", "fp64"): 1012736, ("sweep", "fp32"): 12330000000}


def algorithmic_flops_per_step(spin_x2: int, tau: int, n_tones: int = 0) -> float:
    """Algorithmic FP32 flops of one spin-one CF4 step (FMA = 2 flops): two
    Lie-Trotter exponentials with tau residual squarings of a 3x3 complex
    matrix (27 complex MACs = 216 flops each) plus ~100 flops to build T, two
    3x3 complex products (216 each) and the field at two nodes: 432 tau + 650.
    Each further drive tone adds its two phasors at both nodes (a 3-term
    sine/cosine series and four complex multiply-adds, ~40 flops per node) and
    its share of both exponents (8): 88 per tone.  The timed workloads are
    spin-one only."""
    if spin_x2 != 2:
        raise ValueError("the flop model covers spin-one steps only")
    return 432.0 * tau + 650.0 + 88.0 * n_tones


def su3_flops_per_step(degree: int, squarings: int = 0) -> float:
    """Algorithmic FP64 flops of one CF4 step with quadrupole drives (full
    su(3), spin-one; FMA = 2, add or multiply = 1).  Per exponential: the
    Hermitian exponent and its norm (40), B^2 with its six distinct entries
    (108), floor((degree - 1) / 2) products of the Hermitian B^2 with a general
    matrix (162 each) and the blocks I/(2j)! + B/(2j+1)! added in (54), and
    the rest beyond the J and Q first order: with no halving formed directly
    (12), else T + B (18), 252 per squaring and the first-order split (36).  Per step: two
    exponentials, two residual products (262 each) and, at both nodes, the
    field (the co-rotating drive and quadrupole-drive phasors by their sine
    and cosine series, the counter-rotating ones turned by one step, the
    Gaussian pulse: ~190) and the weighted exponents (46)."""
    per_exp = 40.0 + 108.0 + 162.0 * ((degree - 1) // 2) + 54.0 + (12.0 if squarings == 0 else
                                                                    18.0 + 252.0 * squarings + 36.0)
    return 2 * per_exp + 2 * 262.0 + 2 * (190.0 + 46.0)


# Taylor degree of the su(3) exponential on the su3 workload: every CF4
# exponent's max-row norm stays below 1.5e-4 there (under the 2.0e-4 switch to 5).
SU3_DEGREE = 4


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return None
        mhz = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": mhz[len(mhz) // 2] if mhz else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier_max(value: float, world: int, device: str = "cuda"):
    """Maximum of `value` over all ranks (the slowest rank's time)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier_sum(value: float, world: int, device: str = "cuda"):
    """Sum of `value` over all ranks."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_per_rank_step: int, steps: int, world: int, max_seconds: float) -> float:
    """Whole-job throughput: the units every rank processed (each rank runs
    its own copy of the workload) divided by the slowest rank's time."""
    return units_per_rank_step * steps * world / max_seconds


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------- workloads
SWEEP_PER_RANK = 4096
SUBSET = 16          # simulations of the sweep compared with the oracle (stratified by duration)
SERVE_SAMPLE = 32    # served requests compared with the oracle
SERVE_RATES = (2000.0, 20000.0, 100000.0)


def make_workload(name, world, rank, sweep_per_rank=0):
    """(requests of this rank, description, parallelism) of a named workload."""
    from paper_2204_05586_gb300 import sharded, workloads as W
    if name == "sweep":
        n = (sweep_per_rank or SWEEP_PER_RANK) * world
        reqs = W.sweep(n, seed=W.SEED)
        mine = sharded.partition(reqs, world)[rank] if world > 1 else list(range(n))
        desc = (f"batched spin-one sweep: {n} simulations in one persistent launch per GPU, bias U(600,800) kHz, "
                "Rabi U(0.5,2) kHz, detuning U(-500,500) Hz, q U(0,600) Hz, Gaussian pulse U(0,100) Hz / 1 ms at "
                "U(0,T), T log-uniform [1,100] ms; dt 10 ns, dt_out 1 us; FP32 bulk, FP64 chain")
        par = (f"{n} simulations split over {world} ranks by estimated steps (longest first), "
               "no data-path collective" if world > 1 else "one GPU")
        return [reqs[i] for i in mine], desc, par
    par = f"weak x{world}, independent copies per GPU"
    if name == "sensing":
        return [W.spin_one_sensing()], ("spin-one sensing: bias 700 kHz, drive 2x1 kHz at 700 kHz, q 400 Hz, "
                                        "Gaussian z pulse 50 Hz / 1 ms at 50 ms; 100 ms, dt 10 ns, dt_out 1 us "
                                        "(1e5 samples x 100 CF4 steps)"), par
    if name == "neural":
        return [W.neural_pulse()], ("spin-one, the paper's benchmark field (Eq. neural_pulse): bias 700 kHz, drive "
                                    "2x1 kHz at 700 kHz, 70 Hz single sine cycle of 1 ms on J_z at 50 ms; 100 ms, "
                                    "dt 100 ns, dt_out 1 us (1e5 samples x 10 CF4 steps)"), par
    if name == "multitone":
        return [W.multitone_sensing()], ("spin-one sensing field plus three further drive tones (1 kHz circular at "
                                         "+500 Hz, 0.5 kHz linear at -2 kHz, 0.8 kHz y at +5 kHz); 100 ms, dt 10 ns, "
                                         "dt_out 1 us (1e5 samples x 100 CF4 steps)"), par
    if name == "su3":
        return [W.su3_sensing()], ("spin-one sensing field plus two quadrupole drives (full su(3)): 1 kHz circular "
                                   "on (D_xz, D_yz) at 700.3 kHz, 0.5 kHz circular on (D_x2y2, D_xy) at 1400.2 kHz; "
                                   "100 ms, dt 10 ns, dt_out 1 us (1e5 samples x 100 CF4 steps), FP64"), par
    raise ValueError(name)


def samples_of(r):
    return int(round((r["t_end"] - r["t_start"]) / r["dt_out"]))


def chain_run(K):
    """The library's lane-run length of the chain (a function of K alone)."""
    return min(8, max(6 if K >= 16384 else 4, -(-K // (32 * 608))))


def stratified(reqs, n):
    """n requests spread over the range of durations: the ones at the
    quantiles (i + 1/2) / n of the sorted durations, i = 0 .. n - 1."""
    import numpy as np
    T = np.array([r["t_end"] - r["t_start"] for r in reqs])
    order = np.argsort(T, kind="stable")
    n = min(n, len(reqs))
    return [int(order[int((i + 0.5) * len(reqs) / n)]) for i in range(n)]


def host_chain_norm_drift(ops, psi0):
    """max_k | ||U_k ... U_1 psi0|| - 1 | of operators chained in FP64 on the
    host without renormalisation: the drift the written states would carry
    if the chain did not renormalise them (FP32-bulk operators are stored as
    computed)."""
    import numpy as np
    psi = np.asarray(psi0, dtype=np.complex128)
    worst = 0.0
    for U in ops:
        psi = U @ psi
        worst = max(worst, abs(float(np.vdot(psi, psi).real) ** 0.5 - 1.0))
    return worst


def unitarity_defect(ops):
    """max_k ||U_k^H U_k - I||_max of a stack of operators."""
    import numpy as np
    n = ops.shape[-1]
    g = np.einsum("kji,kjl->kil", ops.conj(), ops) - np.eye(n)
    return float(np.abs(g).max()) if len(ops) else 0.0


# ----------------------------------------------------------------- our arm
def measure_batch(args, reqs, prec, dev, local, world, tag):
    """Time one batch: `args.steps` CUDA graph replays with the L2 flushed
    between them, the kernels' live times, the rooflines, and the end-to-end
    rate through spinsim_simulate with pinned host buffers."""
    import numpy as np
    import torch

    from paper_2204_05586_gb300 import spinsim as S, workloads as W

    steps_per_pass = W.total_steps(reqs)
    # replayed as one CUDA graph per step (the first call tunes, runs eagerly and captures)
    sim = S.Simulator(precision=prec, tau=args.tau, profile=True, device=local, use_graphs=True)
    outs = sim.allocate(reqs, device=dev, one_buffer=True)
    stream = torch.cuda.current_stream()
    raw_stream = stream.cuda_stream
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    # the requests marshalled once: every timed step is one spinsim_simulate call
    req_arr = (S.spinsim_request * len(reqs))(*[S.make_request(q) for q in reqs])
    res_dev = sim.results_struct(outs)
    for _ in range(args.warmup):
        if S.spinsim_simulate(sim.handle, req_arr, res_dev, raw_stream) != S.OK:
            raise RuntimeError("spinsim_simulate failed in the warm-up")
    torch.cuda.synchronize()
    # the squarings the automatic choice gave each request (they can differ per request)
    taus = [v["trotter_squares"] for v in sim.simulate(reqs, outs=outs)]

    # ---- timed region: K steps, L2 flushed between steps
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    integ_ms, chain_ms, launches = [], [], 0
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        if S.spinsim_simulate(sim.handle, req_arr, res_dev, raw_stream) != S.OK:
            raise RuntimeError("spinsim_simulate failed in the timed loop")
        ev[i][1].record(stream)
        li = sim.last_launch()          # reads the library's kernel events (waits for them)
        integ_ms.append(li["integrate_ms"])
        chain_ms.append(li["chain_ms"])
        launches += li["kernels_launched"]
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = barrier_max(sum(step_ms) / 1e3, world)
    all_steps = barrier_sum(steps_per_pass, world)
    value = all_steps * args.steps / total_s
    ms_per_step = total_s * 1e3 / args.steps

    # ---- roofline of the dominant kernel (integrate), from its live CUDA events
    su3 = any(r["field"].get("qdrives") for r in reqs)
    if su3:
        flops = sum(W.total_steps([r]) * su3_flops_per_step(SU3_DEGREE) for r in reqs)
    else:
        flops = sum(W.total_steps([r]) * algorithmic_flops_per_step(r["spin_x2"], t, len(r["field"].get("tones", ())))
                    for r, t in zip(reqs, taus))
    mean_int = float(np.mean(integ_ms))
    achieved = flops / (mean_int / 1e3) / 1e12
    # FP32-bulk spin-one requests in the rotating frame take the small-angle
    # variants, which run in the paired kernel (two samples per thread)
    paired = prec == S.PREC_FP32_BULK and all(r["spin_x2"] == 2 for r in reqs)
    kernel = ("integrate_su3_kernel" if su3 else
              "integrate_tones_kernel" if any(r["field"].get("tones") for r in reqs) else
              "integrate_pair_kernel" if paired else "integrate_kernel")
    roofline = {"bound": "alu", "kernel": kernel, "achieved": round(achieved, 3),
                "peak": round(FP32_PEAK_TFLOPS, 2), "unit": "TFLOP/s", "frac": round(achieved / FP32_PEAK_TFLOPS, 4),
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                "traffic": INTEGRATE_TRAFFIC_BYTES.get((tag, args.precision)),
                "integrate_ms": round(mean_int, 4), "chain_ms": round(float(np.mean(chain_ms)), 4),
                "flops_per_step": round(flops / steps_per_pass, 1)}
    if prec == S.PREC_FP64:
        roofline.update({"bound": "fp64", "peak": round(FP64_DERIVED_TFLOPS, 3),
                         "frac": round(achieved / FP64_DERIVED_TFLOPS, 4), "peak_source": FP64_PEAK_SOURCE})
    # the chain's share of the step against the FP64 rate (the chain always runs in FP64)
    cflops = sum(samples_of(r) * chain_flops_per_sample(r["spin_x2"], chain_run(samples_of(r))) for r in reqs)
    mean_chain = float(np.mean(chain_ms))
    chain_tf = cflops / (mean_chain / 1e3) / 1e12
    chain_roofline = {"bound": "fp64", "kernels": "chain_up_kernel, chain_apply_kernel",
                      "achieved": round(chain_tf, 4), "peak": round(FP64_DERIVED_TFLOPS, 3), "unit": "TFLOP/s",
                      "frac": round(chain_tf / FP64_DERIVED_TFLOPS, 4), "peak_source": FP64_PEAK_SOURCE,
                      "flops_per_sample": round(cflops / max(1, sum(samples_of(r) for r in reqs)), 1),
                      "chain_ms": round(mean_chain, 4)}
    # the write-out: psi_k (N complex) and <J>_k (3 doubles) per sample
    out_bytes = sum(samples_of(r) * (16 * (r["spin_x2"] + 1) + 24) for r in reqs)
    chain_roofline["output_bytes"] = out_bytes
    chain_roofline["output_gbs"] = round(out_bytes / (mean_chain / 1e3) / 1e9, 1)

    # ---- end to end through the C ABI with pinned host buffers (e2e_measure)
    sim.close()
    e2e = e2e_measure(args, reqs, prec, dev, local, world, all_steps)
    return {"value": value, "ms_per_step": ms_per_step, "roofline": roofline, "chain_roofline": chain_roofline,
            "e2e": e2e, "gpu_launches": launches, "wall_s_timed_loop": wall, "clocks": clk, "taus": taus,
            "outs": outs, "steps_per_pass": steps_per_pass}


def e2e_measure(args, reqs, prec, dev, local, world, all_steps):
    """The metric end to end through spinsim_simulate with pinned host
    buffers: every step one call that takes new parameters (two parameter
    sets alternate, so each call validates the requests, fills and uploads
    the parameter tables), runs the kernels and delivers states and <J> to
    host memory.  Timed one call at a time (serial) and double-buffered (two
    handles on two streams, a buffer reused only after its previous pass
    completed), for the two ways results reach host memory: staged in device
    memory and copied back, and written directly by the kernels into the
    mapped pinned buffers (direct_host_outputs).  The faster double-buffered
    form is the line's e2e value; all four are reported."""
    import copy

    import torch

    from paper_2204_05586_gb300 import spinsim as S

    alt = copy.deepcopy(reqs)
    for q in alt:                        # the second parameter set: another drive phase
        q["field"]["drive_phase"] = float(q["field"].get("drive_phase", 0.0)) + 0.25
    sets = [(S.spinsim_request * len(reqs))(*[S.make_request(q) for q in reqs]),
            (S.spinsim_request * len(alt))(*[S.make_request(q) for q in alt])]
    e2e_steps = max(3, min(args.steps, 200))
    streams = [torch.cuda.current_stream(), torch.cuda.Stream(device=dev)]
    probe = S.Simulator(precision=prec, tau=args.tau, device=local)
    bufs = [probe.allocate(reqs, device="cpu", pin_memory=True, one_buffer=True) for _ in range(2)]
    probe.close()
    out = {}
    for direct in (False, True):
        sims = [S.Simulator(precision=prec, tau=args.tau, device=local, use_graphs=True, direct_host_outputs=direct)
                for _ in range(2)]
        res = [sm.results_struct(b) for sm, b in zip(sims, bufs)]
        for j in range(2):               # first calls: tuning, scratch, graph capture
            for q in sets:
                if S.spinsim_simulate(sims[j].handle, q, res[j], streams[j].cuda_stream) != S.OK:
                    raise RuntimeError("spinsim_simulate failed before the end-to-end loop")
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            if S.spinsim_simulate(sims[0].handle, sets[i % 2], res[0], streams[0].cuda_stream) != S.OK:
                raise RuntimeError("spinsim_simulate failed in the end-to-end loop")
            streams[0].synchronize()
        serial_s = barrier_max(time.perf_counter() - t0, world)
        li = sims[0].last_launch()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            j = i % 2
            streams[j].synchronize()      # this buffer's previous pass is complete
            if S.spinsim_simulate(sims[j].handle, sets[(i // 2) % 2], res[j], streams[j].cuda_stream) != S.OK:
                raise RuntimeError("spinsim_simulate failed in the end-to-end loop")
        for st in streams:
            st.synchronize()
        piped_s = barrier_max(time.perf_counter() - t0, world)
        out[direct] = {"value": all_steps * e2e_steps / piped_s, "serial_value": all_steps * e2e_steps / serial_s,
                       "h2d": int(li["h2d_bytes"]), "d2h": int(li["d2h_bytes"])}
        for sm in sims:
            sm.close()
    best = True if out[True]["value"] >= out[False]["value"] else False
    b = out[best]
    return {"value": b["value"], "unit": UNIT, "h2d_bytes_per_step": b["h2d"], "d2h_bytes_per_step": b["d2h"],
            "steps": e2e_steps,
            "calling": ("each step one spinsim_simulate call with new parameters (two sets alternate: validation, "
                        "parameter tables filled and uploaded), states and <J> into pinned host buffers; two "
                        "handles on two streams, a buffer reused after its pass completes; results "
                        + ("written directly into the mapped pinned buffers by the kernels (direct_host_outputs = 1)"
                           if best else "staged in device memory and copied back")),
            "serial_value": b["serial_value"], "serial_calling": "one handle, a wait after every call",
            "staged": {"value": out[False]["value"], "serial_value": out[False]["serial_value"]},
            "direct_host_outputs": {"value": out[True]["value"], "serial_value": out[True]["serial_value"]}}


def fp64_plain(reqs, local, dev, ref_states, value_fp32_per_gpu, tau=-1):
    """The plain FP64 path on the same GPU and requests: rate, error against
    the oracle (the compared prefix of each request), norm drift."""
    import numpy as np
    import torch

    from paper_2204_05586_gb300 import spinsim as S, workloads as W
    sim64 = S.Simulator(precision=S.PREC_FP64, tau=tau, device=local)
    o64 = sim64.allocate(reqs, device=dev, one_buffer=True)
    sim64.simulate(reqs, outs=o64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        sim64.simulate(reqs, outs=o64, sync=False)
    e1.record()
    torch.cuda.synchronize()
    rate = W.total_steps(reqs) * 3 / (e0.elapsed_time(e1) / 1e3)
    err = drift = 0.0
    for o, ref in zip(o64, ref_states):
        s64 = torch.view_as_complex(o["states"][:o["K"]]).cpu().numpy()[:len(ref)]
        err = max(err, float(np.abs(s64 - ref).max()))
        drift = max(drift, float(np.abs(np.linalg.norm(s64, axis=1) - 1.0).max()))
    sim64.close()
    out = {"value": rate, "unit": UNIT, "state_err_vs_oracle": err, "norm_drift": drift,
           "speedup_fp32_bulk_over_fp64": value_fp32_per_gpu / rate}
    if tau >= 0:
        out["trotter_squares"] = tau
    return out


def accuracy_single(args, reqs, prec, local, dev, outs, value_per_gpu, tag):
    """One simulation against the FP64 oracle over all host cores (also the
    CPU baseline), the FP64-plain path, and the multicore CPU backend."""
    import numpy as np
    import torch

    from oracle import oracle as O   # the CPU baseline leg: the oracle as it stands
    from paper_2204_05586_gb300 import spinsim as S, workloads as W
    O.build()
    r = dict(reqs[0])
    cores = os.cpu_count() or 1
    sample = ("the full workload once (1e5 sample operators over all host cores, then the sequential "
              "chain), tau = 24, FP64")
    if tag == "su3":   # the oracle's 30-term su(3) series: a bounded prefix of the run
        r["t_end"] = r["t_start"] + 1e4 * r["dt_out"]
        sample = ("the first 1e4 of 1e5 output samples (10 ms, 1e6 CF4 steps) over all host cores, then "
                  "the sequential chain, FP64; states compared over that prefix")
    t0 = time.perf_counter()
    ref = O.simulate(r["spin_x2"], r["field"], r["t_start"], r["t_end"], r["dt"], r["dt_out"], r["psi0"],
                     threads=cores)
    t_cpu = time.perf_counter() - t0
    out = {"cpu_baseline": {"value": W.total_steps([r]) / t_cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample}}
    gpu_states = torch.view_as_complex(outs[0]["states"][:len(ref["states"])]).cpu().numpy()
    out["state_err_vs_oracle"] = float(np.abs(gpu_states - ref["states"]).max())
    # the paper's own error measure (Eq. error, 1/K outside the root as printed) and the
    # states' norm drift, beside the primary max |dpsi|
    out["paper_error_metric_vs_oracle"] = float(O.error_metric(np.ascontiguousarray(gpu_states), ref["states"]))
    out["norm_drift"] = float(np.abs(np.linalg.norm(gpu_states, axis=1) - 1.0).max())
    if prec == S.PREC_FP32_BULK:
        # the drift the FP32-bulk operators would give without the chain's renormalisation
        with S.Simulator(precision=prec, tau=args.tau, device=local) as sop:
            (o,) = sop.simulate(reqs, want_ops=True)
            ops = o["ops"].cpu().numpy()
        out["norm_drift_before_renormalisation"] = host_chain_norm_drift(ops[1:], reqs[0]["psi0"])
        out["operator_unitarity_defect"] = unitarity_defect(ops)
        out["fp64_plain"] = fp64_plain(reqs, local, dev, [ref["states"]], value_per_gpu)
        out["fp64_plain_tau0"] = fp64_plain(reqs, local, dev, [ref["states"]], value_per_gpu, tau=0)
        # the multicore CPU backend (same algorithm and precision, every host core)
        from paper_2204_05586_gb300 import cpu_backend as CB
        CB.simulate([W.spin_one_sensing(t_end=1e-5)], precision=prec)   # loads the library
        t0 = time.perf_counter()
        (cb,) = CB.simulate(reqs, precision=prec, tau=args.tau)
        t_cb = time.perf_counter() - t0
        out["cpu_backend"] = {"value": W.total_steps(reqs) / t_cb, "unit": UNIT, "cores": cores,
                              "precision": args.precision, "kind": "libspinsim_cpu (same algorithm on host cores)",
                              "sample": "the full workload once, all host cores",
                              "state_err_vs_oracle": float(np.abs(cb["states"][:len(ref["states"])] -
                                                                  ref["states"]).max())}
    return out


def accuracy_sweep(args, reqs, prec, local, dev, outs, value_per_gpu):
    """A stratified subset of the sweep (SUBSET simulations across the
    durations) against the FP64 oracle on every sample; the oracle's time on
    it, over all host cores, is the CPU baseline, extrapolated to the whole
    sweep by step count."""
    import numpy as np
    import torch

    from oracle import oracle as O   # the CPU baseline leg: the oracle as it stands
    from paper_2204_05586_gb300 import spinsim as S, workloads as W
    O.build()
    cores = os.cpu_count() or 1
    pick = stratified(reqs, SUBSET)
    sub = [reqs[i] for i in pick]
    refs = []
    t0 = time.perf_counter()
    for r in sub:
        refs.append(O.simulate(r["spin_x2"], r["field"], r["t_start"], r["t_end"], r["dt"], r["dt_out"], r["psi0"],
                               threads=cores)["states"])
    t_cpu = time.perf_counter() - t0
    sub_steps = W.total_steps(sub)
    rate = sub_steps / t_cpu
    out = {"cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{len(sub)} of {len(reqs)} simulations stratified by duration "
                                      f"({sub_steps:.3e} CF4 steps, sample operators over all host cores, then each "
                                      "chain in order), tau = 24, FP64; the whole sweep extrapolated by step count",
                            "extrapolated_sweep_s": W.total_steps(reqs) / rate}}
    err = pm = drift = 0.0
    for i, ref in zip(pick, refs):
        g = torch.view_as_complex(outs[i]["states"][:outs[i]["K"]]).cpu().numpy()
        err = max(err, float(np.abs(g - ref).max()))
        pm = max(pm, float(O.error_metric(np.ascontiguousarray(g), ref)))
        drift = max(drift, float(np.abs(np.linalg.norm(g, axis=1) - 1.0).max()))
    out["state_err_vs_oracle"] = err
    out["state_err_subset"] = {"simulations": len(sub), "durations_ms": [round(1e3 * (r["t_end"] - r["t_start"]), 3)
                                                                          for r in sub],
                               "compared": "every sample and component of each"}
    out["paper_error_metric_vs_oracle"] = pm
    out["norm_drift"] = drift
    if prec == S.PREC_FP32_BULK:
        with S.Simulator(precision=prec, tau=args.tau, device=local) as sop:
            got = sop.simulate(sub, want_ops=True)
            nd = ud = 0.0
            for q, o in zip(sub, got):
                ops = o["ops"].cpu().numpy()
                nd = max(nd, host_chain_norm_drift(ops[1:], q["psi0"]))
                ud = max(ud, unitarity_defect(ops))
        out["norm_drift_before_renormalisation"] = nd
        out["operator_unitarity_defect"] = ud
        out["fp64_plain"] = fp64_plain(sub, local, dev, refs, value_per_gpu)
        out["fp64_plain"]["sample"] = "the same stratified subset as one batch"
        out["fp64_plain_tau0"] = fp64_plain(sub, local, dev, refs, value_per_gpu, tau=0)
        out["fp64_plain_tau0"]["sample"] = "the same stratified subset as one batch"
    return out


def run_ours(args, world, rank, local):
    import torch

    from paper_2204_05586_gb300 import spinsim as S

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if args.workload == "serve":
        sv = serving_summary(args, world, rank, local, rates=(2000.0,))
        line = {"metric": METRIC, "value": sv["served_steps_per_s"], "unit": UNIT, "n_gpus": world,
                "steps": args.serve_requests, "warmup": 8, "ms_per_step": sv["span_s"] * 1e3 / args.serve_requests,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 bulk / f64 chain",
                "data": "synthetic", "config": {"workload": sv["workload"]}, "serving": sv}
        if sv.get("clocks"):
            line["clocks"] = sv["clocks"]      # sampled over the served stream
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    prec = S.PREC_FP32_BULK if args.precision == "fp32" else S.PREC_FP64
    if args.workload == "su3":
        prec, args.precision = S.PREC_FP64, "fp64"      # full su(3) runs in FP64 only
    reqs, workload, parallelism = make_workload(args.workload, world, rank, args.sweep_sims)
    m = measure_batch(args, reqs, prec, dev, local, world, args.workload)
    taus = m["taus"]
    line = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 bulk / f64 chain" if prec == S.PREC_FP32_BULK else "f64",
            "data": "synthetic (seeded field parameters shaped like the paper's sensing benchmark)",
            "config": {"workload": workload, "precision": args.precision, "trotter_squares": max(taus),
                       "steps_by_trotter_squares": {str(t): sum(W_steps(r) for r, u in zip(reqs, taus) if u == t)
                                                    for t in sorted(set(taus))},
                       "rotating_frame": True, "method": "CF4", "simulations_per_gpu": len(reqs),
                       "cf4_steps_per_pass": m["steps_per_pass"],
                       "l2": "flushed between timed steps (256 MiB device write outside the step events)",
                       "launch": "each step one CUDA graph replay (integrate + chain kernels)",
                       "parallelism": parallelism},
            "roofline": m["roofline"], "chain_roofline": m["chain_roofline"], "e2e": m["e2e"],
            "gpu_launches": m["gpu_launches"], "wall_s_timed_loop": m["wall_s_timed_loop"]}
    if args.workload == "su3":      # the general exponential takes no Lie-Trotter squarings
        line["config"].pop("steps_by_trotter_squares")
        line["config"]["trotter_squares"] = None
        line["config"]["taylor_degree"] = SU3_DEGREE
    if m["clocks"]:
        line["clocks"] = m["clocks"]
    per_gpu = m["value"] / world
    # ---- rank 0: accuracy vs the FP64 oracle, oracle CPU baseline, FP64-plain kernel
    if rank == 0 and not args.no_cpu_baseline:
        if args.workload == "sweep":
            line.update(accuracy_sweep(args, reqs, prec, local, dev, m["outs"], per_gpu))
        else:
            line.update(accuracy_single(args, reqs, prec, local, dev, m["outs"], per_gpu, args.workload))
    del m
    if args.workload == "sweep" and not args.no_extras:
        # the served stream (config of the metric's latency half) and the
        # single long sensing simulation, both measured in the same run
        line["serving"] = serving_summary(args, world, rank, local, rates=SERVE_RATES)
        sreqs, sdesc, _ = make_workload("sensing", world, rank)
        ms = measure_batch(args, sreqs, prec, dev, local, world, "sensing")
        sens = {"workload": sdesc, "value": ms["value"], "unit": UNIT, "ms_per_step": ms["ms_per_step"],
                "trotter_squares": max(ms["taus"]), "roofline": ms["roofline"],
                "chain_roofline": ms["chain_roofline"], "e2e": ms["e2e"], "gpu_launches": ms["gpu_launches"]}
        if ms["clocks"]:
            sens["clocks"] = ms["clocks"]
        if rank == 0 and not args.no_cpu_baseline:
            sens.update(accuracy_single(args, sreqs, prec, local, dev, ms["outs"], ms["value"] / world, "sensing"))
        line["sensing"] = sens
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def W_steps(r):
    from paper_2204_05586_gb300 import workloads as W
    return W.total_steps([r])


# ------------------------------------------------------------------ serving
def serve_once(sim, creqs, res, arrivals):
    """Submit requests at their arrival times and collect completions with
    spinsim_poll_any; returns (latency per request in s, span in s)."""
    import ctypes

    import numpy as np

    from paper_2204_05586_gb300 import spinsim as S
    n = len(creqs)
    lat = np.zeros(n)
    index = {}
    buf = (ctypes.c_int64 * 4096)()
    done = nxt = 0
    t0 = time.perf_counter()
    while done < n:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            st, t = S.spinsim_submit(sim.handle, creqs[nxt], res[nxt])
            if st != S.OK:
                raise RuntimeError(f"spinsim_submit: {S.status_string(st)}")
            index[t] = nxt
            nxt += 1
        st, k = S.spinsim_poll_any(sim.handle, buf, 0)
        if k:
            tnow = time.perf_counter() - t0
            for t in buf[:k]:
                i = index.pop(t)
                lat[i] = tnow - arrivals[i]
            done += k
        elif nxt < n and not index:
            time.sleep(max(0.0, min(arrivals[nxt] - (time.perf_counter() - t0), 0.001)))
    return lat, time.perf_counter() - t0


def serving_summary(args, world, rank, local, rates=SERVE_RATES):
    """The served Poisson stream (70% spin-one / 30% spin-half, durations
    log-uniform [0.1, 100] ms, FP32-bulk): latency percentiles and served
    steps/s at each offered rate (the same requests, arrival times scaled),
    and a seeded sample of served requests against the FP64 oracle."""
    import numpy as np
    import torch

    from paper_2204_05586_gb300 import spinsim as S, workloads as W
    n = args.serve_requests
    arrivals, reqs = W.serving_stream(n, seed=W.SEED + 1 + rank)
    total = W.total_steps(reqs)
    sim = S.Simulator(precision=S.PREC_FP32_BULK, device=local)
    outs = sim.allocate(reqs, one_buffer=True)
    res = sim.results_struct(outs)
    creqs = [S.make_request(q) for q in reqs]
    # warm-up (tuning, pool growth) on a few requests outside the measured stream
    lat, _ = serve_once(sim, creqs[:64], res[:64], np.zeros(64))
    torch.cuda.synchronize()
    loads = []
    clocks = ClockSampler(local)
    clocks.start()
    for rate in rates:
        barrier(world)
        lat, span = serve_once(sim, creqs, res, arrivals * (2000.0 / rate))
        span = barrier_max(span, world)
        served = barrier_sum(total, world)
        loads.append({"offered_req_per_s": rate, "offered_steps_per_s": served / float(arrivals[-1] * 2000.0 / rate),
                      "served_steps_per_s": served / span, "span_s": span,
                      "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3),
                                     "p99": float(np.percentile(lat, 99) * 1e3), "mean": float(lat.mean() * 1e3)}})
        if rate == rates[0]:
            statuses = [r.status for r in res]
    clk = clocks.stop()
    mem = S.spinsim_memory(sim.handle)
    out = {"workload": f"served Poisson stream: {n} requests, 70% spin-one / 30% spin-half, fields as the sweep, "
                       "durations log-uniform [0.1,100] ms, dt 10 ns, dt_out 1 us, FP32-bulk, admitted by device-memory "
                       "footprint into one serving pool",
           "requests": n, "latency_ms": loads[0]["latency_ms"], "served_steps_per_s": loads[0]["served_steps_per_s"],
           "offered_steps_per_s": loads[0]["offered_steps_per_s"], "span_s": loads[0]["span_s"],
           "loads": loads, "all_ok": all(s == S.OK for s in statuses),
           "pool_bytes": mem["pool"], "peak_held_bytes": mem["peak_held"]}
    if clk:
        out["clocks"] = clk
    if rank == 0 and not args.no_cpu_baseline:
        # the last load's results (every request ran again) against the FP64 oracle
        from oracle import oracle as O
        O.build()
        rng = np.random.Generator(np.random.PCG64(W.SEED + 7))
        pick = sorted(rng.choice(n, size=min(SERVE_SAMPLE, n), replace=False).tolist())
        err = 0.0
        cores = os.cpu_count() or 1
        for i in pick:
            r = reqs[i]
            ref = O.simulate(r["spin_x2"], r["field"], r["t_start"], r["t_end"], r["dt"], r["dt_out"], r["psi0"],
                             threads=cores)["states"]
            g = torch.view_as_complex(outs[i]["states"][:outs[i]["K"]]).cpu().numpy()
            err = max(err, float(np.abs(g - ref).max()))
        out["state_err_vs_oracle"] = err
        out["state_err_sample"] = (f"{len(pick)} served requests drawn with a seeded generator "
                                   f"({sum(1 for i in pick if reqs[i]['spin_x2'] == 1)} spin-half), every sample")
    sim.close()
    return out


# ---------------------------------------------------------- reference arm
def run_reference(args, world, rank, local):
    """The FP64 CPU oracle, as it stands, on the host cores, on the same
    workload: each step is a bounded window of it (sweep: the first 2000
    output samples of one simulation of the stratified subset, in turn;
    single simulations: the first 1000 output samples)."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2204_05586_gb300 import workloads as W
    O.build()
    cores = os.cpu_count() or 1
    if args.workload == "sweep":
        reqs, desc, _ = make_workload("sweep", 1, 0, args.sweep_sims)
        window = 2000
        sub = [reqs[i] for i in stratified(reqs, SUBSET)]
        windows = []
        for r in sub:
            q = dict(r)
            q["t_end"] = min(r["t_end"], r["t_start"] + window * r["dt_out"])
            windows.append(q)
        config = (f"{desc}; each step: the first {window} output samples of one of {len(sub)} simulations "
                  "stratified by duration, in turn; tau = 24")
        sample = f"first {window} output samples of one sweep simulation per step"
    else:
        window = 1000
        full, desc, _ = make_workload(args.workload, 1, 0)
        q = dict(full[0])
        q["t_end"] = q["t_start"] + window * q["dt_out"]
        windows = [q]
        config = f"{desc}; each step: the first {window} output samples; tau = 24"
        sample = f"first {window} output samples per step"

    def one(i):
        q = windows[i % len(windows)]
        O.simulate(q["spin_x2"], q["field"], q["t_start"], q["t_end"], q["dt"], q["dt_out"], q["psi0"],
                   threads=cores)
        return W.total_steps([q])

    for i in range(args.warmup):
        one(i)
    t0 = time.perf_counter()
    steps = sum(one(i) for i in range(args.steps))
    dt = time.perf_counter() - t0
    value = steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded field parameters shaped like the paper's sensing benchmark)",
            "config": {"workload": config},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("sweep", "sensing", "serve", "neural", "multitone", "su3"), default="sweep")
    ap.add_argument("--precision", choices=("fp32", "fp64"), default="fp32")
    ap.add_argument("--tau", type=int, default=-1)
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="sweep only: skip the serving and sensing keys")
    ap.add_argument("--sweep-sims", type=int, default=0,
                    help="simulations per GPU of the sweep (default 4096, the configured sweep; smaller for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
