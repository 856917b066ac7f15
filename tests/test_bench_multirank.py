"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

Under torchrun every rank runs its own copy of the workload (weak scaling):
the timed region is closed by a max over ranks, served step counts are summed,
and only rank 0 prints.  These tests run that logic on gloo ranks without a
GPU; the per-rank simulations themselves are covered by the GPU tests."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_setup()
        seconds = [0.75, 1.25][r]                  # rank 1 is the slow one
        t = bench.barrier_max(seconds, w, device="cpu")
        served = bench.barrier_sum(1000 * (r + 1), w, device="cpu")
        rate = bench.job_rate(9_999_900, 10, w, t)
        bench.barrier(w)
        q.put((r, w, local, t, served, rate))
    finally:
        dist.destroy_process_group()


def test_max_sum_and_rate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    for _, _, _, t, served, rate in out:
        assert t == 1.25                            # the slowest rank decides the time
        assert served == 3000.0                     # served steps add up over ranks
        assert rate == pytest.approx(9_999_900 * 10 * 2 / 1.25, rel=1e-15)


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.barrier_max(2.5, 1) == 2.5
    assert bench.barrier_sum(7, 1) == 7
    assert bench.job_rate(100, 3, 1, 0.5) == 600.0
    with pytest.raises(ValueError):
        bench.algorithmic_flops_per_step(1, 0)
    assert bench.algorithmic_flops_per_step(2, 1) == 1082.0


def test_ranks_get_distinct_sweep_inputs():
    sys.path.insert(0, ROOT)
    from paper_2204_05586_gb300 import workloads as W
    a, b = W.sweep(8, seed=W.SEED), W.sweep(8, seed=W.SEED + 1)
    assert [r["field"]["bias_hz"] for r in a] != [r["field"]["bias_hz"] for r in b]
    assert [r["field"]["bias_hz"] for r in a] == [r["field"]["bias_hz"] for r in W.sweep(8, seed=W.SEED)]


def test_reference_arm_under_torchrun_prints_once():
    """`bench.py --impl reference` launched under torchrun with N = 2:
    rank 0 times the oracle and prints one line, rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 1
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
