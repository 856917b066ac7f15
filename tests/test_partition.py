"""A batch of independent simulations split over processes
(paper_2204_05586_gb300.sharded.partition), on the CPU.

The partitioner assigns requests to ranks greedily, longest first, by
estimated steps; each rank runs its share as one batch and nothing passes
between ranks.  Because a request's result does not depend on the batch it
runs in, the union of the ranks' results must equal the single-process batch
bit for bit.  Here every rank runs its share through the library's multicore
CPU backend (the same per-sample arithmetic as the GPU path) on gloo ranks of
world size 2 and 3.
"""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2204_05586_gb300 import sharded as SH, workloads as W  # noqa: E402


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def small_sweep():
    """A short sweep of uneven lengths (20 us to 1 ms, 100 ns steps), mixed spins."""
    reqs = W.sweep(10, t_min=2e-5, t_max=1e-3, dt=1e-7)
    _, served = W.serving_stream(6, t_min=2e-5, t_max=5e-4, dt=1e-7)
    return reqs + served


def test_partition_is_a_balanced_cover():
    reqs = W.sweep(200, t_min=1e-4, t_max=1e-2, dt=1e-7)
    steps = [SH.estimated_steps(r) for r in reqs]
    for world in (1, 2, 3, 8):
        parts = SH.partition(reqs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(reqs)))             # every request exactly once
        assert all(p == sorted(p) for p in parts)
        loads = [sum(steps[i] for i in p) for p in parts]
        # longest-first greedy: no rank exceeds the lightest by more than the longest request
        assert max(loads) - min(loads) <= max(steps)
    assert SH.partition([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        SH.partition(reqs, 0)


def test_partition_follows_longest_first():
    reqs = [W.spin_one_sensing(t_end=t, dt=1e-7) for t in (5e-4, 3e-4, 3e-4, 2e-4, 1e-4)]
    # steps 4990, 2990, 2990, 1990, 990: 0 -> r0; 1 -> r1; 2 -> r1 (2990 < 4990);
    # 3 -> r0 (4990 < 5980); 4 -> r1 (5980 < 6980)
    assert [SH.estimated_steps(r) for r in reqs] == [4990, 2990, 2990, 1990, 990]
    assert SH.partition(reqs, 2) == [[0, 3], [1, 2, 4]]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_2204_05586_gb300 import cpu_backend as CB, sharded as SH2
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        reqs = small_sweep()
        mine = SH2.partition(reqs, world)[rank]
        outs = CB.simulate([reqs[i] for i in mine], threads=2) if mine else []
        got = [None] * world
        dist.all_gather_object(got, [(i, o["states"]) for i, o in zip(mine, outs)])
        if rank == 0:
            q.put([pair for part in got for pair in part])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_union_of_ranks_equals_one_batch(world):
    from paper_2204_05586_gb300 import cpu_backend as CB
    try:
        CB.load()
    except Exception as e:   # the host backend is built with the GPU library
        pytest.skip(f"CPU backend unavailable: {e}")
    reqs = small_sweep()
    whole = CB.simulate(reqs, threads=4)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    pairs = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(i for i, _ in pairs) == list(range(len(reqs)))
    for i, states in pairs:
        assert np.array_equal(states, whole[i]["states"]), i
