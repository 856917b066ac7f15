"""Work split over processes: a batch of independent simulations
(``partition``), and one long simulation split into ranges (Sec. 1.2.4).

The sample operators U_k depend only on the field, so contiguous ranges of
output samples can be computed by different processes (one per GPU).  What
the ranges share is the ordered product: the state entering range r is
    psi(t_{k_r}) = A_{r-1} ... A_1 A_0 psi_init,
A_j the propagator over range j.  So each process

  1. computes its range's operators and their ordered product A_r
     (``spinsim_range_begin``; the operators stay on its GPU),
  2. exchanges A_r with every other process (one all-gather of one N x N
     FP64 complex matrix per range),
  3. forms its entering state from the gathered products
     (``spinsim_range_entering_state``: every process does the same tiny
     product, in FP64, in range order) and
  4. writes its states from that entering state (``spinsim_range_finish``).

A range r < last is run as the request for its samples plus one: its K
operators then carry psi(t_{k_r}) to psi(t_{k_{r+1}}), the next range's first
sample, and that extra sample's state is dropped.

``run_range`` takes the exchange as a callable, so the same code runs with
``torch.distributed`` (``torch_all_gather``; gloo or NCCL) or any other
transport.
"""
from __future__ import annotations

import numpy as np


def estimated_steps(req: dict) -> int:
    """Integration steps of a request, (K - 1) L: the sample operators U_1 ..
    U_{K-1} of L steps each (U_0 is the identity); the measure of work by
    which a batch is split."""
    K = int(round((req["t_end"] - req["t_start"]) / req["dt_out"]))
    L = int(round(req["dt_out"] / req["dt"]))
    return max(K - 1, 0) * L


def partition(reqs, world: int):
    """Split a batch of independent simulations over `world` processes by
    estimated steps, greedily longest first: requests in decreasing order of
    steps (ties: lower index first), each to the process with the fewest
    steps so far (ties: lower rank).  Returns one ascending index list per
    rank.  Every process then runs its share as one batch; no data passes
    between them (a request's result does not depend on its batch)."""
    if world < 1:
        raise ValueError("world >= 1 required")
    load = [0] * world
    parts = [[] for _ in range(world)]
    steps = [estimated_steps(r) for r in reqs]
    for i in sorted(range(len(reqs)), key=lambda j: (-steps[j], j)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += steps[i]
    return [sorted(p) for p in parts]


def ranges(K: int, world: int):
    """Contiguous ranges [k0, k1) of K output samples over `world` processes,
    as even as possible (the first K % world ranges one sample longer)."""
    if K < 0 or world < 1:
        raise ValueError("K >= 0 and world >= 1 required")
    base, extra = divmod(K, world)
    out, k = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((k, k + n))
        k += n
    return out


def range_request(req: dict, k0: int, k1: int, last: bool) -> dict:
    """The request for output samples [k0, k1) of `req` (plus one sample unless
    `last`, so that its operators reach the next range's first sample)."""
    t0, dt_out = req["t_start"], req["dt_out"]
    k_end = k1 if last else k1 + 1
    r = dict(req)
    r["t_start"] = t0 + k0 * dt_out
    r["t_end"] = t0 + k_end * dt_out
    return r


def entering_states(aggs, psi_init):
    """States entering every range: psi_0 = psi_init, psi_{r+1} = A_r psi_r,
    formed by the library (spinsim_range_entering_state: FP64, in range
    order, renormalised after each range as every written state is)."""
    from . import spinsim as S
    psi_init = np.asarray(psi_init, dtype=np.complex128)
    spin_x2 = psi_init.shape[0] - 1
    out = []
    for r in range(len(aggs)):
        st, psi = S.spinsim_range_entering_state(spin_x2, aggs, r, psi_init)
        if st != S.OK:
            raise S.SpinsimError(st, "spinsim_range_entering_state")
        out.append(psi)
    return out


def run_range(backend, req: dict, rank: int, world: int, all_gather):
    """Run this process's range of `req` through `backend` and return
    (k0, k1, states) with states the complex128 [k1 - k0, N] array.

    backend.begin(request) -> A (complex128 [N, N]) computes the range's
    operators and their ordered product; backend.finish(psi_in) -> states of
    that request from the entering state psi_in.  all_gather(A) returns the
    list of every process's A in rank order."""
    K = int(round((req["t_end"] - req["t_start"]) / req["dt_out"]))
    k0, k1 = ranges(K, world)[rank]
    last = rank == world - 1
    sub = range_request(req, k0, k1, last)
    A = backend.begin(sub)
    aggs = all_gather(A)
    psi_in = entering_states(aggs, req["psi0"])[rank]
    states = backend.finish(psi_in)
    return k0, k1, np.asarray(states)[: k1 - k0]


def torch_all_gather(device: str = "cpu"):
    """An all_gather over the default torch.distributed process group for
    N x N complex matrices (gloo on the CPU, NCCL with device='cuda')."""
    import torch
    import torch.distributed as dist

    def gather(A):
        a = np.ascontiguousarray(np.asarray(A, dtype=np.complex128))
        n = a.shape[0]
        t = torch.from_numpy(a.view(np.float64).reshape(-1).copy()).to(device)
        out = [torch.empty_like(t) for _ in range(dist.get_world_size())]
        dist.all_gather(out, t)
        return [o.cpu().numpy().view(np.complex128).reshape(n, n) for o in out]

    return gather


class CudaRange:
    """The library as a range backend: one handle, one open range at a time."""

    def __init__(self, **cfg):
        from . import spinsim as S
        self.S = S
        self.sim = S.Simulator(**cfg)
        self.outs = None
        self.res = None
        self.req = None

    def begin(self, req: dict):
        S = self.S
        self.outs = self.sim.allocate([req])
        self.res = S.Simulator.results_struct(self.outs)
        self.req = S.make_request(req)
        st, A = S.spinsim_range_begin(self.sim.handle, self.req, self.res[0], 0)
        if st != S.OK:
            raise S.SpinsimError(st, "spinsim_range_begin")
        return A

    def finish(self, psi_in):
        import torch
        S = self.S
        st = S.spinsim_range_finish(self.sim.handle, psi_in, 0)
        if st != S.OK:
            raise S.SpinsimError(st, "spinsim_range_finish")
        torch.cuda.synchronize()
        o = self.outs[0]
        return torch.view_as_complex(o["states"][: o["K"]]).cpu().numpy()

    def close(self):
        self.sim.close()
