"""One long simulation split over processes (paper_2204_05586_gb300.sharded),
on the CPU: range planning, the entering states, and the whole exchange on
gloo ranks (world size 2 and 3) with the oracle as every rank's backend,
against the oracle's unsplit run.  The library's own range entry points are
covered by the GPU tests."""
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


class OracleRange:
    """The oracle as a range backend: the range's operators and their ordered
    product, then the states from a given entering state."""

    def __init__(self, O, threads=1):
        self.O, self.threads, self.req = O, threads, None

    def begin(self, req):
        self.req = req
        out = self.O.simulate(req["spin_x2"], req["field"], req["t_start"], req["t_end"], req["dt"], req["dt_out"],
                              req["psi0"], want_ops=True, threads=self.threads)
        A = np.eye(out["ops"].shape[1], dtype=np.complex128)
        for U in out["ops"]:
            A = U @ A
        return A

    def finish(self, psi_in):
        r = self.req
        return self.O.simulate(r["spin_x2"], r["field"], r["t_start"], r["t_end"], r["dt"], r["dt_out"],
                               psi_in, threads=self.threads)["states"]


def long_request(spin_x2):
    f = W.field(bias_hz=40e3, drive_x_hz=3e3, drive_hz=40.2e3, quad_hz=300.0 if spin_x2 == 2 else 0.0,
                pulses=[(200.0, 0.4e-3, 0.1e-3), (150.0, 0.9e-3, 0.25e-3, "sine")])
    rng = np.random.default_rng(3 + spin_x2)
    return W.request(spin_x2, f, 0.0, 1.3e-3, 1e-7, 1e-6, psi0=W.random_state(spin_x2 + 1, rng))


def test_ranges_partition():
    for K, world in [(0, 1), (1, 3), (10, 3), (100000, 8), (7, 7), (5, 8)]:
        rs = SH.ranges(K, world)
        assert len(rs) == world and rs[0][0] == 0 and rs[-1][1] == K
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        sizes = [b - a for a, b in rs]
        assert max(sizes) - min(sizes) <= 1


def test_range_requests_cover_the_run_with_one_sample_of_overlap():
    req = long_request(2)
    rs = SH.ranges(1300, 3)
    for r, (k0, k1) in enumerate(rs):
        sub = SH.range_request(req, k0, k1, last=r == 2)
        K = round((sub["t_end"] - sub["t_start"]) / sub["dt_out"])
        assert abs(sub["t_start"] - k0 * 1e-6) < 1e-18
        assert K == (k1 - k0 if r == 2 else k1 - k0 + 1)


def test_entering_states_are_the_ordered_products():
    rng = np.random.default_rng(5)
    mats = []
    for _ in range(4):
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3)))
        mats.append(q)
    psi0 = W.random_state(3, rng)
    psis = SH.entering_states(mats, psi0)
    assert len(psis) == 4
    assert np.allclose(psis[0], psi0)
    assert np.allclose(psis[3], mats[2] @ mats[1] @ mats[0] @ psi0)   # later ranges on the left


def test_entering_state_entry_point():
    """spinsim_range_entering_state (host arithmetic in the library, no GPU):
    the ordered products renormalised after each range, both spins, and its
    argument checks."""
    from paper_2204_05586_gb300 import spinsim as S
    rng = np.random.default_rng(9)
    for n in (2, 3):
        mats = [1.01 * np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))[0] for _ in range(3)]
        psi0 = W.random_state(n, rng)
        psi = psi0.copy()
        for r in range(4):
            st, got = S.spinsim_range_entering_state(n - 1, mats, r, psi0)
            assert st == S.OK
            assert np.abs(got - psi).max() < 1e-14 and abs(np.linalg.norm(got) - 1) < 1e-15
            if r < 3:
                psi = mats[r] @ psi
                psi = psi / np.linalg.norm(psi)      # the 1.01 scale is taken out at every range
    one = [np.eye(3, dtype=np.complex128)]
    assert S.spinsim_range_entering_state(3, one, 1, W.UP_ONE)[0] == S.E_ARG
    assert S.spinsim_range_entering_state(2, one, -1, W.UP_ONE)[0] == S.E_ARG
    assert S.spinsim_range_entering_state(2, one, 1, 1.1 * W.UP_ONE)[0] == S.E_NORM
    assert S.spinsim_range_entering_state(2, [np.full((3, 3), np.nan)], 1, W.UP_ONE)[0] == S.E_ARG


def test_split_equals_unsplit_in_one_process(oracle_mod):
    """The split with an in-process exchange: every range's states equal the
    unsplit oracle run (spin-one and spin-half, 1 to 4 ranges)."""
    for spin_x2 in (2, 1):
        req = long_request(spin_x2)
        full = OracleRange(oracle_mod, threads=4)
        full_states = full.O.simulate(req["spin_x2"], req["field"], req["t_start"], req["t_end"], req["dt"],
                                      req["dt_out"], req["psi0"], threads=4)["states"]
        for world in (1, 2, 4):
            backends = [OracleRange(oracle_mod, threads=4) for _ in range(world)]
            K = full_states.shape[0]
            subs = [SH.range_request(req, k0, k1, r == world - 1) for r, (k0, k1) in enumerate(SH.ranges(K, world))]
            aggs = [b.begin(s) for b, s in zip(backends, subs)]
            psis = SH.entering_states(aggs, req["psi0"])
            got = np.concatenate([b.finish(p)[: k1 - k0] for b, p, (k0, k1) in
                                  zip(backends, psis, SH.ranges(K, world))])
            assert got.shape == full_states.shape
            assert np.abs(got - full_states).max() < 1e-12, (spin_x2, world)


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_2204_05586_gb300 import sharded as SH2
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for spin_x2 in (2, 1):
            req = long_request(spin_x2)
            k0, k1, states = SH2.run_range(OracleRange(O), req, rank, world, SH2.torch_all_gather("cpu"))
            np.save(os.path.join(outdir, f"s{spin_x2}_r{rank}.npy"), states)
            np.save(os.path.join(outdir, f"s{spin_x2}_r{rank}_k.npy"), np.array([k0, k1]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_over_gloo_ranks(oracle_mod, tmp_path, world):
    """Each gloo rank runs the oracle on its range; the ranks exchange their
    range products with torch.distributed.all_gather; the concatenated states
    equal the unsplit run."""
    ctx = mp.get_context("spawn")
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    for spin_x2 in (2, 1):
        req = long_request(spin_x2)
        full = oracle_mod.simulate(req["spin_x2"], req["field"], req["t_start"], req["t_end"], req["dt"],
                                   req["dt_out"], req["psi0"], threads=4)["states"]
        parts, ks = [], []
        for r in range(world):
            parts.append(np.load(tmp_path / f"s{spin_x2}_r{r}.npy"))
            ks.append(tuple(np.load(tmp_path / f"s{spin_x2}_r{r}_k.npy")))
        assert ks == SH.ranges(full.shape[0], world)
        got = np.concatenate(parts)
        assert np.abs(got - full).max() < 1e-12
