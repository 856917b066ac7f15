"""Serving through the C ABI: admission by device-memory footprint.

The serving queue (spinsim_submit / spinsim_poll / spinsim_poll_any) carves
every batch's scratch from one pool; the pool and the handle's arena together
never exceed mem_budget, a request waits while its scratch does not fit, and a
request that could never fit is refused (the paper's counterpart: Sec. 1.2.4,
the simulator raises an out-of-memory error for a job larger than the GPU's
memory).  Every served result must equal the request's run alone, bit for bit.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2204_05586_gb300 import spinsim as S, workloads as W  # noqa: E402


def alone_states(reqs, **cfg):
    out = []
    for q in reqs:
        with S.Simulator(**cfg) as sim:
            (o,) = sim.simulate([q])
            out.append(o["states"].cpu().numpy())
    return out


def footprint(sim, q):
    return S.spinsim_footprint(sim.handle, [S.make_request(q)])


def test_small_budget_queues_requests_and_bounds_memory():
    """A budget of 1.6x the largest request's footprint: requests queue while
    earlier batches hold the pool, the handle never holds more than the
    budget, and every result equals its run alone."""
    _, reqs = W.serving_stream(40, t_max=3e-3)
    alone = alone_states(reqs, precision=S.PREC_FP32_BULK)
    with S.Simulator(precision=S.PREC_FP32_BULK) as probe:
        big = max(footprint(probe, q) for q in reqs)
    budget = int(1.6 * big)
    with S.Simulator(precision=S.PREC_FP32_BULK, mem_budget=budget) as sim:
        outs = sim.allocate(reqs)
        res = sim.results_struct(outs)
        creqs = [S.make_request(q) for q in reqs]
        tickets = []
        waited_behind_work = 0
        for q, r in zip(creqs, res):
            st, t = S.spinsim_submit(sim.handle, q, r)
            assert st == S.OK
            tickets.append(t)
            m = S.spinsim_memory(sim.handle)
            assert m["budget"] == budget and m["held"] <= budget
            if m["pending"] > 0 and m["in_flight"] > 0:
                waited_behind_work += 1
        left = set(tickets)
        while left:
            for t in list(left):
                st = S.spinsim_poll(sim.handle, t, 0)
                assert st in (S.OK, S.PENDING)
                if st == S.OK:
                    left.discard(t)
            m = S.spinsim_memory(sim.handle)
            assert m["held"] <= budget and m["pool_in_use"] <= m["pool"]
        m = S.spinsim_memory(sim.handle)
        assert m["peak_held"] <= budget
        assert m["pending"] == 0 and m["in_flight"] == 0 and m["pool_in_use"] == 0
    assert waited_behind_work > 0, "the budget never made a request wait"
    for o, r, a in zip(outs, res, alone):
        assert r.status == S.OK
        assert np.array_equal(torch.view_as_complex(o["states"][:o["K"]]).cpu().numpy(), a)


def test_over_budget_request_is_refused_everywhere():
    q = W.spin_one_sensing(t_end=5e-3)
    with S.Simulator(precision=S.PREC_FP32_BULK) as probe:
        need = footprint(probe, q)
    budget = need // 2
    with S.Simulator(precision=S.PREC_FP32_BULK, mem_budget=budget) as sim:
        assert footprint(sim, q) == need > budget
        outs = sim.allocate([q])
        res = sim.results_struct(outs)
        st, t = S.spinsim_submit(sim.handle, S.make_request(q), res[0])
        assert st == S.E_NOMEM and res[0].status == S.E_NOMEM
        assert S.spinsim_poll(sim.handle, t, 0) == S.OK      # completed at once, with its error
        assert S.spinsim_simulate(sim.handle, [S.make_request(q)], res) == S.E_NOMEM
        assert res[0].status == S.E_NOMEM
        m = S.spinsim_memory(sim.handle)
        assert m["held"] == 0 and m["peak_held"] == 0
        # a request that fits still runs on the same handle
        small = W.spin_one_sensing(t_end=2e-4)
        (o,) = sim.simulate([small])
        assert o["status"] == S.OK
        assert S.spinsim_memory(sim.handle)["held"] <= budget


def test_poll_times_out_then_completes():
    """A long FP64 request (2e6 CF4 steps at tau = 24, tens of ms on the
    device): a 1 us wait runs out, a zero wait reports it pending, a long wait
    sees it complete."""
    q = W.spin_one_sensing(t_end=0.02)
    with S.Simulator(precision=S.PREC_FP64) as sim:
        outs = sim.allocate([q])
        res = sim.results_struct(outs)
        st, t = S.spinsim_submit(sim.handle, S.make_request(q), res[0])
        assert st == S.OK
        assert S.spinsim_poll(sim.handle, t, 1) == S.E_TIMEOUT
        assert S.spinsim_poll(sim.handle, t, 0) == S.PENDING
        buf = (ctypes.c_int64 * 4)()
        assert S.spinsim_poll_any(sim.handle, buf, 1)[0] == S.E_TIMEOUT
        assert S.spinsim_poll(sim.handle, t, 30_000_000) == S.OK
        assert res[0].status == S.OK
        states = torch.view_as_complex(outs[0]["states"][:outs[0]["K"]]).cpu().numpy()
    (a,) = alone_states([q], precision=S.PREC_FP64)
    assert np.array_equal(states, a)


def test_poll_any_reports_each_ticket_once():
    _, reqs = W.serving_stream(24, t_max=2e-3)
    alone = alone_states(reqs, precision=S.PREC_FP32_BULK)
    with S.Simulator(precision=S.PREC_FP32_BULK) as sim:
        outs = sim.allocate(reqs)
        res = sim.results_struct(outs)
        tickets = {}
        for i, (q, r) in enumerate(zip(reqs, res)):
            st, t = S.spinsim_submit(sim.handle, S.make_request(q), r)
            assert st == S.OK
            tickets[t] = i
        # one ticket reported by spinsim_poll is not reported again by poll_any
        first = next(iter(tickets))
        assert S.spinsim_poll(sim.handle, first, 10_000_000) == S.OK
        seen = [first]
        buf = (ctypes.c_int64 * 5)()
        while len(seen) < len(tickets):
            st, n = S.spinsim_poll_any(sim.handle, buf, 10_000_000)
            assert st == S.OK and 1 <= n <= 5
            seen.extend(buf[:n])
        assert sorted(seen) == sorted(tickets)
        assert S.spinsim_poll_any(sim.handle, buf, 0) == (S.PENDING, 0)
    for o, r, a in zip(outs, res, alone):
        assert r.status == S.OK
        assert np.array_equal(torch.view_as_complex(o["states"][:o["K"]]).cpu().numpy(), a)


def test_arena_and_pool_share_the_budget():
    """After serving, a batch through spinsim_simulate that needs more than the
    budget minus the pool still runs: the idle pool is given back first."""
    _, reqs = W.serving_stream(8, t_max=2e-3)
    batch = [W.spin_one_sensing(t_end=8e-3)]
    with S.Simulator(precision=S.PREC_FP32_BULK) as probe:
        need = footprint(probe, batch[0])
        serve_need = max(footprint(probe, q) for q in reqs)
    budget = int(max(need, serve_need) * 1.2)
    with S.Simulator(precision=S.PREC_FP32_BULK, mem_budget=budget) as sim:
        outs = sim.allocate(reqs)
        res = sim.results_struct(outs)
        for q, r in zip(reqs, res):
            st, t = S.spinsim_submit(sim.handle, S.make_request(q), r)
            assert st == S.OK
            assert S.spinsim_poll(sim.handle, t, 10_000_000) == S.OK
        assert S.spinsim_memory(sim.handle)["pool"] > 0
        (o,) = sim.simulate(batch)
        assert o["status"] == S.OK
        m = S.spinsim_memory(sim.handle)
        assert m["held"] <= budget and m["peak_held"] <= budget and m["arena"] >= need
    (a,) = alone_states(batch, precision=S.PREC_FP32_BULK)
    assert np.array_equal(o["states"].cpu().numpy(), a)


@pytest.mark.parametrize("prec", [S.PREC_FP32_BULK, S.PREC_FP64])
@pytest.mark.parametrize("tones", [False, True])
def test_footprint_is_what_the_arena_takes(prec, tones):
    """On a fresh handle the arena is the batch's footprint rounded up to 1 MiB,
    with requests with further tones (whose phasor tables follow the drive's)
    in the batch too."""
    reqs = W.sweep(6, t_min=1e-4, t_max=3e-3)
    if tones:
        reqs += [W.multitone_sensing(t_end=3e-3), W.multitone_sensing(t_end=1.3e-3)]
    with S.Simulator(precision=prec) as sim:
        need = S.spinsim_footprint(sim.handle, [S.make_request(q) for q in reqs])
        outs = sim.simulate(reqs)
        m = S.spinsim_memory(sim.handle)
    assert all(o["status"] == S.OK for o in outs)
    mib = 1 << 20
    assert m["arena"] == -(-need // mib) * mib


def test_magnus_warning_bit():
    """||H|| delta_t at or above the Magnus radius xi = 1.0868687 (Sec. 1.2.2)
    sets SPINSIM_WARN_MAGNUS; the sensing field at delta_t = 1e-6 s in the lab
    frame has ||H|| delta_t = 4.4, at 1e-8 s 0.044."""
    coarse = W.spin_one_sensing(t_end=2e-4, dt=1e-6, dt_out=1e-6)
    fine = W.spin_one_sensing(t_end=2e-4)
    with S.Simulator(precision=S.PREC_FP64, rotating_frame=False) as sim:
        a, b = sim.simulate([coarse, fine])
    assert a["status"] == S.OK and a["flags"] & S.WARN_MAGNUS
    assert b["status"] == S.OK and not b["flags"] & S.WARN_MAGNUS
