"""Failure handling through the C ABI, driven by host-side fault injection.

SPINSIM_FAIL_ALLOC / SPINSIM_FAIL_LAUNCH (read at spinsim_create) make the
handle's n-th device allocation or kernel launch report failure without
being made, so no GPU fault is involved.  The batch (or the served batch)
must return the error, every request in it must carry it, and the handle
must stay usable: the next call runs and equals a clean run bit for bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2204_05586_gb300 import spinsim as S, workloads as W  # noqa: E402

REQS = [W.spin_one_sensing(t_end=1e-3), W.spin_half_rabi(t_end=2e-3), W.spin_one_sensing(t_end=4e-4)]


def clean_states(reqs):
    with S.Simulator(precision=S.PREC_FP32_BULK) as sim:
        return [o["states"].cpu().numpy() for o in sim.simulate(reqs)]


@pytest.mark.parametrize("var,n,expect", [("SPINSIM_FAIL_ALLOC", 1, S.E_NOMEM),
                                          ("SPINSIM_FAIL_LAUNCH", 1, S.E_CUDA),    # first integrate launch
                                          ("SPINSIM_FAIL_LAUNCH", 2, S.E_CUDA),    # first chain launch
                                          ("SPINSIM_FAIL_LAUNCH", 3, S.E_CUDA)])   # second group's integrate
def test_injected_failure_then_recovery(monkeypatch, var, n, expect):
    ref = clean_states(REQS)
    monkeypatch.setenv(var, str(n))
    with S.Simulator(precision=S.PREC_FP32_BULK) as sim:
        monkeypatch.delenv(var)
        outs = sim.allocate(REQS)
        got = sim.simulate(REQS, outs=outs, check=False)
        assert all(o["status"] == expect for o in got), [o["status"] for o in got]
        again = sim.simulate(REQS, outs=outs)
        assert all(o["status"] == S.OK for o in again)
        for o, r in zip(again, ref):
            assert np.array_equal(o["states"].cpu().numpy(), r)


@pytest.mark.parametrize("var,expect", [("SPINSIM_FAIL_ALLOC", S.E_NOMEM), ("SPINSIM_FAIL_LAUNCH", S.E_CUDA)])
def test_injected_failure_in_serving(monkeypatch, var, expect):
    """The first served batch fails (its pool allocation, or its first
    launch); the requests after it are served normally."""
    ref = clean_states(REQS)
    monkeypatch.setenv(var, "1")
    with S.Simulator(precision=S.PREC_FP32_BULK) as sim:
        monkeypatch.delenv(var)
        outs = sim.allocate(REQS)
        res = sim.results_struct(outs)
        tickets = []
        for q, r in zip(REQS, res):
            st, t = S.spinsim_submit(sim.handle, S.make_request(q), r)
            tickets.append(t)
            assert S.spinsim_poll(sim.handle, t, 10_000_000) == S.OK   # one at a time
        assert res[0].status == expect
        for i in (1, 2):
            assert res[i].status == S.OK
            got = torch.view_as_complex(outs[i]["states"][:outs[i]["K"]]).cpu().numpy()
            assert np.array_equal(got, ref[i])
        assert S.spinsim_memory(sim.handle)["in_flight"] == 0
