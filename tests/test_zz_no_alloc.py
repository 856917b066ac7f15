"""The allocation-free entry point spinsim_simulate_static.

It serves callers that cannot let a library allocate (real-time loops where a
cudaMalloc/cudaFree would synchronise the device, frameworks whose own pooled
allocator owns all device memory).  Its scratch is a fixed file-scope device
array, so these tests check, through the C ABI, that its results equal
spinsim_simulate's bit for bit on three consecutive calls whose chain trees
have different heights (each call runs over the previous call's leftovers in
the array), that a warmed call changes the device's free memory by nothing,
that the caller's current device is left as it was, and that it refuses
requests it cannot serve without allocating.  The file name makes pytest
collect it after every other test file.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2204_05586_gb300 import spinsim as S, workloads as W  # noqa: E402


def static_outputs(req, want_ops):
    K = S.spinsim_counts(S.make_request(req))[1]
    n = req["spin_x2"] + 1
    states = torch.full((K, n, 2), float("nan"), dtype=torch.float64, device="cuda")
    spin = torch.full((K, 3), float("nan"), dtype=torch.float64, device="cuda")
    ops = torch.full((K, n, n, 2), float("nan"), dtype=torch.float64, device="cuda") if want_ops else None
    res = S.spinsim_result()
    res.states, res.spin = states.data_ptr(), spin.data_ptr()
    res.ops = ops.data_ptr() if want_ops else None
    res.capacity = K
    return K, res, states, spin, ops


def static_run(cfg, req, want_ops=False):
    K, res, states, spin, ops = static_outputs(req, want_ops)
    st = S.spinsim_simulate_static(cfg, S.make_request(req), res, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == S.OK and res.status == S.OK and res.n_samples == K
    return {"states": torch.view_as_complex(states).cpu().numpy(), "spin": spin.cpu().numpy(),
            "ops": torch.view_as_complex(ops).cpu().numpy() if want_ops else None}


# Per spin, three lengths whose chain trees have top levels 2, 1 and 0.
CASES = {2: [W.spin_one_sensing(t_end=6e-3), W.spin_one_sensing(t_end=2.5e-3), W.spin_one_sensing(t_end=1e-4)],
         1: [W.spin_half_rabi(t_end=5e-2), W.spin_half_rabi(t_end=4e-3), W.spin_half_rabi(t_end=5e-4)]}


@pytest.mark.parametrize("prec", [S.PREC_FP32_BULK, S.PREC_FP64])
@pytest.mark.parametrize("spin_x2", [2, 1])
def test_static_equals_simulate_on_consecutive_calls(prec, spin_x2):
    reqs = CASES[spin_x2]
    cfg = S.make_config(precision=prec)
    with S.Simulator(precision=prec) as sim:
        refs = sim.simulate(reqs, want_ops=True)
    for req, ref in zip(reqs, refs):   # calls in a row, each over the previous one's leftovers
        got = static_run(cfg, req, want_ops=True)
        assert np.array_equal(got["states"], ref["states"].cpu().numpy())
        assert np.array_equal(got["spin"], ref["spin"].cpu().numpy())
        assert np.array_equal(got["ops"], ref["ops"].cpu().numpy())


def test_warm_call_allocates_nothing_and_keeps_the_device():
    cfg = S.make_config()
    req = W.spin_one_sensing(t_end=3e-3)
    static_run(cfg, req)                                   # first call: set-up, modules loaded
    K, res, states, spin, _ = static_outputs(req, False)   # outputs allocated before the measurement
    torch.cuda.synchronize()
    dev_before = torch.cuda.current_device()
    free_before = torch.cuda.mem_get_info()[0]
    st = S.spinsim_simulate_static(cfg, S.make_request(req), res, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == S.OK and res.status == S.OK
    assert torch.cuda.mem_get_info()[0] == free_before
    assert torch.cuda.current_device() == dev_before


def test_static_rejects_what_it_cannot_serve():
    cfg = S.make_config()
    req = W.spin_one_sensing(t_end=0.2)     # 200,000 samples: beyond the fixed scratch
    K = S.spinsim_counts(S.make_request(req))[1]
    big = torch.empty((K, 3, 2), dtype=torch.float64, device="cuda")
    res = S.spinsim_result()
    res.states, res.capacity = big.data_ptr(), K
    assert S.spinsim_simulate_static(cfg, S.make_request(req), res, 0) == S.E_NOMEM
    small = W.spin_one_sensing(t_end=1e-4)
    host = torch.empty((100, 3, 2), dtype=torch.float64)   # host memory would need staging
    res = S.spinsim_result()
    res.states, res.capacity = host.data_ptr(), 100
    assert S.spinsim_simulate_static(cfg, S.make_request(small), res, 0) == S.E_ARG
    res.states, res.capacity = big.data_ptr(), 50             # capacity below K
    assert S.spinsim_simulate_static(cfg, S.make_request(small), res, 0) == S.E_CAPACITY
