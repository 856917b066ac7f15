"""The allocation-free entry point spinsim_simulate_static.

It serves callers that cannot let a library allocate (real-time loops where a
cudaMalloc/cudaFree would synchronise the device, frameworks whose own pooled
allocator owns all device memory).  Its scratch is a fixed file-scope device
array, so these tests check, through the C ABI, that its results match
spinsim_simulate's on two consecutive calls (the second call reuses the
array with the first call's contents still in it), and that it refuses
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

TOL = {S.PREC_FP64: 1e-10, S.PREC_FP32_BULK: 1e-5}   # the tolerances of the parity tests


def static_run(cfg, req, want_ops=False):
    K = S.spinsim_counts(S.make_request(req))[1]
    n = req["spin_x2"] + 1
    states = torch.full((K, n, 2), float("nan"), dtype=torch.float64, device="cuda")
    spin = torch.full((K, 3), float("nan"), dtype=torch.float64, device="cuda")
    ops = torch.full((K, n, n, 2), float("nan"), dtype=torch.float64, device="cuda") if want_ops else None
    res = S.spinsim_result()
    res.states, res.spin = states.data_ptr(), spin.data_ptr()
    res.ops = ops.data_ptr() if want_ops else None
    res.capacity = K
    st = S.spinsim_simulate_static(cfg, S.make_request(req), res, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == S.OK and res.status == S.OK and res.n_samples == K
    return {"states": torch.view_as_complex(states).cpu().numpy(), "spin": spin.cpu().numpy(),
            "ops": torch.view_as_complex(ops).cpu().numpy() if want_ops else None}


@pytest.mark.parametrize("prec", [S.PREC_FP32_BULK, S.PREC_FP64])
@pytest.mark.parametrize("spin_x2", [2, 1])
def test_static_matches_simulate_on_two_calls(prec, spin_x2):
    reqs = [W.spin_one_sensing(t_end=6e-3), W.spin_one_sensing(t_end=2.5e-3)] if spin_x2 == 2 else \
        [W.spin_half_rabi(t_end=4e-3), W.spin_half_rabi(t_end=1.7e-3)]
    cfg = S.make_config(precision=prec)
    with S.Simulator(precision=prec) as sim:
        refs = sim.simulate(reqs, want_ops=True)
    for req, ref in zip(reqs, refs):   # two calls in a row, the second over the first's leftovers
        got = static_run(cfg, req, want_ops=True)
        tol = TOL[prec]
        assert np.abs(got["states"] - ref["states"].cpu().numpy()).max() <= tol
        assert np.abs(got["spin"] - ref["spin"].cpu().numpy()).max() <= 2 * tol
        assert np.abs(got["ops"] - ref["ops"].cpu().numpy()).max() <= tol


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
