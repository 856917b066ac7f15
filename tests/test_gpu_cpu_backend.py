"""The multicore CPU backend and the GPU library run the same algorithm: on
the same requests their results agree to the rounding of the host's and the
device's maths library (FP64) or to FP32 rounding (FP32-bulk)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2204_05586_gb300 import cpu_backend as C, spinsim as S, workloads as W  # noqa: E402


@pytest.mark.parametrize("prec,tol", [(S.PREC_FP64, 1e-12), (S.PREC_FP32_BULK, 2e-6)])
def test_cpu_backend_equals_gpu(prec, tol):
    reqs = W.sweep(32, t_min=1e-4, t_max=2e-3) + [W.spin_half_rabi(), W.neural_pulse(t_end=2e-3, t_p=0.5e-3),
                                                  W.multitone_sensing(t_end=1e-3)]
    with S.Simulator(precision=prec) as sim:
        gpu = sim.simulate(reqs)
    cpu = C.simulate(reqs, precision=prec)
    for g, c in zip(gpu, cpu):
        assert g["status"] == S.OK and c["status"] == S.OK
        d = np.abs(g["states"].cpu().numpy() - c["states"]).max()
        assert d <= tol, d
        assert c["trotter_squares"] == g["trotter_squares"]
