"""The roofline models of bench.py: the algorithmic flop counts and derived
peaks that the bench line reports and the design notes quote, pinned so that
a change to one shows up here."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_models", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_derived_peaks(bench):
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert bench.FP64_DERIVED_TFLOPS == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)
    assert bench.FP64_DERIVED_TFLOPS == pytest.approx(bench.FP32_PEAK_TFLOPS / 64)


def test_spin_one_step_model(bench):
    # two Lie-Trotter exponentials with tau squarings, two products, the field
    assert bench.algorithmic_flops_per_step(2, 0) == 650.0
    assert bench.algorithmic_flops_per_step(2, 24) == 432.0 * 24 + 650.0
    assert bench.algorithmic_flops_per_step(2, 1, n_tones=3) - bench.algorithmic_flops_per_step(2, 1) == 264.0
    with pytest.raises(ValueError):
        bench.algorithmic_flops_per_step(1, 0)


def test_su3_step_model(bench):
    assert bench.SU3_DEGREE == 4
    assert bench.su3_flops_per_step(4) == 1748.0
    # one more Hermitian-times-general product every two degrees
    assert bench.su3_flops_per_step(5) - bench.su3_flops_per_step(4) == 2 * 162.0
    assert bench.su3_flops_per_step(6) == bench.su3_flops_per_step(5)
    # a halving adds the full-matrix tail and one squaring per exponential
    assert bench.su3_flops_per_step(4, 1) - bench.su3_flops_per_step(4) == 2 * (18.0 + 252.0 + 36.0 - 12.0)


def test_chain_model(bench):
    assert bench.chain_flops_per_sample(2, 6) == pytest.approx(5 / 6 * 216 + 72 + 60)
    assert bench.chain_flops_per_sample(1, 6) == pytest.approx(5 / 6 * 32 + 16 + 30)
