"""GPU test of sigkernel_fma_peak, the measured FMA rate that the benchmark's roofline fractions
divide by: a finite rate of the right order for a GB300 (nominal FP32 about 80 TFLOP/s from 152 SMs
x 128 lanes x 2 FLOP x 2.07 GHz; FP64 about 1.2 TFLOP/s), and argument checks."""
import pytest
import torch

pytestmark = pytest.mark.gpu
sk = pytest.importorskip("paper_2502_08470_gb300.sigkernel")


@pytest.fixture(scope="module", autouse=True)
def _cuda_available():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_fma_peaks_have_the_expected_order():
    f32 = sk.fma_peak("f32", reps=2)
    f32p = sk.fma_peak("f32", packed=True, reps=2)
    f64 = sk.fma_peak("f64", reps=2)
    assert 10.0 < f32 < 200.0
    assert 10.0 < f32p < 200.0
    assert 0.1 < f64 < 20.0
    assert f64 < f32


def test_fma_peak_rejects_bad_arguments():
    with pytest.raises(sk.SigKernelError):
        sk.fma_peak("f64", packed=True)
    with pytest.raises(sk.SigKernelError):
        sk.fma_peak("f32", reps=0)
