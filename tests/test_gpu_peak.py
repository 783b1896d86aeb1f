"""clb_peak_fma: the fused multiply-add throughput microbenchmark that the
sweeps' measured FLOP rates are reported against.  Checks that it runs in both
precisions, that the FP32 rate is well above the FP64 rate (GB300), and that
other storages are refused."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_01955_gb300.clb as clb

    return clb


def test_peak_fma_rates(clb):
    f32 = clb.clb_peak_fma(clb.CLB_FP32_SHIFTED)
    f64 = clb.clb_peak_fma(clb.CLB_FP64)
    # nominal GB300: 152 SMs x 128 FP32 FMA lanes x 2 FLOP x ~2 GHz ~ 80 TFLOP/s; FP64 ~ 1.2
    assert 10.0 < f32 < 200.0
    assert 0.1 < f64 < 20.0
    assert f32 > 10 * f64


def test_peak_fma_refuses_other_storages(clb):
    with pytest.raises(clb.CLBError) as e:
        clb.clb_peak_fma(clb.CLB_FP16_SCALED)
    assert e.value.status == clb.CLB_EINVAL
