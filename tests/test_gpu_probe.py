"""The FMA throughput probe that gives the measured ALU roof: FP64 and FP32
rates within a factor of the GB300's lane counts (2 FP64 and 128 FP32 FMA
lanes per SM at up to 2.07 GHz: 1.26 and 80.5 TFLOP/s), FP64 far below FP32."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10103_gb300 import build
    build.build()
    from paper_2509_10103_gb300 import _lib
    return _lib


def test_fma_probe_rates(L):
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    f64 = L.pnop_measure_fma_peak(L.PNOP_FP64, 0.02)
    f32 = L.pnop_measure_fma_peak(L.PNOP_MIXED, 0.02)
    print(f"FMA probe: FP64 {f64:.3f} TFLOP/s, FP32 {f32:.2f} TFLOP/s on {nsm} SMs")
    assert 0 < f64 < f32
    if nsm == 152:  # GB300
        assert 0.6 < f64 < 1.4
        assert 30 < f32 < 90
