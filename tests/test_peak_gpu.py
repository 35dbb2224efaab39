"""kf_measure_peak: the measured FP32 and FP64 fused multiply-add rates used
as roofline denominators are plausible for the device (positive, FP32 well
above FP64, FP32 within the SM count x 128 lanes x 2 flop x a 3 GHz clock)."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible(cuda_ctx_factory):
    import torch
    from paper_1605_05508_gb300 import kf
    ctx = cuda_ctx_factory((4.0, 8.0, 12.0))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f32 = kf.kf_measure_peak(ctx, kf.PEAK_FP32)
    f64 = kf.kf_measure_peak(ctx, kf.PEAK_FP64)
    print(f"FP32 {f32 / 1e12:.1f} TFLOP/s, FP64 {f64 / 1e12:.2f} TFLOP/s on {sms} SMs")
    assert 0 < f64 < f32 <= sms * 128 * 2 * 3.0e9
    assert f32 > sms * 128 * 2 * 0.5e9  # at least half the lanes' rate at 1 GHz
    with pytest.raises(kf.KfError):
        kf.kf_measure_peak(ctx, 7)
