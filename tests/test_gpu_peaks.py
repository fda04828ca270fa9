"""The measured FMA throughput (denominator of the ALU rooflines) is
plausible for the device: FP32 within the range set by the SM count, 128
FP32 lanes per SM and the maximum SM clock, FP64 below FP32."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2005_08736_gb300.solver import measure_fp_peaks  # noqa: E402


def test_measured_fma_peaks_are_plausible():
    p = measure_fp_peaks()
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12  # upper bound, 2.2 GHz
    print(p, f"nominal bound {nominal:.1f}")
    assert 0.3 * nominal < p["fp32"] <= nominal
    assert 0.3 * nominal < p["fp32x2"] <= 2 * nominal
    assert 0.0 < p["fp64"] < p["fp32"]
