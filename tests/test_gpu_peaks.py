"""The measured FMA peaks (hfd_measure_fma_peaks) that the FP64 path's arithmetic roofline uses."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_measured_fma_peaks_are_plausible_for_the_device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_01286_gb300 import measure_fma_peaks
    m = measure_fma_peaks()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    assert m["sm_count"] == props.multi_processor_count
    # per SM and clock: at most 64 FP64 and 128 FP32 FMAs on any current NVIDIA part, at most
    # 2.2 GHz; FP32 must outrun FP64 (GB300 issues FP32 FMAs many times faster)
    per_sm_ghz = 2.2e9 * m["sm_count"] * 2
    assert 0 < m["fp64_flops"] <= 64 * per_sm_ghz
    assert 0 < m["fp32_flops"] <= 128 * per_sm_ghz
    assert m["fp32_flops"] > 4 * m["fp64_flops"]
    again = measure_fma_peaks()
    assert abs(again["fp64_flops"] - m["fp64_flops"]) < 0.1 * m["fp64_flops"]
