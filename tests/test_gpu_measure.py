"""The library's FP32 FMA throughput measurement (the denominator of the tick
kernels' ALU roofline): a plausible rate for the device and argument checks."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_02318_gb300 import build, mpmi
    build.build()
    return mpmi


def test_fp32_peak_is_plausible(lib):
    import torch
    props = torch.cuda.get_device_properties(0)
    tflops = lib.measure_fp32_peak(0, 0.2)
    # 128 FP32 lanes x 2 flops per SM and cycle; clocks between 0.5 and 3.5 GHz
    per_sm_ghz = tflops * 1e3 / (props.multi_processor_count * 256)
    assert 0.5 < per_sm_ghz < 3.5, (tflops, per_sm_ghz)


def test_fp32_peak_argument_checks(lib):
    for bad in (0.0, -1.0, 11.0, float("nan")):
        with pytest.raises(lib.MpmiError) as e:
            lib.measure_fp32_peak(0, bad)
        assert e.value.code == -1
