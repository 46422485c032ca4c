"""The library's microbenchmarks (include/tcbf_peak.h), measurement
infrastructure behind the benchmark's roofline denominators: they run and
return plausible rates on the GPU."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_stream_mix_runs():
    """An HBM stream of 0.25 GB read and 1 GB written: every block count
    finishes, above 100 GB/s and below 20 TB/s (no work skipped)."""
    from paper_2505_03269_gb300 import peaks
    r = peaks.stream(0.25, 1.0)
    for per_sm in (4, 8, 16):
        gbs = r[f"blocks_per_sm_{per_sm}"]["gbs"]
        assert 100 < gbs < 20000, (per_sm, gbs)


def test_fp16_tensor_peak_runs():
    """The kind::f16 M128 N256 microbenchmark: a positive rate below 5000
    TeraOps/s (the nominal dense peak is 2250)."""
    from paper_2505_03269_gb300 import peaks
    tops = peaks.measure(0)
    assert 100 < tops < 5000
