"""The benchmark's FMA-throughput probe (the measured denominators of the
ALU rooflines) runs and gives rates within a factor of two of GB300's
nominal FP64 and FP32 multiply-add throughput."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_probe_rates():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_00762_gb300 import build
    build.build()
    import bench
    r = bench.fma_peaks()
    assert r is not None
    print(f"FMA probe: FP64 {r[64]:.0f} GFLOP/s, FP32 {r[32]:.0f} GFLOP/s")
    assert 0.5 * bench.FP64_PEAK_NOMINAL < r[64] < 2.0 * bench.FP64_PEAK_NOMINAL
    assert 0.5 * bench.FP32_PEAK_NOMINAL < r[32] < 2.0 * bench.FP32_PEAK_NOMINAL
