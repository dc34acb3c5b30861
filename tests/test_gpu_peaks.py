"""The throughput probes behind the roofline denominators (qlr_peak_probe): every kind runs and
reports a positive rate; the MMA loop of N = 64 runs at most at the dense rate's share, since an
MMA of M = 128 takes at least as long as one of N ~ 100 (so a thin sketch's MMA width, not the
dense peak, bounds its tensor time); argument errors are reported without a launch."""
import pytest

from paper_2507_13731_gb300 import qlr


def test_peak_probe_rejects_bad_arguments():
    with pytest.raises(qlr.QlrError):
        qlr.peak_probe(99, 0, 10)
    with pytest.raises(qlr.QlrError):
        qlr.peak_probe(qlr.PEAK_TF32_MMA, 0, 0)
    with pytest.raises(qlr.QlrError):
        qlr.peak_probe(qlr.PEAK_BF16_MMA_N64, 0, 400001)


@pytest.mark.gpu
def test_peak_probes_run_and_order():
    r = {k: qlr.measure_peak(k, 0, target_ms=10.0, reps=2) for k in
         (qlr.PEAK_TF32_MMA, qlr.PEAK_BF16_MMA, qlr.PEAK_TF32_MMA_N64, qlr.PEAK_BF16_MMA_N64, qlr.PEAK_FP32_FMA)}
    assert all(v > 0 for v in r.values())
    # BF16 runs K = 16 per MMA where TF32 runs K = 8: about twice the rate at the same N
    assert 1.5 < r[qlr.PEAK_BF16_MMA] / r[qlr.PEAK_TF32_MMA] < 2.5
    # N = 64: at most the N = 256 rate, and no faster than N ~ 100 would allow
    for dense, n64 in ((qlr.PEAK_TF32_MMA, qlr.PEAK_TF32_MMA_N64), (qlr.PEAK_BF16_MMA, qlr.PEAK_BF16_MMA_N64)):
        assert r[n64] < 0.8 * r[dense]
    assert r[qlr.PEAK_FP32_FMA] < r[qlr.PEAK_TF32_MMA]
