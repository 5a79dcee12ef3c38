"""Pipe throughput probes used as roofline denominators: they run and give rates in the range a
GB300-class part allows (the exact figures are reported by bench.py, not asserted here)."""
import os

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_10270_gb300 as pkg
    if not os.path.exists(pkg.LIB_PATH):
        from paper_1811_10270_gb300 import build
        build.build()
    pkg.lib()
    return pkg


def test_probes_report_plausible_rates(S):
    # (kind, short iteration count, lower bound, upper bound) in ops/s
    cases = [(S.PROBE_FFMA, 20000, 5e12, 2e14), (S.PROBE_DFMA, 300, 1e11, 1e13),
             (S.PROBE_RSQRT, 2500, 5e11, 5e13), (S.PROBE_HMMA_BF16, 30000, 5e13, 5e15),
             (S.PROBE_DMMA_F64, 300, 1e11, 1e13)]
    for kind, iters, lo, hi in cases:
        rate, ms = S.probe_peak(kind, iters)
        assert ms > 0 and lo < rate < hi, (kind, rate)
    with pytest.raises(S.ShbimError):
        S.probe_peak(99, 10)
