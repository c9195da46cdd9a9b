"""FP64 throughput probe (lbm_fp64_rates): the measured ceilings that the
FP64-bound step kernels are reported against."""
import pytest

torch = pytest.importorskip("torch")

from paper_1110_0270_gb300 import lbm  # noqa: E402

pytestmark = pytest.mark.gpu


def test_fp64_rates_are_measured_and_plausible():
    r = lbm.fp64_rates()
    # a GB300 runs FP64 FMAs at about 1.2 TFLOP/s and a log costs tens of
    # FMAs: both rates far from zero and below the FP32 tensor-free peak
    assert 1e10 < r["dfma_flops"] < 1e14, r
    assert 1e8 < r["log_per_s"] < r["dfma_flops"], r
