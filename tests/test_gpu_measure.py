"""The measured FP64 FMA rate (mfs_fp64_rate), the denominator of the float64
kernels' roofline.  GB300's nominal FP64 rate is about 1.25 TFLOP/s (152 SMs
at up to 2.07 GHz); the measurement must land in a physically plausible band
around it and repeat within a few per cent.  Needs a GB300.
"""
import pytest

torch = pytest.importorskip("torch")

from paper_1605_01522_gb300 import mfs

pytestmark = pytest.mark.gpu


def test_fp64_rate_is_plausible_and_repeatable():
    a = mfs.fp64_rate()
    b = mfs.fp64_rate()
    assert 0.3 < a < 4.0, a
    assert abs(a - b) <= 0.1 * max(a, b), (a, b)
