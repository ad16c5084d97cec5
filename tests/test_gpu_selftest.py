"""The library's exact float -> double widening (used by every double-precision inner
product of the count rule, Def. 1) against the GPU's own conversion, over all 2^32 float
bit patterns: normals, subnormals, signed zeros, infinities and NaNs."""
import pytest

pytestmark = pytest.mark.gpu


def test_f2d_widening_matches_hardware(sah):
    assert sah.selftest_f2d() == 0
