"""The stencils divide by 5 and 7 with Markstein's correction step instead of
an IEEE division; the sequence must give the correctly rounded quotient for
every float input (checked on the device against __fdiv_rn, all 2^32 bit
patterns)."""
import ctypes as C

import pytest

from paper_2202_05549_gb300 import _lib as L


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.gpu
@pytest.mark.parametrize("divisor", [5, 7])
def test_constant_division_is_correctly_rounded_for_every_float(divisor):
    bad = C.c_uint64(123)
    assert L.load().lt_selftest_div_const(0, divisor, C.byref(bad)) == L.LT_OK
    assert bad.value == 0


def test_selftest_rejects_other_divisors():
    bad = C.c_uint64(0)
    assert L.load().lt_selftest_div_const(0, 3, C.byref(bad)) == L.LT_ERR_INVALID_ARG
