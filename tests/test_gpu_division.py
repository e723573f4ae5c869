"""The library's binary64 division on the integer units, bit for bit against
the hardware binary64 division over a few hundred million drawn operand pairs
(random significands, the rounding-deciding patterns, exponents across the
normal range and beyond, zeros, infinities and NaNs)."""
import pytest

from paper_2403_12345_gb300 import gbmc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [1, 2])
def test_integer_division_is_correctly_rounded(seed):
    ctx = gbmc.Context(0)
    try:
        bad, first = ctx.check_division(1 << 27, seed)
    finally:
        ctx.close()
    assert bad == 0, (bad, first)
