"""The library's binary64 division on the integer units, bit for bit against
the hardware binary64 division:
- kind 0: div_rn over a few hundred million drawn operand pairs (random
  significands, the rounding-deciding patterns, exponents across the normal
  range and beyond, zeros, infinities and NaNs);
- kind 1: the lookup's interpolation factor (E - e0) / (e1 - e0) formed from
  the binary64 interval records (exact integer E - e0, table reciprocal)
  over grid-like intervals, E at, next to, inside, below and above them."""
import pytest

from paper_2403_12345_gb300 import gbmc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,seed", [(0, 1), (0, 2), (1, 1), (1, 2)])
def test_integer_division_is_correctly_rounded(kind, seed):
    ctx = gbmc.Context(0)
    try:
        bad, first = ctx.check_division(1 << 27, seed, kind=kind)
    finally:
        ctx.close()
    assert bad == 0, (bad, first)
