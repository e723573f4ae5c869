"""GB300-native event-based continuous-energy Monte Carlo transport hot path.

The compute runs in libgbmc.so (hand-written CUDA for sm_103a behind the C
ABI of include/gbmc.h); `gbmc` is its Python binding.
"""
from . import gbmc  # noqa: F401
from .gbmc import Context, geometry, geometry_from, problem  # noqa: F401
