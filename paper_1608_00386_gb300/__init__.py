"""GB300-native MCAO closed-loop step (arXiv:1608.00386 hot path).

``mcao`` is the ctypes binding of libmcao.so (C ABI in include/mcao.h); ``build`` compiles it
for sm_103a; ``inputs`` draws the seeded synthetic configurations, screens and reconstructors.
"""
from . import build, inputs  # noqa: F401
from .mcao import McaoError, Sim, make_sim  # noqa: F401
