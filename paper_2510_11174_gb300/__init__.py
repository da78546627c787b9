"""GB300-native hybrid fluid-kinetic laser-plasma step (arXiv 2510.11174).

The compute path is libhyb.so (hand-written CUDA for sm_103a, C ABI in
include/hyb.h); this package is its thin Python binding plus seeded input
generators.
"""
from ._abi import HybError, load  # noqa: F401
from .sim import Batch, Simulation  # noqa: F401
from .model import Classifier, Surrogate, SwitchNet  # noqa: F401
