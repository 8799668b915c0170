"""GB300-native bitslice custom-precision floating point (arXiv 1602.04716).

The compute path is libbsfp.so (CUDA for sm_103a, C ABI in include/bsfp.h);
this package is its thin Python binding.
"""
from .bsfp import *  # noqa: F401,F403
from .bsfp import BsfpError, Format, bsfp_format  # noqa: F401
