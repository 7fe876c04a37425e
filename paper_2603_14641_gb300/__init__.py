"""GB300-native stabilizer-tableau simulator (arXiv 2603.14641 hot path).

The compute path is libqs.so (hand-written CUDA for sm_103a, C ABI in
include/qs.h); `paper_2603_14641_gb300.qs` is its Python binding.
"""
from . import qs  # noqa: F401
from .qs import Simulator, QsError  # noqa: F401
