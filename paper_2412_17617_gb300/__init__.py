"""GB300-native pre-computed MoM candidate evaluator (arXiv 2412.17617 hot path).

The compute lives in the CUDA library built from csrc/ (C ABI in include/pmom.h); `pmom`
is its thin ctypes binding.
"""
from .pmom import Evaluator, band_codes, load_library, PmomError  # noqa: F401
