"""GB300-native multibody acoustic scattering via MFS scattering matrices.

The compute path lives in libmbs.so (hand-written CUDA for sm_103a behind the
C ABI of include/mbs.h); this package is its Python binding.  Importing the
package does not load the library; the first call does, and fails loudly if
the library has not been built (there is no CPU fallback).
"""
from .api import (  # noqa: F401
    PREC_FP32,
    PREC_FP64,
    PREC_MIXED,
    Context,
    MbsError,
    Server,
    default_options,
    launch_count,
    measure_peaks,
    shapes_bodies_from_workload,
)
from . import _lib  # noqa: F401


def load_library():
    """Load libmbs.so (raises ImportError if it is missing)."""
    return _lib.load()
