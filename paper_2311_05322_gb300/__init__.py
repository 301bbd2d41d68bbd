"""GB300-native hot path of the microwave-tomography method of arXiv 2311.05322.

The compute path is libmw.so (hand-written sm_103a CUDA behind a C ABI, declared in
include/mw.h); `mw` is its thin ctypes binding.  Importing the binding does not load the
library; `mw.load_library()` (called by `mw.Context`) fails loudly when it is not built.
"""
from . import mw  # noqa: F401

__all__ = ["mw"]
