"""GB300-native maximal biclique enumeration (arXiv 2401.05039, MBEA on the GPU).

The computation lives in the CUDA library built from ``csrc/`` (C ABI in
``include/mbe.h``); ``mbe`` is its ctypes binding.
"""
from . import build  # noqa: F401
from .mbe import (Bicliques, BicliqueBuffer, Graph, MBEError, Options, Result, copy_bandwidth,  # noqa: F401
                  enumerate_batch, enumerate_noalloc, library_path, load, options, release_workspace)
