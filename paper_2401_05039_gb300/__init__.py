"""GB300-native maximal biclique enumeration (arXiv 2401.05039, MBEA on the GPU).

The computation lives in the CUDA library built from ``csrc/`` (C ABI in
``include/mbe.h``); ``mbe`` is its ctypes binding.
"""
from . import build  # noqa: F401
from .mbe import (N_CLASSES, Bicliques, BicliqueBuffer, ClassParams, Graph, MBEError, Model, Options,  # noqa: F401
                  Result, autotune_batch, batch_class, copy_bandwidth, enumerate_batch, enumerate_noalloc,
                  library_path, load, options, release_workspace, training_set, shard_bounds, allreduce_totals,
                  sharded_enumerate, lpt_shards, static_root_cost)
