"""GB300-native (sm_103a) kd-tree construction and exact k-nearest-neighbour
query after PANDA (Patwary et al., arXiv 1607.08220).

The compute path is the CUDA library ``_lib/libpanda.so`` behind the C ABI in
``include/panda.h``; :mod:`.panda` is its Python binding.  Build the library
with :func:`paper_1607_08220_gb300.build_ext.build`.
"""
from .panda import (Batch, PandaError, Server, Tree, build, build_host, kernel_launches, knn, knn_host,
                    knn_mean, knn_self, knn_self_host, knn_self_sync, knn_sync, knn_visits, knn_vote, load, load_tree, refit, save,
                    phase_times,
                    set_phase_timing, tune, tune_lookup, version)

__all__ = ["Batch", "PandaError", "Server", "Tree", "build", "build_host", "knn", "knn_host", "knn_self",
           "knn_self_host", "knn_self_sync", "knn_sync", "knn_visits", "knn_vote", "knn_mean", "load", "load_tree", "refit", "save", "phase_times",
           "set_phase_timing", "kernel_launches", "tune", "tune_lookup", "version"]
