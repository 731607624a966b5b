"""GB300-native index-based SCAN (Tseng, Dhulipala, Shun, SIGMOD 2021).

The computation lives in the CUDA library libscan.so (C ABI in include/scan.h);
this package builds it in-tree and exposes a thin ctypes binding.
"""
from .scan import (COSINE, COUNTS_AUTO, COUNTS_DENSE, COUNTS_SPARSE, JACCARD, Q_HUBS, ScanError,
                   ScanIndex, Server, kernel_launches, last_build_timings, library_path, load,
                   make_lsh, paper_sigma, set_wide_index, use_torch_allocator)
from ._build import build

__all__ = ["COSINE", "COUNTS_AUTO", "COUNTS_DENSE", "COUNTS_SPARSE", "JACCARD", "Q_HUBS",
           "ScanError", "ScanIndex", "Server", "build", "kernel_launches", "last_build_timings",
           "library_path", "load", "make_lsh", "paper_sigma", "set_wide_index",
           "use_torch_allocator"]
