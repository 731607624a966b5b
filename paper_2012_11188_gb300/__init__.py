"""GB300-native index-based SCAN (Tseng, Dhulipala, Shun, SIGMOD 2021).

The computation lives in the CUDA library libscan.so (C ABI in include/scan.h);
this package builds it in-tree and exposes a thin ctypes binding.
"""
from .scan import (COSINE, COUNTS_AUTO, COUNTS_DENSE, COUNTS_SPARSE, DEFAULT_COUNT_CONFIG, JACCARD,
                   Q_HUBS, ScanError,
                   ScanIndex, Server, autotune_batch, closed_counts_range, count_config_for,
                   kernel_launches,
                   last_count_kernel_ms,
                   last_build_timings, library_path, load, make_lsh, paper_sigma,
                   set_count_config, set_wide_index, sort_segments_desc, tuning_clear, tuning_load,
                   tuning_save,
                   use_torch_allocator)
from ._build import build

__all__ = ["COSINE", "COUNTS_AUTO", "COUNTS_DENSE", "COUNTS_SPARSE", "DEFAULT_COUNT_CONFIG",
           "JACCARD", "Q_HUBS",
           "ScanError", "ScanIndex", "Server", "autotune_batch", "build", "closed_counts_range",
           "count_config_for",
           "kernel_launches", "last_build_timings", "last_count_kernel_ms", "library_path", "load",
           "make_lsh",
           "paper_sigma", "set_count_config", "set_wide_index", "sort_segments_desc",
           "tuning_clear", "tuning_load",
           "tuning_save", "use_torch_allocator"]
