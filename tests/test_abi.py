"""The C-ABI library builds, loads, and exports every symbol declared in include/*.h.

No compute call is made here (no GPU on this host); only calls that return
before touching the device (argument validation, status names).
"""
import ctypes
import glob
import os
import re

import pytest

import paper_2012_11188_gb300 as gs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(scan_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    # typedef'd function pointer types are not symbols
    return sorted(n for n in names if not n.endswith("_fn"))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("scan_index_build", "scan_query", "scan_query_batch", "scan_index_export",
                 "scan_index_free", "scan_strerror", "scan_index_build_batch"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(gs.library_path() if os.path.exists(gs.library_path()) else gs.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_argument_checks_without_gpu():
    lib = gs.load()
    assert lib.scan_strerror(0) == b"ok"
    assert lib.scan_strerror(-3) == b"not a simple undirected CSR graph"
    # NULL csr / NULL out are rejected before any device work
    h = ctypes.c_void_p()
    assert lib.scan_index_build(None, 0, None, 0, ctypes.byref(h)) == -1
    assert lib.scan_index_build(None, 0, None, 0, None) == -1
    assert lib.scan_query(None, 5, 0.5, None, 0, 0) == -1
    # allocator hooks must come in pairs
    assert lib.scan_set_allocator(ctypes.c_void_p(1), None, None) == -1
    assert lib.scan_set_allocator(None, None, None) == 0


def test_range_count_argument_checks_without_gpu():
    lib = gs.load()
    import graphgen
    from paper_2012_11188_gb300.scan import _csr_struct
    g = graphgen.from_edges(4, [(0, 1), (1, 2), (2, 0), (2, 3)])
    c, keep = _csr_struct(g, device=False)
    out = (ctypes.c_uint32 * g.arcs)()
    assert lib.scan_closed_counts_range(None, 0, 4, out, 0) == -1
    for v0, v1 in [(-1, 2), (3, 2), (0, 5)]:  # outside [0, n] or reversed
        assert lib.scan_closed_counts_range(ctypes.byref(c), v0, v1, out, 0) == -1
    assert lib.scan_closed_counts_range(ctypes.byref(c), 0, 4, None, 0) == -1
    del keep


def test_build_script_targets_sm103a():
    from paper_2012_11188_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.NVCC_FLAGS)


def test_weighted_argument_checks_without_gpu():
    """The weighted entry point rejects missing arguments before any device
    work, and the binding rejects weights of the wrong length or with a
    similarity or counting mode that weighted builds do not have."""
    import numpy as np

    import graphgen
    lib = gs.load()
    h = ctypes.c_void_p()
    assert lib.scan_index_build_weighted(None, None, None, 0, ctypes.byref(h)) == -1
    assert lib.scan_index_build_weighted(None, None, None, 0, None) == -1
    g = graphgen.from_edges(4, [(0, 1), (1, 2), (2, 3)])
    c, keep = gs.scan._csr_struct(g, False)
    # arcs but no weights
    assert lib.scan_index_build_weighted(ctypes.byref(c), None, None, 0, ctypes.byref(h)) == -1
    w = np.ones(g.arcs)
    with pytest.raises(ValueError):
        gs.ScanIndex.build(g, gs.COSINE, weights=w[:-1])
    with pytest.raises(gs.ScanError):
        gs.ScanIndex.build(g, gs.JACCARD, weights=w)
    with pytest.raises(gs.ScanError):
        gs.ScanIndex.build(g, gs.COSINE, counts=gs.COUNTS_DENSE, weights=w)


def test_count_config_table_on_the_host(tmp_path):
    """Counting configurations and the tuning table (host-side only)."""
    gs.tuning_clear()
    gs.set_count_config(None)
    default = dict(gs.DEFAULT_COUNT_CONFIG)
    # class of a batch whose largest graph has 1000 vertices (10 bits) and whose
    # average degree is 20 (5 bits)
    assert gs.count_config_for(1000, 5000, 100000) == default
    for bad in ({"warp_deg": 8}, {"cta_chunk": 1000}, {"long_list": 0}, {"rounds": 5},
                {"dense_div": -1}, {"dense_min_n": 1}, {"dense_min_n": 70000}):
        with pytest.raises(gs.ScanError):
            gs.set_count_config(bad)
    with pytest.raises(gs.ScanError):
        gs.count_config_for(10, 5, 100)  # total below the largest graph
    f = tmp_path / "tune.txt"
    f.write_text("# comment\n10 5 256 2048 128 8 0 4096\n")
    gs.tuning_load(str(f))
    tuned = {"warp_deg": 256, "cta_chunk": 2048, "long_list": 128, "rounds": 8, "dense_div": 0,
             "dense_min_n": 4096}
    assert gs.count_config_for(1000, 5000, 100000) == tuned
    assert gs.count_config_for(1000, 5000, 200000) == default  # another class (average 40)
    # a process-wide setting wins over the table; missing fields take the defaults
    gs.set_count_config({"warp_deg": 1024})
    assert gs.count_config_for(1000, 5000, 100000) == {**default, "warp_deg": 1024}
    gs.set_count_config(None)
    # save and reload round trip; a malformed file changes nothing
    out = tmp_path / "saved.txt"
    gs.tuning_save(str(out))
    gs.tuning_clear()
    assert gs.count_config_for(1000, 5000, 100000) == default
    gs.tuning_load(str(out))
    assert gs.count_config_for(1000, 5000, 100000) == tuned
    bad = tmp_path / "bad.txt"
    bad.write_text("10 5 256 2048 128 8\n")
    with pytest.raises(gs.ScanError):
        gs.tuning_load(str(bad))
    assert gs.count_config_for(1000, 5000, 100000) == tuned
    with pytest.raises(gs.ScanError):
        gs.tuning_load(str(tmp_path / "missing.txt"))
    gs.tuning_clear()
