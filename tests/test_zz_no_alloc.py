"""The allocation-free query entry point (scan_query_noalloc).

Some callers cannot allocate device memory while they serve a query -- their
device memory already belongs to their own pool, or an allocation could stall
a latency-critical loop. scan_query_noalloc answers the same (mu, eps) query
as scan_query using scratch compiled into the library, so it allocates
nothing. Here it is called through the C ABI twice in a row and must return
exactly the labels scan_query returns; an index above its vertex limit is
refused. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import paper_2012_11188_gb300 as gs

pytestmark = pytest.mark.gpu

MAX_VERTICES = 4194304  # SCAN_NOALLOC_MAX_VERTICES in include/scan.h


def noalloc_fn():
    lib = gs.load()
    f = lib.scan_query_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_size_t]
    return f


def test_noalloc_query_equals_scan_query_on_consecutive_calls():
    import torch
    f = noalloc_fn()
    g = graphgen.rmat(15, 16, seed=7)
    stream = torch.cuda.current_stream()
    with gs.ScanIndex.build(g, gs.COSINE) as ix:
        labels = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
        for mu, eps, hubs in ((3, 0.4, True), (5, 0.6, False)):
            rc = f(ix._h, mu, eps, labels.data_ptr(), 1 if hubs else 0, stream.cuda_stream)
            assert rc == 0
            torch.cuda.synchronize()
            want = ix.query(mu, eps, hubs=hubs)
            assert np.array_equal(labels.cpu().numpy(), want), (mu, eps)


def test_noalloc_refuses_what_it_cannot_hold():
    import torch
    f = noalloc_fn()
    n = MAX_VERTICES + 1
    g = graphgen.CSR(np.zeros(n + 1, np.int64), np.zeros(0, np.int32))  # isolated vertices
    with gs.ScanIndex.build(g, gs.COSINE) as ix:
        labels = torch.empty(n, dtype=torch.int32, device="cuda")
        assert f(ix._h, 3, 0.5, labels.data_ptr(), 0, 0) == -1
    small = graphgen.from_edges(3, [(0, 1), (1, 2)])
    with gs.ScanIndex.build(small, gs.COSINE) as ix:
        host = np.empty(3, np.int32)
        assert f(ix._h, 2, 0.5, host.ctypes.data, 0, 0) == -1  # labels must be device memory
