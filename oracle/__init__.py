"""CPU oracle for index-based SCAN -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA library
and never imports it. The arithmetic lives in ``scan_oracle.cpp`` (exact path)
and ``lsh_oracle.cpp`` (sketches); this module only compiles them and marshals
numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("scan_oracle.cpp", "lsh_oracle.cpp")]
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None

COSINE, JACCARD = 0, 1
FLAG_HUBS = 1


def build(force: bool = False) -> str:
    srcs = [s for s in _SRCS if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    cmd = ["g++", "-O2", "-std=c++17", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared",
           *srcs, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        _lib = bind(ctypes.CDLL(build()))
    return _lib


def bind(lib):
    """Attach argument and result types to a loaded oracle library."""
    P, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "orc_closed_counts": (i32, [i64, P, P, P]),
        "orc_count_pairs": (i32, [i64, P, P, i64, P, P, P]),
        "orc_similarities": (i32, [i32, i64, P, P, P, P]),
        "orc_weighted_similarities": (i32, [i64, P, P, P, P]),
        "orc_weighted_vertex_similarities": (i32, [i64, P, P, P, i32, P]),
        "orc_neighbor_order": (i32, [i64, P, P, P, P, P]),
        "orc_core_order": (i32, [i64, P, P, i64, P, P, P]),
        "orc_query_index": (i32, [i64, P, P, P, P, i64, P, P, P, i32, f64, i32, P]),
        "orc_query_definition": (i32, [i64, P, P, P, i32, f64, i32, P]),
        "orc_vertex_similarities": (i32, [i32, i64, P, P, i32, P]),
        "orc_ari": (f64, [i64, P, P]),
        "orc_modularity": (f64, [i64, P, P, P]),
    }
    if os.path.exists(_SRCS[1]):
        u64 = ctypes.c_uint64
        sig.update({
            "orc_lsh_select": (i64, [i64, P, P, i64, P]),
            "orc_simhash_sketch": (i32, [i64, P, P, P, i64, i32, u64, P]),
            "orc_simhash_sketch_weighted": (i32, [i64, P, P, P, P, i64, i32, u64, P]),
            "orc_minhash_sketch": (i32, [i64, P, P, P, i64, i32, i32, u64, P]),
            "orc_lsh_similarities": (i32, [i32, i64, P, P, P, P, P, i32, i32, i32, P]),
            "orc_simhash_table": (i32, [i32, P]),
            "orc_splitmix64": (u64, [u64, u64]),
        })
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data


def _csr(g):
    off = np.ascontiguousarray(g.off, dtype=np.int64)
    adj = np.ascontiguousarray(g.adj, dtype=np.int32)
    return off, adj


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def closed_counts(g) -> np.ndarray:
    off, adj = _csr(g)
    cnt = np.zeros(g.arcs, dtype=np.int32)
    _check(_load().orc_closed_counts(g.n, _p(off), _p(adj), _p(cnt)), "closed_counts")
    return cnt


def count_pairs(g, us, vs) -> np.ndarray:
    off, adj = _csr(g)
    us = np.ascontiguousarray(us, dtype=np.int32)
    vs = np.ascontiguousarray(vs, dtype=np.int32)
    out = np.zeros(us.shape[0], dtype=np.int32)
    _check(_load().orc_count_pairs(g.n, _p(off), _p(adj), us.shape[0], _p(us), _p(vs), _p(out)),
           "count_pairs")
    return out


def similarities(g, cnt: np.ndarray, kind: int = COSINE) -> np.ndarray:
    off, adj = _csr(g)
    cnt = np.ascontiguousarray(cnt, dtype=np.int32)
    sim = np.zeros(g.arcs, dtype=np.float64)
    _check(_load().orc_similarities(kind, g.n, _p(off), _p(adj), _p(cnt), _p(sim)), "similarities")
    return sim


def weighted_similarities(g, w: np.ndarray) -> np.ndarray:
    """Weighted cosine similarity of every arc (Section 4.1.1, w(x, x) = 1)."""
    off, adj = _csr(g)
    w = np.ascontiguousarray(w, dtype=np.float64)
    assert w.shape[0] == g.arcs
    sim = np.zeros(g.arcs, dtype=np.float64)
    _check(_load().orc_weighted_similarities(g.n, _p(off), _p(adj), _p(w), _p(sim)),
           "weighted_similarities")
    return sim


def weighted_vertex_similarities(g, w: np.ndarray, v: int) -> np.ndarray:
    """Weighted cosine similarities of the arcs of vertex v (Section 4.1.1)."""
    off, adj = _csr(g)
    w = np.ascontiguousarray(w, dtype=np.float64)
    assert w.shape[0] == g.arcs
    d = int(off[v + 1] - off[v])
    out = np.zeros(d, dtype=np.float64)
    _check(_load().orc_weighted_vertex_similarities(g.n, _p(off), _p(adj), _p(w), v, _p(out)),
           "weighted_vertex_similarities")
    return out


def neighbor_order(g, sim: np.ndarray):
    off, adj = _csr(g)
    sim = np.ascontiguousarray(sim, dtype=np.float64)
    no_id = np.zeros(g.arcs, dtype=np.int32)
    no_sim = np.zeros(g.arcs, dtype=np.float64)
    _check(_load().orc_neighbor_order(g.n, _p(off), _p(adj), _p(sim), _p(no_id), _p(no_sim)),
           "neighbor_order")
    return no_id, no_sim


def max_degree(g) -> int:
    return int(np.diff(g.off).max()) if g.n > 0 else 0


def core_order(g, no_sim: np.ndarray):
    off, _ = _csr(g)
    maxdeg = max_degree(g)
    no_sim = np.ascontiguousarray(no_sim, dtype=np.float64)
    co_off = np.zeros(maxdeg + 1, dtype=np.int64)
    co_id = np.zeros(g.arcs, dtype=np.int32)
    co_thr = np.zeros(g.arcs, dtype=np.float64)
    _check(_load().orc_core_order(g.n, _p(off), _p(no_sim), maxdeg, _p(co_off), _p(co_id),
                                  _p(co_thr)), "core_order")
    return co_off, co_id, co_thr


class Index:
    """The oracle's own index: counts, similarities, NO and CO."""

    def __init__(self, g, kind: int = COSINE, cnt=None, sim=None):
        self.g, self.kind = g, kind
        self.cnt = closed_counts(g) if cnt is None and sim is None else cnt
        self.sim = similarities(g, self.cnt, kind) if sim is None else np.asarray(sim, np.float64)
        self.no_id, self.no_sim = neighbor_order(g, self.sim)
        self.co_off, self.co_id, self.co_thr = core_order(g, self.no_sim)
        self.maxdeg = max_degree(g)

    def query(self, mu: int, eps: float, hubs: bool = False) -> np.ndarray:
        g = self.g
        off, adj = _csr(g)
        labels = np.zeros(g.n, dtype=np.int32)
        _check(_load().orc_query_index(g.n, _p(off), _p(adj), _p(self.no_id), _p(self.no_sim),
                                       self.maxdeg, _p(self.co_off), _p(self.co_id),
                                       _p(self.co_thr), mu, eps, FLAG_HUBS if hubs else 0,
                                       _p(labels)), "query_index")
        return labels

    def query_definition(self, mu: int, eps: float, hubs: bool = False) -> np.ndarray:
        return query_definition(self.g, self.sim, mu, eps, hubs)


def query_definition(g, sim: np.ndarray, mu: int, eps: float, hubs: bool = False) -> np.ndarray:
    off, adj = _csr(g)
    sim = np.ascontiguousarray(sim, dtype=np.float64)
    labels = np.zeros(g.n, dtype=np.int32)
    _check(_load().orc_query_definition(g.n, _p(off), _p(adj), _p(sim), mu, eps,
                                        FLAG_HUBS if hubs else 0, _p(labels)), "query_definition")
    return labels


def vertex_similarities(g, v: int, kind: int = COSINE) -> np.ndarray:
    off, adj = _csr(g)
    d = int(off[v + 1] - off[v])
    out = np.zeros(d, dtype=np.float64)
    _check(_load().orc_vertex_similarities(kind, g.n, _p(off), _p(adj), v, _p(out)),
           "vertex_similarities")
    return out


def vertex_neighbor_order(g, v: int, kind: int = COSINE):
    """NO[v] alone: the neighbours of v stably sorted by non-increasing sigma."""
    s = vertex_similarities(g, v, kind)
    ids = g.adj[g.off[v]:g.off[v + 1]]
    order = np.argsort(-s, kind="stable")
    return ids[order].astype(np.int32), s[order]


def ari(a: np.ndarray, b: np.ndarray) -> float:
    a = np.ascontiguousarray(a, dtype=np.int32)
    b = np.ascontiguousarray(b, dtype=np.int32)
    return float(_load().orc_ari(a.shape[0], _p(a), _p(b)))


def modularity(g, labels: np.ndarray) -> float:
    off, adj = _csr(g)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    return float(_load().orc_modularity(g.n, _p(off), _p(adj), _p(labels)))


# ---------------------------------------------------------------- LSH mode
SIMHASH, MINHASH = 0, 1


def lsh_select(g, T: int = 128):
    """row[v] >= 0 numbers the sketched vertices (degree > T with a neighbour of degree > T)."""
    off, adj = _csr(g)
    row = np.zeros(g.n, dtype=np.int32)
    nH = int(_load().orc_lsh_select(g.n, _p(off), _p(adj), T, _p(row)))
    return row, nH


def simhash_sketch(g, row, nH: int, k: int, seed: int, weights=None) -> np.ndarray:
    """SimHash sketches of the sketched vertices; weights (per arc) selects the
    weighted closed neighbourhood."""
    off, adj = _csr(g)
    row = np.ascontiguousarray(row, dtype=np.int32)
    sig = np.zeros((max(nH, 0), k // 64), dtype=np.uint64)
    if weights is None:
        _check(_load().orc_simhash_sketch(g.n, _p(off), _p(adj), _p(row), nH, k, seed, _p(sig)),
               "simhash_sketch")
    else:
        w = np.ascontiguousarray(weights, dtype=np.float64)
        assert w.shape[0] == g.arcs
        _check(_load().orc_simhash_sketch_weighted(g.n, _p(off), _p(adj), _p(w), _p(row), nH, k,
                                                   seed, _p(sig)), "simhash_sketch_weighted")
    return sig


def minhash_sketch(g, row, nH: int, k: int, seed: int, kpartition: bool = True) -> np.ndarray:
    off, adj = _csr(g)
    row = np.ascontiguousarray(row, dtype=np.int32)
    mh = np.zeros((max(nH, 0), k), dtype=np.uint32)
    _check(_load().orc_minhash_sketch(g.n, _p(off), _p(adj), _p(row), nH, k,
                                      1 if kpartition else 0, seed, _p(mh)), "minhash_sketch")
    return mh


def splitmix64(key: int, c: int) -> int:
    """Output number c of the SplitMix64 stream whose state starts at key."""
    return int(_load().orc_splitmix64(key, c))


def simhash_table(k: int) -> np.ndarray:
    tab = np.zeros(k + 1, dtype=np.float64)
    _check(_load().orc_simhash_table(k, _p(tab)), "simhash_table")
    return tab


def lsh_similarities(g, scheme: int, row, sketch: np.ndarray, exact: np.ndarray, k: int,
                     kpartition: bool = True) -> np.ndarray:
    off, adj = _csr(g)
    row = np.ascontiguousarray(row, dtype=np.int32)
    sketch = np.ascontiguousarray(sketch)
    exact = np.ascontiguousarray(exact, dtype=np.float64)
    out = np.zeros(g.arcs, dtype=np.float64)
    _check(_load().orc_lsh_similarities(scheme, g.n, _p(off), _p(adj), _p(row), _p(sketch),
                                        _p(exact), k, 1 if kpartition else 0, 0, _p(out)),
           "lsh_similarities")
    return out


class LSHIndex(Index):
    """Oracle index in LSH mode: SimHash for cosine, MinHash for Jaccard (Section 5)."""

    def __init__(self, g, kind: int, k: int, T: int = 128, seed: int = 1,
                 kpartition: bool = True, exact_sim=None, weights=None):
        assert weights is None or kind == COSINE
        if exact_sim is not None:
            exact = exact_sim
        elif weights is not None:
            exact = weighted_similarities(g, weights)
        else:
            exact = similarities(g, closed_counts(g), kind)
        self.row, self.nH = lsh_select(g, T)
        if kind == COSINE:
            self.sketch = simhash_sketch(g, self.row, self.nH, k, seed, weights)
            sim = lsh_similarities(g, SIMHASH, self.row, self.sketch, exact, k)
        else:
            self.sketch = minhash_sketch(g, self.row, self.nH, k, seed, kpartition)
            sim = lsh_similarities(g, MINHASH, self.row, self.sketch, exact, k, kpartition)
        self.exact_sim = exact
        super().__init__(g, kind, cnt=None, sim=sim)
