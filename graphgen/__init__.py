"""Seeded synthetic graph inputs: R-MAT and stochastic-block-model graphs as CSR.

This package is the single input producer for the CPU oracle, the tests and the
benchmark. It contains no part of the clustering method (no intersections,
similarities, orders or queries); see ``graphgen.c`` for the generator
definitions. Graphs are simple and undirected (Section 2.2 of the paper), with
each adjacency list sorted by vertex id; vertex ids are 0-based.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into a shared library (host C, OpenMP)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i64, u64, i32, f64 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    lib.gg_rmat.restype = P
    lib.gg_rmat.argtypes = [i32, i64, f64, f64, f64, u64, i32]
    lib.gg_sbm.restype = P
    lib.gg_sbm.argtypes = [i64, i64, f64, f64, u64]
    lib.gg_clean_pairs.restype = P
    lib.gg_clean_pairs.argtypes = [i64, i64, P, P]
    lib.gg_n.restype = i64
    lib.gg_n.argtypes = [P]
    lib.gg_arcs.restype = i64
    lib.gg_arcs.argtypes = [P]
    lib.gg_copy_out.restype = i32
    lib.gg_copy_out.argtypes = [P, P, P]
    lib.gg_free.restype = None
    lib.gg_free.argtypes = [P]
    lib.gg_key.restype = u64
    lib.gg_key.argtypes = [u64, u64]
    lib.gg_draw.restype = u64
    lib.gg_draw.argtypes = [u64, u64]
    lib.gg_uniform.restype = f64
    lib.gg_uniform.argtypes = [u64, u64]
    lib.gg_set_threads.restype = i32
    lib.gg_set_threads.argtypes = [i32]
    lib.gg_permutation.restype = i32
    lib.gg_permutation.argtypes = [i64, u64, P]
    _lib = lib
    return lib


@dataclass
class CSR:
    """Simple undirected graph: off int64[n+1], adj int32[arcs], lists id-sorted."""

    off: np.ndarray
    adj: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def arcs(self) -> int:
        return int(self.adj.shape[0])

    @property
    def edges(self) -> int:
        return self.arcs // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.off).astype(np.int64)

    def off32(self) -> np.ndarray:
        assert self.arcs < 2**31
        return self.off.astype(np.int32)


def _take(g) -> CSR:
    lib = _load()
    if not g:
        raise MemoryError("graph generation failed")
    try:
        n = lib.gg_n(g)
        arcs = lib.gg_arcs(g)
        off = np.empty(n + 1, dtype=np.int64)
        adj = np.empty(max(arcs, 0), dtype=np.int32)
        lib.gg_copy_out(g, off.ctypes.data, adj.ctypes.data)
    finally:
        lib.gg_free(g)
    return CSR(off, adj)


def rmat(scale: int, edgefactor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, permute: bool = True) -> CSR:
    """R-MAT graph with 2**scale vertices from edgefactor * 2**scale samples, cleaned."""
    g = _take(_load().gg_rmat(scale, edgefactor, a, b, c, seed, 1 if permute else 0))
    g.name = f"rmat-s{scale}-ef{edgefactor}-seed{seed}"
    return g


def sbm(n: int, blocks: int, p_in: float, p_out: float, seed: int = 1) -> CSR:
    """Stochastic block model: `blocks` near-equal contiguous blocks over n vertices."""
    g = _take(_load().gg_sbm(n, blocks, p_in, p_out, seed))
    g.name = f"sbm-n{n}-b{blocks}-seed{seed}"
    return g


def from_edges(n: int, edges) -> CSR:
    """Clean an explicit edge list (any order, duplicates and self-loops allowed)."""
    e = np.asarray(edges if isinstance(edges, np.ndarray) else list(edges),
                   dtype=np.int64).reshape(-1, 2)
    src = np.ascontiguousarray(e[:, 0].astype(np.int32))
    dst = np.ascontiguousarray(e[:, 1].astype(np.int32))
    return _take(_load().gg_clean_pairs(n, src.shape[0], src.ctypes.data, dst.ctypes.data))


def from_dense(A: np.ndarray) -> CSR:
    """CSR of the simple graph whose adjacency is the symmetric 0/1 matrix A."""
    n = A.shape[0]
    iu, ju = np.nonzero(np.triu(A, 1))
    return from_edges(n, zip(iu.tolist(), ju.tolist()))


def _mix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea and Flood 2014), elementwise on uint64."""
    x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return x ^ (x >> np.uint64(31))


def edge_weights(g: CSR, seed: int = 1, dist: str = "uniform") -> np.ndarray:
    """Symmetric per-arc weights, aligned with g.adj: both arcs of an edge
    {a, b} carry the value drawn from the hash of (min, max, seed).

    dist: "uniform" (U[0.05, 3)), "int" (1, 2, 3 or 4) or "exp" (0.01 plus an
    exponential of mean 1, a heavier tail)."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.off))
    dst = g.adj.astype(np.int64)
    lo, hi = np.minimum(src, dst).astype(np.uint64), np.maximum(src, dst).astype(np.uint64)
    with np.errstate(over="ignore"):
        k = lo * np.uint64(0x9E3779B97F4A7C15) ^ (hi + np.uint64(seed) * np.uint64(0xD1B54A32D192ED03))
        u = (_mix64(_mix64(k)) >> np.uint64(11)).astype(np.float64) * (1.0 / 2**53)
    if dist == "uniform":
        return 0.05 + 2.95 * u
    if dist == "int":
        return 1.0 + np.floor(4.0 * u)
    if dist == "exp":
        return 0.01 - np.log1p(-u)
    raise ValueError(dist)


def permutation(n: int, seed: int) -> np.ndarray:
    p = np.empty(n, dtype=np.int32)
    _load().gg_permutation(n, seed, p.ctypes.data)
    return p


def uniform(key: int, ctr: int) -> float:
    return float(_load().gg_uniform(key, ctr))


def key(seed: int, tag: int) -> int:
    return int(_load().gg_key(seed, tag))


def draw(key_: int, ctr: int) -> int:
    return int(_load().gg_draw(key_, ctr))


def set_threads(t: int) -> int:
    return int(_load().gg_set_threads(t))


@dataclass
class SBMParams:
    n: int
    blocks: int
    p_in: float
    p_out: float
    seed: int


def batch_sbm_params(count: int, seed: int = 1, n_lo: int = 100, n_hi: int = 20000,
                     b_lo: int = 2, b_hi: int = 64, p_lo: float = 0.02, p_hi: float = 0.2,
                     out_ratio: float = 50.0) -> list[SBMParams]:
    """Parameters of a batch of independent SBM graphs: n log-uniform in [n_lo, n_hi],
    blocks uniform in {b_lo..b_hi} (capped at n), p_in uniform in [p_lo, p_hi],
    p_out = p_in / out_ratio; per-graph seeds are distinct draws."""
    k = key(seed, 0x6261746368)  # "batch"
    out = []
    for i in range(count):
        u0, u1, u2 = uniform(k, 4 * i), uniform(k, 4 * i + 1), uniform(k, 4 * i + 2)
        n = int(round(math.exp(math.log(n_lo) + u0 * (math.log(n_hi) - math.log(n_lo)))))
        nb = min(n, b_lo + int(u1 * (b_hi - b_lo + 1)))
        p_in = p_lo + u2 * (p_hi - p_lo)
        gseed = draw(k, 4 * i + 3) & 0x7FFFFFFFFFFFFFFF
        out.append(SBMParams(n, nb, p_in, p_in / out_ratio, gseed))
    return out


def batch_queries(count: int, per_graph: int = 8, seed: int = 1, mu_lo: int = 2, mu_hi: int = 16,
                  k_lo: int = 2, k_hi: int = 18):
    """(mu, eps) queries for a batch of graphs: per graph `per_graph` pairs with mu
    uniform in {mu_lo..mu_hi} and eps = k / 20 for k uniform in {k_lo..k_hi} (the
    0.05 grid, each value the correctly rounded double of the decimal).

    Returns (mus int32[count, per_graph], epss float64[count, per_graph])."""
    k = key(seed, 0x7175657279)  # "query"
    mus = np.empty((count, per_graph), dtype=np.int32)
    epss = np.empty((count, per_graph), dtype=np.float64)
    for i in range(count):
        for j in range(per_graph):
            c = 2 * (i * per_graph + j)
            mus[i, j] = mu_lo + draw(k, c) % (mu_hi - mu_lo + 1)
            epss[i, j] = (k_lo + draw(k, c + 1) % (k_hi - k_lo + 1)) / 20.0
    return mus, epss
