"""Pins of the oracle's weighted cosine similarity (Section 4.1.1,
WeightedCosineSim of closed neighbourhoods with w(x, x) = 1).

The oracle walks the two closed lists with two pointers; the pins reach the
same numbers another way: the matrix identity of Section 4.1.1 with W[x][x]
= 1 ((W^2)[u][v] is the numerator and (W^2)[x][x] the squared norm), the
reduction to the unweighted cosine when every weight is 1, exact symmetry,
and a hand-computed triangle.
"""
import math

import numpy as np
import pytest

import graphgen
import oracle


def random_weights(g, seed):
    """Symmetric positive weights: w(u,v) = w(v,u) drawn once per edge."""
    rng = np.random.default_rng(seed)
    off, adj = g.off, g.adj
    src = np.repeat(np.arange(g.n), np.diff(off))
    lo, hi = np.minimum(src, adj), np.maximum(src, adj)
    key = lo.astype(np.int64) * g.n + hi
    uniq, inv = np.unique(key, return_inverse=True)
    per_edge = rng.uniform(0.05, 3.0, size=uniq.shape[0])
    return per_edge[inv]


@pytest.mark.parametrize("n,p,seed", [(30, 0.2, 1), (60, 0.1, 2), (25, 0.6, 3)])
def test_weighted_equals_matrix_identity(n, p, seed):
    g = graphgen.sbm(n, 1, p, p, seed=seed)
    w = random_weights(g, seed)
    W = np.eye(g.n)
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    W[src, g.adj] = w
    W2 = W @ W
    want = W2[src, g.adj] / np.sqrt(np.diag(W2)[src] * np.diag(W2)[g.adj])
    got = oracle.weighted_similarities(g, w)
    assert np.allclose(got, want, rtol=1e-13, atol=0)


def test_unit_weights_reduce_to_cosine():
    g = graphgen.sbm(200, 4, 0.2, 0.02, seed=5)
    got = oracle.weighted_similarities(g, np.ones(g.arcs))
    want = oracle.similarities(g, oracle.closed_counts(g), oracle.COSINE)
    assert np.allclose(got, want, rtol=4e-16, atol=0)


def test_weighted_symmetric():
    g = graphgen.sbm(120, 3, 0.3, 0.03, seed=6)
    w = random_weights(g, 6)
    sim = oracle.weighted_similarities(g, w)
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    pos = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(src, g.adj))}
    for (a, b), i in pos.items():
        assert sim[i] == sim[pos[(b, a)]]


def test_weighted_triangle_closed_form():
    # u=0, v=1, x=2: w(u,v)=a, w(u,x)=b, w(v,x)=c
    a, b, c = 0.5, 2.0, 1.5
    g = graphgen.from_edges(3, [(0, 1), (0, 2), (1, 2)])
    w = np.empty(g.arcs)
    weight = {(0, 1): a, (0, 2): b, (1, 2): c}
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    for i, (s, t) in enumerate(zip(src, g.adj)):
        w[i] = weight[(min(s, t), max(s, t))]
    sim = oracle.weighted_similarities(g, w)
    i01 = int(np.flatnonzero((src == 0) & (g.adj == 1))[0])
    want = (2 * a + b * c) / (math.sqrt(1 + a * a + b * b) * math.sqrt(1 + a * a + c * c))
    assert abs(sim[i01] - want) <= 1e-15 * want


@pytest.mark.parametrize("seed", [1, 2])
def test_vertex_routine_equals_matrix_identity_and_all_arcs(seed):
    """The per-vertex routine (sampled checks on large graphs) against the
    matrix identity, and bit for bit against the all-arcs routine, whose
    numerators add the same terms in the same (id) order."""
    g = graphgen.sbm(80, 2, 0.3, 0.05, seed=seed)
    w = graphgen.edge_weights(g, seed, "exp")
    W = np.eye(g.n)
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    W[src, g.adj] = w
    W2 = W @ W
    full = oracle.weighted_similarities(g, w)
    for v in range(g.n):
        row = slice(g.off[v], g.off[v + 1])
        got = oracle.weighted_vertex_similarities(g, w, v)
        nb = g.adj[row]
        want = W2[v, nb] / np.sqrt(W2[v, v] * np.diag(W2)[nb])
        assert np.allclose(got, want, rtol=1e-13, atol=0)
        assert np.array_equal(got, full[row])


def test_weighted_bipartite_closed_form():
    """K_{a,b} with one weight c on every edge has no triangles: the common
    closed neighbourhood of an edge is its two ends, so
    sigma = 2c / (sqrt(1 + b c^2) sqrt(1 + a c^2))."""
    a, b, c = 5, 7, 1.75
    g = graphgen.from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)])
    w = np.full(g.arcs, c)
    want = 2 * c / (math.sqrt(1 + b * c * c) * math.sqrt(1 + a * c * c))
    sim = oracle.weighted_similarities(g, w)
    assert np.allclose(sim, want, rtol=1e-15, atol=0)
    assert np.allclose(oracle.weighted_vertex_similarities(g, w, 0), want, rtol=1e-15, atol=0)


def test_edge_weights_are_symmetric_and_in_range():
    g = graphgen.rmat(10, 8, seed=3)
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    order = np.lexsort((g.adj, src))
    rev = np.lexsort((src, g.adj))  # arc (b, a) at the place of (a, b)
    for dist, lo, hi in (("uniform", 0.05, 3.0), ("int", 1.0, 4.0), ("exp", 0.01, 50.0)):
        w = graphgen.edge_weights(g, 9, dist)
        assert np.array_equal(w[order], w[rev])
        assert w.min() >= lo and w.max() <= hi
    assert set(np.unique(graphgen.edge_weights(g, 9, "int"))) <= {1.0, 2.0, 3.0, 4.0}
