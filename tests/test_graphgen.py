"""Input generators: valid simple undirected CSR, determinism, expected sizes."""
import numpy as np
import pytest

import graphgen


def check_simple(g):
    assert g.off[0] == 0 and g.off[-1] == g.arcs and np.all(np.diff(g.off) >= 0)
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    assert np.all(g.adj >= 0) and np.all(g.adj < g.n)
    assert not np.any(src == g.adj), "self-loop"
    # strictly ascending inside every list (sorted, no duplicates)
    same = src[1:] == src[:-1]
    assert np.all(g.adj[1:][same] > g.adj[:-1][same])
    # symmetric
    fwd = src.astype(np.int64) * g.n + g.adj
    rev = g.adj.astype(np.int64) * g.n + src
    assert np.array_equal(np.sort(fwd), np.sort(rev))


def test_rmat_valid_and_deterministic():
    a = graphgen.rmat(14, 16, seed=3)
    b = graphgen.rmat(14, 16, seed=3)
    c = graphgen.rmat(14, 16, seed=4)
    check_simple(a)
    assert a.n == 1 << 14
    assert np.array_equal(a.off, b.off) and np.array_equal(a.adj, b.adj)
    assert not (a.arcs == c.arcs and np.array_equal(a.adj, c.adj))
    # 16 * 2^14 samples; duplicates and self-loops only remove edges
    assert 0.8 * 16 * (1 << 14) < a.edges <= 16 * (1 << 14)


def test_rmat_thread_count_does_not_matter():
    old = graphgen.set_threads(0)
    graphgen.set_threads(1)
    a = graphgen.rmat(12, 8, seed=9)
    graphgen.set_threads(old)
    b = graphgen.rmat(12, 8, seed=9)
    assert np.array_equal(a.adj, b.adj)


def test_permutation_is_bijection():
    p = graphgen.permutation(1000, 5)
    assert np.array_equal(np.sort(p), np.arange(1000))


def test_sbm_expected_edges():
    # 10,000 vertices in 50 blocks of 200, p_in 0.05, p_out 0.0004
    g = graphgen.sbm(10000, 50, 0.05, 0.0004, seed=1)
    check_simple(g)
    pin = 50 * 200 * 199 // 2
    pout = 10000 * 9999 // 2 - pin
    mean = pin * 0.05 + pout * 0.0004
    sd = (pin * 0.05 * 0.95 + pout * 0.0004 * 0.9996) ** 0.5
    assert abs(g.edges - mean) < 5 * sd
    # blocks are contiguous: most edges stay inside a block
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    inside = (src // 200) == (g.adj // 200)
    assert inside.mean() > 0.6


def test_sbm_extremes():
    g = graphgen.sbm(30, 3, 1.0, 0.0, seed=1)
    check_simple(g)
    assert g.edges == 3 * 45
    g = graphgen.sbm(30, 3, 0.0, 0.0, seed=1)
    assert g.arcs == 0


def test_batch_params_ranges():
    ps = graphgen.batch_sbm_params(300, seed=2)
    assert all(100 <= p.n <= 20000 for p in ps)
    assert all(2 <= p.blocks <= 64 for p in ps)
    assert all(0.02 <= p.p_in <= 0.2 and p.p_out == pytest.approx(p.p_in / 50) for p in ps)
    assert len({p.seed for p in ps}) == 300


def test_from_edges_cleans():
    g = graphgen.from_edges(4, [(0, 1), (1, 0), (2, 2), (3, 1), (0, 1)])
    check_simple(g)
    assert g.edges == 2
