"""GPU parity: the CUDA library through its C ABI against the CPU oracle.

Exact mode is compared bit for bit: closed counts and similarities (IEEE
doubles), the neighbour order, the core order and every label of every query.
Graphs are sized so the oracle finishes in seconds while the GPU path still
runs every kernel variant: warp, block and merge-path segment sorts (rows
longer than 4096), the shared-memory and the global (out-degree > 4096)
counting kernels, ragged tails, isolated vertices and empty graphs.
"""
import itertools
import math
import os

import numpy as np
import pytest

import graphgen
import oracle
import paper_2012_11188_gb300 as gs

pytestmark = pytest.mark.gpu

EPS_GRID = [k / 10 for k in range(1, 10)]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def build(g, kind=gs.COSINE, **kw):
    return gs.ScanIndex.build(g, kind, **kw)


def assert_index_equal(ix, ox):
    ex = ix.export()
    assert np.array_equal(ex["sim"], ox.sim), "similarities differ"
    assert np.array_equal(ex["no_id"], ox.no_id), "NO ids differ"
    assert np.array_equal(ex["no_sim"], ox.no_sim), "NO sims differ"
    assert np.array_equal(ex["co_off"], ox.co_off), "CO offsets differ"
    assert np.array_equal(ex["co_id"], ox.co_id), "CO ids differ"
    assert np.array_equal(ex["co_thr"], ox.co_thr), "CO thresholds differ"


def assert_queries_equal(ix, ox, mus, epss, hubs=True):
    for mu in mus:
        for eps in epss:
            got = ix.query(mu, eps, hubs=hubs)
            want = ox.query(mu, eps, hubs=hubs)
            assert np.array_equal(got, want), (mu, eps)


@pytest.mark.parametrize("kind", [gs.COSINE, gs.JACCARD])
def test_sbm_10k_full_parity(kind):
    # 10,000 vertices, 50 blocks of 200, p_in 0.05, p_out 0.0004
    g = graphgen.sbm(10000, 50, 0.05, 0.0004, seed=1)
    ox = oracle.Index(g, kind)
    with build(g, kind) as ix:
        assert (ix.n, ix.arcs, ix.maxdeg) == (g.n, g.arcs, ox.maxdeg)
        assert_index_equal(ix, ox)
        assert_queries_equal(ix, ox, [5], EPS_GRID)
        assert_queries_equal(ix, ox, [2, 3, 8, 16, ox.maxdeg + 1, ox.maxdeg + 2], [0.0, 0.2, 0.5, 1.0])
        # the index query also equals the definition-only query
        for eps in (0.1, 0.3, 0.5):
            assert np.array_equal(ix.query(5, eps, hubs=True), ox.query_definition(5, eps, hubs=True))


@pytest.mark.parametrize("kind", [gs.COSINE, gs.JACCARD])
def test_rmat_s16_full_parity(kind):
    # power-law rows longer than 4096 exercise the merge-path passes
    g = graphgen.rmat(16, 16, seed=2)
    assert np.diff(g.off).max() > 4096
    ox = oracle.Index(g, kind)
    with build(g, kind) as ix:
        assert_index_equal(ix, ox)
        assert_queries_equal(ix, ox, [2, 4, 8, 16, 32], [0.1, 0.3, 0.5, 0.7, 0.9])


def test_device_inputs_and_int32_offsets():
    import torch
    g = graphgen.rmat(12, 8, seed=3)
    ox = oracle.Index(g)
    off32 = torch.from_numpy(g.off.astype(np.int32)).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    with build((off32, adj)) as ix:
        assert_index_equal(ix, ox)
        lab = torch.empty(g.n, dtype=torch.int32, device="cuda")
        ix.query(3, 0.4, hubs=True, out=lab)
        assert np.array_equal(lab.cpu().numpy(), ox.query(3, 0.4, hubs=True))
    with build((g.off.astype(np.int32), g.adj)) as ix:
        assert_index_equal(ix, ox)


def test_query_batch_equals_single_queries():
    g = graphgen.sbm(3000, 15, 0.08, 0.002, seed=4)
    ox = oracle.Index(g)
    rng = np.random.default_rng(0)
    mus = rng.integers(2, 17, 40).astype(np.int32)
    epss = np.round(rng.integers(2, 19, 40) * 0.05, 2)
    with build(g) as ix:
        lab = ix.query_batch(mus, epss, hubs=True)
        for i in range(40):
            assert np.array_equal(lab[i], ox.query(int(mus[i]), float(epss[i]), hubs=True))
            assert np.array_equal(lab[i], ix.query(int(mus[i]), float(epss[i]), hubs=True))


def golden_graph(name):
    edges = []
    for line in open(os.path.join(GOLDEN, name)):
        f = line.split("#", 1)[0].split()
        if f and f[0] == "edge":
            edges.append((int(f[1]) - 1, int(f[2]) - 1))
    return graphgen.from_edges(max(max(e) for e in edges) + 1, edges)


def test_small_and_degenerate_graphs():
    cases = [
        graphgen.CSR(np.zeros(1, np.int64), np.zeros(0, np.int32)),          # n = 0
        graphgen.CSR(np.zeros(6, np.int64), np.zeros(0, np.int32)),          # no edges
        graphgen.from_edges(2, [(0, 1)]),                                     # one edge
        graphgen.from_edges(7, [(0, 1), (1, 2), (2, 0)]),                     # triangle + isolated
        graphgen.from_edges(6, [(0, 1), (0, 2), (0, 3), (1, 4), (1, 5)]),     # sigma = eps ties
        graphgen.from_edges(40, itertools.combinations(range(40), 2)),       # clique
        graphgen.from_edges(10001, [(0, i) for i in range(1, 10001)]),       # star, long row
        golden_graph("figure1_consistent.txt"),
        golden_graph("worked_example_sigma.txt"),
    ]
    for g in cases:
        for kind in (gs.COSINE, gs.JACCARD):
            ox = oracle.Index(g, kind)
            with build(g, kind) as ix:
                assert_index_equal(ix, ox)
                md = max(ox.maxdeg, 1)
                assert_queries_equal(ix, ox, [2, 3, md + 1, md + 2], [0.0, 0.5, 0.6, 0.75, 1.0])


def test_figure1_captions_on_gpu():
    g = golden_graph("figure1_consistent.txt")
    with build(g) as ix:
        lab = ix.query(3, 0.6, hubs=True)
    # captions of Figure 1 (paper ids 1..11 -> 0..10)
    assert list(lab) == [0, 0, 0, 0, -2, 5, 5, 5, -1, -1, 5]


def test_big_out_degree_closed_form():
    # complete bipartite K_{a,b}, a < b: every edge points from the b side to
    # the a side, so out-degree a > 4096 takes the global-memory counting path.
    # Closed form: N̄(u) ∩ N̄(v) = {u, v}, sigma = 2 / sqrt((a+1)(b+1)).
    a, b = 4200, 4300
    A = np.arange(a)
    B = np.arange(a, a + b)
    n = a + b
    off = np.zeros(n + 1, np.int64)
    off[1:a + 1] = b
    off[a + 1:] = a
    off = np.cumsum(off)
    adj = np.concatenate([np.tile(B, a), np.tile(A, b)]).astype(np.int32)
    g = graphgen.CSR(off, adj)
    with build(g) as ix:
        ex = ix.export()
    want = 2.0 / math.sqrt((a + 1) * (b + 1))
    assert np.all(ex["sim"] == want)
    # the oracle agrees on sampled rows
    for v in (0, a - 1, a, n - 1):
        assert np.array_equal(oracle.vertex_similarities(g, v), ex["sim"][off[v]:off[v + 1]])


def bad_graph(kind):
    g = graphgen.from_edges(5, [(0, 1), (1, 2), (2, 3), (3, 4), (0, 4)])
    off, adj = g.off.copy(), g.adj.copy()
    if kind == "unsorted":
        adj[off[1]:off[2]] = adj[off[1]:off[2]][::-1]
    elif kind == "selfloop":
        adj[0] = 0
    elif kind == "asymmetric":
        adj[off[0]] = 2  # 0 lists 2, but 2 does not list 0 (and 1 lists 0)
        adj[off[0]:off[1]] = np.sort(adj[off[0]:off[1]])
    elif kind == "range":
        adj[-1] = 9
    elif kind == "odd":
        return graphgen.CSR(np.array([0, 1, 1], np.int64), np.array([1], np.int32))
    return graphgen.CSR(off, adj)


@pytest.mark.parametrize("kind", ["unsorted", "selfloop", "asymmetric", "range", "odd"])
def test_bad_graphs_rejected(kind):
    with pytest.raises(gs.ScanError) as e:
        build(bad_graph(kind))
    assert e.value.status == -3


def long_row_graph(kind=None):
    # a hub of degree 5099 (a row longer than 4096) in the middle of a group
    # of 32 rows, and a path through the other vertices
    n, hub = 5100, 40
    edges = [(hub, x) for x in range(n) if x != hub]
    edges += [(x, x + 1) for x in range(n - 1) if hub not in (x, x + 1)]
    g = graphgen.from_edges(n, edges)
    off, adj = g.off.copy(), g.adj.copy()
    h0, h1 = off[hub], off[hub + 1]
    if kind == "unsorted_hub":
        adj[h0 + 3000], adj[h0 + 3001] = adj[h0 + 3001], adj[h0 + 3000]
    elif kind == "selfloop_hub":
        adj[h0 + 39] = hub  # the entry 39 sits between 38 and 41: still ascending
    elif kind == "range_hub":
        adj[h1 - 1] = n + 5
    elif kind == "unsorted_after":  # the row right after the hub, same group
        r0, r1 = off[hub + 1], off[hub + 2]
        adj[r0:r1] = adj[r0:r1][::-1]
    return graphgen.CSR(off, adj)


def test_long_row_graph_builds_like_the_oracle():
    g = long_row_graph()
    with build(g) as ix:
        ex = ix.export()
    ox = oracle.Index(g)
    assert np.array_equal(ex["sim"], ox.sim) and np.array_equal(ex["co_id"], ox.co_id)


@pytest.mark.parametrize("kind", ["unsorted_hub", "selfloop_hub", "range_hub", "unsorted_after"])
def test_bad_long_rows_rejected(kind):
    with pytest.raises(gs.ScanError) as e:
        build(long_row_graph(kind))
    assert e.value.status == -3


def test_bad_query_arguments():
    g = graphgen.from_edges(4, [(0, 1), (1, 2), (2, 3)])
    with build(g) as ix:
        for mu, eps in [(1, 0.5), (0, 0.5), (2, -0.1), (2, 1.5), (2, float("nan"))]:
            with pytest.raises(gs.ScanError) as e:
                ix.query(mu, eps)
            assert e.value.status == -1


def dense_sbm():
    return graphgen.sbm(1200, 3, 0.35, 0.08, seed=4)


@pytest.mark.parametrize("k", [64, 256])
def test_lsh_simhash_bit_exact(k):
    g = dense_sbm()
    ox = oracle.LSHIndex(g, oracle.COSINE, k, T=128, seed=7)
    assert ox.nH > 100
    with build(g, gs.COSINE, lsh=gs.make_lsh(gs.COSINE, k, 128, seed=7)) as ix:
        assert_index_equal(ix, ox)
        assert_queries_equal(ix, ox, [3, 5, 20], [0.3, 0.5, 0.7])


@pytest.mark.parametrize("kpartition", [True, False])
def test_lsh_minhash_bit_exact(kpartition):
    g = dense_sbm()
    ox = oracle.LSHIndex(g, oracle.JACCARD, 64, T=128, seed=5, kpartition=kpartition)
    with build(g, gs.JACCARD, lsh=gs.make_lsh(gs.JACCARD, 64, 128, seed=5, kpartition=kpartition)) as ix:
        assert_index_equal(ix, ox)
        assert_queries_equal(ix, ox, [3, 5, 20], [0.3, 0.5, 0.7])


def test_lsh_threshold_zero_and_huge():
    g = graphgen.rmat(12, 16, seed=8)
    exact = oracle.Index(g)
    # threshold above every degree: nothing is approximated, the index is exact
    with build(g, gs.COSINE, lsh=gs.make_lsh(gs.COSINE, 64, 10 ** 6)) as ix:
        assert_index_equal(ix, exact)
    # threshold 0: every edge between vertices of degree >= 1 is approximated
    ox = oracle.LSHIndex(g, oracle.COSINE, 64, T=0, seed=1)
    with build(g, gs.COSINE, lsh=gs.make_lsh(gs.COSINE, 64, 0, seed=1)) as ix:
        assert_index_equal(ix, ox)


@pytest.fixture
def wide_index():
    """Count with 64-bit element indices, the path of graphs with 2^31 arcs or
    more, on small graphs (process-wide switch, restored afterwards)."""
    gs.set_wide_index(True)
    yield
    gs.set_wide_index(False)


@pytest.mark.parametrize("kind", [gs.COSINE, gs.JACCARD])
def test_wide_index_path_matches_oracle(wide_index, kind):
    g = graphgen.rmat(14, 16, seed=3)  # rows for the warp and the CTA kernels
    ox = oracle.Index(g, kind)
    with build(g, kind, counts=gs.COUNTS_SPARSE) as ix:
        assert_index_equal(ix, ox)
        assert_queries_equal(ix, ox, [2, 5, 16], [0.2, 0.5, 0.8])


def test_wide_index_big_out_degree_and_weights(wide_index):
    # out-degree > 4096 (the global-memory kernel): the closed form of K_{a,b}
    a, b = 4200, 4300
    n = a + b
    off = np.zeros(n + 1, np.int64)
    off[1:a + 1] = b
    off[a + 1:] = a
    off = np.cumsum(off)
    adj = np.concatenate([np.tile(np.arange(a, n), a), np.tile(np.arange(a), b)]).astype(np.int32)
    with build(graphgen.CSR(off, adj)) as ix:
        assert np.all(ix.export()["sim"] == 2.0 / math.sqrt((a + 1) * (b + 1)))
    # weighted, integer weights: bit exact
    g = graphgen.sbm(3000, 6, 0.08, 0.004, seed=12)
    w = graphgen.edge_weights(g, 3, "int")
    ox = oracle.Index(g, oracle.COSINE, sim=oracle.weighted_similarities(g, w))
    with build(g, weights=w) as ix:
        assert_index_equal(ix, ox)
