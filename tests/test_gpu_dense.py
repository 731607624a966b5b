"""GPU parity of the dense path: closed counts as ((A+I)^2)[u][v] from one
bf16 GEMM with fp32 accumulation (Section 4.1.1), exact because the operands
are 0/1 and every sum is an integer below 2^24. The resulting index must be
the oracle's bit for bit, and the same as the sparse path's."""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2012_11188_gb300 as gs

pytestmark = pytest.mark.gpu


def export_equal(a, b):
    ea, eb = a.export(), b.export()
    return all(np.array_equal(ea[k], eb[k]) for k in ea)


def assert_index_equal(ix, ox):
    ex = ix.export()
    assert np.array_equal(ex["sim"], ox.sim), "similarities differ"
    assert np.array_equal(ex["no_id"], ox.no_id), "NO ids differ"
    assert np.array_equal(ex["no_sim"], ox.no_sim), "NO sims differ"
    assert np.array_equal(ex["co_off"], ox.co_off), "CO offsets differ"
    assert np.array_equal(ex["co_id"], ox.co_id), "CO ids differ"
    assert np.array_equal(ex["co_thr"], ox.co_thr), "CO thresholds differ"


@pytest.mark.parametrize("kind", [gs.COSINE, gs.JACCARD])
@pytest.mark.parametrize("n,blocks,p_in,p_out", [(1500, 1, 0.3, 0.3), (2049, 7, 0.4, 0.05),
                                                 (333, 3, 0.9, 0.2)])
def test_dense_counts_match_oracle(kind, n, blocks, p_in, p_out):
    g = graphgen.sbm(n, blocks, p_in, p_out, seed=n)
    ox = oracle.Index(g, kind)
    with gs.ScanIndex.build(g, kind, counts=gs.COUNTS_DENSE) as ix:
        assert_index_equal(ix, ox)
        for mu, eps in ((2, 0.3), (5, 0.5), (20, 0.6)):
            assert np.array_equal(ix.query(mu, eps, hubs=True), ox.query(mu, eps, hubs=True))


def test_dense_equals_sparse_and_auto():
    """A graph with isolated vertices, a dense core and a sparse fringe."""
    rng = np.random.default_rng(4)
    n = 4000
    core = rng.choice(n, 600, replace=False)
    edges = [(int(a), int(b)) for a in core for b in core if a < b and rng.random() < 0.5]
    edges += [(int(rng.integers(n)), int(rng.integers(n))) for _ in range(20000)]
    g = graphgen.from_edges(n, edges)
    with gs.ScanIndex.build(g, gs.COSINE, counts=gs.COUNTS_DENSE) as d, \
            gs.ScanIndex.build(g, gs.COSINE, counts=gs.COUNTS_SPARSE) as sp, \
            gs.ScanIndex.build(g, gs.COSINE) as auto:
        assert export_equal(d, sp)
        assert export_equal(auto, sp)


@pytest.mark.parametrize("kind", [gs.COSINE, gs.JACCARD])
def test_dense_many_tiles_per_cta(kind):
    """n = 5000 pads to 5120: 420 upper tiles of 128 x 256 over at most one
    CTA per SM, so every CTA runs several tiles and both TMEM accumulators;
    rows of both a dense and a sparse block, and isolated vertices."""
    rng = np.random.default_rng(11)
    n = 5000
    a = graphgen.sbm(3000, 1, 0.3, 0.3, seed=5)
    src = np.repeat(np.arange(3000), np.diff(a.off))
    edges = np.stack([src, a.adj], 1)
    edges = edges[edges[:, 0] < edges[:, 1]]
    extra = rng.integers(0, 4900, (40000, 2))  # vertices 4900.. stay isolated
    g = graphgen.from_edges(n, np.concatenate([edges, extra]))
    ox = oracle.Index(g, kind)
    with gs.ScanIndex.build(g, kind, counts=gs.COUNTS_DENSE) as ix:
        assert_index_equal(ix, ox)
        assert np.array_equal(ix.query(4, 0.4, hubs=True), ox.query(4, 0.4, hubs=True))


def test_auto_takes_the_sparse_path_below_the_size_threshold():
    """A small dense graph (n < 4096) goes through the sparse enumeration
    under the automatic choice: its launches are those of the sparse path."""
    g = graphgen.sbm(1500, 1, 0.3, 0.3, seed=2)

    def launches(mode):
        k0 = gs.kernel_launches()
        with gs.ScanIndex.build(g, gs.COSINE, counts=mode):
            pass
        return gs.kernel_launches() - k0

    sparse, dense, auto = (launches(m) for m in (gs.COUNTS_SPARSE, gs.COUNTS_DENSE,
                                                 gs.COUNTS_AUTO))
    assert auto == sparse and dense != sparse


def test_dense_with_lsh_equals_sparse_with_lsh():
    g = graphgen.sbm(3000, 4, 0.2, 0.02, seed=8)  # degrees ~ 180: most edges approximated
    lsh = gs.make_lsh(gs.COSINE, 64, 128, seed=3)
    with gs.ScanIndex.build(g, gs.COSINE, lsh=lsh, counts=gs.COUNTS_DENSE) as d, \
            gs.ScanIndex.build(g, gs.COSINE, lsh=lsh, counts=gs.COUNTS_SPARSE) as sp:
        assert export_equal(d, sp)
    ox = oracle.LSHIndex(g, oracle.COSINE, 64, T=128, seed=3)
    with gs.ScanIndex.build(g, gs.COSINE, lsh=lsh, counts=gs.COUNTS_DENSE) as d:
        assert np.array_equal(d.export()["sim"], ox.sim)


def test_dense_size_limit_and_bad_mode():
    g = graphgen.from_edges(70000, [(0, 1), (1, 2)])
    with pytest.raises(gs.ScanError):
        gs.ScanIndex.build(g, gs.COSINE, counts=gs.COUNTS_DENSE)
    with pytest.raises(gs.ScanError):
        gs.ScanIndex.build(g, gs.COSINE, counts=7)
    with gs.ScanIndex.build(g, gs.COSINE) as ix:  # auto: sparse for this graph
        assert ix.query(2, 0.5)[0] >= 0


def _bad_graph(kind):
    g = graphgen.from_edges(5, [(0, 1), (1, 2), (2, 3), (3, 4), (0, 4)])
    off, adj = g.off.copy(), g.adj.copy()
    if kind == "asymmetric":
        adj[off[0]] = 2  # 0 lists 2, but 2 does not list 0 (and 1 lists 0)
        adj[off[0]:off[1]] = np.sort(adj[off[0]:off[1]])
    elif kind == "selfloop":
        adj[0] = 0
    elif kind == "unsorted":
        adj[off[1]:off[2]] = adj[off[1]:off[2]][::-1]
    return graphgen.CSR(off, adj)


@pytest.mark.parametrize("mode", [gs.COUNTS_SPARSE, gs.COUNTS_DENSE])
@pytest.mark.parametrize("kind", ["asymmetric", "selfloop", "unsorted"])
def test_bad_graphs_rejected_by_both_paths(mode, kind):
    with pytest.raises(gs.ScanError) as e:
        gs.ScanIndex.build(_bad_graph(kind), gs.COSINE, counts=mode)
    assert e.value.status == -3
