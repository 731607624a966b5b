"""GPU parity of the weighted cosine index (Section 4.1.1, w(x, x) = 1) against
the oracle.

The GPU adds a numerator's triangle terms with atomics, in no fixed order,
and may fuse a product into the sum; the oracle adds them in id order
without fusion. Every term is a product of two non-negative weights, so each
side's numerator is within (c + 1) u of the exact sum (c terms, u = 2^-53),
and each norm, a square root of d + 1 non-negative squares, within
((d + 1) / 2 + 1) u; with the product of the norms and the division this
bounds the relative difference of the two results by
    2 (du + dv + 8) u,
the per-arc tolerance of arc_tolerance below. With integer
weights every product and sum is an exact integer, so the two sides agree
bit for bit, and so do the neighbour order, the core order and the labels.
With real weights the neighbour and core orders are checked for validity
(the oracle's orders of the GPU's own similarities, bit for bit) and the
labels against the oracle's at thresholds at least the tolerance away from
every similarity.
"""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2012_11188_gb300 as gs

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def assert_index_equal(ex, ox):
    assert np.array_equal(ex["sim"], ox.sim), "similarities differ"
    assert np.array_equal(ex["no_id"], ox.no_id), "NO ids differ"
    assert np.array_equal(ex["no_sim"], ox.no_sim), "NO sims differ"
    assert np.array_equal(ex["co_off"], ox.co_off), "CO offsets differ"
    assert np.array_equal(ex["co_id"], ox.co_id), "CO ids differ"
    assert np.array_equal(ex["co_thr"], ox.co_thr), "CO thresholds differ"


def arc_tolerance(g, want):
    deg = np.diff(g.off)
    src = np.repeat(np.arange(g.n), deg)
    return 2.0 * (deg[src] + deg[g.adj] + 8) * U * np.abs(want)


def safe_eps(sim, tol, grid):
    """Thresholds of the grid moved off every similarity by more than tol."""
    out = []
    s = np.sort(sim)
    t = float(tol.max()) * 4 + 1e-15
    for e in grid:
        while True:
            i = np.searchsorted(s, e)
            near = (i < s.size and abs(s[i] - e) <= t) or (i > 0 and abs(s[i - 1] - e) <= t)
            if not near:
                break
            e += 3 * t
        out.append(e)
    return out


GRAPHS = {
    "sbm_10k": lambda: graphgen.sbm(10_000, 40, 0.04, 0.0005, seed=21),
    # power-law rows: the CTA kernel (out-lists up to 4096) and long sort rows
    "rmat_s15": lambda: graphgen.rmat(15, 16, seed=22),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_integer_weights_bit_exact(name):
    g = GRAPHS[name]()
    w = graphgen.edge_weights(g, 5, "int")
    ox = oracle.Index(g, oracle.COSINE, sim=oracle.weighted_similarities(g, w))
    with gs.ScanIndex.build(g, gs.COSINE, weights=w) as ix:
        assert_index_equal(ix.export(), ox)
        for mu, eps in ((2, 0.3), (4, 0.5), (8, 0.4), (16, 0.2)):
            assert np.array_equal(ix.query(mu, eps, hubs=True), ox.query(mu, eps, hubs=True))


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("dist", ["uniform", "exp"])
def test_real_weights_within_tolerance(name, dist):
    g = GRAPHS[name]()
    w = graphgen.edge_weights(g, 7, dist)
    want = oracle.weighted_similarities(g, w)
    tol = arc_tolerance(g, want)
    with gs.ScanIndex.build(g, gs.COSINE, weights=w) as ix:
        ex = ix.export()
        got = ex["sim"]
        bad = np.abs(got - want) > tol
        assert not bad.any(), (int(bad.sum()), float(np.abs(got - want).max()))
        # the orders are the oracle's orders of the GPU's own similarities
        mine = oracle.Index(g, oracle.COSINE, sim=got)
        assert_index_equal(ex, mine)
        ox = oracle.Index(g, oracle.COSINE, sim=want)
        for mu in (2, 5, 12):
            for eps in safe_eps(want, tol, [0.15, 0.3, 0.45, 0.6]):
                assert np.array_equal(ix.query(mu, eps, hubs=True), ox.query(mu, eps, hubs=True))


def test_unit_weights_match_unweighted_cosine():
    """All weights 1: the weighted cosine is the cosine of Section 3.1; the
    two differ only in rounding (c / sqrt(p q) against c / (sqrt p sqrt q))."""
    g = graphgen.rmat(14, 16, seed=23)
    with gs.ScanIndex.build(g, gs.COSINE, weights=np.ones(g.arcs)) as wx, \
            gs.ScanIndex.build(g, gs.COSINE, counts=gs.COUNTS_SPARSE) as ux:
        a, b = wx.export()["sim"], ux.export()["sim"]
        assert np.all(np.abs(a - b) <= 8 * U * b)


def test_big_out_degree_rows():
    """Out-lists longer than the shared table (4096 entries): in K_{4300,4200}
    the 4300 vertices of side A have degree 4200 and point to side B, so
    their out-degree is 4200. A fringe C of low-degree vertices, each joined
    to a few vertices of both sides, makes triangles c < a < b whose middle
    vertex a is counted by the global-memory kernel. Integer weights: bit
    exact on sampled rows against the oracle's per-vertex routine."""
    a_n, b_n, c_n = 4300, 4200, 64
    rng = np.random.default_rng(3)
    A = np.arange(a_n)
    B = np.arange(a_n, a_n + b_n)
    n = a_n + b_n + c_n
    bip = np.stack(np.meshgrid(A, B, indexing="ij"), -1).reshape(-1, 2)
    fringe = []
    for i in range(c_n):
        c = a_n + b_n + i
        fringe += [(c, int(x)) for x in rng.choice(B, 3, replace=False)]
        fringe += [(c, int(x)) for x in rng.choice(A, 20, replace=False)]
    g = graphgen.from_edges(n, np.concatenate([bip, np.array(fringe)]))
    deg = np.diff(g.off)
    assert deg[:a_n].max() < deg[a_n:a_n + b_n].min()  # A points to B
    w = graphgen.edge_weights(g, 11, "int")
    with gs.ScanIndex.build(g, gs.COSINE, weights=w) as ix:
        sim = ix.export()["sim"]
    fringe_a = sorted({e[1] for e in fringe if e[1] < a_n})[:4]
    for v in [0, a_n - 1, a_n, a_n + b_n - 1, n - c_n, n - 1] + fringe_a:
        row = slice(g.off[v], g.off[v + 1])
        assert np.array_equal(sim[row], oracle.weighted_vertex_similarities(g, w, v)), v


@pytest.mark.parametrize("k,T", [(128, 200), (256, 190)])
def test_weighted_simhash(k, T):
    """LSH mode (Section 5) on a weighted graph: SimHash of the weighted
    closed neighbourhoods. The sketch bits are decided by double-precision
    sums in the same fixed order on both sides, so approximated arcs match
    the oracle bit for bit; the other arcs are exact within the tolerance."""
    g = graphgen.sbm(1200, 3, 0.35, 0.08, seed=4)
    w = graphgen.edge_weights(g, 6, "exp")
    ox = oracle.LSHIndex(g, oracle.COSINE, k, T=T, seed=3, weights=w)
    deg = np.diff(g.off)
    src = np.repeat(np.arange(g.n), deg)
    approx = (deg[src] > T) & (deg[g.adj] > T)
    assert approx.mean() > 0.3 and (~approx).any()
    with gs.ScanIndex.build(g, gs.COSINE, lsh=gs.make_lsh(gs.COSINE, k, T, seed=3),
                            weights=w) as ix:
        ex = ix.export()
    got = ex["sim"]
    assert np.array_equal(got[approx], ox.sim[approx])
    tol = arc_tolerance(g, ox.sim)
    assert np.all(np.abs(got[~approx] - ox.sim[~approx]) <= tol[~approx])
    assert_index_equal(ex, oracle.Index(g, oracle.COSINE, sim=got))


def test_device_inputs_and_index_api():
    torch = pytest.importorskip("torch")
    g = graphgen.sbm(3000, 10, 0.05, 0.002, seed=24)
    w = graphgen.edge_weights(g, 2, "uniform")
    want = oracle.weighted_similarities(g, w)
    tol = arc_tolerance(g, want)
    eps = safe_eps(want, tol, [0.4])[0]
    ox = oracle.Index(g, oracle.COSINE, sim=want)
    labels = ox.query(3, eps)
    q_want = oracle.modularity(g, labels)
    dg = (torch.from_numpy(g.off).cuda(), torch.from_numpy(g.adj).cuda())
    with gs.ScanIndex.build(g, gs.COSINE, weights=w) as hx, \
            gs.ScanIndex.build(dg, gs.COSINE, weights=torch.from_numpy(w).cuda()) as dx:
        for ix in (hx, dx):
            assert np.all(np.abs(ix.export()["sim"] - want) <= tol)
            assert np.array_equal(ix.query(3, eps), labels)
            assert abs(ix.modularity(labels) - q_want) <= 1e-12
            q = ix.sweep([3, 3], [eps, eps])
            assert np.all(np.abs(q - q_want) <= 1e-12)


def test_empty_and_edgeless_graphs():
    for g in (graphgen.from_edges(0, []), graphgen.from_edges(6, [])):
        with gs.ScanIndex.build(g, gs.COSINE, weights=np.zeros(0)) as ix:
            assert np.all(ix.query(2, 0.5) == -1)
    g = graphgen.from_edges(3, [(0, 1)])
    with gs.ScanIndex.build(g, gs.COSINE, weights=np.array([0.0, 0.0])) as ix:
        # zero weight: sigma = 0 / (1 * 1)
        assert np.array_equal(ix.export()["sim"], np.zeros(2))


def _weighted_path():
    g = graphgen.from_edges(5, [(0, 1), (1, 2), (2, 3), (3, 4), (0, 4), (1, 3)])
    return g, graphgen.edge_weights(g, 1, "uniform")


@pytest.mark.parametrize("what", ["negative", "nan", "inf", "asymmetric"])
def test_bad_weights_rejected(what):
    g, w = _weighted_path()
    w = w.copy()
    if what == "negative":
        w[3] = -0.5
    elif what == "nan":
        w[-1] = np.nan
    elif what == "inf":
        w[0] = np.inf
    else:
        w[2] += 0.25  # one arc of an edge differs from its twin
    with pytest.raises(gs.ScanError) as e:
        gs.ScanIndex.build(g, gs.COSINE, weights=w)
    assert e.value.status == -1


def test_weighted_argument_errors():
    g, w = _weighted_path()
    with pytest.raises(ValueError):
        gs.ScanIndex.build(g, gs.COSINE, weights=w[:-1])
    for kw in ({"kind": gs.JACCARD}, {"counts": gs.COUNTS_DENSE}):
        kind = kw.pop("kind", gs.COSINE)
        with pytest.raises(gs.ScanError):
            gs.ScanIndex.build(g, kind, weights=w, **kw)
    # a bad graph is still a bad graph
    off, adj = g.off.copy(), g.adj.copy()
    adj[0] = 0
    with pytest.raises(gs.ScanError) as e:
        gs.ScanIndex.build(graphgen.CSR(off, adj), gs.COSINE, weights=w)
    assert e.value.status == -3


@pytest.mark.parametrize("name", ["rmat_s22", "blood_vessel_like"])
def test_weighted_bench_sizes_sampled(name):
    """The weighted workloads bench.py times (R-MAT s22 and the blood-vessel
    shape, n = 25,825 with average degree 5.4K; weights U[0.05, 3)), built
    from device-resident inputs as there. Sampled rows (random vertices and
    the three of highest degree) are within the tolerance of the oracle's
    per-vertex routine; their neighbour order is the order of the GPU's own
    similarities; the core order has its properties at several mu."""
    from test_gpu_fullsize import check_core_order, device_csr
    if name == "rmat_s22":
        g = graphgen.rmat(22, 16, seed=1)
    else:
        g = graphgen.sbm(25825, 1, 5400 / 25824, 5400 / 25824, seed=1)
    w = graphgen.edge_weights(g, 1, "uniform")
    import torch
    deg = np.diff(g.off)
    with gs.ScanIndex.build(device_csr(g), gs.COSINE, weights=torch.from_numpy(w).cuda()) as ix:
        ex = ix.export()
    rng = np.random.default_rng(22)
    nz = np.nonzero(deg)[0]
    sample = list(rng.choice(nz, 12, replace=False)) + list(np.argsort(deg)[-3:])
    for v in sample:
        s = slice(g.off[v], g.off[v + 1])
        want = oracle.weighted_vertex_similarities(g, w, int(v))
        got = ex["sim"][s]
        tol = 2.0 * (deg[v] + deg[g.adj[s]] + 8) * U * want
        assert np.all(np.abs(got - want) <= tol), v
        order = np.lexsort((g.adj[s], -got))
        assert np.array_equal(ex["no_id"][s], g.adj[s][order]), v
        assert np.array_equal(ex["no_sim"][s], got[order]), v
    md = int(deg.max())
    check_core_order(g, ex, [2, 3, 5, 17, 128, md + 1])
