"""Parity at the benchmark's sizes, in the launch configuration bench.py times.

R-MAT scale 20 (15.7M edges) is compared with the full CPU oracle. R-MAT scale
24 (260M edges) is too large for it, so there the oracle checks sampled rows
(similarities and the neighbour order of random and of the highest-degree
vertices), and properties that hold at any size check the rest: the core
order's membership, sizes, order and thresholds, and, for queries, the core
set, the connected components of the core eps-graph (scipy), canonical labels,
the border rule and the hub rule.
"""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2012_11188_gb300 as gs

pytestmark = pytest.mark.gpu


def device_csr(g):
    import torch
    return torch.from_numpy(g.off).cuda(), torch.from_numpy(g.adj).cuda()


def rows(off):
    return np.repeat(np.arange(off.shape[0] - 1), np.diff(off))


def check_core_order(g, ex, mus):
    deg = np.diff(g.off)
    co_off, co_id, co_thr = ex["co_off"], ex["co_id"], ex["co_thr"]
    assert co_off.shape[0] == deg.max() + 1 and co_off[-1] == g.arcs
    sizes = np.diff(co_off)
    cnt_ge = np.bincount(deg, minlength=deg.max() + 1)[::-1].cumsum()[::-1]  # #{d >= k}
    assert np.array_equal(sizes, cnt_ge[1:])  # |CO[mu]| = #{d >= mu-1}, mu = 2..
    for mu in mus:
        s = slice(co_off[mu - 2], co_off[mu - 1])
        ids, thr = co_id[s], co_thr[s]
        assert np.array_equal(np.sort(ids), np.nonzero(deg + 1 >= mu)[0])
        assert np.array_equal(thr, ex["no_sim"][g.off[ids] + mu - 2])
        ok = (thr[:-1] > thr[1:]) | ((thr[:-1] == thr[1:]) & (ids[:-1] < ids[1:]))
        assert ok.all()


def check_query(g, ex, lab, mu, eps, hubs=True):
    """Labels of (mu, eps) against the definitions, using the (verified) NO."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    off, n = g.off, g.n
    deg = np.diff(off)
    no_id, no_sim = ex["no_id"], ex["no_sim"]
    src = rows(off)
    ge = no_sim >= eps
    # core iff |N_eps(v)| >= mu, v itself included
    n_eps = np.bincount(src[ge], minlength=n) + 1
    core = n_eps >= mu
    # components of the eps-similar core-core graph, labelled by their smallest id
    m = ge & core[src] & core[no_id]
    A = csr_matrix((np.ones(int(m.sum()), np.int8), (src[m], no_id[m])), shape=(n, n))
    ncomp, comp = connected_components(A, directed=False)
    cores = np.nonzero(core)[0]
    mins = np.full(ncomp, np.iinfo(np.int64).max)
    np.minimum.at(mins, comp[cores], cores)
    assert np.array_equal(lab[cores], mins[comp[cores]])
    # borders: the first core of the eps-prefix of NO[v] (most similar, smallest id)
    cand = ge & core[no_id] & ~core[src]
    pos = np.nonzero(cand)[0]
    first = np.full(n, -1, np.int64)
    # first candidate per row: positions are increasing, keep the first per row
    rv = src[pos]
    keep = np.ones(pos.shape[0], bool)
    keep[1:] = rv[1:] != rv[:-1]
    first[rv[keep]] = pos[keep]
    noncore = ~core
    has = noncore & (first >= 0)
    assert np.array_equal(lab[has], lab[no_id[first[has]]])
    un = noncore & (first < 0)
    if not hubs:
        assert np.all(lab[un] == -1)
        return
    # hubs: unclustered vertices whose neighbours carry two distinct labels
    final = np.where(lab >= 0, lab, -1).astype(np.int64)
    nl = final[g.adj]
    big = np.iinfo(np.int64).max
    lo = np.where(nl >= 0, nl, big)
    hi = np.where(nl >= 0, nl, -1)
    mn = np.full(n, big)
    mx = np.full(n, -1)
    nz = deg > 0
    mn[nz] = np.minimum.reduceat(lo, off[:-1][nz])
    mx[nz] = np.maximum.reduceat(hi, off[:-1][nz])
    hub = un & (mx >= 0) & (mn != mx)
    assert np.all(lab[hub] == -2)
    assert np.all(lab[un & ~hub] == -1)


@pytest.fixture(scope="module")
def rmat20():
    return graphgen.rmat(20, 16, seed=1)


@pytest.mark.parametrize("kind", [gs.COSINE, gs.JACCARD])
def test_rmat_s20_full_oracle(rmat20, kind):
    g = rmat20
    ox = oracle.Index(g, kind)
    with gs.ScanIndex.build(device_csr(g), kind) as ix:
        ex = ix.export()
        for key in ("sim", "no_id", "no_sim", "co_off", "co_id", "co_thr"):
            assert np.array_equal(ex[key], getattr(ox, key)), key
        for mu in (2, 4, 8, 16, 32):
            for eps in (0.1, 0.3, 0.5, 0.7, 0.9):
                lab = ix.query(mu, eps, hubs=True)
                assert np.array_equal(lab, ox.query(mu, eps, hubs=True)), (mu, eps)
        mus = np.array([2, 4, 8, 16, 32] * 5, np.int32)
        epss = np.repeat([0.1, 0.3, 0.5, 0.7, 0.9], 5)
        labs = ix.query_batch(mus, epss, hubs=True)
        for i in range(25):
            assert np.array_equal(labs[i], ox.query(int(mus[i]), float(epss[i]), hubs=True))


@pytest.fixture(scope="module")
def rmat24():
    return graphgen.rmat(24, 16, seed=1)


def test_rmat_s24_sampled_and_properties(rmat24):
    g = rmat24
    deg = np.diff(g.off)
    with gs.ScanIndex.build(device_csr(g), gs.COSINE) as ix:
        ex = ix.export()
        rng = np.random.default_rng(24)
        nz = np.nonzero(deg)[0]
        sample = list(rng.choice(nz, 48, replace=False)) + list(np.argsort(deg)[-3:])
        for v in sample:
            s = slice(g.off[v], g.off[v + 1])
            assert np.array_equal(ex["sim"][s], oracle.vertex_similarities(g, int(v))), v
            ids, sims = oracle.vertex_neighbor_order(g, int(v))
            assert np.array_equal(ex["no_id"][s], ids) and np.array_equal(ex["no_sim"][s], sims), v
        md = int(deg.max())
        check_core_order(g, ex, [2, 3, 5, 17, 128, 1000, 30000, md + 1])
        for eps in (0.3, 0.5, 0.7):
            lab = ix.query(5, eps, hubs=True)
            check_query(g, ex, lab, 5, eps, hubs=True)
        lab = ix.query_batch(np.array([5, 5], np.int32), np.array([0.3, 0.7]), hubs=False)
        check_query(g, ex, lab[0], 5, 0.3, hubs=False)
        check_query(g, ex, lab[1], 5, 0.7, hubs=False)
