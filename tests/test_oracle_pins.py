"""Pins for the CPU oracle: facts fixed by the paper and by independent mathematics.

Each test checks the oracle against something other than itself: the paper's
worked example and figure captions (tests/golden), dense (A+I)^2 products,
triangle counts from trace(A^3), closed forms on cliques, stars and bridged
cliques, brute force over every graph on five vertices, and library routines
for ARI and modularity.
"""
import itertools
import math
import os

import numpy as np
import pytest

import graphgen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense(g):
    A = np.zeros((g.n, g.n), dtype=np.int64)
    for v in range(g.n):
        A[v, g.adj[g.off[v]:g.off[v + 1]]] = 1
    return A


def arc_pairs(g):
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    return src, g.adj.astype(np.int64)


def random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    A = (rng.random((n, n)) < p).astype(np.int64)
    A = np.triu(A, 1)
    return graphgen.from_dense(A + A.T)


def load_golden(name):
    edges, facts = [], []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "edge":
                edges.append((int(line[1]) - 1, int(line[2]) - 1))
            else:
                facts.append(line)
    n = max(max(e) for e in edges) + 1
    return graphgen.from_edges(n, edges), facts


# ------------------------------------------------------------------ counts

@pytest.mark.parametrize("n,p,seed", [(12, 0.3, 1), (25, 0.2, 2), (40, 0.5, 3), (33, 0.08, 4)])
def test_counts_equal_dense_square(n, p, seed):
    # Section 4.1.1: for adjacent u, v the numerator is ((A+I)^2)_{uv}.
    g = random_graph(n, p, seed)
    A = dense(g) + np.eye(g.n, dtype=np.int64)
    C = A @ A
    src, dst = arc_pairs(g)
    assert np.array_equal(oracle.closed_counts(g), C[src, dst])
    assert np.array_equal(oracle.count_pairs(g, src, dst), C[src, dst])


def test_triangle_identity():
    # Section 3.1: |N(u) ∩ N(v)| is the number of triangles on edge {u,v};
    # summed over arcs each triangle is seen 6 times; #triangles = trace(A^3)/6.
    g = random_graph(60, 0.25, 7)
    A = dense(g)
    tri = int(np.trace(A @ A @ A)) // 6
    cnt = oracle.closed_counts(g)
    assert int((cnt.astype(np.int64) - 2).sum()) == 6 * tri


# ------------------------------------------------------- closed-form graphs

def test_clique_all_one():
    n = 9
    g = graphgen.from_edges(n, itertools.combinations(range(n), 2))
    for kind in (oracle.COSINE, oracle.JACCARD):
        ix = oracle.Index(g, kind)
        assert np.all(ix.sim == 1.0)
        for mu in range(2, n + 1):
            assert np.all(ix.query(mu, 1.0) == 0)
        assert np.all(ix.query(n + 1, 0.0) == -1)


@pytest.mark.parametrize("k", [3, 7, 40])
def test_star(k):
    g = graphgen.from_edges(k + 1, [(0, i) for i in range(1, k + 1)])
    ix = oracle.Index(g)
    want = 2.0 / math.sqrt(2 * (k + 1))
    assert np.allclose(ix.sim, want, rtol=0, atol=1e-15)
    jx = oracle.Index(g, oracle.JACCARD)
    assert np.allclose(jx.sim, 2.0 / (k + 1), rtol=0, atol=1e-15)
    # eps above the leaf-centre similarity: nobody is a core, everyone an outlier
    lab = ix.query(2, min(1.0, want + 1e-9), hubs=True)
    assert np.all(lab == -1)
    # eps at it and mu=2: the whole star is one cluster
    assert np.all(ix.query(2, want) == 0)


def test_bridged_cliques_hub():
    a = 5
    A = list(range(a))
    B = list(range(a, 2 * a))
    h = 2 * a
    edges = list(itertools.combinations(A, 2)) + list(itertools.combinations(B, 2))
    edges += [(h, A[0]), (h, B[0])]
    g = graphgen.from_edges(2 * a + 1, edges)
    ix = oracle.Index(g)
    s = dict(zip(zip(*arc_pairs(g)), ix.sim))
    assert s[(h, A[0])] == pytest.approx(2 / math.sqrt(3 * (a + 1)), abs=1e-15)
    assert s[(A[0], A[1])] == pytest.approx(math.sqrt(a / (a + 1)), abs=1e-15)
    assert s[(A[1], A[2])] == 1.0
    lab = ix.query(3, 0.6, hubs=True)
    assert list(lab[A]) == [A[0]] * a and list(lab[B]) == [B[0]] * a
    assert lab[h] == -2


def test_vertex_next_to_one_cluster_is_outlier():
    # Section 4.3: a hub needs neighbours in at least two clusters. Vertex 5
    # touches two members of the clique cluster {0..4}: sigma = 3/sqrt(18) < .8.
    edges = list(itertools.combinations(range(5), 2)) + [(5, 0), (5, 1)]
    g = graphgen.from_edges(6, edges)
    ix = oracle.Index(g)
    lab = ix.query(3, 0.8, hubs=True)
    assert list(lab) == [0, 0, 0, 0, 0, -1]


def test_sigma_exactly_eps_counts():
    # Section 3.1: eps-similar means sigma >= eps. Two adjacent degree-3
    # vertices with no common neighbour have sigma = 2/sqrt(16) = 0.5 exactly.
    edges = [(0, 1), (0, 2), (0, 3), (1, 4), (1, 5)]
    g = graphgen.from_edges(6, edges)
    ix = oracle.Index(g)
    s = dict(zip(zip(*arc_pairs(g)), ix.sim))
    assert s[(0, 1)] == 0.5
    lab = ix.query(2, 0.5)
    assert lab[0] == lab[1] >= 0
    lab = ix.query(2, np.nextafter(0.5, 1.0))
    assert not (lab[0] == lab[1] >= 0)


def test_isolated_vertices_are_outliers():
    g = graphgen.from_edges(5, [(0, 1)])
    ix = oracle.Index(g)
    lab = ix.query(2, 0.1, hubs=True)
    assert list(lab) == [0, 0, -1, -1, -1]


# --------------------------------------------------- the paper's own values

def test_worked_example_sigma():
    g, facts = load_golden("worked_example_sigma.txt")
    ix = oracle.Index(g)
    s = dict(zip(zip(*arc_pairs(g)), ix.sim))
    for f in facts:
        assert f[0] == "sigma"
        u, v, num, prod = (int(x) for x in f[1:])
        assert s[(u - 1, v - 1)] == num / math.sqrt(prod)
        assert round(s[(u - 1, v - 1)], 2) == 0.58


def test_figure_captions():
    g, facts = load_golden("figure1_consistent.txt")
    ix = oracle.Index(g)
    lab = ix.query(3, 0.6, hubs=True)
    lab_def = ix.query_definition(3, 0.6, hubs=True)
    assert np.array_equal(lab, lab_def)
    s = dict(zip(zip(*arc_pairs(g)), ix.sim))
    for f in facts:
        ids = [int(x) - 1 for x in f[1:]] if f[0] in ("cluster", "hub", "outlier", "border") else None
        if f[0] == "cluster":
            assert len({lab[i] for i in ids}) == 1 and lab[ids[0]] == min(ids)
            assert set(np.nonzero(lab == lab[ids[0]])[0]) == set(ids)
        elif f[0] == "hub":
            assert all(lab[i] == -2 for i in ids)
        elif f[0] == "outlier":
            assert all(lab[i] == -1 for i in ids)
        elif f[0] == "border":
            deg = np.diff(g.off)
            for i in ids:  # clustered, but |N̄| < mu so not a core
                assert lab[i] >= 0 and deg[i] + 1 < 3
        elif f[0] == "co_size":
            mu, size = int(f[1]), int(f[2])
            assert ix.co_off[mu - 1] - ix.co_off[mu - 2] == size
        elif f[0] == "co_threshold":
            mu, v, thr = int(f[1]), int(f[2]) - 1, float(f[3])
            seg = slice(ix.co_off[mu - 2], ix.co_off[mu - 1])
            pos = list(ix.co_id[seg]).index(v)
            assert round(ix.co_thr[seg][pos], 2) == thr
        elif f[0] == "no_entry":
            v, u, val = int(f[1]) - 1, int(f[2]) - 1, float(f[3])
            seg = slice(g.off[v], g.off[v + 1])
            pos = list(ix.no_id[seg]).index(u)
            assert round(ix.no_sim[seg][pos], 2) == val
        elif f[0] == "sigma":
            u, v, num, prod = (int(x) for x in f[1:])
            assert s[(u - 1, v - 1)] == num / math.sqrt(prod)


# ------------------------------------------------------ orders: invariants

def check_orders(g, ix):
    deg = np.diff(g.off)
    for v in range(g.n):
        seg = slice(g.off[v], g.off[v + 1])
        ids, sims = ix.no_id[seg], ix.no_sim[seg]
        assert sorted(ids) == list(g.adj[seg])
        ref = dict(zip(g.adj[seg], ix.sim[seg]))
        assert all(ref[i] == s for i, s in zip(ids, sims))
        for j in range(len(ids) - 1):
            assert sims[j] > sims[j + 1] or (sims[j] == sims[j + 1] and ids[j] < ids[j + 1])
    maxdeg = deg.max() if g.n else 0
    assert ix.co_off.shape[0] == maxdeg + 1 and ix.co_off[-1] == g.arcs
    for mu in range(2, maxdeg + 2):
        seg = slice(ix.co_off[mu - 2], ix.co_off[mu - 1])
        ids, thr = ix.co_id[seg], ix.co_thr[seg]
        assert sorted(ids) == list(np.nonzero(deg + 1 >= mu)[0])
        for i, t in zip(ids, thr):
            assert ix.no_sim[g.off[i] + mu - 2] == t
        for j in range(len(ids) - 1):
            assert thr[j] > thr[j + 1] or (thr[j] == thr[j + 1] and ids[j] < ids[j + 1])


@pytest.mark.parametrize("kind", [oracle.COSINE, oracle.JACCARD])
def test_order_invariants(kind):
    g = graphgen.sbm(300, 6, 0.2, 0.02, seed=3)
    check_orders(g, oracle.Index(g, kind))


# ----------------------------------------------- brute force on tiny graphs

def all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        yield graphgen.from_edges(n, [p for b, p in enumerate(pairs) if mask >> b & 1]) \
            if mask else graphgen.CSR(np.zeros(n + 1, np.int64), np.zeros(0, np.int32))


def test_exhaustive_five_vertices():
    # every simple graph on 5 vertices: counts against (A+I)^2, and the index
    # query (Algorithms 3-5) against the definition-only query for all mu and
    # for eps over a grid that includes every similarity value that occurs
    n = 5
    for g in all_graphs(n):
        if g.arcs:
            A = dense(g) + np.eye(n, dtype=np.int64)
            src, dst = arc_pairs(g)
            assert np.array_equal(oracle.closed_counts(g), (A @ A)[src, dst])
        ix = oracle.Index(g) if g.arcs else None
        if ix is None:
            continue
        epss = sorted(set(np.round(np.linspace(0, 1, 11), 10)) | set(ix.sim.tolist()))
        for mu in range(2, n + 2):
            for eps in epss:
                for hubs in (False, True):
                    a = ix.query(mu, eps, hubs)
                    b = ix.query_definition(mu, eps, hubs)
                    assert np.array_equal(a, b), (g.adj, mu, eps)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_index_query_equals_definition_sbm(seed):
    g = graphgen.sbm(400, 8, 0.15, 0.01, seed=seed)
    for kind in (oracle.COSINE, oracle.JACCARD):
        ix = oracle.Index(g, kind)
        for mu in (2, 3, 5, 8, 16, 40):
            for eps in np.arange(1, 10) / 10:
                assert np.array_equal(ix.query(mu, eps, True), ix.query_definition(mu, eps, True))


def test_vertex_helpers_match_full_index():
    g = graphgen.rmat(10, 8, seed=5)
    ix = oracle.Index(g)
    for v in (0, 17, int(np.argmax(np.diff(g.off)))):
        seg = slice(g.off[v], g.off[v + 1])
        assert np.array_equal(oracle.vertex_similarities(g, v), ix.sim[seg])
        ids, sims = oracle.vertex_neighbor_order(g, v)
        assert np.array_equal(ids, ix.no_id[seg]) and np.array_equal(sims, ix.no_sim[seg])


# ------------------------------------------------------ quality measures

def test_ari_basic_cases():
    a = np.array([0, 0, 0, 3, 3, 5, 5, 5], dtype=np.int32)
    assert oracle.ari(a, a) == pytest.approx(1.0)
    perm = {0: 7, 3: 1, 5: 4}
    assert oracle.ari(a, np.array([perm[x] for x in a], np.int32)) == pytest.approx(1.0)
    # hand-computed: sizes {3,3} vs {2,4} on 6 items, n_ij = [[2,1],[0,3]]
    x = np.array([0, 0, 0, 1, 1, 1], np.int32)
    y = np.array([0, 0, 1, 1, 1, 1], np.int32)
    sij = 1 + 0 + 0 + 3
    si, sj, tot = 3 + 3, 1 + 6, 15
    exp = si * sj / tot
    assert oracle.ari(x, y) == pytest.approx((sij - exp) / ((si + sj) / 2 - exp))


def test_ari_matches_sklearn():
    metrics = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(1)
    for _ in range(5):
        a = rng.integers(-1, 6, 300).astype(np.int32)
        b = rng.integers(-1, 4, 300).astype(np.int32)
        b[:150] = a[:150]
        # negative labels are singletons
        ua = np.where(a >= 0, a, 1000 + np.arange(300))
        ub = np.where(b >= 0, b, 1000 + np.arange(300))
        assert oracle.ari(a, b) == pytest.approx(metrics.adjusted_rand_score(ua, ub), abs=1e-12)


def test_modularity_matches_networkx():
    nx = pytest.importorskip("networkx")
    g = graphgen.sbm(200, 4, 0.2, 0.02, seed=9)
    ix = oracle.Index(g)
    lab = ix.query(3, 0.3)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    src, dst = arc_pairs(g)
    G.add_edges_from((int(u), int(v)) for u, v in zip(src, dst) if u < v)
    comms = {}
    for v in range(g.n):
        comms.setdefault(int(lab[v]) if lab[v] >= 0 else -1 - v, set()).add(v)
    want = nx.community.modularity(G, list(comms.values()))
    assert oracle.modularity(g, lab) == pytest.approx(want, abs=1e-12)
