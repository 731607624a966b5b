"""GPU parity of the modularity passes and of the (mu, eps) sweep (Sections
7.2 and 7.3.4) against the oracle's modularity of the oracle's clusterings.

The GPU sums the inside arcs, the clustered vertices' squared degrees and
the squared cluster degree sums as exact 64-bit integers and converts once;
the oracle adds the same integers in double precision, exactly as long as
every partial sum stays below 2^53 (true for these graphs), so the two
results are the same double. The tolerance below (1e-12) only covers a
different rounding of the final two divisions.
"""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2012_11188_gb300 as gs

pytestmark = pytest.mark.gpu

TOL = 1e-12


def test_modularity_of_query_labels_matches_oracle():
    g = graphgen.sbm(10_000, 50, 0.05, 0.0004, seed=3)
    ox = oracle.Index(g, oracle.COSINE)
    with gs.ScanIndex.build(g, gs.COSINE) as ix:
        for mu, eps in ((2, 0.2), (4, 0.3), (5, 0.5), (8, 0.25), (3, 0.9)):
            labels = ix.query(mu, eps, hubs=True)
            assert np.array_equal(labels, ox.query(mu, eps, hubs=True))
            want = oracle.modularity(g, labels)
            got = ix.modularity(labels)
            assert abs(got - want) <= TOL, (mu, eps, got, want)


def test_modularity_of_arbitrary_labels():
    """Cluster ids need not be core ids: random ids, negatives as singletons."""
    g = graphgen.rmat(13, 16, seed=5)
    rng = np.random.default_rng(11)
    with gs.ScanIndex.build(g, gs.COSINE) as ix:
        for ncl in (1, 7, 300):
            labels = rng.integers(0, ncl, size=g.n).astype(np.int32)
            labels[rng.random(g.n) < 0.2] = -1
            labels[rng.random(g.n) < 0.05] = -2
            assert abs(ix.modularity(labels) - oracle.modularity(g, labels)) <= TOL
        # all singletons and one cluster: closed forms
        deg = np.diff(g.off).astype(np.float64)
        two_m = float(g.arcs)
        single = np.full(g.n, -1, np.int32)
        assert abs(ix.modularity(single) - (-(deg ** 2).sum() / two_m ** 2)) <= TOL
        assert abs(ix.modularity(np.zeros(g.n, np.int32)) - 0.0) <= TOL


def test_modularity_device_labels_and_bad_label():
    torch = pytest.importorskip("torch")
    g = graphgen.sbm(2000, 10, 0.1, 0.002, seed=2)
    with gs.ScanIndex.build(g, gs.COSINE) as ix:
        host = ix.query(3, 0.4)
        dev = torch.from_numpy(host).cuda()
        assert ix.modularity(dev) == ix.modularity(host)
        bad = host.copy()
        bad[7] = g.n
        with pytest.raises(gs.ScanError):
            ix.modularity(bad)


def test_sweep_matches_oracle_queries():
    g = graphgen.sbm(6000, 30, 0.06, 0.0005, seed=9)
    ox = oracle.Index(g, oracle.COSINE)
    mus = np.repeat(np.array([2, 4, 8, 16, 64], np.int32), 9)
    epss = np.tile(np.arange(1, 10) / 10.0, 5)
    with gs.ScanIndex.build(g, gs.COSINE) as ix:
        q = ix.sweep(mus, epss)
    for i in range(mus.shape[0]):
        want = oracle.modularity(g, ox.query(int(mus[i]), float(epss[i]), hubs=False))
        assert abs(q[i] - want) <= TOL, (mus[i], epss[i], q[i], want)


def test_sweep_over_paper_sigma_picks_the_blocks():
    """Over the paper's full parameter set the best clustering of a planted
    partition with dense blocks is (close to) the blocks themselves."""
    g = graphgen.sbm(4000, 20, 0.3, 0.001, seed=4)
    mus, epss = gs.paper_sigma()
    assert mus.shape == (1782,) and epss.shape == (1782,)
    with gs.ScanIndex.build(g, gs.COSINE) as ix:
        q = ix.sweep(mus, epss)
        best = int(np.argmax(q))
        labels = ix.query(int(mus[best]), float(epss[best]))
    truth = np.arange(g.n) // (g.n // 20)
    # planted blocks: 59.7 of 63.5 expected neighbours inside, 20 equal blocks,
    # so Q of the block partition is about 0.94 - 0.05
    assert q[best] > 0.85
    assert oracle.ari(truth.astype(np.int32), labels) > 0.99
    # spot-check a few pairs against the oracle
    ox = oracle.Index(g, oracle.COSINE)
    for i in (0, 98, 99 * 3 + 40, best):
        want = oracle.modularity(g, ox.query(int(mus[i]), float(epss[i]), hubs=False))
        assert abs(q[i] - want) <= TOL


def test_sweep_empty_and_argument_errors():
    g = graphgen.from_edges(5, [])
    with gs.ScanIndex.build(g, gs.COSINE) as ix:
        assert np.array_equal(ix.sweep([2, 3], [0.5, 0.5]), np.zeros(2))
        with pytest.raises(gs.ScanError):
            ix.sweep([1], [0.5])
        with pytest.raises(gs.ScanError):
            ix.sweep([2], [1.5])
