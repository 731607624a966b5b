"""Pins for the LSH part of the oracle (Sections 2.1.2, 5 and 6.3).

The sketches are random, so beyond exact special cases these pins are
statistical: the MinHash collision probability equals the Jaccard similarity
(Section 2.1.2), Hoeffding bounds as in Theorem 5.2, and SimHash estimates that
track the exact cosine on large neighbourhoods.
"""
import itertools
import math

import numpy as np
import pytest

import graphgen
import oracle


def test_splitmix64_published_vectors():
    # SplitMix64 (Steele, Lea, Flood 2014) seeded with 0: its first three outputs
    assert oracle.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64(0, 2) == 0x06C45D188009454F


def test_selection_rule():
    g = graphgen.rmat(12, 16, seed=2)
    T = 40
    row, nH = oracle.lsh_select(g, T)
    deg = np.diff(g.off)
    src = np.repeat(np.arange(g.n), deg)
    hi_nbr = np.zeros(g.n, bool)
    np.logical_or.at(hi_nbr, src, deg[g.adj] > T)
    want = (deg > T) & hi_nbr
    assert np.array_equal(row >= 0, want)
    assert np.array_equal(row[want], np.arange(nH))


def clique(n):
    return graphgen.from_edges(n, itertools.combinations(range(n), 2))


@pytest.mark.parametrize("k", [64, 256])
def test_identical_neighbourhoods_estimate_one(k):
    # every closed neighbourhood of K_n is the same set: sketches coincide
    g = clique(140)
    exact = oracle.similarities(g, oracle.closed_counts(g))
    row, nH = oracle.lsh_select(g, 128)
    assert nH == g.n
    sig = oracle.simhash_sketch(g, row, nH, k, seed=5)
    assert (sig == sig[0]).all()
    s = oracle.lsh_similarities(g, oracle.SIMHASH, row, sig, exact, k)
    assert np.all(s == 1.0)
    for kp in (True, False):
        mh = oracle.minhash_sketch(g, row, nH, 64, seed=5, kpartition=kp)
        assert (mh == mh[0]).all()
        s = oracle.lsh_similarities(g, oracle.MINHASH, row, mh, exact, 64, kp)
        assert np.all(s == 1.0)


def test_simhash_table():
    for k in (64, 256):
        tab = oracle.simhash_table(k)
        assert tab[0] == 1.0 and tab[k] == 0.0 and np.all(tab >= 0)
        assert np.all(np.diff(tab) <= 0)
        assert tab[k // 3] == pytest.approx(0.5, abs=0.02)


def test_rademacher_signs_balanced():
    g = clique(200)
    row, nH = oracle.lsh_select(g, 1)
    # a single-vertex view: sketch bits over many vertices are ~ fair coins
    sig = oracle.simhash_sketch(g, row, nH, 256, seed=11)
    bits = np.unpackbits(sig.view(np.uint8), axis=1)
    assert abs(bits.mean() - 0.5) < 0.1  # all rows equal here: 256 fair bits


def dense_sbm():
    # high-degree vertices with a spread of Jaccard values
    return graphgen.sbm(1200, 3, 0.35, 0.08, seed=4)


def approx_arcs(g, row):
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    m = (row[src] >= 0) & (row[g.adj] >= 0) & (src < g.adj)
    return m


def test_standard_minhash_unbiased_and_hoeffding():
    # Section 2.1.2: P[min-hashes equal] = Jaccard similarity; Theorem 5.2 uses
    # Hoeffding: P(|estimate - J| >= delta) <= 2 exp(-2 k delta^2) per edge
    g = dense_sbm()
    exact = oracle.similarities(g, oracle.closed_counts(g), oracle.JACCARD)
    row, nH = oracle.lsh_select(g, 128)
    k = 64
    mh = oracle.minhash_sketch(g, row, nH, k, seed=3, kpartition=False)
    est = oracle.lsh_similarities(g, oracle.MINHASH, row, mh, exact, k, kpartition=False)
    m = approx_arcs(g, row)
    err = est[m] - exact[m]
    assert m.sum() > 10000
    # mean error: the per-edge estimates have variance <= 1/(4k)
    assert abs(err.mean()) < 0.01
    delta = 0.3
    assert (np.abs(err) >= delta).mean() <= 2 * math.exp(-2 * k * delta * delta) * 50 + 1e-4


def test_kpartition_minhash_close():
    g = dense_sbm()
    exact = oracle.similarities(g, oracle.closed_counts(g), oracle.JACCARD)
    row, nH = oracle.lsh_select(g, 128)
    mh = oracle.minhash_sketch(g, row, nH, 64, seed=3, kpartition=True)
    est = oracle.lsh_similarities(g, oracle.MINHASH, row, mh, exact, 64, kpartition=True)
    m = approx_arcs(g, row)
    assert abs((est[m] - exact[m]).mean()) < 0.03
    assert np.abs(est[m] - exact[m]).mean() < 0.08
    # arcs that are not approximated keep their exact value
    src = np.repeat(np.arange(g.n), np.diff(g.off))
    keep = (row[src] < 0) | (row[g.adj] < 0)
    assert np.array_equal(est[keep], exact[keep])


def test_simhash_tracks_cosine():
    # Section 2.1.2: P[sign differs] = theta/pi for Gaussian directions; the
    # Rademacher projections of these large neighbourhoods are close to that.
    g = dense_sbm()
    exact = oracle.similarities(g, oracle.closed_counts(g), oracle.COSINE)
    row, nH = oracle.lsh_select(g, 128)
    k = 256
    sig = oracle.simhash_sketch(g, row, nH, k, seed=9)
    est = oracle.lsh_similarities(g, oracle.SIMHASH, row, sig, exact, k)
    m = approx_arcs(g, row)
    theta = np.arccos(np.clip(exact[m], 0, 1))
    # estimated angle from the estimate (clamped cosines are at theta >= pi/2)
    theta_hat = np.arccos(np.clip(est[m], 0, 1))
    assert abs((theta_hat - theta).mean()) < 0.02
    assert np.abs(theta_hat - theta).mean() < 0.1


def test_weighted_simhash_unit_weights_equal_unweighted():
    g = dense_sbm()
    row, nH = oracle.lsh_select(g, 128)
    a = oracle.simhash_sketch(g, row, nH, 128, seed=5)
    b = oracle.simhash_sketch(g, row, nH, 128, seed=5, weights=np.ones(g.arcs))
    assert np.array_equal(a, b)


def test_weighted_simhash_brute_force_definition():
    """s_j(v) = sum over N̄(v) of rho_j(x) w(v,x) with w(v,v) = 1, written
    out with numpy from the SplitMix64 stream (pinned to its published
    vectors); integer weights make every sum exact, so the bits must agree."""
    g = graphgen.sbm(120, 2, 0.3, 0.05, seed=8)
    w = graphgen.edge_weights(g, 4, "int")
    row, nH = oracle.lsh_select(g, 10)
    assert nH > 20
    k, seed = 128, 13
    sig = oracle.simhash_sketch(g, row, nH, k, seed, weights=w)
    # key_s = mix(seed ^ "SIMH"); output 0 of SplitMix64 started at state
    # z - gamma is mix(z)
    gamma = 0x9E3779B97F4A7C15
    key = oracle.splitmix64(((seed ^ 0x53494D48) - gamma) % 2**64, 0)

    def rho(x):
        words = [oracle.splitmix64(key, x * 1024 + q) for q in range(k // 64)]
        return np.array([1.0 if (words[j // 64] >> (j % 64)) & 1 else -1.0 for j in range(k)])

    for v in np.flatnonzero(row >= 0)[:25]:
        s = rho(int(v)) * 1.0
        for i in range(g.off[v], g.off[v + 1]):
            s = s + rho(int(g.adj[i])) * w[i]
        bits = np.zeros(k // 64, dtype=np.uint64)
        for j in range(k):
            if s[j] >= 0:
                bits[j // 64] |= np.uint64(1) << np.uint64(j % 64)
        assert np.array_equal(sig[row[v]], bits), v


def test_weighted_simhash_tracks_weighted_cosine():
    g = dense_sbm()
    w = graphgen.edge_weights(g, 6, "exp")
    exact = oracle.weighted_similarities(g, w)
    row, nH = oracle.lsh_select(g, 128)
    k = 256
    sig = oracle.simhash_sketch(g, row, nH, k, seed=9, weights=w)
    est = oracle.lsh_similarities(g, oracle.SIMHASH, row, sig, exact, k)
    m = approx_arcs(g, row)
    theta = np.arccos(np.clip(exact[m], 0, 1))
    theta_hat = np.arccos(np.clip(est[m], 0, 1))
    assert abs((theta_hat - theta).mean()) < 0.03
    assert np.abs(theta_hat - theta).mean() < 0.12
    # the unweighted sketch of the same graph is a worse estimate of the
    # weighted cosine: the weights are used
    sig_u = oracle.simhash_sketch(g, row, nH, k, seed=9)
    est_u = oracle.lsh_similarities(g, oracle.SIMHASH, row, sig_u, exact, k)
    theta_u = np.arccos(np.clip(est_u[m], 0, 1))
    assert np.abs(theta_hat - theta).mean() < np.abs(theta_u - theta).mean()
