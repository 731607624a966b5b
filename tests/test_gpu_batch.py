"""Batched multi-graph build: every graph's index, built in one pass over the
packed graphs, equals the index built alone and the CPU oracle's."""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2012_11188_gb300 as gs

pytestmark = pytest.mark.gpu

KEYS = ("sim", "no_id", "no_sim", "co_off", "co_id", "co_thr")


def batch_graphs(count, seed, n_hi=3000):
    ps = graphgen.batch_sbm_params(count, seed=seed, n_hi=n_hi)
    gl = [graphgen.sbm(p.n, p.blocks, p.p_in, p.p_out, p.seed) for p in ps]
    # degenerate members: no vertices, no edges, one edge
    gl.insert(3, graphgen.CSR(np.zeros(1, np.int64), np.zeros(0, np.int32)))
    gl.insert(7, graphgen.CSR(np.zeros(9, np.int64), np.zeros(0, np.int32)))
    gl.insert(11, graphgen.from_edges(2, [(0, 1)]))
    return gl


@pytest.mark.parametrize("kind", [gs.COSINE, gs.JACCARD])
def test_batch_equals_single_and_oracle(kind):
    gl = batch_graphs(40, seed=1)
    hs = gs.ScanIndex.build_batch(gl, kind)
    try:
        for i, (g, h) in enumerate(zip(gl, hs)):
            assert (h.n, h.arcs) == (g.n, g.arcs)
            with gs.ScanIndex.build(g, kind) as single:
                a, b = h.export(), single.export()
                for k in KEYS:
                    assert np.array_equal(a[k], b[k]), (i, k)
                for mu, eps in ((2, 0.3), (5, 0.5), (8, 0.7)):
                    assert np.array_equal(h.query(mu, eps, hubs=True), single.query(mu, eps, hubs=True))
            if i % 8 == 0:
                ox = oracle.Index(g, kind)
                a = h.export()
                for k in KEYS:
                    assert np.array_equal(a[k], getattr(ox, k)), (i, k)
    finally:
        for h in hs:
            h.free()


def test_batch_device_inputs_and_handle_lifetimes():
    import torch
    gl = batch_graphs(12, seed=2)
    dev = [(torch.from_numpy(g.off.astype(np.int32)).cuda(), torch.from_numpy(g.adj).cuda()) for g in gl]
    hs = gs.ScanIndex.build_batch(dev, gs.COSINE)
    refs = [oracle.Index(g) for g in gl[:4]]
    # free every other handle; the rest stay valid
    for h in hs[1::2]:
        h.free()
    for i in (0, 2):
        a = hs[i].export()
        for k in KEYS:
            assert np.array_equal(a[k], getattr(refs[i], k)), (i, k)
        assert np.array_equal(hs[i].query(3, 0.4, hubs=True), refs[i].query(3, 0.4, hubs=True))
    for h in hs[0::2]:
        h.free()


def test_batch_query_batch_on_member():
    gl = batch_graphs(6, seed=3)
    hs = gs.ScanIndex.build_batch(gl, gs.COSINE)
    try:
        mus = np.array([2, 3, 5, 8], np.int32)
        epss = np.array([0.2, 0.4, 0.6, 0.8])
        for g, h in zip(gl, hs):
            ox = oracle.Index(g)
            lab = h.query_batch(mus, epss, hubs=True)
            for i in range(4):
                assert np.array_equal(lab[i], ox.query(int(mus[i]), float(epss[i]), hubs=True))
    finally:
        for h in hs:
            h.free()


def test_batch_rejects_a_bad_member():
    gl = batch_graphs(5, seed=4)
    bad = gl[1]
    adj = bad.adj.copy()
    adj[0] = bad.n + 5  # out of the graph's own range (but inside the packed range)
    gl[1] = graphgen.CSR(bad.off, adj)
    with pytest.raises(gs.ScanError) as e:
        gs.ScanIndex.build_batch(gl, gs.COSINE)
    assert e.value.status == -3


CONFIGS = [
    {"warp_deg": 128, "cta_chunk": 1024, "long_list": 32, "rounds": 8},
    {"warp_deg": 2048, "cta_chunk": 8192, "long_list": 256, "rounds": 4, "dense_div": 0},
    {"warp_deg": 256, "cta_chunk": 256, "long_list": 1, "rounds": 8},
    # batch members of 2048+ vertices and degree >= n/64 go to the dense path
    {"dense_div": 64, "dense_min_n": 2048},
]


def test_batch_with_dense_members_is_the_oracle():
    """Members routed to the dense GEMM path and members of the union build
    come back in the caller's order, each equal to the oracle."""
    gl = batch_graphs(12, seed=9)
    gl.insert(2, graphgen.sbm(2500, 2, 0.3, 0.01, seed=3))   # dense under the setting below
    gl.insert(6, graphgen.sbm(2100, 1, 0.2, 0.2, seed=4))
    gs.set_count_config({"dense_div": 16, "dense_min_n": 2048})
    try:
        hs = gs.ScanIndex.build_batch(gl, gs.COSINE)
    finally:
        gs.set_count_config(None)
    try:
        for i in (0, 2, 5, 6, 9, len(gl) - 1):
            ox = oracle.Index(gl[i])
            a = hs[i].export()
            for k in KEYS:
                assert np.array_equal(a[k], getattr(ox, k)), (i, k)
            assert np.array_equal(hs[i].query(3, 0.4, hubs=True), ox.query(3, 0.4, hubs=True))
    finally:
        for h in hs:
            h.free()


@pytest.mark.parametrize("cfg", CONFIGS)
def test_every_count_config_gives_the_same_index(cfg):
    """The per-degree-bucket strategy changes only the speed: the index of a
    skewed graph and of a batch is identical under every configuration."""
    g = graphgen.rmat(14, 16, seed=3)
    gl = batch_graphs(10, seed=4)
    with gs.ScanIndex.build(g, gs.COSINE) as ref:
        want = ref.export()
    refs = [h.export() for h in gs.ScanIndex.build_batch(gl, gs.COSINE)]
    gs.set_count_config(cfg)
    try:
        with gs.ScanIndex.build(g, gs.COSINE) as ix:
            got = ix.export()
        hs = gs.ScanIndex.build_batch(gl, gs.COSINE)
        outs = [h.export() for h in hs]
        for h in hs:
            h.free()
    finally:
        gs.set_count_config(None)
    for k in KEYS:
        assert np.array_equal(got[k], want[k]), k
    for a, b in zip(outs, refs):
        for k in KEYS:
            assert np.array_equal(a[k], b[k]), k


def test_autotune_batch_records_and_uses_its_choice(tmp_path):
    gs.tuning_clear()
    gl = batch_graphs(30, seed=6)
    res = gs.autotune_batch(gl, gs.COSINE, reps=1)
    assert res["best_ms"] <= res["default_ms"] and res["best_ms"] > 0
    best = res["best"]
    # the batch's degree class now maps to the tuned configuration
    n = sum(g.n for g in gl)
    arcs = sum(g.arcs for g in gl)
    nmax = max(g.n for g in gl)
    assert gs.count_config_for(nmax, n, arcs) == best
    path = tmp_path / "tune.txt"
    gs.tuning_save(str(path))
    gs.tuning_clear()
    gs.tuning_load(str(path))
    assert gs.count_config_for(nmax, n, arcs) == best
    # a tuned batched build is the oracle's
    hs = gs.ScanIndex.build_batch(gl, gs.COSINE)
    try:
        for i in (0, 5, 17):
            ox = oracle.Index(gl[i])
            a = hs[i].export()
            for k in KEYS:
                assert np.array_equal(a[k], getattr(ox, k)), (i, k)
    finally:
        for h in hs:
            h.free()
        gs.tuning_clear()
