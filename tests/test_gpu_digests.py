"""Full-size bit-exact parity through digests.

The CPU oracle's index and labels at full size take minutes to hours to
compute, so ``tests/golden/make_digests.py`` computed them once (oracle and
input generators only) and stored SHA-256 digests of every array. Here the
CUDA library builds the same inputs in the launch configuration bench.py
times, and the digest of every exported array and label vector must equal the
oracle's:

* R-MAT scale 24, edge factor 16, seed 1: the exact cosine index (sim, NO,
  CO), the labels of 54 (mu, eps) queries with hubs, and the LSH indexes
  (SimHash 64 and 256, k-partition MinHash 64; degree threshold 128, seed 1)
  with their labels at mu = 5, eps in {.3, .5, .7};
* all 2048 graphs of the batched SBM build, built in one batched call, each
  graph's index and the labels of its 8 queries.

A digest of each input graph is checked first, so that an input generated
differently on this machine is reported as such and not as a parity failure.
"""
import json
import os
import sys

import numpy as np
import pytest

import graphgen
import paper_2012_11188_gb300 as gs

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import digests  # noqa: E402

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_rmat_s24_exact_and_lsh_indexes_equal_oracle_digests():
    import torch
    exp = load("digests_rmat_s24.json")
    w = exp["workload"]
    g = graphgen.rmat(w["scale"], w["edgefactor"], seed=w["seed"])
    assert (g.n, g.arcs) == (exp["n"], exp["arcs"])
    assert digests.graph_digest(g) == exp["graph"], "input graph differs from the one hashed"
    off = torch.from_numpy(g.off).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    with gs.ScanIndex.build((off, adj), gs.COSINE) as ix:
        ex = ix.export()
        for k in digests.INDEX_KEYS:
            assert digests.array_digest(k, ex[k]) == exp["cosine"][k], k
        del ex
        qs = exp["queries"]
        for s in range(0, len(qs), 9):
            part = qs[s:s + 9]
            mus = np.array([q[0] for q in part], np.int32)
            epss = np.array([q[1] for q in part], np.float64)
            labs = ix.query_batch(mus, epss, hubs=exp["hubs"])
            for i, q in enumerate(part):
                assert digests.labels_digest([labs[i]]) == exp["cosine_labels"][s + i], q
        # the single-query entry point gives the same labels
        lab = ix.query(5, 0.5, hubs=True)
        assert digests.labels_digest([lab]) == exp["cosine_labels"][qs.index([5, 0.5])]
    lsh = exp["lsh"]
    lq = lsh["queries"]
    for name, kind, k in (("simhash64", gs.COSINE, 64), ("simhash256", gs.COSINE, 256),
                          ("minhash64", gs.JACCARD, 64)):
        p = gs.make_lsh(kind, k, lsh["threshold"], seed=lsh["seed"], kpartition=lsh["kpartition"])
        with gs.ScanIndex.build((off, adj), kind, lsh=p) as ix:
            assert digests.index_digest(ix.export()) == lsh[name]["index"], name
            labs = ix.query_batch(np.array([q[0] for q in lq], np.int32),
                                  np.array([q[1] for q in lq], np.float64), hubs=True)
            for i, q in enumerate(lq):
                assert digests.labels_digest([labs[i]]) == lsh[name]["labels"][i], (name, q)


def test_batch_2048_graphs_equal_oracle_digests():
    import torch
    exp = load("digests_batch_2048.json")
    w, hx = exp["workload"], exp["hex"]
    rows = exp["graphs"]
    ps = graphgen.batch_sbm_params(w["count"], seed=w["seed"])
    gl = [graphgen.sbm(p.n, p.blocks, p.p_in, p.p_out, p.seed) for p in ps]
    for i, g in enumerate(gl):
        assert [g.n, g.arcs] == rows[i][:2], i
        assert digests.graph_digest(g, hx) == rows[i][2], f"input graph {i} differs"
    mus, epss = graphgen.batch_queries(w["count"], w["queries_per_graph"], seed=w["query_seed"])
    dev = [(torch.from_numpy(g.off).cuda(), torch.from_numpy(g.adj).cuda()) for g in gl]
    hs = gs.ScanIndex.build_batch(dev, gs.COSINE)
    try:
        bad = []
        for i, h in enumerate(hs):
            if digests.index_digest(h.export(), hx) != rows[i][3]:
                bad.append(("index", i))
                continue
            labs = h.query_batch(mus[i], epss[i], hubs=exp["hubs"])
            if digests.labels_digest(list(labs), hx) != rows[i][4]:
                bad.append(("labels", i))
        assert not bad, f"{len(bad)} graphs differ, first {bad[:8]}"
    finally:
        for h in hs:
            h.free()
