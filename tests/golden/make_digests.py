#!/usr/bin/env python
"""Writes the expected full-size digests from the CPU oracle alone.

The GPU parity tests at full size hash what the CUDA library exports and
compare with these digests. Everything here runs on the CPU and calls only
``oracle`` (the index, the queries) and ``graphgen`` (the seeded inputs);
the CUDA library is never loaded.

    python tests/golden/make_digests.py rmat24   # about 20 min, ~30 GB of RAM
    python tests/golden/make_digests.py batch    # a few minutes on 8 cores

Outputs: ``digests_rmat_s24.json`` and ``digests_batch_2048.json`` beside
this file. Workloads:

* R-MAT scale 24, edge factor 16, (a, b, c) = (.57, .19, .19), seed 1: the
  exact cosine index (counts by Section 3.1's definition, NO and CO by
  Algorithm 2) and the labels (hubs flagged, Section 4.3) of every
  (mu, eps) with mu in {2, 4, 5, 8, 16, 32} and eps = k/10, k = 1..9; the
  LSH indexes (Section 5) with degree threshold 128 and seed 1: SimHash 64
  and 256 bits (cosine), k-partition MinHash 64 (Jaccard), with their labels
  at mu = 5, eps in {.3, .5, .7}.
* The 2048-graph SBM batch (n log-uniform in [100, 20000], 2-64 blocks,
  p_in uniform in [.02, .2], p_out = p_in/50, batch seed 1): per graph the
  exact cosine index and the labels of its 8 queries from
  ``graphgen.batch_queries(2048, 8, seed=1)``.
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import numpy as np  # noqa: E402

import digests  # noqa: E402
import graphgen  # noqa: E402
import oracle  # noqa: E402

RMAT24 = {"scale": 24, "edgefactor": 16, "seed": 1}
S24_QUERIES = [(mu, k / 10) for mu in (2, 4, 5, 8, 16, 32) for k in range(1, 10)]
LSH_QUERIES = [(5, 0.3), (5, 0.5), (5, 0.7)]
LSH_MODES = [("simhash64", oracle.COSINE, 64), ("simhash256", oracle.COSINE, 256),
             ("minhash64", oracle.JACCARD, 64)]
LSH_T, LSH_SEED = 128, 1
BATCH = {"count": 2048, "seed": 1, "queries_per_graph": 8, "query_seed": 1}
BATCH_HEX = 24


def _ix_dict(ox):
    return {k: getattr(ox, k) for k in digests.INDEX_KEYS}


def _log(*a):
    print(time.strftime("%H:%M:%S"), *a, flush=True)


def rmat24():
    g = graphgen.rmat(RMAT24["scale"], RMAT24["edgefactor"], seed=RMAT24["seed"])
    _log("graph", g.n, g.arcs)
    out = {"workload": RMAT24, "n": g.n, "arcs": g.arcs, "graph": digests.graph_digest(g),
           "queries": [[mu, eps] for mu, eps in S24_QUERIES], "hubs": True}
    cnt = oracle.closed_counts(g)
    _log("counts")
    sims = {oracle.COSINE: oracle.similarities(g, cnt, oracle.COSINE)}
    sims[oracle.JACCARD] = oracle.similarities(g, cnt, oracle.JACCARD)
    del cnt
    ox = oracle.Index(g, oracle.COSINE, sim=sims[oracle.COSINE])
    _log("exact index")
    out["cosine"] = {k: digests.array_digest(k, getattr(ox, k)) for k in digests.INDEX_KEYS}
    out["cosine_labels"] = [digests.labels_digest([ox.query(mu, eps, hubs=True)])
                            for mu, eps in S24_QUERIES]
    _log("exact queries")
    del ox
    out["lsh"] = {"threshold": LSH_T, "seed": LSH_SEED, "kpartition": True,
                  "queries": [[mu, eps] for mu, eps in LSH_QUERIES]}
    for name, kind, k in LSH_MODES:
        ox = oracle.LSHIndex(g, kind, k, T=LSH_T, seed=LSH_SEED, exact_sim=sims[kind])
        out["lsh"][name] = {"index": digests.index_digest(_ix_dict(ox)),
                            "labels": [digests.labels_digest([ox.query(mu, eps, hubs=True)])
                                       for mu, eps in LSH_QUERIES]}
        _log(name)
        del ox
    return out


def _batch_one(args):
    i, p, mus, epss = args
    g = graphgen.sbm(p.n, p.blocks, p.p_in, p.p_out, p.seed)
    ox = oracle.Index(g, oracle.COSINE)
    labs = [ox.query(int(mu), float(eps), hubs=True) for mu, eps in zip(mus, epss)]
    return i, [g.n, g.arcs, digests.graph_digest(g, BATCH_HEX),
               digests.index_digest(_ix_dict(ox), BATCH_HEX),
               digests.labels_digest(labs, BATCH_HEX)]


def batch(workers: int):
    ps = graphgen.batch_sbm_params(BATCH["count"], seed=BATCH["seed"])
    mus, epss = graphgen.batch_queries(BATCH["count"], BATCH["queries_per_graph"],
                                       seed=BATCH["query_seed"])
    oracle.build()
    jobs = [(i, p, mus[i], epss[i]) for i, p in enumerate(ps)]
    jobs.sort(key=lambda j: -j[1].n * j[1].n * j[1].p_in / j[1].blocks)  # large graphs first
    rows = [None] * len(jobs)
    with mp.get_context("spawn").Pool(workers) as pool:
        for done, (i, row) in enumerate(pool.imap_unordered(_batch_one, jobs, chunksize=1)):
            rows[i] = row
            if done % 256 == 0:
                _log("batch", done)
    return {"workload": BATCH, "kind": "cosine", "hubs": True, "hex": BATCH_HEX,
            "columns": ["n", "arcs", "graph", "index", "labels"], "graphs": rows}


def main():
    what = sys.argv[1] if len(sys.argv) > 1 else ""
    if what == "rmat24":
        res, name = rmat24(), "digests_rmat_s24.json"
    elif what == "batch":
        res, name = batch(int(sys.argv[2]) if len(sys.argv) > 2 else max(1, os.cpu_count() - 1)), \
            "digests_batch_2048.json"
    else:
        print(__doc__)
        return 2
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(res, f, indent=None, separators=(",", ":"))
        f.write("\n")
    _log("wrote", name)
    return 0


if __name__ == "__main__":
    sys.exit(main())
