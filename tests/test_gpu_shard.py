"""Device steps of the sharded build: the counting restricted to each rank's
middle vertices adds up to the oracle's counts, the library's segmented sort
sorts and merges CO runs exactly like a plain lexicographic sort, and the
per-rank runs of a one-rank plan on the GPU give the oracle's core order."""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2012_11188_gb300 as gs
from paper_2012_11188_gb300 import shard

pytestmark = pytest.mark.gpu


def test_sort_segments_matches_lexsort():
    import torch
    rng = np.random.default_rng(5)
    lens = np.concatenate([rng.integers(0, 40, 300), [1, 0, 5000, 9000, 20000]])
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    keys = np.round(rng.random(off[-1]), 2)  # many ties
    ids = rng.permutation(off[-1]).astype(np.int32)
    want_k, want_i = keys.copy(), ids.copy()
    for a, b in zip(off[:-1], off[1:]):
        o = np.lexsort((want_i[a:b], -want_k[a:b]))
        want_k[a:b], want_i[a:b] = want_k[a:b][o], want_i[a:b][o]
    k = torch.from_numpy(keys).cuda()
    v = torch.from_numpy(ids).cuda()
    gs.sort_segments_desc(k, v, torch.from_numpy(off).cuda())
    assert np.array_equal(k.cpu().numpy(), want_k) and np.array_equal(v.cpu().numpy(), want_i)
    # host arrays are refused (SCAN_EINVAL)
    assert gs.load().scan_sort_segments_desc(keys.ctypes.data, ids.ctypes.data, off.ctypes.data,
                                             len(lens), int(off[-1]), 20000, 0) == -1


def test_one_rank_plan_with_device_sorts_is_the_oracle_core_order():
    g = graphgen.rmat(13, 16, seed=4)
    ox = oracle.Index(g)
    deg = np.diff(g.off)
    mu_b = shard.mu_ranges(deg, 1)
    ids, thr, dest, per_mu = shard.local_runs(g.off.astype(np.int64), ox.no_sim, deg, 0, g.n,
                                              mu_b, shard.device_sort)
    run_len = per_mu.reshape(-1, 1)
    seg_off, mid, mthr = shard.merge_runs(ids, thr, run_len, shard.device_sort)
    assert np.array_equal(mid, ox.co_id) and np.array_equal(mthr, ox.co_thr)
    assert np.array_equal(seg_off, ox.co_off)


@pytest.mark.parametrize("world", [1, 3, 5])
def test_range_counts_of_a_partition_add_up_to_the_oracle(world):
    # R-MAT rows longer than 512 (the CTA kernel's items) and short rows (the
    # warp kernel) fall on both sides of the range bounds
    g = graphgen.rmat(15, 16, seed=3)
    want = oracle.closed_counts(g).astype(np.int64) - 2
    bounds = shard.partition_by_arcs(g.off, world)
    total = np.zeros(g.arcs, dtype=np.int64)
    for r in range(world):
        part = shard.device_counts(g, int(bounds[r]), int(bounds[r + 1]))
        assert part.dtype == np.uint32 and part.shape == (g.arcs,)
        total += part
    assert np.array_equal(total, want)


def test_range_counts_device_output_and_empty_range():
    import torch
    g = graphgen.sbm(600, 3, 0.2, 0.02, seed=2)
    host = gs.closed_counts_range(g, 100, 400)
    dev = torch.zeros(g.arcs, dtype=torch.int32, device="cuda")
    gs.closed_counts_range(g, 100, 400, out=dev)
    assert np.array_equal(dev.cpu().numpy().view(np.uint32), host)
    assert not gs.closed_counts_range(g, 250, 250).any()
    # both arcs of an edge carry the same count
    off, adj = g.off, g.adj
    for u in (0, 150, 599):
        for i in range(off[u], off[u + 1]):
            v = adj[i]
            j = off[v] + np.searchsorted(adj[off[v]:off[v + 1]], u)
            assert host[i] == host[j]


def middle_vertex_counts(g, v0, v1):
    """Plain restatement: every triangle, ordered by (degree, id), adds one to
    both arcs of its three edges when its middle vertex lies in [v0, v1)."""
    off, adj = g.off, g.adj
    deg = np.diff(off)
    pos = {}
    for u in range(g.n):
        for i in range(off[u], off[u + 1]):
            pos[(u, int(adj[i]))] = i
    nbr = [set(int(x) for x in adj[off[u]:off[u + 1]]) for u in range(g.n)]
    cnt = np.zeros(g.arcs, dtype=np.int64)
    for a in range(g.n):
        for b in nbr[a]:
            if b <= a:
                continue
            for c in nbr[a] & nbr[b]:
                if c <= b:
                    continue
                mid = sorted((a, b, c), key=lambda x: (deg[x], x))[1]
                if v0 <= mid < v1:
                    for x, y in ((a, b), (b, c), (a, c)):
                        cnt[pos[(x, y)]] += 1
                        cnt[pos[(y, x)]] += 1
    return cnt


def test_range_counts_equal_the_middle_vertex_definition():
    g = graphgen.sbm(300, 3, 0.25, 0.03, seed=7)
    for v0, v1 in ((0, 300), (0, 1), (37, 180), (180, 300), (299, 300)):
        assert np.array_equal(gs.closed_counts_range(g, v0, v1).astype(np.int64),
                              middle_vertex_counts(g, v0, v1)), (v0, v1)
