"""The sharded build's host-side plan and exchanges, with two gloo ranks on CPU.

Each rank owns a range of vertices balanced by arcs. The per-rank device steps
(triangle enumeration for the owned middle vertices, sorting and merging
runs) are emulated here with plain numpy; the product's plan and exchange
functions of paper_2012_11188_gb300.shard do the rest. The merged core order
and the all-reduced counts must equal the single-process oracle's.
"""
import os
import socket

import numpy as np
import pytest

import graphgen
import oracle
from paper_2012_11188_gb300 import shard


def sort_segments(keys, ids, seg_off):
    """Emulated device sort: each segment by key descending, id ascending."""
    for a, b in zip(seg_off[:-1], seg_off[1:]):
        if b - a > 1:
            o = np.lexsort((ids[a:b], -keys[a:b]))
            keys[a:b] = keys[a:b][o]
            ids[a:b] = ids[a:b][o]


def owned_triangle_counts(g, v0, v1):
    """Emulated device step: every triangle u < v < w of the degree
    orientation whose middle vertex v is owned adds one to both arcs of its
    three edges."""
    off, adj = g.off, g.adj
    deg = np.diff(off)
    key = lambda x: (deg[x], x)  # noqa: E731
    pos = {}
    for u in range(g.n):
        for i in range(off[u], off[u + 1]):
            pos[(u, int(adj[i]))] = i
    cnt = np.zeros(g.arcs, dtype=np.int64)
    outs = [set(int(x) for x in adj[off[u]:off[u + 1]] if key(int(x)) > key(u)) for u in range(g.n)]
    for v in range(v0, v1):
        ins = [int(x) for x in adj[off[v]:off[v + 1]] if key(int(x)) < key(v)]
        for u in ins:
            for w in outs[u] & outs[v]:
                for a, b in ((u, v), (v, w), (u, w)):
                    cnt[pos[(a, b)]] += 1
                    cnt[pos[(b, a)]] += 1
    return cnt


def run_rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = graphgen.sbm(400, 4, 0.2, 0.02, seed=1)  # replicated input
        ox = oracle.Index(g)
        deg = np.diff(g.off)
        # counts: partial per rank (the device step emulated), one all-reduce
        bounds, cnt = shard.sharded_counts(dist, g, rank, world, count_fn=owned_triangle_counts)
        v0, v1 = int(bounds[rank]), int(bounds[rank + 1])
        counts_ok = bool(np.array_equal(cnt.numpy() + 2, oracle.closed_counts(g)))
        # core order: local runs, one exchange, merge per mu (the device sort
        # emulated)
        no_off = g.off[v0:v1 + 1].astype(np.int64)
        mu_b, seg_off, mid, mthr = shard.sharded_core_order(dist, no_off, ox.no_sim, deg, v0, v1,
                                                            rank, world, sort_fn=sort_segments)
        lo, hi = int(mu_b[rank]), int(mu_b[rank + 1])
        a, b = int(ox.co_off[lo - 2]), int(ox.co_off[hi - 2])
        co_ok = bool(np.array_equal(mid, ox.co_id[a:b]) and np.array_equal(mthr, ox.co_thr[a:b])
                     and np.array_equal(seg_off + a, ox.co_off[lo - 2:hi - 1]))
        # replicas: the whole core order on every rank
        full = shard.allgather_v(dist, torch.from_numpy(mid), world).numpy()
        replica_ok = bool(np.array_equal(full, ox.co_id))
        q.put((rank, counts_ok, co_ok, replica_ok, v1 - v0, hi - lo))
    finally:
        dist.destroy_process_group()


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [1, 2, 3])
def test_sharded_core_order_and_counts_equal_single_process(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=run_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, counts_ok, co_ok, replica_ok, nv, nmu in res:
        assert counts_ok, f"rank {rank}: all-reduced counts differ from the oracle"
        assert co_ok, f"rank {rank}: merged CO of its mu range differs from the oracle"
        assert replica_ok, f"rank {rank}: gathered CO differs from the oracle"
        assert nv > 0 and nmu > 0


def test_partition_and_mu_ranges_cover_everything_once():
    g = graphgen.rmat(12, 16, seed=2)
    deg = np.diff(g.off)
    for world in (1, 2, 3, 8):
        b = shard.partition_by_arcs(g.off, world)
        assert b[0] == 0 and b[-1] == g.n and np.all(np.diff(b) >= 0)
        arcs = np.diff(g.off[b])
        assert arcs.sum() == g.arcs
        assert arcs.max() <= g.arcs / world + deg.max()  # balanced up to one row
        owners = shard.owner_of(np.arange(g.n), b)
        assert np.all(np.bincount(owners, minlength=world) == np.diff(b))
        m = shard.mu_ranges(deg, world)
        assert m[0] == 2 and m[-1] == deg.max() + 2 and np.all(np.diff(m) >= 0)
        sizes = shard.co_sizes(deg)
        assert sizes.sum() == g.arcs
        per = [sizes[m[r] - 2:m[r + 1] - 2].sum() for r in range(world)]
        assert sum(per) == g.arcs and max(per) <= g.arcs / world + sizes.max()
        # each rank's per-mu run lengths sum, over ranks, to |CO[mu]|
        runs = sum(shard.local_run_counts(deg[b[r]:b[r + 1]], 2, int(deg.max()) + 2)
                   for r in range(world))
        assert np.array_equal(runs, sizes)
