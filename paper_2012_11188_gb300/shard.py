"""Sharded index build over ranks: the host-side plan and its exchanges.

One process per GPU. The CSR is replicated on every rank (R-MAT scale 24 is
2.2 GB). The build shards as follows:

1. Vertices are split into contiguous ranges of about equal arc count
   (``partition_by_arcs``); rank r owns the vertices [b_r, b_{r+1}).
2. Closed counts (Section 3.1): every triangle u < v < w of the degree
   orientation (Section 6.1) has exactly one middle vertex v, and the rank
   that owns v enumerates it, adding one to the three oriented edges
   (u,v), (v,w), (u,w). Each rank therefore holds partial counts of edges
   anywhere in the graph; one sum all-reduce of the per-arc counts
   (``allreduce_counts``) gives every rank the full counts of every edge.
3. Similarities and the neighbour order (Algorithm 2, MakeNeighborOrder) are
   local to a vertex: each rank computes them for the rows it owns.
4. Core order (Algorithm 2, MakeCoreOrder): the segments CO[mu],
   mu = 2..maxdeg+1, are split into contiguous mu ranges of about equal total
   size (``mu_ranges``); rank r sorts, for every mu, the entries
   (NO_sim[v][mu-2], v) of the vertices it owns into one run, sends the runs
   of each mu range to the rank that owns the range (``exchange_runs``, one
   all-to-all), and that rank merges, for every mu of its range, the runs it
   received from all ranks.
5. Queries cross the shards (the union-find of Algorithm 5 follows edges
   anywhere), so the index is replicated for serving: one all-gather of the
   owned NO rows and of the CO segments (``allgather_v``).

Exchanges run over ``torch.distributed`` (NCCL on GPUs, gloo on the CPU):
an all-reduce of 4 bytes per arc and all-to-alls of 12 bytes per CO entry.
The counting, sorting and merging are device work: ``device_counts`` is the
library's counting restricted to a range of middle vertices, and the
functions that sort take the sort as a callable (``device_sort`` is the
library's segmented sort). Not measured on more than one GPU: every run of
this project has one.
"""
from __future__ import annotations

import numpy as np


def partition_by_arcs(off: np.ndarray, world: int) -> np.ndarray:
    """Vertex bounds b[0..world] (b[0] = 0, b[world] = n), non-decreasing, such
    that rank r's vertices [b[r], b[r+1]) hold about A / world arcs."""
    off = np.asarray(off, dtype=np.int64)
    n = off.shape[0] - 1
    A = int(off[-1])
    targets = (np.arange(world + 1, dtype=np.int64) * A) // max(world, 1)
    b = np.searchsorted(off, targets, side="left").astype(np.int64)
    b[0], b[-1] = 0, n
    return np.minimum.accumulate(b[::-1])[::-1] if world > 0 else b


def owner_of(v: np.ndarray, bounds: np.ndarray) -> np.ndarray:
    """Rank owning each vertex id."""
    return np.searchsorted(bounds, np.asarray(v), side="right") - 1


def co_sizes(deg: np.ndarray) -> np.ndarray:
    """|CO[mu]| = #{v : d_v + 1 >= mu} for mu = 2..maxdeg+1 (index mu - 2)."""
    deg = np.asarray(deg, dtype=np.int64)
    if deg.shape[0] == 0 or deg.max() == 0:
        return np.zeros(0, dtype=np.int64)
    h = np.bincount(deg)  # h[d] = #{v : d_v = d}
    ge = h[::-1].cumsum()[::-1]  # ge[d] = #{v : d_v >= d}
    return ge[1:].astype(np.int64)  # mu - 1 = d, d = 1..maxdeg


def mu_ranges(deg: np.ndarray, world: int) -> np.ndarray:
    """mu bounds m[0..world] over 2..maxdeg+2: rank r owns CO[mu] for
    m[r] <= mu < m[r+1], the ranges of about equal total size."""
    sizes = co_sizes(deg)
    total = int(sizes.sum())
    pref = np.concatenate([[0], np.cumsum(sizes)])
    targets = (np.arange(world + 1, dtype=np.int64) * total) // max(world, 1)
    idx = np.searchsorted(pref, targets, side="left")
    idx[0], idx[-1] = 0, sizes.shape[0]
    idx = np.minimum.accumulate(idx[::-1])[::-1]
    return (idx + 2).astype(np.int64)


def local_run_counts(deg_owned: np.ndarray, mu_lo: int, mu_hi: int) -> np.ndarray:
    """For mu = mu_lo..mu_hi-1: how many owned vertices are in CO[mu]."""
    if mu_hi <= mu_lo:
        return np.zeros(0, dtype=np.int64)
    d1 = np.asarray(deg_owned, dtype=np.int64) + 1  # vertex in CO[mu] iff d + 1 >= mu
    mus = np.arange(mu_lo, mu_hi, dtype=np.int64)
    return (d1.shape[0] - np.searchsorted(np.sort(d1), mus, side="left")).astype(np.int64)


def local_runs(no_off: np.ndarray, no_sim: np.ndarray, deg: np.ndarray, v0: int, v1: int,
               mu_bounds: np.ndarray, sort_runs):
    """The CO runs of the owned vertices [v0, v1), grouped by destination rank.

    no_off / no_sim: the owned rows of the neighbour order (no_off[v - v0]
    indexes no_sim for the row of v, n_owned + 1 entries). sort_runs(keys,
    ids, seg_off) sorts each segment by key descending, id ascending, in
    place (device work). Returns (ids, thr, per-destination entry counts,
    per-mu counts in mu order)."""
    world = mu_bounds.shape[0] - 1
    deg_o = np.asarray(deg[v0:v1], dtype=np.int64)
    mu_lo, mu_hi = int(mu_bounds[0]), int(mu_bounds[-1])
    # vertex v of degree d contributes (NO_sim[v][mu-2], v) to CO[mu] for
    # mu = 2..d+1: its whole NO row, in order (rows are contiguous)
    no_off = np.asarray(no_off, dtype=np.int64)
    total = int(no_off[-1] - no_off[0])
    verts = np.repeat(np.arange(v0, v1, dtype=np.int64), deg_o)
    rank_in_row = np.arange(total, dtype=np.int64) - np.repeat(no_off[:-1] - no_off[0], deg_o)
    mu = rank_in_row + 2
    order = np.argsort(mu, kind="stable")
    ids = verts[order].astype(np.int32)
    thr = np.asarray(no_sim[no_off[0]:no_off[-1]], dtype=np.float64)[order]
    per_mu = np.bincount(mu - mu_lo, minlength=mu_hi - mu_lo).astype(np.int64)[:mu_hi - mu_lo]
    seg_off = np.concatenate([[0], np.cumsum(per_mu)]).astype(np.int64)
    sort_runs(thr, ids, seg_off)
    dest = np.array([int(seg_off[mu_bounds[r + 1] - mu_lo] - seg_off[mu_bounds[r] - mu_lo])
                     for r in range(world)], dtype=np.int64)
    return ids, thr, dest, per_mu


def exchange_runs(dist, ids: np.ndarray, thr: np.ndarray, dest_counts: np.ndarray,
                  per_mu: np.ndarray, mu_bounds: np.ndarray, rank: int, world: int, group=None):
    """One all-to-all of the runs (12 bytes per entry) and one of their per-mu
    lengths. Returns, for this rank's mu range, ids and thresholds in
    (mu, source rank) order and the per-(mu, source) run lengths [n_mu, world]."""
    import torch
    lo, hi = int(mu_bounds[rank]), int(mu_bounds[rank + 1])
    # per-mu lengths: to rank r, the lengths of this rank's runs of r's range
    send_len = per_mu.astype(np.int64)
    len_splits = [int(mu_bounds[r + 1] - mu_bounds[r]) for r in range(world)]
    recv_len = torch.empty(world * (hi - lo), dtype=torch.int64)
    dist.all_to_all_single(recv_len, torch.from_numpy(np.ascontiguousarray(send_len)),
                           [hi - lo] * world, len_splits, group=group)
    run_len = recv_len.numpy().reshape(world, hi - lo)  # [source, mu]
    # counts of entries each source sends here
    recv_counts = run_len.sum(axis=1)
    out_ids = torch.empty(int(recv_counts.sum()), dtype=torch.int32)
    out_thr = torch.empty(int(recv_counts.sum()), dtype=torch.float64)
    send_splits = [int(c) for c in dest_counts]
    recv_splits = [int(c) for c in recv_counts]
    dist.all_to_all_single(out_ids, torch.from_numpy(np.ascontiguousarray(ids)), recv_splits,
                           send_splits, group=group)
    dist.all_to_all_single(out_thr, torch.from_numpy(np.ascontiguousarray(thr)), recv_splits,
                           send_splits, group=group)
    # reorder from (source, mu) to (mu, source)
    src_ids = np.split(out_ids.numpy(), np.cumsum(recv_counts)[:-1])
    src_thr = np.split(out_thr.numpy(), np.cumsum(recv_counts)[:-1])
    ids_m, thr_m = [], []
    for j in range(hi - lo):
        for s in range(world):
            a = int(run_len[s, :j].sum())
            b = a + int(run_len[s, j])
            ids_m.append(src_ids[s][a:b])
            thr_m.append(src_thr[s][a:b])
    cat_i = np.concatenate(ids_m) if ids_m else np.zeros(0, np.int32)
    cat_t = np.concatenate(thr_m) if thr_m else np.zeros(0, np.float64)
    return cat_i, cat_t, run_len.T.copy()


def merge_runs(ids: np.ndarray, thr: np.ndarray, run_len: np.ndarray, merge_fn):
    """For every mu of the range, merge its sorted runs (one per source rank)
    into CO[mu]: merge_fn(keys, ids, seg_off) orders each segment by key
    descending, id ascending (device work). Returns (co_off_local, ids, thr)."""
    per_mu = run_len.sum(axis=1)
    seg_off = np.concatenate([[0], np.cumsum(per_mu)]).astype(np.int64)
    merge_fn(thr, ids, seg_off)
    return seg_off, ids, thr


def device_sort(keys, ids, seg_off):
    """The library's segmented sort (scan_sort_segments_desc) as the sort and
    merge step of local_runs / merge_runs, on the current CUDA device."""
    import torch
    from .scan import sort_segments_desc
    k = torch.from_numpy(np.ascontiguousarray(keys)).cuda()
    v = torch.from_numpy(np.ascontiguousarray(ids)).cuda()
    o = torch.from_numpy(np.ascontiguousarray(seg_off, dtype=np.int64)).cuda()
    sort_segments_desc(k, v, o)
    keys[:] = k.cpu().numpy()
    ids[:] = v.cpu().numpy()


def device_counts(g, v0: int, v1: int, out=None):
    """Step 2 on this rank's GPU: per-arc triangle counts of the triangles
    whose middle vertex lies in [v0, v1) (scan_closed_counts_range)."""
    from .scan import closed_counts_range
    return closed_counts_range(g, v0, v1, out=out)


def sharded_core_order(dist, no_off, no_sim, deg, v0: int, v1: int, rank: int, world: int,
                       sort_fn=device_sort, group=None):
    """Step 4 on one rank: the runs of its vertices [v0, v1) (no_off / no_sim:
    its NO rows, as for local_runs), one exchange by mu range, and the merge
    of the runs of every mu of its range. Returns (mu_bounds, co_off_local,
    ids, thr): CO[mu] for mu_bounds[rank] <= mu < mu_bounds[rank + 1]."""
    mu_b = mu_ranges(deg, world)
    ids, thr, dest, per_mu = local_runs(no_off, no_sim, deg, v0, v1, mu_b, sort_fn)
    rid, rthr, run_len = exchange_runs(dist, ids, thr, dest, per_mu, mu_b, rank, world, group=group)
    seg_off, mid, mthr = merge_runs(rid, rthr, run_len, sort_fn)
    return mu_b, seg_off, mid, mthr


def allreduce_counts(dist, counts, group=None):
    """Sum the per-arc partial counts of all ranks, in place (step 2)."""
    dist.all_reduce(counts, group=group)
    return counts


def sharded_counts(dist, g, rank: int, world: int, count_fn=device_counts, group=None):
    """Steps 1 and 2 on one rank: this rank's vertex range by arcs, its partial
    counts (count_fn(g, v0, v1): the device counting by default), and the sum
    over all ranks. Returns (bounds, t) with t[arc] = |N(u) ∩ N(v)| (int64
    tensor) on every rank."""
    import torch
    bounds = partition_by_arcs(g.off, world)
    part = np.asarray(count_fn(g, int(bounds[rank]), int(bounds[rank + 1])))
    t = torch.from_numpy(part.astype(np.int64))
    allreduce_counts(dist, t, group=group)
    return bounds, t


def allgather_v(dist, local, world: int, group=None):
    """Concatenation over ranks of arrays of different lengths (replicas)."""
    import torch
    t = torch.as_tensor(local)
    n = torch.tensor([t.shape[0]], dtype=torch.int64)
    sizes = torch.empty(world, dtype=torch.int64)
    dist.all_to_all_single(sizes, n.repeat(world), [1] * world, [1] * world, group=group)
    out = torch.empty(int(sizes.sum()), dtype=t.dtype)
    dist.all_to_all_single(out, t.repeat(world), [int(x) for x in sizes],
                           [t.shape[0]] * world, group=group)
    return out
