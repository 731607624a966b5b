"""The multi-GPU benchmark path runs independent replicas: the timed region is
the slowest rank's and the value counts every rank's edges. Checked with two
gloo ranks on the CPU (no GPU involved)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    mx = bench.replica_max_ms(times[rank], ws, "cpu")
    out[rank] = (mx, bench.replica_value(1000, 5, ws, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    times = [120.0, 180.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        mx, val = out[r]
        assert mx == 180.0
        assert val == pytest.approx(1000 * 5 * 2 / 0.18)


def test_single_rank_is_identity():
    assert bench.replica_max_ms(42.0, 1) == 42.0
    assert bench.replica_value(10, 2, 1, 1000.0) == 20.0
