"""Serving runtime: continuous batching of queries and builds (include/scan_serve.h).

Every result obtained through the server, with other queries and builds in
flight, must be bit-identical to the same request made alone.
"""
import numpy as np
import pytest

import graphgen
import paper_2012_11188_gb300 as gs

pytestmark = pytest.mark.gpu


def random_queries(count, seed):
    rng = np.random.default_rng(seed)
    mus = rng.integers(2, 33, count).astype(np.int32)
    epss = np.round(rng.integers(2, 19, count) * 0.05, 2)
    return mus, epss


@pytest.fixture(scope="module")
def index():
    g = graphgen.rmat(16, 16, seed=5)
    ix = gs.ScanIndex.build(g, gs.COSINE)
    yield g, ix
    ix.free()


@pytest.mark.parametrize("max_batch", [64, 1])
def test_queries_and_builds_in_the_mix_equal_alone(index, max_batch):
    g, ix = index
    mus, epss = random_queries(120, 1)
    builds = [graphgen.sbm(3000 + 1000 * i, 10, 0.08, 0.002, seed=10 + i) for i in range(3)]
    with gs.Server(max_batch=max_batch) as srv:
        outs, tickets = [], []
        bt = {}
        for i in range(len(mus)):
            out = np.empty(g.n, np.int32)
            tickets.append(srv.submit_query(ix, int(mus[i]), float(epss[i]), out, hubs=i % 2 == 0))
            outs.append(out)
            if i % 40 == 0:
                bg = builds[i // 40]
                bt[srv.submit_build(bg, gs.COSINE)] = bg
        for t in tickets:
            assert srv.wait(t, timeout_ms=120000) is None
        built = {t: srv.wait(t, timeout_ms=120000) for t in bt}
        st = srv.stats()
        assert st["completed"] == len(mus) and st["p99_ms"] >= st["p50_ms"] > 0
    for i in range(len(mus)):
        alone = ix.query(int(mus[i]), float(epss[i]), hubs=i % 2 == 0)
        assert np.array_equal(outs[i], alone), i
    for t, bix in built.items():
        with gs.ScanIndex.build(bt[t], gs.COSINE) as ref:
            a, b = bix.export(), ref.export()
            for key in a:
                assert np.array_equal(a[key], b[key]), key
        bix.free()


def test_replay_trace_matches_direct_queries(index):
    import torch
    g, ix = index
    mus, epss = random_queries(300, 2)
    rate = 2000.0
    rng = np.random.default_rng(3)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, mus.shape[0]))
    labels = torch.empty((mus.shape[0], g.n), dtype=torch.int32, device="cuda")
    bgraphs = [graphgen.sbm(5000, 20, 0.05, 0.001, seed=4)]
    with gs.Server(max_batch=128) as srv:
        lat = srv.replay(ix, arrivals, mus, epss, labels=labels, build_arrivals=[arrivals[150]],
                         build_graphs=bgraphs)
    assert np.all(lat > 0)
    lab = labels.cpu().numpy()
    direct = ix.query_batch(mus, epss)
    assert np.array_equal(lab, direct)


@pytest.mark.parametrize("where", ["device", "host"])
def test_replay_ring_of_label_rows(index, where):
    """A ring of 16 label rows under a trace of 400 queries arriving faster
    than one batch completes: rows are reused only after their previous query
    completed, so the last 16 queries' rows hold exactly their own labels."""
    import torch
    g, ix = index
    mus, epss = random_queries(400, 5)
    rng = np.random.default_rng(6)
    arrivals = np.cumsum(rng.exponential(1.0 / 50000.0, mus.shape[0]))
    R = 16
    if where == "device":
        ring = torch.full((R, g.n), -7, dtype=torch.int32, device="cuda")
    else:
        ring = torch.full((R, g.n), -7, dtype=torch.int32).pin_memory()
    with gs.Server(max_batch=8) as srv:
        lat = srv.replay(ix, arrivals, mus, epss, hubs=True, labels=ring, label_rows=R)
    assert np.all(lat > 0)
    direct = ix.query_batch(mus[-R:], epss[-R:], hubs=True)
    got = ring.cpu().numpy()
    for q in range(mus.shape[0] - R, mus.shape[0]):
        assert np.array_equal(got[q % R], direct[q - (mus.shape[0] - R)]), q


def test_replay_library_ring(index):
    """labels=None: the library's own device ring; every query completes."""
    g, ix = index
    mus, epss = random_queries(500, 7)
    arrivals = np.arange(mus.shape[0]) * 2e-5
    with gs.Server(max_batch=64) as srv:
        lat = srv.replay(ix, arrivals, mus, epss, label_rows=4)
        lat2 = srv.replay(ix, arrivals, mus, epss)
    assert np.all(lat > 0) and np.all(lat2 > 0)
    with gs.Server(max_batch=4) as srv:
        with pytest.raises(gs.ScanError) as e:
            srv.replay(ix, arrivals[:3], mus[:3], epss[:3], label_rows=-1)
        assert e.value.status == -1


def test_admission_and_arguments(index):
    g, ix = index
    with gs.Server(memory_budget=1 << 20, max_batch=8) as srv:
        big = graphgen.rmat(14, 16, seed=1)
        with pytest.raises(gs.ScanError) as e:
            srv.submit_build(big, gs.COSINE)
        assert e.value.status == -6  # SCAN_EBUSY: the build alone exceeds the budget
        out = np.empty(g.n, np.int32)
        with pytest.raises(gs.ScanError) as e:
            srv.submit_query(ix, 1, 0.5, out)
        assert e.value.status == -1
        with pytest.raises(gs.ScanError) as e:
            srv.wait(987654321, timeout_ms=10)
        assert e.value.status == -1
