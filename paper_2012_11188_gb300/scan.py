"""Python binding of libscan.so: argument marshalling only.

Every computation happens in the CUDA library (include/scan.h); this module
loads it with ctypes, turns numpy arrays / torch tensors into pointers and
status codes into exceptions. There is no CPU fallback: if the library cannot
be built or loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

COSINE, JACCARD = 0, 1
Q_HUBS = 1
COUNTS_AUTO, COUNTS_SPARSE, COUNTS_DENSE = 0, 1, 2

STATUS = {0: "SCAN_OK", -1: "SCAN_EINVAL", -2: "SCAN_ENOMEM", -3: "SCAN_EBADGRAPH",
          -4: "SCAN_ECUDA", -5: "SCAN_ETIMEOUT", -6: "SCAN_EBUSY"}


class ScanError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)}")
        self.status = status


class scan_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("num_arcs", ctypes.c_int64), ("offsets", ctypes.c_void_p),
                ("offsets_64", ctypes.c_int), ("adj", ctypes.c_void_p), ("on_device", ctypes.c_int)]


class scan_lsh_params(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int), ("simhash_bits", ctypes.c_int),
                ("minhash_k", ctypes.c_int), ("minhash_kpartition", ctypes.c_int),
                ("degree_threshold", ctypes.c_int), ("seed", ctypes.c_uint64)]


class scan_count_config(ctypes.Structure):
    _fields_ = [("warp_deg", ctypes.c_int), ("cta_chunk", ctypes.c_int),
                ("long_list", ctypes.c_int), ("rounds", ctypes.c_int),
                ("dense_div", ctypes.c_int), ("dense_min_n", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libscan.so, compiling it first if it is missing or stale."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    lib = ctypes.CDLL(path)
    P, i32, i64, f64, u = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
    sigs = {
        "scan_set_allocator": (i32, [P, P, P]),
        "scan_index_build": (i32, [P, i32, P, ctypes.c_size_t, P]),
        "scan_index_build_batch": (i32, [P, i32, i32, P, ctypes.c_size_t, P]),
        "scan_index_build_ex": (i32, [P, i32, P, i32, ctypes.c_size_t, P]),
        "scan_index_build_weighted": (i32, [P, P, P, ctypes.c_size_t, P]),
        "scan_query": (i32, [P, i32, f64, P, i32, ctypes.c_size_t]),
        "scan_query_batch": (i32, [P, i32, P, P, P, i32, ctypes.c_size_t]),
        "scan_index_export": (i32, [P, P, P, P, P, P, P]),
        "scan_modularity": (i32, [P, P, P, ctypes.c_size_t]),
        "scan_sweep": (i32, [P, i32, P, P, P, ctypes.c_size_t]),
        "scan_index_info": (i32, [P, P, P, P, P]),
        "scan_index_free": (None, [P]),
        "scan_strerror": (ctypes.c_char_p, [i32]),
        "scan_last_build_timings": (i32, [P]),
        "scan_last_count_kernel_ms": (i32, [P]),
        "scan_kernel_launches": (i32, [P]),
        "scan_set_wide_index": (i32, [i32]),
        "scan_set_count_config": (i32, [P]),
        "scan_autotune_batch": (i32, [P, i32, i32, i32, ctypes.c_size_t, P, P, P]),
        "scan_count_config_for": (i32, [i64, i64, i64, P]),
        "scan_tuning_save": (i32, [ctypes.c_char_p]),
        "scan_tuning_load": (i32, [ctypes.c_char_p]),
        "scan_tuning_clear": (i32, []),
        "scan_sort_segments_desc": (i32, [P, P, P, i64, i64, i64, ctypes.c_size_t]),
        "scan_closed_counts_range": (i32, [P, i64, i64, P, ctypes.c_size_t]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    _lib = lib
    return lib


def set_count_config(cfg=None):
    """Set (a dict with any of the fields of DEFAULT_COUNT_CONFIG; missing
    ones take the default) or clear (None) the process-wide counting
    configuration."""
    if cfg is None:
        _check(load().scan_set_count_config(None), "scan_set_count_config")
        return
    c = scan_count_config(**{**DEFAULT_COUNT_CONFIG, **cfg})
    _check(load().scan_set_count_config(ctypes.byref(c)), "scan_set_count_config")


def autotune_batch(graphs, kind: int = COSINE, reps: int = 2, stream=None, device: bool = False):
    """Autotune the counting strategy per degree bucket on a batch of graphs
    (include/scan.h); returns {"best": cfg, "best_ms": t, "default_ms": t0}."""
    structs, keep = [], []
    for g in graphs:
        c, k = _csr_struct(g, device)
        structs.append(c)
        keep.append(k)
    arr = (scan_csr * len(structs))(*structs)
    best = scan_count_config()
    bms, dms = ctypes.c_double(), ctypes.c_double()
    _check(load().scan_autotune_batch(arr, len(structs), kind, int(reps), _stream_handle(stream),
                                      ctypes.byref(best), ctypes.byref(bms), ctypes.byref(dms)),
           "scan_autotune_batch")
    return {"best": best.as_dict(), "best_ms": bms.value, "default_ms": dms.value}


DEFAULT_COUNT_CONFIG = {"warp_deg": 512, "cta_chunk": 32768, "long_list": 64, "rounds": 4,
                        "dense_div": 16, "dense_min_n": 4096}


def count_config_for(max_n: int, total_n: int, arcs: int) -> dict:
    """The configuration a build would use (a single graph: max_n = total_n = n)."""
    c = scan_count_config()
    _check(load().scan_count_config_for(int(max_n), int(total_n), int(arcs), ctypes.byref(c)),
           "scan_count_config_for")
    return c.as_dict()


def tuning_save(path: str):
    _check(load().scan_tuning_save(os.fsencode(path)), "scan_tuning_save")


def tuning_load(path: str):
    _check(load().scan_tuning_load(os.fsencode(path)), "scan_tuning_load")


def tuning_clear():
    _check(load().scan_tuning_clear(), "scan_tuning_clear")


def sort_segments_desc(keys, ids, seg_off, max_len: int = 0, stream=None):
    """Sort every segment of (keys, ids) in place, key descending then id
    ascending; CUDA tensors (float64, int32, int64 offsets)."""
    nseg = int(seg_off.shape[0]) - 1
    total = int(keys.shape[0])
    if max_len <= 0:
        max_len = int((seg_off[1:] - seg_off[:-1]).max().item()) if nseg > 0 else 0
    _check(load().scan_sort_segments_desc(_ptr(keys), _ptr(ids), _ptr(seg_off), nseg, total,
                                          int(max_len), _stream_handle(stream)),
           "scan_sort_segments_desc")


def closed_counts_range(g, v_begin: int, v_end: int, out=None, stream=None):
    """Triangle counts per arc from the triangles whose middle vertex (degree
    order) lies in [v_begin, v_end): a rank's share of a sharded count (the
    shares of a partition of [0, n) sum to |N(u) ∩ N(v)|). g as for
    ScanIndex.build; out: None (a new uint32 numpy array) or a uint32 array
    or CUDA tensor of num_arcs entries."""
    c, keep = _csr_struct(g, device=False)
    if out is None:
        out = np.zeros(c.num_arcs, dtype=np.uint32)
    _check(load().scan_closed_counts_range(ctypes.byref(c), int(v_begin), int(v_end), _ptr(out),
                                           _stream_handle(stream)),
           "scan_closed_counts_range")
    del keep
    return out


def paper_sigma():
    """The parameter set of the paper's sweep: mu in {2, 4, ..., 2^18} x
    eps in {.01, .02, ..., .99} (1782 pairs), as (mus, epss) arrays."""
    mus = np.repeat(2 ** np.arange(1, 19, dtype=np.int32), 99)
    epss = np.tile(np.arange(1, 100, dtype=np.float64) / 100.0, 18)
    return mus, epss


def _check(rc: int, what: str):
    if rc != 0:
        raise ScanError(rc, what)


def _stream_handle(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _ptr(a) -> int:
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a.data_ptr())  # torch tensor


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


_torch_hooks = None


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through torch's caching allocator."""
    global _torch_hooks
    lib = load()
    if not enable:
        _check(lib.scan_set_allocator(None, None, None), "scan_set_allocator")
        _torch_hooks = None
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0))
        except RuntimeError:
            return None

    def _free(p, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(p)

    hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(lib.scan_set_allocator(ctypes.cast(hooks[0], ctypes.c_void_p),
                                  ctypes.cast(hooks[1], ctypes.c_void_p), None), "scan_set_allocator")
    _torch_hooks = hooks


def make_lsh(kind: int, k: int, threshold: int = 128, seed: int = 1, kpartition: bool = True):
    p = scan_lsh_params()
    p.enabled = 1
    p.simhash_bits = k if kind == COSINE else 64
    p.minhash_k = k if kind == JACCARD else 64
    p.minhash_kpartition = 1 if kpartition else 0
    p.degree_threshold = threshold
    p.seed = seed
    return p


def _csr_struct(g, device: bool):
    """scan_csr for a graphgen.CSR-like (off, adj numpy) or a pair of torch tensors.

    Returns (struct, keepalive)."""
    c = scan_csr()
    if isinstance(g, tuple):
        off, adj = g
    else:
        off, adj = g.off, g.adj
    if _is_torch(off):
        c.on_device = 1 if off.is_cuda else 0
    elif device:
        import torch
        off = torch.from_numpy(np.ascontiguousarray(off)).cuda()
        adj = torch.from_numpy(np.ascontiguousarray(adj)).cuda()
        c.on_device = 1
    else:
        off = np.ascontiguousarray(off)
        adj = np.ascontiguousarray(adj)
        c.on_device = 0
    dt = str(off.dtype)
    if dt.endswith("int64"):
        c.offsets_64 = 1
    elif dt.endswith("int32"):
        c.offsets_64 = 0
    else:
        raise TypeError("offsets must be int32 or int64")
    if not str(adj.dtype).endswith("int32"):
        raise TypeError("adjacency must be int32")
    c.n = int(off.shape[0]) - 1
    c.num_arcs = int(adj.shape[0])
    c.offsets = _ptr(off)
    c.adj = _ptr(adj)
    return c, (off, adj)


@dataclass
class BuildTimings:
    orient_ms: float
    count_ms: float
    sims_ms: float
    neighbor_order_ms: float
    core_order_ms: float
    lsh_ms: float
    total_ms: float


def kernel_launches() -> int:
    c = ctypes.c_uint64()
    _check(load().scan_kernel_launches(ctypes.byref(c)), "scan_kernel_launches")
    return c.value


def set_wide_index(on: bool) -> None:
    """Test hook: count with 64-bit element indices (the path of graphs with
    at least 2**31 arcs) at every size, process-wide."""
    _check(load().scan_set_wide_index(1 if on else 0), "scan_set_wide_index")


def last_count_kernel_ms() -> float:
    """Duration of the last build's CTA counting kernel (CUDA events)."""
    v = ctypes.c_double()
    _check(load().scan_last_count_kernel_ms(ctypes.byref(v)), "scan_last_count_kernel_ms")
    return v.value


def last_build_timings() -> BuildTimings:
    t = (ctypes.c_double * 7)()
    _check(load().scan_last_build_timings(t), "scan_last_build_timings")
    return BuildTimings(*[float(x) for x in t])


class ScanIndex:
    """A SCAN index resident on the GPU (neighbour order NO and core order CO)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        n, arcs = ctypes.c_int64(), ctypes.c_int64()
        md, nb = ctypes.c_int32(), ctypes.c_size_t()
        _check(load().scan_index_info(self._h, ctypes.byref(n), ctypes.byref(arcs),
                                      ctypes.byref(md), ctypes.byref(nb)), "scan_index_info")
        self.n, self.arcs, self.maxdeg, self.device_bytes = n.value, arcs.value, md.value, nb.value

    @classmethod
    def build(cls, g, kind: int = COSINE, lsh=None, stream=None, device: bool = False,
              counts: int = None, weights=None) -> "ScanIndex":
        """Build from a CSR (graphgen.CSR, or (offsets, adj) numpy/torch).

        device=True uploads numpy inputs with torch first; torch CUDA tensors are
        passed as device pointers; numpy arrays are copied in by the library.
        counts: COUNTS_AUTO (default), COUNTS_SPARSE or COUNTS_DENSE.
        weights: float64 per arc, aligned with adj, for the weighted cosine
        index (Section 4.1.1); cosine only (SimHash for lsh), sparse counts."""
        lib = load()
        c, keep = _csr_struct(g, device)
        h = ctypes.c_void_p()
        if weights is not None:
            if kind != COSINE or counts not in (None, COUNTS_AUTO, COUNTS_SPARSE):
                raise ScanError(-1, "weighted builds are cosine and sparse")
            if c.on_device:
                import torch
                w = weights if _is_torch(weights) else torch.from_numpy(np.asarray(weights))
                w = w.to(device="cuda", dtype=torch.float64).contiguous()
            else:
                if _is_torch(weights):
                    weights = weights.cpu().numpy()
                w = np.ascontiguousarray(weights, dtype=np.float64)
            if int(w.shape[0]) != c.num_arcs:
                raise ValueError("one weight per arc is needed")
            rc = lib.scan_index_build_weighted(ctypes.byref(c), _ptr(w),
                                               ctypes.byref(lsh) if lsh else None,
                                               _stream_handle(stream), ctypes.byref(h))
            del keep, w
            _check(rc, "scan_index_build_weighted")
            return cls(h.value)
        rc = lib.scan_index_build_ex(ctypes.byref(c), kind, ctypes.byref(lsh) if lsh else None,
                                     COUNTS_AUTO if counts is None else int(counts),
                                     _stream_handle(stream), ctypes.byref(h))
        del keep
        _check(rc, "scan_index_build_ex")
        return cls(h.value)

    @staticmethod
    def build_batch(graphs, kind: int = COSINE, lsh=None, stream=None, device: bool = False):
        lib = load()
        structs, keep = [], []
        for g in graphs:
            c, k = _csr_struct(g, device)
            structs.append(c)
            keep.append(k)
        arr = (scan_csr * len(structs))(*structs)
        out = (ctypes.c_void_p * len(structs))()
        rc = lib.scan_index_build_batch(arr, len(structs), kind,
                                        ctypes.byref(lsh) if lsh else None,
                                        _stream_handle(stream), out)
        _check(rc, "scan_index_build_batch")
        return [ScanIndex(h) for h in out]

    def query(self, mu: int, eps: float, hubs: bool = False, out=None, stream=None):
        """Labels of one (mu, eps) query; `out` may be a numpy array or torch tensor."""
        if out is None:
            out = np.empty(self.n, dtype=np.int32)
        _check(load().scan_query(self._h, int(mu), float(eps), _ptr(out), Q_HUBS if hubs else 0,
                                 _stream_handle(stream)), "scan_query")
        return out

    def query_batch(self, mus, epss, hubs: bool = False, out=None, stream=None):
        mus = np.ascontiguousarray(mus, dtype=np.int32)
        epss = np.ascontiguousarray(epss, dtype=np.float64)
        q = mus.shape[0]
        if out is None:
            out = np.empty((q, self.n), dtype=np.int32)
        _check(load().scan_query_batch(self._h, q, mus.ctypes.data, epss.ctypes.data, _ptr(out),
                                       Q_HUBS if hubs else 0, _stream_handle(stream)),
               "scan_query_batch")
        return out

    def modularity(self, labels, stream=None) -> float:
        """Modularity of a clustering of this graph (unclustered = singletons)."""
        if isinstance(labels, np.ndarray):
            labels = np.ascontiguousarray(labels, dtype=np.int32)
        q = ctypes.c_double(0.0)
        _check(load().scan_modularity(self._h, _ptr(labels), ctypes.byref(q),
                                      _stream_handle(stream)), "scan_modularity")
        return q.value

    def sweep(self, mus, epss, stream=None) -> np.ndarray:
        """Modularity of the clustering of every (mu, eps) pair (no hub marks)."""
        mus = np.ascontiguousarray(mus, dtype=np.int32)
        epss = np.ascontiguousarray(epss, dtype=np.float64)
        q = np.empty(mus.shape[0], dtype=np.float64)
        _check(load().scan_sweep(self._h, mus.shape[0], mus.ctypes.data, epss.ctypes.data,
                                 q.ctypes.data, _stream_handle(stream)), "scan_sweep")
        return q

    def export(self) -> dict:
        A = self.arcs
        out = {
            "sim": np.empty(A, np.float64), "no_id": np.empty(A, np.int32),
            "no_sim": np.empty(A, np.float64), "co_off": np.empty(self.maxdeg + 1, np.int64),
            "co_id": np.empty(A, np.int32), "co_thr": np.empty(A, np.float64),
        }
        _check(load().scan_index_export(self._h, *[_ptr(out[k]) for k in
                                                   ("sim", "no_id", "no_sim", "co_off", "co_id",
                                                    "co_thr")]), "scan_index_export")
        return out

    def free(self):
        if self._h is not None and self._h.value:
            load().scan_index_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()


# ---------------------------------------------------------------- serving
class scan_serve_params(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_int),
                ("max_pending", ctypes.c_int), ("device", ctypes.c_int)]


def _load_serve():
    lib = load()
    if getattr(lib, "_serve_bound", False):
        return lib
    P, i32, i64, f64, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
    sigs = {
        "scan_serve_create": (i32, [P, P]),
        "scan_serve_submit_query": (i32, [P, P, i32, f64, P, i32, P]),
        "scan_serve_submit_build": (i32, [P, P, i32, P, P]),
        "scan_serve_wait": (i32, [P, u64, i32, P]),
        "scan_serve_stats": (i32, [P, P, P, P, P]),
        "scan_serve_reset_stats": (i32, [P]),
        "scan_serve_replay": (i32, [P, P, i64, P, P, P, i32, P, i64, P, i64, P, P, i32, i32]),
        "scan_serve_destroy": (None, [P]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    lib._serve_bound = True
    return lib


class Server:
    """Continuous-batching query/build server (include/scan_serve.h)."""

    def __init__(self, memory_budget: int = 0, max_batch: int = 64, max_pending: int = 0,
                 device: int = 0):
        lib = _load_serve()
        p = scan_serve_params(memory_budget, max_batch, max_pending, device)
        h = ctypes.c_void_p()
        _check(lib.scan_serve_create(ctypes.byref(p), ctypes.byref(h)), "scan_serve_create")
        self._h = h
        self._keep = {}

    def submit_query(self, index: "ScanIndex", mu: int, eps: float, out, hubs: bool = False) -> int:
        t = ctypes.c_uint64()
        _check(_load_serve().scan_serve_submit_query(self._h, index._h, int(mu), float(eps), _ptr(out),
                                                     Q_HUBS if hubs else 0, ctypes.byref(t)),
               "scan_serve_submit_query")
        self._keep[t.value] = out
        return t.value

    def submit_build(self, g, kind: int = COSINE, lsh=None, device: bool = False) -> int:
        c, keep = _csr_struct(g, device)
        t = ctypes.c_uint64()
        _check(_load_serve().scan_serve_submit_build(self._h, ctypes.byref(c), kind,
                                                     ctypes.byref(lsh) if lsh else None,
                                                     ctypes.byref(t)), "scan_serve_submit_build")
        self._keep[t.value] = (c, keep)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        h = ctypes.c_void_p()
        rc = _load_serve().scan_serve_wait(self._h, ticket, timeout_ms, ctypes.byref(h))
        if rc != -5:
            self._keep.pop(ticket, None)
        _check(rc, "scan_serve_wait")
        return ScanIndex(h.value) if h.value else None

    def stats(self) -> dict:
        p50, p99, qps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        done = ctypes.c_int64()
        _check(_load_serve().scan_serve_stats(self._h, ctypes.byref(p50), ctypes.byref(p99),
                                              ctypes.byref(qps), ctypes.byref(done)), "scan_serve_stats")
        return {"p50_ms": p50.value, "p99_ms": p99.value, "qps": qps.value, "completed": done.value}

    def reset_stats(self):
        _check(_load_serve().scan_serve_reset_stats(self._h), "scan_serve_reset_stats")

    def replay(self, index: "ScanIndex", arrivals, mus, epss, hubs: bool = False, labels=None,
               label_rows: int = 0, build_arrivals=None, build_graphs=None,
               build_kind: int = COSINE, timeout_ms: int = 600000):
        """Open-loop trace replay driven by a C++ thread; returns per-query
        latencies (ms, scheduled arrival to completion).

        labels: None (a device ring of `label_rows` rows owned by the library
        for the call; 0 = its default), or a host/device buffer of rows of n
        int32 of which query i writes row i % label_rows (label_rows = 0: one
        row per query). Each query in flight has its own row."""
        arrivals = np.ascontiguousarray(arrivals, dtype=np.float64)
        mus = np.ascontiguousarray(mus, dtype=np.int32)
        epss = np.ascontiguousarray(epss, dtype=np.float64)
        nq = arrivals.shape[0]
        lat = np.zeros(nq, dtype=np.float64)
        nb = 0
        barr, bstructs, keep = None, None, []
        if build_graphs:
            nb = len(build_graphs)
            barr = np.ascontiguousarray(build_arrivals, dtype=np.float64)
            structs = []
            for g in build_graphs:
                c, k = _csr_struct(g, False)
                structs.append(c)
                keep.append(k)
            bstructs = (scan_csr * nb)(*structs)
        rc = _load_serve().scan_serve_replay(
            self._h, index._h, nq, arrivals.ctypes.data, mus.ctypes.data, epss.ctypes.data,
            Q_HUBS if hubs else 0, _ptr(labels), int(label_rows), lat.ctypes.data, nb,
            barr.ctypes.data if barr is not None else None, bstructs, build_kind, timeout_ms)
        _check(rc, "scan_serve_replay")
        return lat

    def close(self):
        if self._h is not None and self._h.value:
            _load_serve().scan_serve_destroy(self._h)
        self._h = None
        self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
