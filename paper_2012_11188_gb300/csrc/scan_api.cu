// C ABI of libscan.so: index lifecycle, build orchestration, queries, export.
// Declarations and argument conventions: include/scan.h.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "scan_internal.cuh"

struct scan_index {
  gscan::IndexData d;
};

namespace gscan {

std::atomic<unsigned long long> g_kernel_launches{0};

// ------------------------------------------------------------ allocator hooks
namespace {
scan_alloc_fn g_alloc = nullptr;
scan_free_fn g_free = nullptr;
void* g_ctx = nullptr;
std::mutex g_pool_mu;
bool g_pool_configured[64] = {false};
thread_local double g_timings[8] = {0};

void configure_default_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_pool_configured[dev]) return;
  cudaMemPool_t mp;
  if (cudaDeviceGetDefaultMemPool(&mp, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  g_pool_configured[dev] = true;
}
}  // namespace

void* dev_alloc(size_t bytes, cudaStream_t s) {
  if (g_alloc) return g_alloc(bytes, (uintptr_t)s, g_ctx);
  configure_default_pool();
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (g_free) { g_free(p, bytes, (uintptr_t)s, g_ctx); return; }
  cudaFreeAsync(p, s);
}

void record_timings(const double* ms7) {
  for (int i = 0; i < 7; ++i) g_timings[i] = ms7[i];
}

namespace {

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

__global__ void k_off32_to_64(const int32_t* __restrict__ in, int64_t n1, int64_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

// sim in CSR order from NO: each NO entry finds its neighbour's CSR slot.
__global__ void k_no_to_csr(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                            const int32_t* __restrict__ no_id, const double* __restrict__ no_sim,
                            int64_t n, double* __restrict__ sim) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = w0; v < n; v += nw) {
    const int64_t b = off[v], e = off[v + 1];
    for (int64_t j = b + lane; j < e; j += 32) {
      const int32_t x = no_id[j];
      int64_t lo = b, hi = e;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (adj[mid] < x) lo = mid + 1; else hi = mid;
      }
      if (lo < e) sim[lo] = no_sim[j];
    }
  }
}

struct Events {
  cudaEvent_t e[8] = {};
  int used = 0;
  ~Events() {
    for (int i = 0; i < used; ++i) cudaEventDestroy(e[i]);
  }
  int mark(cudaStream_t s) {
    if (used >= 8) return SCAN_OK;
    GS_CUDA(cudaEventCreate(&e[used]));
    GS_CUDA(cudaEventRecord(e[used], s));
    ++used;
    return SCAN_OK;
  }
  double ms(int a, int b) {
    float t = 0;
    if (a >= used || b >= used) return 0;
    cudaEventElapsedTime(&t, e[a], e[b]);
    return t;
  }
};

int validate_lsh(const scan_lsh_params* p, int kind) {
  if (!p || !p->enabled) return SCAN_OK;
  if (p->degree_threshold < 0) return SCAN_EINVAL;
  if (kind == SCAN_COSINE) {
    if (p->simhash_bits < 64 || p->simhash_bits > 4096 || p->simhash_bits % 64) return SCAN_EINVAL;
  } else {
    const int k = p->minhash_k;
    if (k < 1 || k > 1024) return SCAN_EINVAL;
    if (p->minhash_kpartition && (k & (k - 1))) return SCAN_EINVAL;
  }
  return SCAN_OK;
}

// Build one index into ix; on error every block is released by the pool.
int build_one(const scan_csr* csr, int kind, const scan_lsh_params* lsh, cudaStream_t s,
              IndexData* ix) {
  const int64_t n = csr->n, arcs = csr->num_arcs;
  if (n < 0 || n > 0x7ffffffe || arcs < 0) return SCAN_EINVAL;
  if ((n > 0 && !csr->offsets) || (arcs > 0 && !csr->adj)) return SCAN_EINVAL;
  if (kind != SCAN_COSINE && kind != SCAN_JACCARD) return SCAN_EINVAL;
  GS_TRY(validate_lsh(lsh, kind));
  if (arcs % 2) return SCAN_EBADGRAPH;
  const bool use_lsh = lsh && lsh->enabled;
  Pool pool(s);
  Events ev;
  GS_TRY(ev.mark(s));
  ix->n = n;
  ix->arcs = arcs;
  ix->kind = kind;
  ix->lsh = use_lsh;
  ix->home = 0;  // frees and exports run on the legacy stream after this call has synchronised
  ix->off = pool.get<int64_t>(n + 1);
  ix->deg = pool.get<int32_t>(n > 0 ? n : 1);
  ix->adj = pool.get<int32_t>(arcs > 0 ? arcs : 1);
  ix->no_id = pool.get<int32_t>(arcs > 0 ? arcs : 1);
  ix->no_sim = pool.get<double>(arcs > 0 ? arcs : 1);
  ix->status = pool.get<unsigned>(4);
  if (!ix->off || !ix->deg || !ix->adj || !ix->no_id || !ix->no_sim || !ix->status)
    return SCAN_ENOMEM;
  unsigned* scalars = ix->status;  // [0] status, [1] maxdeg, [2] max out-degree
  GS_CUDA(cudaMemsetAsync(scalars, 0, 4 * sizeof(unsigned), s));
  // ---- inputs into the index's own arrays
  const bool dev_in = csr->on_device != 0;
  const cudaMemcpyKind k_in = dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  std::vector<int64_t> off_host;
  if (csr->offsets_64) {
    GS_CUDA(cudaMemcpyAsync(ix->off, csr->offsets, (n + 1) * sizeof(int64_t), k_in, s));
  } else if (dev_in) {
    k_off32_to_64<<<(unsigned)std::min<int64_t>((n + 256) / 256, 4096), 256, 0, s>>>(
        (const int32_t*)csr->offsets, n + 1, ix->off);
    GS_LAUNCH();
  } else {
    off_host.resize(n + 1);
    const int32_t* o32 = (const int32_t*)csr->offsets;
    for (int64_t i = 0; i <= n; ++i) off_host[i] = o32[i];
    GS_CUDA(cudaMemcpyAsync(ix->off, off_host.data(), (n + 1) * sizeof(int64_t),
                            cudaMemcpyHostToDevice, s));
  }
  if (arcs > 0) GS_CUDA(cudaMemcpyAsync(ix->adj, csr->adj, arcs * sizeof(int32_t), k_in, s));
  int64_t ends[2] = {0, 0};
  GS_CUDA(cudaMemcpyAsync(&ends[0], ix->off, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaMemcpyAsync(&ends[1], ix->off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  // ---- degrees, checks, orientation (Section 6.1)
  GS_TRY(launch_degrees(ix->off, ix->adj, n, arcs, ix->deg, (int32_t*)scalars + 1, scalars, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (ends[0] != 0 || ends[1] != arcs) return SCAN_EBADGRAPH;
  unsigned hs[4];
  GS_CUDA(cudaMemcpy(hs, scalars, sizeof(hs), cudaMemcpyDeviceToHost));
  if (hs[0] & DEV_BADGRAPH) return SCAN_EBADGRAPH;
  ix->maxdeg = (int32_t)hs[1];
  int64_t *oo = nullptr;
  int32_t *oadj = nullptr, *opos = nullptr;
  if (arcs > 0) {
    GS_TRY(launch_orient(ix->off, ix->adj, ix->deg, n, arcs, pool, &oo, &oadj, &opos,
                         (int32_t*)scalars + 2, s));
    GS_CUDA(cudaMemcpyAsync(hs, scalars, sizeof(hs), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
  }
  const int32_t max_od = (int32_t)hs[2];
  GS_TRY(ev.mark(s));
  // ---- LSH selection (Section 6.3)
  int32_t* row = nullptr;
  int64_t nH = 0;
  if (use_lsh && arcs > 0) {
    row = pool.get<int32_t>(n);
    if (!row) return SCAN_ENOMEM;
    GS_TRY(lsh_select(ix->off, ix->adj, ix->deg, n, lsh->degree_threshold, row, &nH, pool, s));
  }
  // ---- counts and similarities (Section 3.1, Section 6.1)
  float count_ms = 0;
  if (arcs > 0) {
    GS_CUDA(cudaMemcpyAsync(ix->no_id, ix->adj, arcs * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    GS_TRY(launch_closed_counts_and_sims(kind, ix->off, ix->adj, ix->deg, n, arcs, oo, oadj, opos,
                                         max_od, use_lsh ? lsh->degree_threshold : -1,
                                         ix->no_sim, scalars, pool, s, &count_ms));
    GS_CUDA(cudaMemcpyAsync(hs, scalars, sizeof(hs), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    if (hs[0] & DEV_BADGRAPH) return SCAN_EBADGRAPH;
    pool.put(oo);
    pool.put(oadj);
    pool.put(opos);
  }
  GS_TRY(ev.mark(s));
  if (use_lsh && nH > 0)
    GS_TRY(lsh_apply(*lsh, kind, ix->off, ix->adj, ix->deg, n, arcs, row, nH, ix->no_sim, pool, s));
  if (row) pool.put(row);
  GS_TRY(ev.mark(s));
  // ---- neighbour order (Algorithm 2)
  GS_TRY(segmented_sort_desc((uint64_t*)ix->no_sim, ix->no_id, ix->off, n, arcs, ix->maxdeg, pool, s));
  GS_TRY(ev.mark(s));
  // ---- core order (Algorithm 2)
  GS_TRY(build_core_order(*ix, pool, s));
  GS_TRY(ev.mark(s));
  GS_CUDA(cudaStreamSynchronize(s));
  GS_CUDA(cudaMemcpy(hs, scalars, sizeof(hs), cudaMemcpyDeviceToHost));
  if (hs[0] & DEV_BADGRAPH) return SCAN_EBADGRAPH;
  if (hs[0] & DEV_LIMIT) return SCAN_ETIMEOUT;
  double t[7];
  t[0] = ev.ms(0, 1);
  t[1] = count_ms;
  t[2] = ev.ms(1, 2) - count_ms;
  t[5] = ev.ms(2, 3);
  t[3] = ev.ms(3, 4);
  t[4] = ev.ms(4, 5);
  t[6] = ev.ms(0, 5);
  record_timings(t);
  ix->blocks = pool.detach();
  ix->bytes = 0;
  for (auto& b : ix->blocks) ix->bytes += b.b;
  return SCAN_OK;
}

void free_index(IndexData* ix) {
  for (auto& b : ix->blocks) dev_free(b.p, b.b, ix->home);
  ix->blocks.clear();
}

int copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!dst || bytes == 0) return SCAN_OK;
  const cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  GS_CUDA(cudaMemcpyAsync(dst, src, bytes, k, s));
  return SCAN_OK;
}

int query_impl(scan_index* index, int q, const int* mu, const double* eps, int32_t* labels,
               int flags, cudaStream_t s) {
  if (!index || q < 0 || (q > 0 && (!mu || !eps || !labels))) return SCAN_EINVAL;
  for (int i = 0; i < q; ++i) {
    if (mu[i] < 2) return SCAN_EINVAL;
    if (!(eps[i] >= 0.0 && eps[i] <= 1.0)) return SCAN_EINVAL;
  }
  if (flags & ~SCAN_Q_HUBS) return SCAN_EINVAL;
  const IndexData& ix = index->d;
  if (q == 0 || ix.n == 0) return SCAN_OK;
  Pool pool(s);
  const size_t bytes = (size_t)q * (size_t)ix.n * sizeof(int32_t);
  const bool dev_out = is_device_ptr(labels);
  int32_t* lab = dev_out ? labels : pool.get<int32_t>((size_t)q * ix.n);
  if (!lab) return SCAN_ENOMEM;
  GS_CUDA(cudaMemsetAsync(ix.status, 0, sizeof(unsigned), s));
  GS_TRY(run_queries(ix, q, mu, eps, lab, flags, pool, s));
  if (!dev_out) GS_CUDA(cudaMemcpyAsync(labels, lab, bytes, cudaMemcpyDeviceToHost, s));
  unsigned st = 0;
  GS_CUDA(cudaMemcpyAsync(&st, ix.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (st & DEV_LIMIT) return SCAN_ETIMEOUT;
  return SCAN_OK;
}

}  // namespace
}  // namespace gscan

using namespace gscan;

extern "C" {

int scan_set_allocator(scan_alloc_fn alloc, scan_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr)) return SCAN_EINVAL;
  g_alloc = alloc;
  g_free = release;
  g_ctx = ctx;
  return SCAN_OK;
}

int scan_index_build(const scan_csr* csr, scan_sim_kind kind, const scan_lsh_params* lsh,
                     uintptr_t stream, scan_index** out) {
  if (!out) return SCAN_EINVAL;
  *out = nullptr;
  if (!csr) return SCAN_EINVAL;
  scan_index* h = new (std::nothrow) scan_index();
  if (!h) return SCAN_ENOMEM;
  const int rc = build_one(csr, (int)kind, lsh, (cudaStream_t)stream, &h->d);
  if (rc != SCAN_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    delete h;  // the build's pool already released every block
    return rc;
  }
  *out = h;
  return SCAN_OK;
}

int scan_index_build_batch(const scan_csr* graphs, int count, scan_sim_kind kind,
                           const scan_lsh_params* lsh, uintptr_t stream, scan_index** out) {
  if (!out || count < 0 || (count > 0 && !graphs)) return SCAN_EINVAL;
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  for (int i = 0; i < count; ++i) {
    const int rc = scan_index_build(&graphs[i], kind, lsh, stream, &out[i]);
    if (rc != SCAN_OK) {
      for (int j = 0; j < i; ++j) { scan_index_free(out[j]); out[j] = nullptr; }
      return rc;
    }
  }
  return SCAN_OK;
}

int scan_query(scan_index* index, int mu, double eps, int32_t* labels, int flags, uintptr_t stream) {
  return query_impl(index, 1, &mu, &eps, labels, flags, (cudaStream_t)stream);
}

int scan_query_batch(scan_index* index, int q, const int* mu, const double* eps, int32_t* labels,
                     int flags, uintptr_t stream) {
  return query_impl(index, q, mu, eps, labels, flags, (cudaStream_t)stream);
}

int scan_index_export(scan_index* index, double* sim, int32_t* no_id, double* no_sim,
                      int64_t* co_off, int32_t* co_id, double* co_thr) {
  if (!index) return SCAN_EINVAL;
  const IndexData& ix = index->d;
  cudaStream_t s = ix.home;
  const size_t A = (size_t)ix.arcs;
  GS_TRY(copy_out(no_id, ix.no_id, A * 4, s));
  GS_TRY(copy_out(no_sim, ix.no_sim, A * 8, s));
  GS_TRY(copy_out(co_id, ix.co_id, A * 4, s));
  GS_TRY(copy_out(co_thr, ix.co_thr, A * 8, s));
  GS_TRY(copy_out(co_off, ix.co_off, ((size_t)ix.maxdeg + 1) * 8, s));
  if (sim && A > 0) {
    Pool pool(s);
    const bool dev = is_device_ptr(sim);
    double* tmp = dev ? sim : pool.get<double>(A);
    if (!tmp) return SCAN_ENOMEM;
    k_no_to_csr<<<(unsigned)std::min<int64_t>((ix.n + 7) / 8, 152 * 32), 256, 0, s>>>(
        ix.off, ix.adj, ix.no_id, ix.no_sim, ix.n, tmp);
    GS_LAUNCH();
    if (!dev) GS_CUDA(cudaMemcpyAsync(sim, tmp, A * 8, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
  }
  GS_CUDA(cudaStreamSynchronize(s));
  return SCAN_OK;
}

int scan_index_info(scan_index* index, int64_t* n, int64_t* num_arcs, int32_t* max_deg,
                    size_t* device_bytes) {
  if (!index) return SCAN_EINVAL;
  if (n) *n = index->d.n;
  if (num_arcs) *num_arcs = index->d.arcs;
  if (max_deg) *max_deg = index->d.maxdeg;
  if (device_bytes) *device_bytes = index->d.bytes;
  return SCAN_OK;
}

void scan_index_free(scan_index* index) {
  if (!index) return;
  free_index(&index->d);
  delete index;
}

const char* scan_strerror(int status) {
  switch (status) {
    case SCAN_OK: return "ok";
    case SCAN_EINVAL: return "invalid argument";
    case SCAN_ENOMEM: return "out of device memory";
    case SCAN_EBADGRAPH: return "not a simple undirected CSR graph";
    case SCAN_ECUDA: return "CUDA runtime error";
    case SCAN_ETIMEOUT: return "bounded wait expired";
    case SCAN_EBUSY: return "admission refused";
    default: return "unknown status";
  }
}

int scan_kernel_launches(uint64_t* count) {
  if (!count) return SCAN_EINVAL;
  *count = g_kernel_launches.load();
  return SCAN_OK;
}

int scan_last_build_timings(double* ms7) {
  if (!ms7) return SCAN_EINVAL;
  for (int i = 0; i < 7; ++i) ms7[i] = g_timings[i];
  return SCAN_OK;
}

}  // extern "C"
