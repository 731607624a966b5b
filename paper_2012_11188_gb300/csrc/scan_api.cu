// C ABI of libscan.so: index lifecycle, build orchestration, queries, export.
// Declarations and argument conventions: include/scan.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "scan_internal.cuh"

namespace gscan {

std::atomic<unsigned long long> g_kernel_launches{0};
std::atomic<int> g_force_wide{0};  // scan_set_wide_index

bool force_wide_index() { return g_force_wide.load(std::memory_order_relaxed) != 0; }

// ------------------------------------------------------------ counting configuration
// Class of a build: (bit length of the vertex count of its largest graph,
// bit length of its average degree), both known before any device work. The
// tuning table maps a class to the configuration the autotuner found fastest
// for it.
namespace {
int bit_length(int64_t x) {
  int b = 0;
  while (x > 0) { ++b; x >>= 1; }
  return b;
}
std::pair<int, int> degree_class(int64_t n_max, int64_t n_total, int64_t arcs) {
  return {bit_length(n_max), bit_length(n_total > 0 ? arcs / n_total : 0)};
}
std::mutex g_tune_mu;
std::map<std::pair<int, int>, CountCfg> g_tune_table;
bool g_cfg_global_set = false;
CountCfg g_cfg_global;
thread_local bool t_cfg_set = false;  // the autotuner's override on its own thread
thread_local CountCfg t_cfg;
}  // namespace

CountCfg count_config_for(int64_t n_max, int64_t n_total, int64_t arcs) {
  if (t_cfg_set) return t_cfg;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_cfg_global_set) return g_cfg_global;
  auto it = g_tune_table.find(degree_class(n_max, n_total, arcs));
  return it != g_tune_table.end() ? it->second : CountCfg{};
}

int sm_count() {
  static std::atomic<int> cached[64];  // zero until looked up
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  int c = cached[dev].load(std::memory_order_relaxed);
  if (c == 0) {
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c < 1) {
      cudaGetLastError();
      return 1;
    }
    cached[dev].store(c, std::memory_order_relaxed);
  }
  return c;
}

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

void record_kernel_ms(double ms) { g_timings[7] = ms; }

void record_timings(const double* ms7) {
  for (int i = 0; i < 7; ++i) g_timings[i] = ms7[i];
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t build_footprint(int64_t n, int64_t arcs) {
  // index 28 B/arc + 12 B/vertex; build temporaries: oriented lists, counts,
  // twins (16 B/edge), sort scratch (a second key/val pair, bucket ids,
  // samples and group counts: 15 B/arc), item and scan arrays (~24 B/vertex)
  return (size_t)arcs * 28 + (size_t)n * 12 + (size_t)(arcs / 2) * 16 + (size_t)arcs * 15 +
         (size_t)n * 24 + (1u << 20);
}

namespace {

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

// Steps shared by the single and the batched build: CSR checks, degrees,
// orientation, counts and similarities, LSH estimates, neighbour order.
// ix holds n, arcs, off (absolute, int64), adj and allocated deg, no_id,
// no_sim and an 8-word status block; on return ix->maxdeg is set.
int run_pipeline(IndexData* ix, int kind, const scan_lsh_params* lsh, Pool& pool, cudaStream_t s,
                 Events& ev, float* count_ms, int counts_mode, const CountCfg& cfg,
                 const double* wcsr = nullptr) {
  const int64_t n = ix->n, arcs = ix->arcs;
  const bool use_lsh = lsh && lsh->enabled;
  unsigned* scalars = ix->status;  // [0] status, [1] maxdeg, [2] max out-degree
  GS_TRY(launch_degrees(ix->off, ix->adj, n, arcs, ix->deg, (int32_t*)scalars + 1, scalars, pool,
                        s));
  unsigned hs[4];
  GS_CUDA(cudaMemcpyAsync(hs, scalars, sizeof(hs), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (hs[0] & DEV_BADGRAPH) return SCAN_EBADGRAPH;
  ix->maxdeg = (int32_t)hs[1];
  // weighted similarities take the sparse enumeration only
  const bool dense = arcs > 0 && !wcsr && (counts_mode == SCAN_COUNTS_DENSE ||
                                  (counts_mode == SCAN_COUNTS_AUTO && dense_counts_pay(n, arcs, cfg)));
  if (dense) {
    // closed counts of every arc from one matrix product (Section 4.1.1)
    if (n > DENSE_MAX_N) return SCAN_EINVAL;
    GS_TRY(ev.mark(s));
    int32_t* row = nullptr;
    int64_t nH = 0;
    if (use_lsh) {
      row = pool.get<int32_t>(n);
      if (!row) return SCAN_ENOMEM;
      GS_TRY(lsh_select(ix->off, ix->adj, ix->deg, n, lsh->degree_threshold, row, &nH, pool, s));
    }
    GS_CUDA(cudaMemcpyAsync(ix->no_id, ix->adj, arcs * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    GS_TRY(dense_counts_and_sims(kind, ix->off, ix->adj, ix->deg, n,
                                 use_lsh ? lsh->degree_threshold : -1, ix->no_sim, scalars, pool,
                                 s, count_ms));
    GS_CUDA(cudaMemcpyAsync(hs, scalars, sizeof(hs), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    if (hs[0] & DEV_BADGRAPH) return SCAN_EBADGRAPH;
    GS_TRY(ev.mark(s));
    if (use_lsh && nH > 0)
      GS_TRY(lsh_apply(*lsh, kind, ix->off, ix->adj, ix->deg, n, arcs, row, nH, ix->no_sim, pool, s));
    if (row) pool.put(row);
    GS_TRY(ev.mark(s));
    GS_TRY(segmented_sort_desc((uint64_t*)ix->no_sim, ix->no_id, ix->off, n, arcs, ix->maxdeg, pool,
                               s));
    GS_TRY(ev.mark(s));
    return SCAN_OK;
  }
  // ---- orientation (Section 6.1)
  int32_t *od = nullptr, *oadj = nullptr, *opos = nullptr;
  if (arcs > 0) {
    unsigned long long* sum_od = (unsigned long long*)(scalars + 4);
    GS_TRY(launch_orient(ix->off, ix->adj, ix->deg, n, arcs, pool, &od, &oadj, &opos,
                         (int32_t*)scalars + 2, sum_od, s));
    unsigned long long hsum = 0;
    GS_CUDA(cudaMemcpyAsync(hs, scalars, sizeof(hs), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaMemcpyAsync(&hsum, sum_od, sizeof(hsum), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    // a symmetric graph orients exactly arcs/2 edges
    if ((int64_t)hsum != arcs / 2) return SCAN_EBADGRAPH;
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
  if (arcs > 0) {
    GS_CUDA(cudaMemcpyAsync(ix->no_id, ix->adj, arcs * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    GS_TRY(launch_closed_counts_and_sims(kind, ix->off, ix->adj, ix->deg, n, arcs, od, oadj, opos,
                                         ix->maxdeg, max_od, use_lsh ? lsh->degree_threshold : -1,
                                         wcsr, ix->no_sim, scalars, pool, s, count_ms, cfg));
    GS_CUDA(cudaMemcpyAsync(hs, scalars, sizeof(hs), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    if (hs[0] & DEV_BADGRAPH) return SCAN_EBADGRAPH;
    if (hs[0] & DEV_BADWEIGHT) return SCAN_EINVAL;
    pool.put(od);
    pool.put(oadj);
    pool.put(opos);
  }
  GS_TRY(ev.mark(s));
  if (use_lsh && nH > 0)
    GS_TRY(lsh_apply(*lsh, kind, ix->off, ix->adj, ix->deg, n, arcs, row, nH, ix->no_sim, pool, s,
                     wcsr));
  if (row) pool.put(row);
  GS_TRY(ev.mark(s));
  // ---- neighbour order (Algorithm 2)
  GS_TRY(segmented_sort_desc((uint64_t*)ix->no_sim, ix->no_id, ix->off, n, arcs, ix->maxdeg, pool, s));
  GS_TRY(ev.mark(s));
  return SCAN_OK;
}

void store_timings(Events& ev, float count_ms) {
  double t[7];
  t[0] = ev.ms(0, 1);
  t[1] = count_ms;
  t[2] = ev.ms(1, 2) - count_ms;
  t[5] = ev.ms(2, 3);
  t[3] = ev.ms(3, 4);
  t[4] = ev.ms(4, 5);
  t[6] = ev.ms(0, 5);
  record_timings(t);
}

int check_final_status(const unsigned* scalars, cudaStream_t s) {
  unsigned hs[4];
  GS_CUDA(cudaMemcpyAsync(hs, scalars, sizeof(hs), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (hs[0] & DEV_BADGRAPH) return SCAN_EBADGRAPH;
  if (hs[0] & DEV_LIMIT) return SCAN_ETIMEOUT;
  return SCAN_OK;
}

int check_csr_args(const scan_csr* csr) {
  const int64_t n = csr->n, arcs = csr->num_arcs;
  if (n < 0 || n > 0x7ffffffe || arcs < 0) return SCAN_EINVAL;
  if ((n > 0 && !csr->offsets) || (arcs > 0 && !csr->adj)) return SCAN_EINVAL;
  if (arcs % 2) return SCAN_EBADGRAPH;
  return SCAN_OK;
}

// Build one index into ix; on error every block is released by the pool.
int build_one(const scan_csr* csr, int kind, const scan_lsh_params* lsh, cudaStream_t s,
              IndexData* ix, int counts_mode = SCAN_COUNTS_AUTO, const double* weights = nullptr,
              const CountCfg* cfg_in = nullptr) {
  if (counts_mode < SCAN_COUNTS_AUTO || counts_mode > SCAN_COUNTS_DENSE) return SCAN_EINVAL;
  GS_TRY(check_csr_args(csr));
  if (kind != SCAN_COSINE && kind != SCAN_JACCARD) return SCAN_EINVAL;
  GS_TRY(validate_lsh(lsh, kind));
  if (weights && (kind != SCAN_COSINE || counts_mode == SCAN_COUNTS_DENSE)) return SCAN_EINVAL;
  const int64_t n = csr->n, arcs = csr->num_arcs;
  Pool pool(s);
  Events ev;
  GS_TRY(ev.mark(s));
  ix->n = n;
  ix->arcs = arcs;
  ix->kind = kind;
  ix->lsh = lsh && lsh->enabled;
  ix->home = 0;  // frees and exports run on the legacy stream after this call has synchronised
  ix->off = pool.get<int64_t>(n + 1);
  ix->deg = pool.get<int32_t>(n > 0 ? n : 1);
  ix->adj = pool.get<int32_t>(arcs > 0 ? arcs : 1);
  ix->no_id = pool.get<int32_t>(arcs > 0 ? arcs : 1);
  ix->no_sim = pool.get<double>(arcs > 0 ? arcs : 1);
  ix->status = pool.get<unsigned>(8);
  if (!ix->off || !ix->deg || !ix->adj || !ix->no_id || !ix->no_sim || !ix->status)
    return SCAN_ENOMEM;
  GS_CUDA(cudaMemsetAsync(ix->status, 0, 8 * sizeof(unsigned), s));
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
  double* wcsr = nullptr;  // arc weights, released with the build's scratch
  if (weights && arcs > 0) {
    wcsr = pool.get<double>(arcs);
    if (!wcsr) return SCAN_ENOMEM;
    GS_CUDA(cudaMemcpyAsync(wcsr, weights, arcs * sizeof(double), k_in, s));
  }
  int64_t ends[2] = {0, 0};
  GS_CUDA(cudaMemcpyAsync(&ends[0], ix->off, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaMemcpyAsync(&ends[1], ix->off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (ends[0] != 0 || ends[1] != arcs) return SCAN_EBADGRAPH;
  float count_ms = 0;
  const CountCfg cfg = cfg_in ? *cfg_in : count_config_for(n, n, arcs);
  GS_TRY(run_pipeline(ix, kind, lsh, pool, s, ev, &count_ms, counts_mode, cfg, wcsr));
  if (wcsr) pool.put(wcsr);
  // ---- core order (Algorithm 2)
  GS_TRY(build_core_order(*ix, pool, s));
  GS_TRY(ev.mark(s));
  GS_TRY(check_final_status(ix->status, s));
  store_timings(ev, count_ms);
  ix->blocks = pool.detach();
  ix->bytes = 0;
  for (auto& b : ix->blocks) ix->bytes += b.b;
  return SCAN_OK;
}

// ---------------------------------------------------------------- batched build
__device__ __forceinline__ int64_t last_le(const int64_t* a, int64_t cnt, int64_t x) {
  int64_t lo = 0, hi = cnt;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// union offsets: off[u] = ab_g + raw[u + g] for u in graph g; off[N] = A.
// raw holds each graph's own n_g+1 offsets, graph g starting at vb_g + g.
__global__ void k_pack_offsets(const int64_t* __restrict__ raw, const int64_t* __restrict__ vb,
                               const int64_t* __restrict__ ab, int G, int64_t N,
                               int64_t* __restrict__ off, unsigned* status) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u <= N;
       u += (int64_t)gridDim.x * blockDim.x) {
    if (u == N) { off[N] = ab[G]; continue; }
    const int64_t g = last_le(vb, G, u);
    const int64_t o = raw[u + g];
    const int64_t na = ab[g + 1] - ab[g];
    if (o < 0 || o > na) { atomicOr(status, (unsigned)DEV_BADGRAPH); off[u] = ab[g]; continue; }
    off[u] = ab[g] + o;
  }
}

__global__ void k_check_ends(const int64_t* __restrict__ raw, const int64_t* __restrict__ vb,
                             const int64_t* __restrict__ ab, int G, unsigned* status) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = vb[g] + g, ng = vb[g + 1] - vb[g];
    if (raw[b] != 0 || raw[b + ng] != ab[g + 1] - ab[g]) atomicOr(status, (unsigned)DEV_BADGRAPH);
  }
}

// local ids -> union ids (checked against the graph's own n)
__global__ void k_shift_adj(int32_t* __restrict__ adj, const int64_t* __restrict__ vb,
                            const int64_t* __restrict__ ab, int G, int64_t A, unsigned* status) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = last_le(ab, G, i);
    const int32_t x = adj[i];
    const int64_t ng = vb[g + 1] - vb[g];
    if (x < 0 || x >= ng) { atomicOr(status, (unsigned)DEV_BADGRAPH); adj[i] = (int32_t)vb[g]; continue; }
    adj[i] = (int32_t)(x + vb[g]);
  }
}

__global__ void k_graph_maxdeg(const int32_t* __restrict__ deg, const int64_t* __restrict__ vb, int G,
                               int64_t N, int32_t* __restrict__ md) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = deg[v];
    if (d > 0) atomicMax(&md[last_le(vb, G, v)], d);
  }
}

// union ids -> local ids in adj and NO
__global__ void k_rebase_ids(int32_t* __restrict__ adj, int32_t* __restrict__ no_id,
                             const int64_t* __restrict__ vb, const int64_t* __restrict__ ab, int G,
                             int64_t A) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = (int32_t)vb[last_le(ab, G, i)];
    adj[i] -= b;
    no_id[i] -= b;
  }
}

// per-graph offsets relative to the graph's first arc: graph g's n_g+1 entries
// start at rb[g] = vb[g] + g (rel_off) / its maxdeg_g+1 CO offsets at cb[g]
__global__ void k_rebase_offsets(const int64_t* __restrict__ src, const int64_t* __restrict__ base,
                                 const int64_t* __restrict__ rb, const int64_t* __restrict__ ab,
                                 int G, int64_t total, int64_t* __restrict__ rel) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < total;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = last_le(rb, G, u);
    rel[u] = src[base[g] + (u - rb[g])] - ab[g];
  }
}

struct Arena {
  std::vector<Pool::Blk> blocks;
  ~Arena() {
    for (auto& b : blocks) dev_free(b.p, b.b, 0);
  }
};

// The G graphs packed into one union CSR and built by one pass of the
// pipeline; the per-graph indexes are views into one shared arena.
int build_union(const scan_csr* graphs, int G, int kind, const scan_lsh_params* lsh,
                cudaStream_t s, const CountCfg& cfg, scan_index** out) {
  std::vector<int64_t> vb(G + 1, 0), ab(G + 1, 0);
  for (int g = 0; g < G; ++g) {
    GS_TRY(check_csr_args(&graphs[g]));
    vb[g + 1] = vb[g] + graphs[g].n;
    ab[g + 1] = ab[g] + graphs[g].num_arcs;
  }
  const int64_t N = vb[G], A = ab[G];
  if (N > 0x7ffffffe) return SCAN_EINVAL;  // union ids are int32
  Pool pool(s);
  Events ev;
  GS_TRY(ev.mark(s));
  IndexData u;
  u.n = N;
  u.arcs = A;
  u.kind = kind;
  u.off = pool.get<int64_t>(N + 1);
  u.deg = pool.get<int32_t>(N > 0 ? N : 1);
  u.adj = pool.get<int32_t>(A > 0 ? A : 1);
  u.no_id = pool.get<int32_t>(A > 0 ? A : 1);
  u.no_sim = pool.get<double>(A > 0 ? A : 1);
  u.status = pool.get<unsigned>(8);
  int64_t* raw = pool.get<int64_t>(N + G);
  int64_t* meta = pool.get<int64_t>(2 * (size_t)(G + 1));
  if (!u.off || !u.deg || !u.adj || !u.no_id || !u.no_sim || !u.status || !raw || !meta)
    return SCAN_ENOMEM;
  GS_CUDA(cudaMemsetAsync(u.status, 0, 8 * sizeof(unsigned), s));
  std::vector<int64_t> hmeta(2 * (size_t)(G + 1));
  std::copy(vb.begin(), vb.end(), hmeta.begin());
  std::copy(ab.begin(), ab.end(), hmeta.begin() + (G + 1));
  GS_CUDA(cudaMemcpyAsync(meta, hmeta.data(), hmeta.size() * 8, cudaMemcpyHostToDevice, s));
  const int64_t* d_vb = meta;
  const int64_t* d_ab = meta + (G + 1);
  // ---- pack: raw offsets (int64) and adjacency of every graph into the arena
  std::vector<std::vector<int64_t>> staged;
  for (int g = 0; g < G; ++g) {
    const scan_csr& c = graphs[g];
    const cudaMemcpyKind k = c.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    int64_t* dst = raw + vb[g] + g;
    if (c.offsets_64) {
      GS_CUDA(cudaMemcpyAsync(dst, c.offsets, (c.n + 1) * 8, k, s));
    } else if (c.on_device) {
      k_off32_to_64<<<(unsigned)std::min<int64_t>((c.n + 256) / 256, 4096), 256, 0, s>>>(
          (const int32_t*)c.offsets, c.n + 1, dst);
      GS_LAUNCH();
    } else {
      staged.emplace_back(c.n + 1);
      const int32_t* o32 = (const int32_t*)c.offsets;
      for (int64_t i = 0; i <= c.n; ++i) staged.back()[i] = o32[i];
      GS_CUDA(cudaMemcpyAsync(dst, staged.back().data(), (c.n + 1) * 8, cudaMemcpyHostToDevice, s));
    }
    if (c.num_arcs > 0) GS_CUDA(cudaMemcpyAsync(u.adj + ab[g], c.adj, c.num_arcs * 4, k, s));
  }
  const unsigned gN = (unsigned)std::max<int64_t>(1, std::min<int64_t>((N + 256) / 256, sm_count() * 16));
  const unsigned gA = (unsigned)std::max<int64_t>(1, std::min<int64_t>((A + 255) / 256, sm_count() * 16));
  const unsigned gG = (unsigned)std::max<int64_t>(1, std::min<int64_t>((G + 255) / 256, sm_count() * 16));
  k_check_ends<<<gG, 256, 0, s>>>(raw, d_vb, d_ab, G, u.status);
  GS_LAUNCH();
  k_pack_offsets<<<gN, 256, 0, s>>>(raw, d_vb, d_ab, G, N, u.off, u.status);
  GS_LAUNCH();
  if (A > 0) {
    k_shift_adj<<<gA, 256, 0, s>>>(u.adj, d_vb, d_ab, G, A, u.status);
    GS_LAUNCH();
  }
  GS_CUDA(cudaStreamSynchronize(s));  // staged host offsets must outlive their copies
  staged.clear();
  pool.put(raw);
  // ---- the shared pipeline over the union (every step is local to a vertex)
  float count_ms = 0;
  GS_TRY(run_pipeline(&u, kind, lsh, pool, s, ev, &count_ms, SCAN_COUNTS_SPARSE, cfg));
  // ---- per-graph core orders
  int32_t* md_dev = pool.get<int32_t>(G);
  if (!md_dev) return SCAN_ENOMEM;
  GS_CUDA(cudaMemsetAsync(md_dev, 0, G * 4, s));
  k_graph_maxdeg<<<gN, 256, 0, s>>>(u.deg, d_vb, G, N, md_dev);
  GS_LAUNCH();
  std::vector<int32_t> md(G);
  GS_CUDA(cudaMemcpyAsync(md.data(), md_dev, G * 4, cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  pool.put(md_dev);
  std::vector<int64_t> sb(G + 1, 0), rb(G + 1, 0), cb(G + 1, 0);
  for (int g = 0; g < G; ++g) {
    sb[g + 1] = sb[g] + md[g];
    rb[g + 1] = rb[g] + (vb[g + 1] - vb[g]) + 1;
    cb[g + 1] = cb[g] + md[g] + 1;
  }
  const int64_t S = sb[G];
  int64_t* co_off_all = pool.get<int64_t>(S + 1);
  int32_t* co_id = pool.get<int32_t>(A > 0 ? A : 1);
  double* co_thr = pool.get<double>(A > 0 ? A : 1);
  int64_t* off_rel = pool.get<int64_t>(N + G);
  int64_t* co_off_rel = pool.get<int64_t>(S + G);
  int64_t* meta2 = pool.get<int64_t>(4 * (size_t)(G + 1));
  if (!co_off_all || !co_id || !co_thr || !off_rel || !co_off_rel || !meta2) return SCAN_ENOMEM;
  GS_TRY(build_core_order_multi(N, A, u.off, u.deg, (const uint64_t*)u.no_sim, vb, md, co_off_all,
                                co_id, (uint64_t*)co_thr, pool, s));
  GS_TRY(ev.mark(s));
  // ---- back to per-graph ids and offsets
  std::vector<int64_t> hm2(4 * (size_t)(G + 1));
  std::copy(rb.begin(), rb.end(), hm2.begin());
  std::copy(vb.begin(), vb.end(), hm2.begin() + (G + 1));
  std::copy(cb.begin(), cb.end(), hm2.begin() + 2 * (G + 1));
  std::copy(sb.begin(), sb.end(), hm2.begin() + 3 * (G + 1));
  GS_CUDA(cudaMemcpyAsync(meta2, hm2.data(), hm2.size() * 8, cudaMemcpyHostToDevice, s));
  if (A > 0) {
    k_rebase_ids<<<gA, 256, 0, s>>>(u.adj, u.no_id, d_vb, d_ab, G, A);
    GS_LAUNCH();
  }
  k_rebase_offsets<<<gN, 256, 0, s>>>(u.off, meta2 + (G + 1), meta2, d_ab, G, N + G, off_rel);
  GS_LAUNCH();
  const unsigned gS = (unsigned)std::max<int64_t>(1, std::min<int64_t>((S + G + 255) / 256, sm_count() * 16));
  k_rebase_offsets<<<gS, 256, 0, s>>>(co_off_all, meta2 + 3 * (G + 1), meta2 + 2 * (G + 1), d_ab, G,
                                      S + G, co_off_rel);
  GS_LAUNCH();
  GS_TRY(check_final_status(u.status, s));
  store_timings(ev, count_ms);
  pool.put(co_off_all);
  pool.put(u.off);
  pool.put(meta2);
  // ---- handles viewing the shared arena
  auto arena = std::make_shared<Arena>();
  size_t total_bytes = 0;
  for (auto& b : pool.blocks) total_bytes += b.b;
  std::vector<scan_index*> hs(G, nullptr);
  for (int g = 0; g < G; ++g) {
    hs[g] = new (std::nothrow) scan_index();
    if (!hs[g]) {
      for (int j = 0; j < g; ++j) delete hs[j];
      return SCAN_ENOMEM;
    }
  }
  arena->blocks = pool.detach();
  for (int g = 0; g < G; ++g) {
    IndexData& d = hs[g]->d;
    d.n = vb[g + 1] - vb[g];
    d.arcs = ab[g + 1] - ab[g];
    d.maxdeg = md[g];
    d.kind = kind;
    d.lsh = lsh && lsh->enabled;
    d.off = off_rel + rb[g];
    d.deg = u.deg + vb[g];
    d.adj = u.adj + ab[g];
    d.no_id = u.no_id + ab[g];
    d.no_sim = u.no_sim + ab[g];
    d.co_off = co_off_rel + cb[g];
    d.co_id = co_id + ab[g];
    d.co_thr = co_thr + ab[g];
    d.status = u.status;
    d.home = 0;
    d.arena = arena;
    d.bytes = A > 0 ? (size_t)((double)total_bytes * (double)d.arcs / (double)A) : 0;
    out[g] = hs[g];
  }
  return SCAN_OK;
}

// Batched build: the members that the counting configuration sends to the
// dense path (one tcgen05 GEMM each) are built one by one, the others packed
// into one union build. The handles come back in the callers' order; the
// phase timings recorded are the sums over the builds.
int build_batch(const scan_csr* graphs, int G, int kind, const scan_lsh_params* lsh,
                cudaStream_t s, scan_index** out) {
  if (kind != SCAN_COSINE && kind != SCAN_JACCARD) return SCAN_EINVAL;
  GS_TRY(validate_lsh(lsh, kind));
  int64_t N = 0, A = 0, nmax = 0;
  for (int g = 0; g < G; ++g) {
    GS_TRY(check_csr_args(&graphs[g]));
    N += graphs[g].n;
    A += graphs[g].num_arcs;
    nmax = std::max<int64_t>(nmax, graphs[g].n);
  }
  const CountCfg cfg = count_config_for(nmax, N, A);
  std::vector<int> dense_ids, sparse_ids;
  for (int g = 0; g < G; ++g)
    (graphs[g].num_arcs > 0 && dense_counts_pay(graphs[g].n, graphs[g].num_arcs, cfg)
         ? dense_ids : sparse_ids).push_back(g);
  if (dense_ids.empty()) return build_union(graphs, G, kind, lsh, s, cfg, out);
  double tsum[7] = {0, 0, 0, 0, 0, 0, 0};
  auto add_timings = [&] {
    for (int i = 0; i < 7; ++i) tsum[i] += g_timings[i];
  };
  std::vector<scan_index*> built;  // released if a later build fails
  auto fail = [&](int rc) {
    for (scan_index* h : built) scan_index_free(h);
    return rc;
  };
  if (!sparse_ids.empty()) {
    std::vector<scan_csr> sp;
    for (int g : sparse_ids) sp.push_back(graphs[g]);
    std::vector<scan_index*> sp_out(sp.size(), nullptr);
    const int rc = build_union(sp.data(), (int)sp.size(), kind, lsh, s, cfg, sp_out.data());
    if (rc != SCAN_OK) return rc;
    add_timings();
    for (size_t i = 0; i < sp.size(); ++i) {
      out[sparse_ids[i]] = sp_out[i];
      built.push_back(sp_out[i]);
    }
  }
  for (int g : dense_ids) {
    scan_index* h = new (std::nothrow) scan_index();
    if (!h) return fail(SCAN_ENOMEM);
    const int rc = build_one(&graphs[g], kind, lsh, s, &h->d, SCAN_COUNTS_DENSE, nullptr, &cfg);
    if (rc != SCAN_OK) {
      delete h;
      return fail(rc);
    }
    add_timings();
    out[g] = h;
    built.push_back(h);
  }
  record_timings(tsum);
  return SCAN_OK;
}

}  // namespace

int build_index(const scan_csr* csr, int kind, const scan_lsh_params* lsh, cudaStream_t s,
                IndexData* ix) {
  return build_one(csr, kind, lsh, s, ix);
}

void free_index_data(IndexData* ix) {
  for (auto& b : ix->blocks) dev_free(b.p, b.b, ix->home);
  ix->blocks.clear();
  ix->arena.reset();  // the last view of a batched build releases its arena
}

namespace {

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
  unsigned* st_dev = pool.get<unsigned>(1);
  if (!st_dev) return SCAN_ENOMEM;
  GS_CUDA(cudaMemsetAsync(st_dev, 0, sizeof(unsigned), s));
  GS_TRY(run_queries(ix, q, mu, eps, lab, flags, pool, s, st_dev));
  if (!dev_out) GS_CUDA(cudaMemcpyAsync(labels, lab, bytes, cudaMemcpyDeviceToHost, s));
  unsigned st = 0;
  GS_CUDA(cudaMemcpyAsync(&st, st_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (st & DEV_LIMIT) return SCAN_ETIMEOUT;
  return SCAN_OK;
}

}  // namespace
}  // namespace gscan

using namespace gscan;

namespace {
// stands in for the weight array of a graph without arcs (never read)
const double k_no_weight = 0.0;
}  // namespace

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
  return scan_index_build_ex(csr, kind, lsh, SCAN_COUNTS_AUTO, stream, out);
}

int scan_index_build_ex(const scan_csr* csr, scan_sim_kind kind, const scan_lsh_params* lsh,
                        int counts, uintptr_t stream, scan_index** out) {
  if (!out) return SCAN_EINVAL;
  *out = nullptr;
  if (!csr) return SCAN_EINVAL;
  scan_index* h = new (std::nothrow) scan_index();
  if (!h) return SCAN_ENOMEM;
  const int rc = build_one(csr, (int)kind, lsh, (cudaStream_t)stream, &h->d, counts);
  if (rc != SCAN_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    delete h;  // the build's pool already released every block
    return rc;
  }
  *out = h;
  return SCAN_OK;
}

int scan_index_build_weighted(const scan_csr* csr, const double* weights,
                              const scan_lsh_params* lsh, uintptr_t stream, scan_index** out) {
  if (!out) return SCAN_EINVAL;
  *out = nullptr;
  if (!csr || (csr->num_arcs > 0 && !weights)) return SCAN_EINVAL;
  scan_index* h = new (std::nothrow) scan_index();
  if (!h) return SCAN_ENOMEM;
  const int rc = build_one(csr, SCAN_COSINE, lsh, (cudaStream_t)stream, &h->d,
                           SCAN_COUNTS_SPARSE, weights ? weights : &k_no_weight);
  if (rc != SCAN_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    delete h;
    return rc;
  }
  *out = h;
  return SCAN_OK;
}

int scan_index_build_batch(const scan_csr* graphs, int count, scan_sim_kind kind,
                           const scan_lsh_params* lsh, uintptr_t stream, scan_index** out) {
  if (!out || count < 0 || (count > 0 && !graphs)) return SCAN_EINVAL;
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  if (count == 0) return SCAN_OK;
  const int rc = build_batch(graphs, count, (int)kind, lsh, (cudaStream_t)stream, out);
  if (rc != SCAN_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    for (int i = 0; i < count; ++i) out[i] = nullptr;
  }
  return rc;
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
    k_no_to_csr<<<(unsigned)std::min<int64_t>((ix.n + 7) / 8, sm_count() * 32), 256, 0, s>>>(
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
  free_index_data(&index->d);
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

int scan_set_wide_index(int on) {
  g_force_wide.store(on ? 1 : 0, std::memory_order_relaxed);
  return SCAN_OK;
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

int scan_last_count_kernel_ms(double* ms) {
  if (!ms) return SCAN_EINVAL;
  *ms = g_timings[7];
  return SCAN_OK;
}

namespace {
bool valid_cfg(const scan_count_config& c) {
  return c.warp_deg >= 32 && c.warp_deg <= 4096 && c.cta_chunk >= 256 && c.cta_chunk <= 65536 &&
         c.cta_chunk % 32 == 0 && c.long_list >= 1 && c.long_list <= (1 << 20) &&
         (c.rounds == 4 || c.rounds == 8) && c.dense_div >= 0 && c.dense_div <= 1024 &&
         c.dense_min_n >= 2 && c.dense_min_n <= gscan::DENSE_MAX_N;
}
gscan::CountCfg to_cfg(const scan_count_config& c) {
  gscan::CountCfg g;
  g.warp_deg = c.warp_deg;
  g.cta_chunk = c.cta_chunk;
  g.long_list = c.long_list;
  g.rounds = c.rounds;
  g.dense_div = c.dense_div;
  g.dense_min_n = c.dense_min_n;
  return g;
}
scan_count_config from_cfg(const gscan::CountCfg& g) {
  return scan_count_config{g.warp_deg, g.cta_chunk, g.long_list, g.rounds, g.dense_div,
                           g.dense_min_n};
}
}  // namespace

int scan_set_count_config(const scan_count_config* cfg) {
  if (cfg && !valid_cfg(*cfg)) return SCAN_EINVAL;
  std::lock_guard<std::mutex> lk(gscan::g_tune_mu);
  gscan::g_cfg_global_set = cfg != nullptr;
  if (cfg) gscan::g_cfg_global = to_cfg(*cfg);
  return SCAN_OK;
}

int scan_autotune_batch(const scan_csr* graphs, int count, scan_sim_kind kind, int reps,
                        uintptr_t stream, scan_count_config* best, double* best_ms,
                        double* default_ms) {
  if (!graphs || count <= 0 || reps <= 0) return SCAN_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<scan_index*> hs((size_t)count, nullptr);
  int64_t N = 0, A = 0, nmax = 0;
  for (int g = 0; g < count; ++g) {
    N += graphs[g].n;
    A += graphs[g].num_arcs;
    nmax = std::max<int64_t>(nmax, graphs[g].n);
  }
  // the fastest of `reps` batched builds (whole build, CUDA events)
  auto measure = [&](const gscan::CountCfg& c, double* ms) -> int {
    gscan::t_cfg_set = true;
    gscan::t_cfg = c;
    double best_t = 1e300;
    int rc = SCAN_OK;
    for (int r = 0; r < reps && rc == SCAN_OK; ++r) {
      rc = gscan::build_batch(graphs, count, kind, nullptr, s, hs.data());
      if (rc != SCAN_OK) break;
      best_t = std::min(best_t, gscan::g_timings[6]);
      for (int g = 0; g < count; ++g) scan_index_free(hs[g]);
    }
    gscan::t_cfg_set = false;
    *ms = best_t;
    return rc;
  };
  gscan::CountCfg cur;
  double cur_ms = 0;
  GS_TRY(measure(cur, &cur_ms));
  if (default_ms) *default_ms = cur_ms;
  // coordinate search: one parameter at a time, keeping any improvement
  const int dense_divs[] = {0, 8, 16, 32, 64};
  const int dense_min_ns[] = {2048, 4096, 8192};
  const int warp_degs[] = {128, 256, 512, 1024, 2048};
  const int chunks[] = {1024, 2048, 4096, 8192, 16384, 32768, 65536};
  const int longs[] = {32, 64, 128, 256};
  const int rounds[] = {4, 8};
  auto try_value = [&](int gscan::CountCfg::*field, int v) -> int {
    if (cur.*field == v) return SCAN_OK;
    gscan::CountCfg c = cur;
    c.*field = v;
    double t = 0;
    GS_TRY(measure(c, &t));
    if (t < cur_ms) {
      cur = c;
      cur_ms = t;
    }
    return SCAN_OK;
  };
  for (int v : dense_divs) GS_TRY(try_value(&gscan::CountCfg::dense_div, v));
  if (cur.dense_div > 0)
    for (int v : dense_min_ns) GS_TRY(try_value(&gscan::CountCfg::dense_min_n, v));
  for (int v : warp_degs) GS_TRY(try_value(&gscan::CountCfg::warp_deg, v));
  for (int v : chunks) GS_TRY(try_value(&gscan::CountCfg::cta_chunk, v));
  for (int v : longs) GS_TRY(try_value(&gscan::CountCfg::long_list, v));
  for (int v : rounds) GS_TRY(try_value(&gscan::CountCfg::rounds, v));
  {
    std::lock_guard<std::mutex> lk(gscan::g_tune_mu);
    gscan::g_tune_table[gscan::degree_class(nmax, N, A)] = cur;
  }
  if (best) *best = from_cfg(cur);
  if (best_ms) *best_ms = cur_ms;
  return SCAN_OK;
}

int scan_count_config_for(int64_t max_n, int64_t total_n, int64_t num_arcs,
                          scan_count_config* cfg) {
  if (!cfg || max_n < 0 || total_n < max_n || num_arcs < 0) return SCAN_EINVAL;
  *cfg = from_cfg(gscan::count_config_for(max_n, total_n, num_arcs));
  return SCAN_OK;
}

int scan_tuning_save(const char* path) {
  if (!path) return SCAN_EINVAL;
  FILE* f = std::fopen(path, "w");
  if (!f) return SCAN_EINVAL;
  std::fprintf(f, "# max_n_bits avg_degree_bits warp_deg cta_chunk long_list rounds dense_div "
                 "dense_min_n\n");
  {
    std::lock_guard<std::mutex> lk(gscan::g_tune_mu);
    for (const auto& kv : gscan::g_tune_table)
      std::fprintf(f, "%d %d %d %d %d %d %d %d\n", kv.first.first, kv.first.second,
                   kv.second.warp_deg, kv.second.cta_chunk, kv.second.long_list, kv.second.rounds,
                   kv.second.dense_div, kv.second.dense_min_n);
  }
  return std::fclose(f) == 0 ? SCAN_OK : SCAN_EINVAL;
}

int scan_tuning_load(const char* path) {
  if (!path) return SCAN_EINVAL;
  FILE* f = std::fopen(path, "r");
  if (!f) return SCAN_EINVAL;
  std::map<std::pair<int, int>, gscan::CountCfg> table;
  char line[256];
  int rc = SCAN_OK;
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    int a, b;
    scan_count_config c;
    if (std::sscanf(line, "%d %d %d %d %d %d %d %d", &a, &b, &c.warp_deg, &c.cta_chunk,
                    &c.long_list, &c.rounds, &c.dense_div, &c.dense_min_n) != 8 ||
        !valid_cfg(c)) {
      rc = SCAN_EINVAL;
      break;
    }
    table[{a, b}] = to_cfg(c);
  }
  std::fclose(f);
  if (rc != SCAN_OK) return rc;
  std::lock_guard<std::mutex> lk(gscan::g_tune_mu);
  for (const auto& kv : table) gscan::g_tune_table[kv.first] = kv.second;
  return SCAN_OK;
}

int scan_closed_counts_range(const scan_csr* csr, int64_t v_begin, int64_t v_end,
                             uint32_t* counts, uintptr_t stream) {
  if (!csr) return SCAN_EINVAL;
  GS_TRY(gscan::check_csr_args(csr));
  const int64_t n = csr->n, arcs = csr->num_arcs;
  if (v_begin < 0 || v_end < v_begin || v_end > n) return SCAN_EINVAL;
  if (arcs > 0 && !counts) return SCAN_EINVAL;
  if (arcs == 0) return SCAN_OK;
  cudaStream_t s = (cudaStream_t)stream;
  gscan::Pool pool(s);
  int64_t* off = pool.get<int64_t>(n + 1);
  int32_t* adj = pool.get<int32_t>(arcs);
  int32_t* deg = pool.get<int32_t>(n > 0 ? n : 1);
  unsigned* scalars = pool.get<unsigned>(8);  // [0] status, [1] maxdeg, [2] max out-degree, [4..5] sum od
  const bool out_dev = gscan::is_device_ptr(counts);
  uint32_t* out = out_dev ? counts : pool.get<uint32_t>(arcs);
  if (!off || !adj || !deg || !scalars || !out) return SCAN_ENOMEM;
  GS_CUDA(cudaMemsetAsync(scalars, 0, 8 * sizeof(unsigned), s));
  GS_CUDA(cudaMemsetAsync(out, 0, arcs * sizeof(uint32_t), s));
  // the CSR into device arrays with int64 offsets
  const bool dev_in = csr->on_device != 0;
  const cudaMemcpyKind k_in = dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  std::vector<int64_t> off_host;
  if (csr->offsets_64) {
    GS_CUDA(cudaMemcpyAsync(off, csr->offsets, (n + 1) * sizeof(int64_t), k_in, s));
  } else if (dev_in) {
    gscan::k_off32_to_64<<<(unsigned)std::min<int64_t>((n + 256) / 256, 4096), 256, 0, s>>>(
        (const int32_t*)csr->offsets, n + 1, off);
    GS_LAUNCH();
  } else {
    off_host.resize(n + 1);
    const int32_t* o32 = (const int32_t*)csr->offsets;
    for (int64_t i = 0; i <= n; ++i) off_host[i] = o32[i];
    GS_CUDA(cudaMemcpyAsync(off, off_host.data(), (n + 1) * sizeof(int64_t),
                            cudaMemcpyHostToDevice, s));
  }
  GS_CUDA(cudaMemcpyAsync(adj, csr->adj, arcs * sizeof(int32_t), k_in, s));
  int64_t ends[2] = {0, 0};
  GS_CUDA(cudaMemcpyAsync(&ends[0], off, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaMemcpyAsync(&ends[1], off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (ends[0] != 0 || ends[1] != arcs) return SCAN_EBADGRAPH;
  // degrees and CSR checks, orientation (Section 6.1)
  GS_TRY(gscan::launch_degrees(off, adj, n, arcs, deg, (int32_t*)scalars + 1, scalars, pool, s));
  unsigned hs[4];
  GS_CUDA(cudaMemcpyAsync(hs, scalars, sizeof(hs), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (hs[0] & gscan::DEV_BADGRAPH) return SCAN_EBADGRAPH;
  const int32_t maxdeg = (int32_t)hs[1];
  int32_t *od = nullptr, *oadj = nullptr, *opos = nullptr;
  unsigned long long* sum_od = (unsigned long long*)(scalars + 4);
  GS_TRY(gscan::launch_orient(off, adj, deg, n, arcs, pool, &od, &oadj, &opos,
                              (int32_t*)scalars + 2, sum_od, s));
  unsigned long long hsum = 0;
  GS_CUDA(cudaMemcpyAsync(hs, scalars, sizeof(hs), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaMemcpyAsync(&hsum, sum_od, sizeof(hsum), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if ((int64_t)hsum != arcs / 2) return SCAN_EBADGRAPH;
  // the counts of the middle vertices in [v_begin, v_end) (Section 3.1)
  const gscan::CountCfg cfg = gscan::count_config_for(n, n, arcs);
  GS_TRY(gscan::launch_closed_counts_and_sims(SCAN_COSINE, off, adj, deg, n, arcs, od, oadj, opos,
                                              maxdeg, (int32_t)hs[2], -1, nullptr, nullptr,
                                              scalars, pool, s, nullptr, cfg, v_begin, v_end,
                                              out));
  GS_CUDA(cudaMemcpyAsync(hs, scalars, sizeof(hs), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (hs[0] & gscan::DEV_BADGRAPH) return SCAN_EBADGRAPH;
  if (!out_dev) {
    GS_CUDA(cudaMemcpyAsync(counts, out, arcs * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
  }
  return SCAN_OK;
}

int scan_sort_segments_desc(double* keys, int32_t* ids, const int64_t* seg_off, int64_t nseg,
                            int64_t total, int64_t max_len, uintptr_t stream) {
  if (nseg < 0 || total < 0 || max_len < 0) return SCAN_EINVAL;
  if (nseg == 0 || total <= 1 || max_len <= 1) return SCAN_OK;
  if (!keys || !ids || !seg_off) return SCAN_EINVAL;
  if (!gscan::is_device_ptr(keys) || !gscan::is_device_ptr(ids) ||
      !gscan::is_device_ptr(seg_off))
    return SCAN_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  gscan::Pool pool(s);
  GS_TRY(gscan::segmented_sort_desc(reinterpret_cast<uint64_t*>(keys), ids, seg_off, nseg, total,
                                    max_len, pool, s));
  GS_CUDA(cudaStreamSynchronize(s));
  return SCAN_OK;
}

int scan_tuning_clear(void) {
  std::lock_guard<std::mutex> lk(gscan::g_tune_mu);
  gscan::g_tune_table.clear();
  return SCAN_OK;
}

}  // extern "C"
