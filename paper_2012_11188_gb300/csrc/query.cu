// (mu, eps) queries on the index (Algorithms 3-5, Section 6.2, Section 4.3).
//
// For a batch of Q queries every phase is one launch over all of them
// (blockIdx.y = query), so CO/NO reads are shared in L2 across the batch:
//  1. GetCores (Algorithm 3): the cores are the prefix of CO[mu] whose
//     threshold is >= eps; its length comes from one binary search (CO[mu] is
//     sorted by non-increasing threshold). The prefix marks parent[v] = v.
//  2. Cluster (Algorithm 5, union-find of Section 6.2): every core u takes the
//     eps-prefix of NO[u] (binary search) and unions with each core neighbour
//     of larger id. The union-find is lock-free: find() halves paths, unite()
//     CASes the larger root under the smaller one, so every root is the
//     smallest id of its component and labels are canonical.
//  3. AssignNonCores (Algorithm 4) with the deterministic rule of Section
//     7.3.4: a non-core takes the label of the first core in its own
//     eps-prefix of NO -- the most similar eps-similar core, smallest id among
//     equal similarities (NO breaks ties by id). Only the non-cores found in
//     the cores' eps-prefixes are visited (each claimed once by a CAS on its
//     label), and a non-core's own eps-prefix is shorter than mu-1, so the
//     query's work follows the eps-edges of its clusters (Theorem 4.3's O(Z))
//     plus two memsets of n words; every other label stays -1.
//  4. With SCAN_Q_HUBS (Section 4.3): an unclustered vertex whose neighbours
//     carry two distinct labels becomes -2.
#include "scan_internal.cuh"

namespace gscan {

namespace {

constexpr int UNITE_LIMIT = 1 << 22;

__device__ __forceinline__ int32_t ld_volatile(const int32_t* p) {
  return *(const volatile int32_t*)p;
}

__device__ __forceinline__ int32_t uf_find(int32_t* parent, int32_t x) {
  for (int it = 0; it < UNITE_LIMIT; ++it) {
    const int32_t p = ld_volatile(parent + x);
    if (p == x) return x;
    const int32_t gp = ld_volatile(parent + p);
    if (gp != p) atomicCAS(parent + x, p, gp);  // path halving; only moves towards the root
    x = gp;
  }
  return x;
}

__device__ __forceinline__ bool uf_unite(int32_t* parent, int32_t a, int32_t b) {
  for (int it = 0; it < UNITE_LIMIT; ++it) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return true;
    if (a > b) { const int32_t t = a; a = b; b = t; }
    if (atomicCAS(parent + b, b, a) == b) return true;  // hook larger root under smaller
  }
  return false;
}

// number of leading entries of the non-increasing array x[0..len) that are >= eps
__device__ __forceinline__ int64_t prefix_ge(const double* x, int64_t len, double eps) {
  int64_t lo = 0, hi = len;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (x[mid] >= eps) lo = mid + 1; else hi = mid;
  }
  return lo;
}

struct QArgs {
  const int64_t* off;
  const int32_t* deg;
  const int32_t* adj;
  const int32_t* no_id;
  const double* no_sim;
  const int64_t* co_off;
  const int32_t* co_id;
  const double* co_thr;
  int64_t n;
  int32_t maxdeg;
  const int* mu;       // Q
  const double* eps;   // Q
  int64_t* ncores;     // Q
  int64_t* ncp;        // Q+1: exclusive prefix of ncores (flattened (query, core) items)
  int Q;
  int32_t* parent;     // Q * n (-1 = not a core)
  int32_t* labels;     // Q * n, used when lab_ptrs is null
  int32_t* const* lab_ptrs;  // Q destinations (device), or null
  unsigned* status;
};

__device__ __forceinline__ int32_t* labels_of(const QArgs& a, int q) {
  return a.lab_ptrs ? a.lab_ptrs[q] : a.labels + (int64_t)q * a.n;
}

__global__ void k_init_labels(QArgs a) {
  int32_t* lab = labels_of(a, blockIdx.y);
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.n;
       v += (int64_t)gridDim.x * blockDim.x)
    lab[v] = -1;
}

// item i of the flattened (query, core) list -> query q, core index i - ncp[q]
__device__ __forceinline__ int item_query(const QArgs& a, int64_t i) {
  int lo = 0, hi = a.Q;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.ncp[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_core_prefix(QArgs a) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int64_t acc = 0;
    for (int q = 0; q < a.Q; ++q) { a.ncp[q] = acc; acc += a.ncores[q]; }
    a.ncp[a.Q] = acc;
  }
}

__global__ void k_get_cores(QArgs a, int Q) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  const int mu = a.mu[q];
  int64_t nc = 0;
  if (mu >= 2 && mu <= a.maxdeg + 1) {
    const int64_t b = a.co_off[mu - 2], e = a.co_off[mu - 1];
    nc = prefix_ge(a.co_thr + b, e - b, a.eps[q]);
  }
  a.ncores[q] = nc;
}

__global__ void k_mark_cores(QArgs a) {
  const int64_t total = a.ncp[a.Q];
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int q = item_query(a, it);
    const int32_t v = a.co_id[a.co_off[a.mu[q] - 2] + (it - a.ncp[q])];
    a.parent[(int64_t)q * a.n + v] = v;
  }
}

// warp per (query, core) item
__global__ void k_union(QArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = a.ncp[a.Q];
  bool fail = false;
  for (int64_t it = w0; it < total; it += nw) {
    const int q = item_query(a, it);
    const double eps = a.eps[q];
    int32_t* parent = a.parent + (int64_t)q * a.n;
    const int32_t u = a.co_id[a.co_off[a.mu[q] - 2] + (it - a.ncp[q])];
    const int64_t rb = a.off[u];
    const int64_t pu = prefix_ge(a.no_sim + rb, a.deg[u], eps);
    for (int64_t j = lane; j < pu; j += 32) {
      const int32_t x = a.no_id[rb + j];
      if (x > u && ld_volatile(parent + x) >= 0) fail |= !uf_unite(parent, u, x);
    }
  }
  if (__any_sync(0xffffffffu, fail) && lane == 0) atomicOr(a.status, (unsigned)DEV_LIMIT);
}

// labels of the cores: their union-find root (the smallest id of the cluster)
__global__ void k_core_labels(QArgs a) {
  const int64_t total = a.ncp[a.Q];
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int q = item_query(a, it);
    const int32_t u = a.co_id[a.co_off[a.mu[q] - 2] + (it - a.ncp[q])];
    labels_of(a, q)[u] = uf_find(a.parent + (int64_t)q * a.n, u);
  }
}

constexpr int32_t CLAIMED = -3;

// warp per core: every non-core x in the core's eps-prefix is a border. The
// first thread to claim x scans x's own eps-prefix of NO for its first core
// (most similar, smallest id on ties); sigma is symmetric, so that prefix
// holds at least this core.
__global__ void k_borders(QArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = a.ncp[a.Q];
  for (int64_t it = w0; it < total; it += nw) {
    const int q = item_query(a, it);
    const double eps = a.eps[q];
    int32_t* parent = a.parent + (int64_t)q * a.n;
    int32_t* lab = labels_of(a, q);
    const int32_t u = a.co_id[a.co_off[a.mu[q] - 2] + (it - a.ncp[q])];
    const int64_t rb = a.off[u];
    const int64_t pu = prefix_ge(a.no_sim + rb, a.deg[u], eps);
    for (int64_t j = lane; j < pu; j += 32) {
      const int32_t x = a.no_id[rb + j];
      if (ld_volatile(parent + x) >= 0) continue;
      if (atomicCAS(lab + x, -1, CLAIMED) != -1) continue;
      int32_t l = -1;
      const int64_t xb = a.off[x], xe = xb + a.deg[x];
      for (int64_t t = xb; t < xe; ++t) {
        if (a.no_sim[t] < eps) break;
        const int32_t y = a.no_id[t];
        if (ld_volatile(parent + y) >= 0) { l = uf_find(parent, y); break; }
      }
      lab[x] = l;
    }
  }
}

// warp per unclustered vertex
__global__ void k_hubs(QArgs a) {
  const int q = blockIdx.y;
  int32_t* lab = labels_of(a, q);
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = w0; v < a.n; v += nw) {
    if (lab[v] != -1) continue;
    const int64_t rb = a.off[v], re = rb + a.deg[v];
    int32_t first = -1;
    bool hub = false;
    for (int64_t j0 = rb; j0 < re && !hub; j0 += 32) {
      const int64_t j = j0 + lane;
      int32_t l = -1;
      if (j < re) l = lab[a.adj[j]];
      if (l == -2) l = -1;  // hub marks are written in this pass; they are not clusters
      // first clustered label in this chunk
      const unsigned m = __ballot_sync(0xffffffffu, l >= 0);
      if (!m) continue;
      if (first < 0) first = __shfl_sync(0xffffffffu, l, __ffs(m) - 1);
      hub = __any_sync(0xffffffffu, l >= 0 && l != first);
    }
    if (hub && lane == 0) lab[v] = -2;
  }
}

}  // namespace

// Launch sequence of a batch of Q queries; every pointer is device memory.
int launch_query_batch(const IndexData& ix, int Q, const int* mu, const double* eps, int64_t* nc,
                       int32_t* parent, int32_t* labels, int32_t* const* lab_ptrs, int flags,
                       cudaStream_t s, unsigned* status_dev) {
  const int64_t n = ix.n;
  GS_CUDA(cudaMemsetAsync(parent, 0xff, sizeof(int32_t) * (size_t)Q * n, s));
  // nc holds 2Q+1 words: Q core counts, then their Q+1 prefix sums
  QArgs a{ix.off, ix.deg, ix.adj, ix.no_id, ix.no_sim, ix.co_off, ix.co_id, ix.co_thr,
          n, ix.maxdeg, mu, eps, nc, nc + Q, Q, parent, labels, lab_ptrs, status_dev};
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sm_count() * 8 / std::min(Q, 8) + 1));
  const unsigned gw = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, sm_count() * 16 / std::min(Q, 16) + 1));
  if (lab_ptrs) {
    k_init_labels<<<dim3(gx, Q), 256, 0, s>>>(a);
    GS_LAUNCH();
  } else {
    GS_CUDA(cudaMemsetAsync(labels, 0xff, sizeof(int32_t) * (size_t)Q * n, s));
  }
  k_get_cores<<<(Q + 127) / 128, 128, 0, s>>>(a, Q);
  GS_LAUNCH();
  k_core_prefix<<<1, 32, 0, s>>>(a);
  GS_LAUNCH();
  // the (query, core) items of the whole batch share one grid
  k_mark_cores<<<sm_count() * 8, 256, 0, s>>>(a);
  GS_LAUNCH();
  k_union<<<sm_count() * 16, 256, 0, s>>>(a);
  GS_LAUNCH();
  k_core_labels<<<sm_count() * 8, 256, 0, s>>>(a);
  GS_LAUNCH();
  k_borders<<<sm_count() * 16, 256, 0, s>>>(a);
  GS_LAUNCH();
  if (flags & SCAN_Q_HUBS) {
    k_hubs<<<dim3(gw, Q), 256, 0, s>>>(a);
    GS_LAUNCH();
  }
  return SCAN_OK;
}

int run_queries(const IndexData& ix, int Q, const int* mu_host, const double* eps_host,
                int32_t* labels_dev, int flags, Pool& pool, cudaStream_t s, unsigned* status_dev) {
  if (Q <= 0) return SCAN_OK;
  const int64_t n = ix.n;
  int* mu = pool.get<int>(Q);
  double* eps = pool.get<double>(Q);
  int64_t* nc = pool.get<int64_t>(2 * (size_t)Q + 1);
  int32_t* parent = pool.get<int32_t>((size_t)Q * (size_t)(n > 0 ? n : 1));
  if (!mu || !eps || !nc || !parent) return SCAN_ENOMEM;
  GS_CUDA(cudaMemcpyAsync(mu, mu_host, sizeof(int) * Q, cudaMemcpyHostToDevice, s));
  GS_CUDA(cudaMemcpyAsync(eps, eps_host, sizeof(double) * Q, cudaMemcpyHostToDevice, s));
  if (n == 0) return SCAN_OK;
  GS_TRY(launch_query_batch(ix, Q, mu, eps, nc, parent, labels_dev, nullptr, flags, s, status_dev));
  pool.put(mu);
  pool.put(eps);
  pool.put(nc);
  pool.put(parent);
  return SCAN_OK;
}

// The same launches as run_queries with every scratch array supplied by the
// caller (mu, eps, core counts and parents already in device memory); used by
// the entry point that must not allocate.
int run_queries_prealloc(const IndexData& ix, int Q, const int* mu_dev, const double* eps_dev,
                         int64_t* nc_dev, int32_t* parent, int32_t* labels_dev, int flags,
                         cudaStream_t s, unsigned* status_dev) {
  if (Q <= 0 || ix.n == 0) return SCAN_OK;
  return launch_query_batch(ix, Q, mu_dev, eps_dev, nc_dev, parent, labels_dev, nullptr, flags, s,
                            status_dev);
}

}  // namespace gscan
