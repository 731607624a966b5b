// Modularity of a clustering (Section 7.2) and the (mu, eps) sweep that
// selects the clustering of highest modularity (Section 7.3.4, over the
// parameter set Sigma: mu in {2, 4, ..., 2^18}, eps in {.01, ..., .99}).
//
// With unclustered vertices as singletons, the modularity of a clustering is
//   Q = I / 2m - (S_c + S_u) / (2m)^2,
// where I counts the arcs (u,v) with u, v in the same cluster, S_c sums
// D_c^2 over the clusters c, D_c being the sum of the degrees in c, and S_u
// sums d_v^2 over the unclustered vertices. All three are integers, summed
// exactly in 64 bits; only the last line is floating point. S_u is the sum
// of d^2 over all vertices (fixed per graph) minus that over the clustered
// ones, so a pass touches the rows of the clustered vertices only.
#include "scan_internal.cuh"

namespace gscan {

namespace {

// Per clustering: acc[0] = I, acc[1] = sum of d^2 over clustered vertices,
// acc[2] = S_c, acc[3] != 0 if a label was not a vertex id. dsum[c] (zero on
// entry and on exit) accumulates D_c at the cluster's label c.
__global__ void k_mod_rows(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                           const int32_t* __restrict__ labels, int64_t n,
                           unsigned long long* __restrict__ dsum,
                           unsigned long long* __restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long inside = 0, dsq = 0;
  bool bad = false;
  for (int64_t v0 = warp * 32; v0 < n; v0 += nwarps * 32) {
    // 32 vertices per step: one label load per lane, then the clustered rows
    const int64_t vl = v0 + lane;
    int32_t ll = vl < n ? labels[vl] : -1;
    if (ll >= n) { bad = true; ll = -1; }
    unsigned todo = __ballot_sync(0xffffffffu, ll >= 0);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const int64_t v = v0 + src;
      const int32_t lv = __shfl_sync(0xffffffffu, ll, src);
      const int64_t b = off[v], e = off[v + 1];
      unsigned cnt = 0;
      for (int64_t i = b + lane; i < e; i += 32) cnt += labels[adj[i]] == lv ? 1u : 0u;
      cnt = __reduce_add_sync(0xffffffffu, cnt);
      if (lane == 0) {
        const unsigned long long d = (unsigned long long)(e - b);
        inside += cnt;
        dsq += d * d;
        if (d) atomicAdd(&dsum[lv], d);
      }
    }
  }
  if (lane == 0) {
    if (inside) atomicAdd(&acc[0], inside);
    if (dsq) atomicAdd(&acc[1], dsq);
  }
  if (bad) atomicOr(&acc[3], 1ull);
}

// S_c = sum over the cluster labels c of D_c^2; dsum is cleared for the next
// clustering.
__global__ void k_mod_clusters(int64_t n, unsigned long long* __restrict__ dsum,
                               unsigned long long* __restrict__ acc) {
  unsigned long long s = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long d = dsum[v];
    if (d) {
      s += d * d;
      dsum[v] = 0;
    }
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(&acc[2], s);
}

// sum of d^2 over all vertices
__global__ void k_deg_sq(const int32_t* __restrict__ deg, int64_t n,
                         unsigned long long* __restrict__ out) {
  unsigned long long s = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long d = (unsigned long long)deg[v];
    s += d * d;
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

unsigned grid_of(int64_t work, int per_block) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > sm_count() * 16) g = sm_count() * 16;
  return (unsigned)g;
}

double modularity_of(const unsigned long long* acc, unsigned long long deg_sq_all, int64_t arcs) {
  if (arcs == 0) return 0.0;
  const double two_m = (double)arcs;
  const unsigned long long su = deg_sq_all - acc[1];  // unclustered singletons
  return (double)acc[0] / two_m - (double)(acc[2] + su) / (two_m * two_m);
}

}  // namespace

// Launches the modularity passes of one clustering (device labels) into the
// four words acc (zeroed by the caller); dsum must be zero on entry.
int launch_modularity(const IndexData& ix, const int32_t* labels_dev, unsigned long long* dsum,
                      unsigned long long* acc, cudaStream_t s) {
  if (ix.n == 0) return SCAN_OK;
  k_mod_rows<<<grid_of(ix.n, 256), 256, 0, s>>>(ix.off, ix.adj, labels_dev, ix.n, dsum, acc);
  GS_LAUNCH();
  k_mod_clusters<<<grid_of(ix.n, 256 * 8), 256, 0, s>>>(ix.n, dsum, acc);
  GS_LAUNCH();
  return SCAN_OK;
}

int modularity_impl(const IndexData& ix, const int32_t* labels, double* q, cudaStream_t s) {
  Pool pool(s);
  const int64_t n = ix.n;
  if (n == 0 || ix.arcs == 0) {
    *q = 0.0;
    return SCAN_OK;
  }
  const bool dev_in = is_device_ptr(labels);
  const int32_t* lab = labels;
  if (!dev_in) {
    int32_t* tmp = pool.get<int32_t>(n);
    if (!tmp) return SCAN_ENOMEM;
    GS_CUDA(cudaMemcpyAsync(tmp, labels, n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    lab = tmp;
  }
  unsigned long long* dsum = pool.get<unsigned long long>(n);
  unsigned long long* acc = pool.get<unsigned long long>(5);  // 4 words + sum of d^2
  if (!dsum || !acc) return SCAN_ENOMEM;
  GS_CUDA(cudaMemsetAsync(dsum, 0, n * sizeof(unsigned long long), s));
  GS_CUDA(cudaMemsetAsync(acc, 0, 5 * sizeof(unsigned long long), s));
  k_deg_sq<<<grid_of(n, 256 * 8), 256, 0, s>>>(ix.deg, n, acc + 4);
  GS_LAUNCH();
  GS_TRY(launch_modularity(ix, lab, dsum, acc, s));
  unsigned long long h[5];
  GS_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (h[3]) return SCAN_EINVAL;  // a label was >= n
  *q = modularity_of(h, h[4], ix.arcs);
  return SCAN_OK;
}

int sweep_impl(const IndexData& ix, int count, const int* mu, const double* eps, double* q,
               cudaStream_t s) {
  const int64_t n = ix.n;
  if (count == 0) return SCAN_OK;
  if (n == 0 || ix.arcs == 0) {
    for (int i = 0; i < count; ++i) q[i] = 0.0;
    return SCAN_OK;
  }
  Pool pool(s);
  // queries are answered SWEEP_BATCH at a time into one label buffer
  constexpr int SWEEP_BATCH = 32;
  const int B = count < SWEEP_BATCH ? count : SWEEP_BATCH;
  int32_t* lab = pool.get<int32_t>((size_t)B * n);
  unsigned long long* dsum = pool.get<unsigned long long>(n);
  unsigned long long* acc = pool.get<unsigned long long>(4 * (size_t)count + 1);
  unsigned* st = pool.get<unsigned>(1);
  if (!lab || !dsum || !acc || !st) return SCAN_ENOMEM;
  GS_CUDA(cudaMemsetAsync(dsum, 0, n * sizeof(unsigned long long), s));
  GS_CUDA(cudaMemsetAsync(acc, 0, (4 * (size_t)count + 1) * sizeof(unsigned long long), s));
  GS_CUDA(cudaMemsetAsync(st, 0, sizeof(unsigned), s));
  k_deg_sq<<<grid_of(n, 256 * 8), 256, 0, s>>>(ix.deg, n, acc + 4 * (size_t)count);
  GS_LAUNCH();
  for (int b0 = 0; b0 < count; b0 += B) {
    const int nb = count - b0 < B ? count - b0 : B;
    GS_TRY(run_queries(ix, nb, mu + b0, eps + b0, lab, 0, pool, s, st));
    for (int i = 0; i < nb; ++i)
      GS_TRY(launch_modularity(ix, lab + (size_t)i * n, dsum, acc + 4 * (size_t)(b0 + i), s));
  }
  std::vector<unsigned long long> h(4 * (size_t)count + 1);
  unsigned hst = 0;
  GS_CUDA(cudaMemcpyAsync(h.data(), acc, h.size() * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaMemcpyAsync(&hst, st, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (hst & DEV_LIMIT) return SCAN_ETIMEOUT;
  for (int i = 0; i < count; ++i) q[i] = modularity_of(&h[4 * (size_t)i], h.back(), ix.arcs);
  return SCAN_OK;
}

}  // namespace gscan

using namespace gscan;

extern "C" {

int scan_modularity(scan_index* index, const int32_t* labels, double* q, uintptr_t stream) {
  if (!index || !q || (index->d.n > 0 && !labels)) return SCAN_EINVAL;
  return modularity_impl(index->d, labels, q, (cudaStream_t)stream);
}

int scan_sweep(scan_index* index, int count, const int* mu, const double* eps, double* q,
               uintptr_t stream) {
  if (!index || count < 0 || (count > 0 && (!mu || !eps || !q))) return SCAN_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (mu[i] < 2) return SCAN_EINVAL;
    if (!(eps[i] >= 0.0 && eps[i] <= 1.0)) return SCAN_EINVAL;
  }
  return sweep_impl(index->d, count, mu, eps, q, (cudaStream_t)stream);
}

}  // extern "C"
