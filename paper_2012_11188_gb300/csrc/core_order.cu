// Core order CO (Section 3.2; Algorithm 2, MakeCoreOrder).
//
// CO[mu], mu = 2..maxdeg+1, lists the vertices with |N̄(v)| >= mu sorted by
// the core threshold sigma(v, NO[v][mu]) -- the mu-th largest similarity over
// N̄(v) with v itself first, i.e. entry mu-2 of the open row NO[v] --
// non-increasing, ties by ascending id. Storage: co_off[maxdeg+1],
// CO[mu] = co_id/co_thr[co_off[mu-2] .. co_off[mu-1]); the sizes add up to the
// number of arcs.
//
// Steps: degree histogram; suffix sums give |CO[mu]| = #{v : d_v >= mu-1};
// vertices placed in non-increasing degree order (the paper's sorted_V, so
// that CO[mu] is a prefix of that order); a tiled transpose copies NO row
// entries r = mu-2 of 32 consecutive vertices into CO[mu]; finally every CO
// segment is sorted by (threshold desc, id asc).
#include "scan_internal.cuh"

namespace gscan {

namespace {

__global__ void k_deg_hist(const int32_t* __restrict__ deg, int64_t n, int32_t maxdeg,
                           unsigned long long* __restrict__ hist) {
  extern __shared__ unsigned long long sh[];  // small degrees privatised
  const int SMALL = 2048;
  for (int i = threadIdx.x; i < SMALL; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = deg[v];
    if (d < SMALL) atomicAdd(&sh[d], 1ull);
    else atomicAdd(&hist[d], 1ull);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < SMALL && i <= maxdeg; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// rev[i] = hist[maxdeg - i], i = 0..maxdeg
__global__ void k_reverse(const unsigned long long* __restrict__ hist, int32_t maxdeg,
                          int64_t* __restrict__ rev) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= maxdeg;
       i += (int64_t)gridDim.x * blockDim.x)
    rev[i] = (int64_t)hist[maxdeg - i];
}

// S = exclusive scan of rev (maxdeg+2 entries); cum[d] = #{deg >= d} = S[maxdeg-d+1].
// sizes[r] = |CO[r+2]| = cum[r+1] = S[maxdeg - r], r = 0..maxdeg-1;
// first[d] = cum[d+1] = position in degree order of the first vertex of degree d.
__global__ void k_co_sizes(const int64_t* __restrict__ S, int32_t maxdeg, int64_t* __restrict__ sizes,
                           int64_t* __restrict__ first) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= maxdeg;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (r < maxdeg) sizes[r] = S[maxdeg - r];
    first[r] = S[maxdeg - r];  // cum[r+1]
  }
}

// Vertices of degree >= 1 in non-increasing degree order (order among equal
// degrees is arbitrary; the final sort does not depend on it).
__global__ void k_place(const int32_t* __restrict__ deg, int64_t n,
                        const int64_t* __restrict__ first, unsigned long long* __restrict__ fill,
                        int32_t* __restrict__ perm) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = deg[v];
    if (d < 1) continue;
    const int64_t pos = first[d] + (int64_t)atomicAdd(&fill[d], 1ull);
    perm[pos] = (int32_t)v;
  }
}

// r-tiles of each 32-vertex q-tile: ceil(deg of its first vertex / 32)
__global__ void k_rtiles(const int32_t* __restrict__ perm, const int32_t* __restrict__ deg,
                         int64_t nq, int64_t* __restrict__ rt) {
  const int64_t qtiles = (nq + 31) / 32;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < qtiles;
       t += (int64_t)gridDim.x * blockDim.x)
    rt[t] = (deg[perm[t * 32]] + 31) / 32;
}

// 32 x 32 tile: rows = 32 consecutive vertices in degree order (q), columns =
// 32 consecutive NO ranks r. Read rows coalesced, write CO columns coalesced.
__global__ void __launch_bounds__(256)
k_co_scatter(const int32_t* __restrict__ perm, const int32_t* __restrict__ deg,
             const int64_t* __restrict__ off, const uint64_t* __restrict__ no_key,
             const int64_t* __restrict__ co_off, const int64_t* __restrict__ rt_prefix,
             int64_t qtiles, int64_t nq, uint64_t* __restrict__ co_key,
             int32_t* __restrict__ co_val) {
  __shared__ uint64_t tk[32][33];
  __shared__ int32_t tv[32];
  __shared__ int32_t td[32];
  __shared__ int64_t to[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int64_t total = rt_prefix[qtiles];
  for (int64_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
    int64_t lo = 0, hi = qtiles;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (rt_prefix[mid] <= tile) lo = mid; else hi = mid;
    }
    const int64_t q0 = lo * 32;
    const int64_t r0 = (tile - rt_prefix[lo]) * 32;
    if (threadIdx.x < 32) {
      const int64_t q = q0 + threadIdx.x;
      if (q < nq) {
        const int32_t v = perm[q];
        tv[threadIdx.x] = v;
        td[threadIdx.x] = deg[v];
        to[threadIdx.x] = off[v];
      } else {
        tv[threadIdx.x] = -1;
        td[threadIdx.x] = 0;
        to[threadIdx.x] = 0;
      }
    }
    __syncthreads();
    for (int row = ty; row < 32; row += 8) {
      const int64_t r = r0 + tx;
      if (r < td[row]) tk[row][tx] = no_key[to[row] + r];
    }
    __syncthreads();
    for (int col = ty; col < 32; col += 8) {
      const int64_t r = r0 + col;
      const int row = tx;
      if (r < td[row]) {
        const int64_t dst = co_off[r] + q0 + row;
        co_key[dst] = tk[row][col];
        co_val[dst] = tv[row];
      }
    }
    __syncthreads();
  }
}

}  // namespace

int build_core_order(IndexData& ix, Pool& pool, cudaStream_t s) {
  const int32_t D = ix.maxdeg;
  ix.co_off = pool.get<int64_t>((size_t)D + 1);
  ix.co_id = pool.get<int32_t>(ix.arcs);
  ix.co_thr = pool.get<double>(ix.arcs);
  if (!ix.co_off || !ix.co_id || !ix.co_thr) return SCAN_ENOMEM;
  if (D == 0) {
    GS_CUDA(cudaMemsetAsync(ix.co_off, 0, sizeof(int64_t), s));
    return SCAN_OK;
  }
  const int64_t n = ix.n;
  unsigned long long* hist = pool.get<unsigned long long>((size_t)D + 1);
  int64_t* rev = pool.get<int64_t>((size_t)D + 1);
  int64_t* S = pool.get<int64_t>((size_t)D + 2);
  int64_t* sizes = pool.get<int64_t>((size_t)D);
  int64_t* first = pool.get<int64_t>((size_t)D + 1);
  unsigned long long* fill = pool.get<unsigned long long>((size_t)D + 1);
  if (!hist || !rev || !S || !sizes || !first || !fill) return SCAN_ENOMEM;
  GS_CUDA(cudaMemsetAsync(hist, 0, ((size_t)D + 1) * 8, s));
  GS_CUDA(cudaMemsetAsync(fill, 0, ((size_t)D + 1) * 8, s));
  const unsigned gn = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16);
  const unsigned gd = (unsigned)std::min<int64_t>(((int64_t)D + 256) / 256, 152 * 16);
  k_deg_hist<<<gn, 256, 2048 * 8, s>>>(ix.deg, n, D, hist);
  GS_LAUNCH();
  k_reverse<<<gd, 256, 0, s>>>(hist, D, rev);
  GS_LAUNCH();
  GS_TRY(exclusive_scan_i64(rev, S, (int64_t)D + 1, pool, s));
  k_co_sizes<<<gd, 256, 0, s>>>(S, D, sizes, first);
  GS_LAUNCH();
  GS_TRY(exclusive_scan_i64(sizes, ix.co_off, D, pool, s));
  // number of vertices with degree >= 1 = cum[1] = first[0]
  int64_t nq = 0;
  GS_CUDA(cudaMemcpyAsync(&nq, first, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  int32_t* perm = pool.get<int32_t>(nq > 0 ? nq : 1);
  const int64_t qtiles = (nq + 31) / 32;
  int64_t* rt = pool.get<int64_t>(qtiles > 0 ? qtiles : 1);
  int64_t* rt_prefix = pool.get<int64_t>(qtiles + 1);
  if (!perm || !rt || !rt_prefix) return SCAN_ENOMEM;
  k_place<<<gn, 256, 0, s>>>(ix.deg, n, first, fill, perm);
  GS_LAUNCH();
  const unsigned gq = (unsigned)std::max<int64_t>(1, std::min<int64_t>((qtiles + 255) / 256, 152 * 16));
  k_rtiles<<<gq, 256, 0, s>>>(perm, ix.deg, nq, rt);
  GS_LAUNCH();
  GS_TRY(exclusive_scan_i64(rt, rt_prefix, qtiles, pool, s));
  k_co_scatter<<<152 * 16, 256, 0, s>>>(perm, ix.deg, ix.off, (const uint64_t*)ix.no_sim,
                                        ix.co_off, rt_prefix, qtiles, nq, (uint64_t*)ix.co_thr,
                                        ix.co_id);
  GS_LAUNCH();
  GS_TRY(segmented_sort_desc((uint64_t*)ix.co_thr, ix.co_id, ix.co_off, D, ix.arcs, nq, pool, s));
  pool.put(hist);
  pool.put(rev);
  pool.put(S);
  pool.put(sizes);
  pool.put(first);
  pool.put(fill);
  pool.put(perm);
  pool.put(rt);
  pool.put(rt_prefix);
  return SCAN_OK;
}

}  // namespace gscan
