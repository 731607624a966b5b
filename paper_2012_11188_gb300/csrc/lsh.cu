// LSH index mode (Sections 2.1.2, 5 and 6.3).
//
// Selection (Section 6.3 heuristic): an edge is approximated iff both of its
// endpoints have degree > T; only vertices of degree > T with at least one
// such neighbour are sketched (row[v] >= 0, numbered in id order).
//
// Random numbers: R(key, c) = output number c of SplitMix64 (Steele, Lea,
// Flood 2014) whose state starts at key, i.e. mix64(key + (c+1) * golden).
//  SimHash (Charikar): hyperplane j gives x in N̄(v) the sign +1 iff bit j%64 of
//    R(ks, x*1024 + j/64) is set, ks = mix64(seed ^ "SIMH"); s_j = sum of the
//    signs over N̄(v) in FP32 (exact: |s_j| <= d+1 < 2^24); bit j = [s_j >= 0].
//    Estimate max(0, cos(pi h / k)) for Hamming distance h, from a table
//    computed on the host in double precision.
//  MinHash: h(x) = low 32 bits of R(km, x), km = mix64(seed ^ "MINH").
//    k-partition (one-permutation hashing): bin = top log2(k) bits, value =
//    the other bits, min per bin, empty = 0xFFFFFFFF; estimate = equal
//    non-empty bins / (k - bins empty in both). Standard: h_j(x) = low 32 bits
//    of R(km ^ ((j+1) * golden), x), min per j; estimate = equal / k.
#include <cmath>

#include <type_traits>

#include "scan_internal.cuh"

namespace gscan {

namespace {

constexpr uint64_t GOLDEN = 0x9E3779B97F4A7C15ULL;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t splitmix_out(uint64_t key, uint64_t c) {
  return mix64(key + (c + 1) * GOLDEN);
}

__global__ void k_select_flags(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                               const int32_t* __restrict__ deg, int64_t n, int T,
                               int32_t* __restrict__ flag) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = w0; v < n; v += nw) {
    bool any = false;
    if (deg[v] > T) {  // uniform across the warp
      for (int64_t j = off[v] + lane; j < off[v + 1]; j += 32)
        if (deg[adj[j]] > T) { any = true; break; }
    }
    any = __any_sync(0xffffffffu, any);
    if (lane == 0) flag[v] = any ? 1 : 0;
  }
}

__global__ void k_select_rows(const int32_t* __restrict__ flag, const int64_t* __restrict__ pre,
                              int64_t n, int32_t* __restrict__ row) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    row[v] = flag[v] ? (int32_t)pre[v] : -1;
}

// One CTA per sketched vertex. Elements of N̄(v) in chunks of SH_T; each thread
// hashes one element into W words, then hyperplane j adds +-1 over the chunk.
// Weighted graphs (WTD): hyperplane j adds +-w(v,x) (w(v,v) = 1) in double
// precision; each thread adds its hyperplanes' terms in the order v, then
// N(v) in id order, a fixed order that decides every sign reproducibly.
constexpr int SH_T = 256;
constexpr int SH_WMAX = 64;  // k <= 4096

template <bool WTD>
__global__ void __launch_bounds__(SH_T)
k_simhash(const int64_t* __restrict__ off, const int32_t* __restrict__ adj, int64_t n,
          const int32_t* __restrict__ hlist, int64_t nH, int W, uint64_t key,
          const double* __restrict__ wcsr, uint64_t* __restrict__ sig) {
  using acc_t = typename std::conditional<WTD, double, float>::type;
  extern __shared__ uint64_t bits[];  // [SH_T][W]
  __shared__ unsigned ballots[SH_WMAX * 2];
  __shared__ double wel[WTD ? SH_T : 1];
  const int k = 64 * W;
  const int per = (k + SH_T - 1) / SH_T;  // hyperplanes per thread (<= 16)
  acc_t s[16];
  for (int64_t h = blockIdx.x; h < nH; h += gridDim.x) {
    const int32_t v = hlist[h];
    const int64_t b = off[v], e = off[v + 1];
    const int64_t cnt = e - b + 1;  // N̄(v)
#pragma unroll
    for (int t = 0; t < 16; ++t) s[t] = (acc_t)0;
    for (int64_t c0 = 0; c0 < cnt; c0 += SH_T) {
      const int64_t c = c0 + threadIdx.x;
      if (c < cnt) {
        const int64_t x = c == 0 ? (int64_t)v : (int64_t)adj[b + c - 1];
        for (int w = 0; w < W; ++w)
          bits[threadIdx.x * W + w] = splitmix_out(key, (uint64_t)x * 1024u + (uint64_t)w);
        if (WTD) wel[threadIdx.x] = c == 0 ? 1.0 : wcsr[b + c - 1];
      }
      __syncthreads();
      const int m = (int)min((int64_t)SH_T, cnt - c0);
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        if (t >= per) break;
        const int j = threadIdx.x + t * SH_T;
        if (j >= k) break;
        const int wj = j >> 6, bj = j & 63;
        acc_t acc = s[t];
        for (int el = 0; el < m; ++el) {
          const bool up = (bits[el * W + wj] >> bj) & 1ull;
          if (WTD) acc = __dadd_rn(acc, up ? wel[el] : -wel[el]);
          else acc += up ? 1.0f : -1.0f;
        }
        s[t] = acc;
      }
      __syncthreads();
    }
    // bit j = [s_j >= 0]; hyperplane j = threadIdx.x + t*SH_T, lanes hold 32 consecutive j
    const int lane = threadIdx.x & 31;
    for (int t = 0; t < per; ++t) {
      const int j = threadIdx.x + t * SH_T;
      const unsigned bal = __ballot_sync(0xffffffffu, j < k && s[t] >= (acc_t)0);
      if (lane == 0 && j < k) ballots[j >> 5] = bal;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < W; w += SH_T)
      sig[h * W + w] = (uint64_t)ballots[2 * w] | ((uint64_t)ballots[2 * w + 1] << 32);
    __syncthreads();
  }
}

// One CTA per sketched vertex; k <= 1024 bins/hashes in shared memory.
__global__ void __launch_bounds__(256)
k_minhash(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
          const int32_t* __restrict__ hlist, int64_t nH, int k, int L, int kpartition,
          uint64_t key, uint32_t* __restrict__ mh) {
  __shared__ uint32_t mins[1024];
  for (int64_t h = blockIdx.x; h < nH; h += gridDim.x) {
    const int32_t v = hlist[h];
    const int64_t b = off[v], e = off[v + 1];
    const int64_t cnt = e - b + 1;
    for (int j = threadIdx.x; j < k; j += blockDim.x) mins[j] = 0xFFFFFFFFu;
    __syncthreads();
    if (kpartition) {
      const uint32_t vmask = L == 0 ? 0x7FFFFFFFu : ((1u << (32 - L)) - 1u);
      for (int64_t c = threadIdx.x; c < cnt; c += blockDim.x) {
        const int64_t x = c == 0 ? (int64_t)v : (int64_t)adj[b + c - 1];
        const uint32_t hv = (uint32_t)splitmix_out(key, (uint64_t)x);
        const uint32_t bin = L == 0 ? 0u : hv >> (32 - L);
        atomicMin(&mins[bin], hv & vmask);
      }
    } else {
      for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const uint64_t kj = key ^ ((uint64_t)(j + 1) * GOLDEN);
        uint32_t mn = 0xFFFFFFFFu;
        for (int64_t c = 0; c < cnt; ++c) {
          const int64_t x = c == 0 ? (int64_t)v : (int64_t)adj[b + c - 1];
          const uint32_t hv = (uint32_t)splitmix_out(kj, (uint64_t)x);
          mn = min(mn, hv);
        }
        mins[j] = mn;
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) mh[h * k + j] = mins[j];
    __syncthreads();
  }
}

// SimHash estimates: overwrite the similarity of every approximated arc
// (warp per sketched vertex, lane per arc; a signature of k/64 words is one
// 32-byte sector at k = 256).
__global__ void k_lsh_sims(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                           const int32_t* __restrict__ row, const int32_t* __restrict__ hlist,
                           int64_t nH, int k, const uint64_t* __restrict__ sig,
                           const double* __restrict__ costab, double* __restrict__ sim_csr) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int W = k / 64;
  for (int64_t h = w0; h < nH; h += nw) {
    const int32_t u = hlist[h];
    for (int64_t j = off[u] + lane; j < off[u + 1]; j += 32) {
      const int32_t r = row[adj[j]];
      if (r < 0) continue;
      int ham = 0;
      for (int w = 0; w < W; ++w) ham += __popcll(sig[h * W + w] ^ sig[(int64_t)r * W + w]);
      sim_csr[j] = costab[ham];
    }
  }
}

// MinHash estimates, lane per arc (warp per sketched vertex): equal
// non-empty bins and bins empty in both; a sketch row whose length is a
// multiple of 4 is read as 16-byte vectors, so that the loads of one arc are
// independent and in flight together.
__device__ __forceinline__ void mh_bin(uint32_t x, uint32_t y, int& match, int& both_empty) {
  if (x == 0xFFFFFFFFu && y == 0xFFFFFFFFu) ++both_empty;
  else if (x == y) ++match;
}

__global__ void k_minhash_sims(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                               const int32_t* __restrict__ row, const int32_t* __restrict__ hlist,
                               int64_t nH, int k, int kpartition, const uint32_t* __restrict__ mh,
                               double* __restrict__ sim_csr) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool vec = (k & 3) == 0;
  for (int64_t h = w0; h < nH; h += nw) {
    const int32_t u = hlist[h];
    for (int64_t j = off[u] + lane; j < off[u + 1]; j += 32) {
      const int32_t r = row[adj[j]];
      if (r < 0) continue;
      int match = 0, both_empty = 0;
      if (vec) {
        const uint4* a4 = reinterpret_cast<const uint4*>(mh + h * k);
        const uint4* b4 = reinterpret_cast<const uint4*>(mh + (int64_t)r * k);
#pragma unroll 16
        for (int t = 0; t < k / 4; ++t) {
          const uint4 x = a4[t], y = b4[t];
          mh_bin(x.x, y.x, match, both_empty);
          mh_bin(x.y, y.y, match, both_empty);
          mh_bin(x.z, y.z, match, both_empty);
          mh_bin(x.w, y.w, match, both_empty);
        }
      } else {
        const uint32_t* a = mh + h * k;
        const uint32_t* bb = mh + (int64_t)r * k;
        for (int t = 0; t < k; ++t) mh_bin(a[t], bb[t], match, both_empty);
      }
      const int denom = kpartition ? k - both_empty : k;
      sim_csr[j] = denom > 0 ? __ddiv_rn((double)match, (double)denom) : 0.0;
    }
  }
}

__global__ void k_hlist(const int32_t* __restrict__ row, int64_t n, int32_t* __restrict__ hlist) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (row[v] >= 0) hlist[row[v]] = (int32_t)v;
}

}  // namespace

int lsh_select(const int64_t* off, const int32_t* adj, const int32_t* deg, int64_t n, int T,
               int32_t* row, int64_t* nH_host, Pool& pool, cudaStream_t s) {
  int32_t* flag = pool.get<int32_t>(n > 0 ? n : 1);
  int64_t* pre = pool.get<int64_t>(n + 1);
  if (!flag || !pre) return SCAN_ENOMEM;
  if (n > 0) {
    k_select_flags<<<(unsigned)std::min<int64_t>((n + 7) / 8, sm_count() * 32), 256, 0, s>>>(off, adj, deg,
                                                                                     n, T, flag);
    GS_LAUNCH();
  }
  GS_TRY(exclusive_scan_i32_to_i64(flag, pre, n, pool, s));
  if (n > 0) {
    k_select_rows<<<(unsigned)std::min<int64_t>((n + 255) / 256, sm_count() * 32), 256, 0, s>>>(flag, pre,
                                                                                       n, row);
    GS_LAUNCH();
  }
  GS_CUDA(cudaMemcpyAsync(nH_host, pre + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  pool.put(flag);
  pool.put(pre);
  return SCAN_OK;
}

int lsh_apply(const scan_lsh_params& p, int kind, const int64_t* off, const int32_t* adj,
              const int32_t* deg, int64_t n, int64_t arcs, const int32_t* row, int64_t nH,
              double* sim_csr, Pool& pool, cudaStream_t s, const double* wcsr) {
  (void)deg;
  (void)arcs;
  if (nH <= 0) return SCAN_OK;
  int32_t* hlist = pool.get<int32_t>(nH);
  if (!hlist) return SCAN_ENOMEM;
  k_hlist<<<(unsigned)std::min<int64_t>((n + 255) / 256, sm_count() * 32), 256, 0, s>>>(row, n, hlist);
  GS_LAUNCH();
  const unsigned gh = (unsigned)std::min<int64_t>(nH, sm_count() * 16);
  const unsigned gw = (unsigned)std::min<int64_t>((nH + 7) / 8, sm_count() * 32);
  if (kind == SCAN_COSINE) {
    const int k = p.simhash_bits, W = k / 64;
    const uint64_t key = mix64(p.seed ^ 0x53494D48ULL);  // "SIMH"
    uint64_t* sig = pool.get<uint64_t>((size_t)nH * W);
    double* tab = pool.get<double>((size_t)k + 1);
    if (!sig || !tab) return SCAN_ENOMEM;
    std::vector<double> htab((size_t)k + 1);
    for (int h = 0; h <= k; ++h) {
      const double c = std::cos(M_PI * (double)h / (double)k);
      htab[h] = c > 0.0 ? c : 0.0;
    }
    GS_CUDA(cudaMemcpyAsync(tab, htab.data(), sizeof(double) * (k + 1), cudaMemcpyHostToDevice, s));
    const size_t smem = (size_t)SH_T * W * sizeof(uint64_t);
    const int smem_max = (int)(SH_T * SH_WMAX * sizeof(uint64_t) > 200 * 1024
                                   ? 200 * 1024
                                   : SH_T * SH_WMAX * sizeof(uint64_t));
    if (wcsr) {
      GS_CUDA(cudaFuncSetAttribute(k_simhash<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   smem_max));
      k_simhash<true><<<gh, SH_T, smem, s>>>(off, adj, n, hlist, nH, W, key, wcsr, sig);
    } else {
      GS_CUDA(cudaFuncSetAttribute(k_simhash<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   smem_max));
      k_simhash<false><<<gh, SH_T, smem, s>>>(off, adj, n, hlist, nH, W, key, nullptr, sig);
    }
    GS_LAUNCH();
    k_lsh_sims<<<gw, 256, 0, s>>>(off, adj, row, hlist, nH, k, sig, tab, sim_csr);
    GS_LAUNCH();
    GS_CUDA(cudaStreamSynchronize(s));  // the host table must outlive the copy
    pool.put(sig);
    pool.put(tab);
  } else {
    const int k = p.minhash_k;
    int L = 0;
    while ((1 << L) < k) ++L;
    const uint64_t key = mix64(p.seed ^ 0x4D494E48ULL);  // "MINH"
    uint32_t* mh = pool.get<uint32_t>((size_t)nH * k);
    if (!mh) return SCAN_ENOMEM;
    k_minhash<<<gh, 256, 0, s>>>(off, adj, hlist, nH, k, L, p.minhash_kpartition, key, mh);
    GS_LAUNCH();
    k_minhash_sims<<<gw, 256, 0, s>>>(off, adj, row, hlist, nH, k, p.minhash_kpartition, mh,
                                      sim_csr);
    GS_LAUNCH();
    pool.put(mh);
  }
  pool.put(hlist);
  return SCAN_OK;
}

}  // namespace gscan
