// Core order CO (Section 3.2; Algorithm 2, MakeCoreOrder), for one graph or
// for G graphs packed into one vertex range (the batched build).
//
// CO[mu], mu = 2..maxdeg+1, lists the vertices with |N̄(v)| >= mu sorted by
// the core threshold sigma(v, NO[v][mu]) -- the mu-th largest similarity over
// N̄(v) with v itself first, i.e. entry mu-2 of the open row NO[v] --
// non-increasing, ties by ascending id. Storage per graph: co_off[maxdeg+1],
// CO[mu] = co_id/co_thr[co_off[mu-2] .. co_off[mu-1]); the sizes add up to the
// graph's number of arcs, so the graphs' core orders sit back to back in the
// same order as their arcs.
//
// Steps (no host synchronisation): a histogram over (graph, degree) keys;
// |CO[mu]| of graph g = #{v in g : d_v >= mu-1} from its prefix sums; the
// vertices of each graph placed in non-increasing degree order (the paper's
// sorted_V, so that CO[mu] is a prefix of it); a tiled transpose copies NO
// row entries r = mu-2 of 32 consecutive vertices into CO[mu]; every CO
// segment is then sorted by (threshold desc, id asc).
#include "scan_internal.cuh"

namespace gscan {

namespace {

// largest i in [0, cnt) with a[i] <= x (a ascending, a[0] <= x)
__device__ __forceinline__ int64_t last_le(const int64_t* a, int64_t cnt, int64_t x) {
  int64_t lo = 0, hi = cnt;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

struct Multi {
  int G;
  const int64_t* vb;  // G+1 vertex bases
  const int64_t* hb;  // G+1 histogram bases: hb[g+1] - hb[g] = maxdeg_g + 1
  const int64_t* sb;  // G+1 segment bases: sb[g+1] - sb[g] = maxdeg_g
  const int64_t* Sx;  // exclusive scan of the histogram, hb[G]+1 entries
};

// #{v in graph g : d_v >= d}, 0 <= d <= maxdeg_g + 1
__device__ __forceinline__ int64_t cum(const Multi& m, int64_t g, int64_t d) {
  const int64_t ng = m.vb[g + 1] - m.vb[g];
  return ng - (m.Sx[m.hb[g] + d] - m.Sx[m.hb[g]]);
}

// Keys below HB_SMALL (the low degrees, where most vertices fall) are
// counted in shared memory first, one global atomic per key and CTA; the
// others by warp-aggregated global atomics.
constexpr int HB_SMALL = 4096;

__global__ void __launch_bounds__(256)
k_hist(const int32_t* __restrict__ deg, int64_t N, Multi m, unsigned long long* __restrict__ hist) {
  __shared__ unsigned sh[HB_SMALL];
  for (int i = threadIdx.x; i < HB_SMALL; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = m.G == 1 ? 0 : last_le(m.vb, m.G, v);
    const int64_t key = m.hb[g] + deg[v];
    if (key < HB_SMALL) {
      atomicAdd(&sh[key], 1u);
    } else {
      // lanes with the same key add once
      const unsigned peers = __match_any_sync(__activemask(), (unsigned long long)key);
      if ((threadIdx.x & 31) == __ffs(peers) - 1)
        atomicAdd(&hist[key], (unsigned long long)__popc(peers));
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < HB_SMALL; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

// sizes[sb_g + r] = |CO[r+2]| of graph g = cum(g, r+1)
__global__ void k_sizes(Multi m, int64_t S, int64_t* __restrict__ sizes) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < S;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = m.G == 1 ? 0 : last_le(m.sb, m.G, k);
    sizes[k] = cum(m, g, k - m.sb[g] + 1);
  }
}

// q-tiles (32 vertices of degree >= 1) per graph
__global__ void k_qtiles(Multi m, int64_t* __restrict__ qt) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < m.G;
       g += (int64_t)gridDim.x * blockDim.x)
    qt[g] = (cum(m, g, 1) + 31) / 32;
}

// Vertices of degree >= 1, per graph, in non-increasing degree order (the
// order among equal degrees is arbitrary; the final sort does not depend on
// it). Each CTA takes a contiguous vertex range: keys below HB_SMALL get one
// global reservation per key and CTA (counted in shared memory first), the
// others one per key and warp.
__global__ void __launch_bounds__(256)
k_place(const int32_t* __restrict__ deg, int64_t N, Multi m, unsigned long long* __restrict__ fill,
        int32_t* __restrict__ perm) {
  __shared__ unsigned long long sbase[HB_SMALL];
  const int lane = threadIdx.x & 31;
  const int64_t per = ((N + gridDim.x - 1) / gridDim.x + 31) & ~(int64_t)31;
  const int64_t v_lo = min(N, (int64_t)blockIdx.x * per), v_hi = min(N, v_lo + per);
  auto key_of = [&](int64_t v, int32_t d, int64_t& g) -> unsigned long long {
    g = (d < 1 || m.G == 1) ? 0 : last_le(m.vb, m.G, v);
    return d >= 1 ? (unsigned long long)(m.hb[g] + d) : ~0ull;
  };
  // 1. counts of the small keys in this range
  for (int i = threadIdx.x; i < HB_SMALL; i += blockDim.x) sbase[i] = 0;
  __syncthreads();
  for (int64_t v = v_lo + threadIdx.x; v < v_hi; v += blockDim.x) {
    int64_t g;
    const unsigned long long key = key_of(v, deg[v], g);
    if (key < (unsigned long long)HB_SMALL) atomicAdd(&sbase[key], 1ull);
  }
  __syncthreads();
  // 2. one reservation per small key
  for (int i = threadIdx.x; i < HB_SMALL; i += blockDim.x) {
    const unsigned long long c = sbase[i];
    if (c) sbase[i] = atomicAdd(&fill[i], c);
  }
  __syncthreads();
  // 3. placement (uniform trip count per warp for the aggregated atomics)
  for (int64_t v0 = v_lo + (threadIdx.x & ~31); v0 < v_hi; v0 += blockDim.x) {
    const int64_t v = v0 + lane;
    const int32_t d = v < v_hi ? deg[v] : 0;
    int64_t g;
    const unsigned long long key = key_of(v, d, g);
    const bool small = key < (unsigned long long)HB_SMALL;
    const bool big = d >= 1 && !small;
    // every lane takes part in the match and the shuffle
    const unsigned peers = __match_any_sync(0xffffffffu, big ? key : ~0ull);
    const int leader = __ffs(peers) - 1;
    unsigned long long gslot = 0;
    if (big && lane == leader) gslot = atomicAdd(&fill[key], (unsigned long long)__popc(peers));
    gslot = __shfl_sync(0xffffffffu, gslot, leader) + __popc(peers & ((1u << lane) - 1u));
    const unsigned long long slot = small ? atomicAdd(&sbase[key], 1ull) : gslot;
    if (d >= 1) {
      const int64_t pos = cum(m, g, d + 1) + (int64_t)slot;
      perm[m.vb[g] + pos] = (int32_t)v;
    }
  }
}

// r-tiles of each q-tile: ceil(degree of its first vertex / 32)
__global__ void k_rtiles(const int32_t* __restrict__ perm, const int32_t* __restrict__ deg, Multi m,
                         const int64_t* __restrict__ qtb, int64_t* __restrict__ rt) {
  const int64_t T = qtb[m.G];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = m.G == 1 ? 0 : last_le(qtb, m.G, t);
    rt[t] = (deg[perm[m.vb[g] + 32 * (t - qtb[g])]] + 31) / 32;
  }
}

// 32 x 32 tile: rows = 32 consecutive vertices of one graph in degree order,
// columns = 32 consecutive NO ranks r. Rows read coalesced, CO columns written
// coalesced. co_val receives ids local to the graph.
__global__ void __launch_bounds__(256)
k_co_scatter(const int32_t* __restrict__ perm, const int32_t* __restrict__ deg,
             const int64_t* __restrict__ off, const uint64_t* __restrict__ no_key, Multi m,
             const int64_t* __restrict__ qtb, const int64_t* __restrict__ co_off,
             const int64_t* __restrict__ rt_prefix, int64_t Tub, uint64_t* __restrict__ co_key,
             int32_t* __restrict__ co_val) {
  __shared__ uint64_t tk[32][33];
  __shared__ int32_t tv[32];
  __shared__ int32_t td[32];
  __shared__ int64_t to[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int64_t total = rt_prefix[Tub];
  // each CTA takes a contiguous range of tiles and walks its q-tile forward
  // (one search per CTA instead of one dependent search per tile)
  const int64_t per = (total + gridDim.x - 1) / gridDim.x;
  const int64_t first = (int64_t)blockIdx.x * per, last = min(total, first + per);
  int64_t t = first < last ? last_le(rt_prefix, Tub, first) : 0;
  // the 32 vertices of a q-tile are looked up once for all its rank tiles
  int64_t cur_t = -1, q0 = 0, sbg = 0;
  for (int64_t tile = first; tile < last; ++tile) {
    while (rt_prefix[t + 1] <= tile) ++t;
    const int64_t r0 = (tile - rt_prefix[t]) * 32;
    if (t != cur_t) {
      cur_t = t;
      const int64_t g = m.G == 1 ? 0 : last_le(qtb, m.G, t);
      q0 = (t - qtb[g]) * 32;
      sbg = m.sb[g];
      const int64_t nq = cum(m, g, 1);
      const int64_t vbg = m.vb[g];
      if (threadIdx.x < 32) {
        const int64_t q = q0 + threadIdx.x;
        if (q < nq) {
          const int32_t v = perm[vbg + q];
          tv[threadIdx.x] = (int32_t)(v - vbg);
          td[threadIdx.x] = deg[v];
          to[threadIdx.x] = off[v];
        } else {
          tv[threadIdx.x] = -1;
          td[threadIdx.x] = 0;
          to[threadIdx.x] = 0;
        }
      }
      __syncthreads();
    }
    for (int row = ty; row < 32; row += 8) {
      const int64_t r = r0 + tx;
      if (r < td[row]) tk[row][tx] = no_key[to[row] + r];
    }
    __syncthreads();
    for (int col = ty; col < 32; col += 8) {
      const int64_t r = r0 + col;
      const int row = tx;
      if (r < td[row]) {
        const int64_t dst = co_off[sbg + r] + q0 + row;
        co_key[dst] = tk[row][col];
        co_val[dst] = tv[row];
      }
    }
    __syncthreads();
  }
}

inline unsigned grid1(int64_t work, int per = 256) {
  int64_t g = (work + per - 1) / per;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, sm_count() * 16));
}

}  // namespace

int build_core_order_multi(int64_t N, int64_t A, const int64_t* off, const int32_t* deg,
                           const uint64_t* no_key, const std::vector<int64_t>& vb,
                           const std::vector<int32_t>& maxdeg, int64_t* co_off_all,
                           int32_t* co_id, uint64_t* co_key, Pool& pool, cudaStream_t s) {
  const int G = (int)maxdeg.size();
  std::vector<int64_t> hb(G + 1), sb(G + 1);
  hb[0] = sb[0] = 0;
  int64_t max_n = 0;
  for (int g = 0; g < G; ++g) {
    hb[g + 1] = hb[g] + maxdeg[g] + 1;
    sb[g + 1] = sb[g] + maxdeg[g];
    max_n = std::max(max_n, vb[g + 1] - vb[g]);
  }
  const int64_t H = hb[G], S = sb[G];
  if (S == 0) {
    GS_CUDA(cudaMemsetAsync(co_off_all, 0, sizeof(int64_t), s));
    return SCAN_OK;
  }
  int64_t* meta = pool.get<int64_t>(3 * (size_t)(G + 1));
  unsigned long long* hist = pool.get<unsigned long long>(H);
  unsigned long long* fill = pool.get<unsigned long long>(H);
  int64_t* Sx = pool.get<int64_t>(H + 1);
  int64_t* sizes = pool.get<int64_t>(S);
  int64_t* qt = pool.get<int64_t>(G);
  int64_t* qtb = pool.get<int64_t>(G + 1);
  const int64_t Tub = N / 32 + G + 1;  // q-tiles upper bound
  int64_t* rt = pool.get<int64_t>(Tub);
  int64_t* rt_prefix = pool.get<int64_t>(Tub + 1);
  int32_t* perm = pool.get<int32_t>(N > 0 ? N : 1);
  if (!meta || !hist || !fill || !Sx || !sizes || !qt || !qtb || !rt || !rt_prefix || !perm)
    return SCAN_ENOMEM;
  std::vector<int64_t> hmeta(3 * (size_t)(G + 1));
  std::copy(vb.begin(), vb.end(), hmeta.begin());
  std::copy(hb.begin(), hb.end(), hmeta.begin() + (G + 1));
  std::copy(sb.begin(), sb.end(), hmeta.begin() + 2 * (G + 1));
  GS_CUDA(cudaMemcpyAsync(meta, hmeta.data(), hmeta.size() * 8, cudaMemcpyHostToDevice, s));
  GS_CUDA(cudaMemsetAsync(hist, 0, H * 8, s));
  GS_CUDA(cudaMemsetAsync(fill, 0, H * 8, s));
  GS_CUDA(cudaMemsetAsync(rt, 0, Tub * 8, s));
  Multi m{G, meta, meta + (G + 1), meta + 2 * (G + 1), Sx};
  k_hist<<<grid1(N), 256, 0, s>>>(deg, N, m, hist);
  GS_LAUNCH();
  GS_TRY(exclusive_scan_i64((const int64_t*)hist, Sx, H, pool, s));
  k_sizes<<<grid1(S), 256, 0, s>>>(m, S, sizes);
  GS_LAUNCH();
  GS_TRY(exclusive_scan_i64(sizes, co_off_all, S, pool, s));
  k_qtiles<<<grid1(G), 256, 0, s>>>(m, qt);
  GS_LAUNCH();
  GS_TRY(exclusive_scan_i64(qt, qtb, G, pool, s));
  k_place<<<grid1(N), 256, 0, s>>>(deg, N, m, fill, perm);
  GS_LAUNCH();
  k_rtiles<<<grid1(Tub), 256, 0, s>>>(perm, deg, m, qtb, rt);
  GS_LAUNCH();
  GS_TRY(exclusive_scan_i64(rt, rt_prefix, Tub, pool, s));
  k_co_scatter<<<sm_count() * 16, 256, 0, s>>>(perm, deg, off, no_key, m, qtb, co_off_all, rt_prefix, Tub,
                                        co_key, co_id);
  GS_LAUNCH();
  GS_TRY(segmented_sort_desc(co_key, co_id, co_off_all, S, A, max_n, pool, s));
  pool.put(meta);
  pool.put(hist);
  pool.put(fill);
  pool.put(Sx);
  pool.put(sizes);
  pool.put(qt);
  pool.put(qtb);
  pool.put(rt);
  pool.put(rt_prefix);
  pool.put(perm);
  return SCAN_OK;
}

int build_core_order(IndexData& ix, Pool& pool, cudaStream_t s) {
  const int32_t D = ix.maxdeg;
  ix.co_off = pool.get<int64_t>((size_t)D + 1);
  ix.co_id = pool.get<int32_t>(ix.arcs);
  ix.co_thr = pool.get<double>(ix.arcs);
  if (!ix.co_off || !ix.co_id || !ix.co_thr) return SCAN_ENOMEM;
  std::vector<int64_t> vb{0, ix.n};
  std::vector<int32_t> md{D};
  return build_core_order_multi(ix.n, ix.arcs, ix.off, ix.deg, (const uint64_t*)ix.no_sim, vb, md,
                                ix.co_off, ix.co_id, (uint64_t*)ix.co_thr, pool, s);
}

}  // namespace gscan
