// Graph preparation: device-wide scans, degrees with CSR checks, and the
// degree orientation of Section 6.1 (every edge directed towards its endpoint
// of larger (degree, id)).
#include "scan_internal.cuh"

namespace gscan {

namespace {

constexpr int SCAN_T = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

template <class T>
__device__ __forceinline__ int64_t load_val(const T* in, int64_t i, int64_t n) {
  return i < n ? (int64_t)in[i] : 0;
}

// Block-wide exclusive scan of one int64 per thread; returns the block total.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* out_excl) {
  __shared__ int64_t warp_tot[SCAN_T / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t w = lane < SCAN_T / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < SCAN_T / 32) warp_tot[lane] = w;  // inclusive
  }
  __syncthreads();
  const int64_t before_warp = wid ? warp_tot[wid - 1] : 0;
  const int64_t total = warp_tot[SCAN_T / 32 - 1];
  *out_excl = before_warp + x - v;
  __syncthreads();
  return total;
}

template <class T>
__global__ void k_tile_sums(const T* in, int64_t n, int64_t* sums) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) s += load_val(in, base + k, n);
  int64_t ex;
  int64_t tot = block_exclusive_scan(s, &ex);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// out has n+1 entries; tile_base[b] is the exclusive prefix of tile b.
template <class T>
__global__ void k_tile_scan(const T* in, int64_t n, const int64_t* tile_base, int64_t* out) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) { v[k] = load_val(in, base + k, n); s += v[k]; }
  int64_t ex;
  block_exclusive_scan(s, &ex);
  int64_t run = ex + (tile_base ? tile_base[blockIdx.x] : 0);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int64_t i = base + k;
    if (i <= n) out[i] = run;
    run += v[k];
  }
}

template <class T>
int scan_impl(const T* in, int64_t* out, int64_t n, Pool& pool, cudaStream_t s) {
  // tiles cover indices 0..n (n+1 outputs)
  const int64_t tiles = (n + 1 + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 1) {
    k_tile_scan<T><<<1, SCAN_T, 0, s>>>(in, n, nullptr, out);
    GS_LAUNCH();
    return SCAN_OK;
  }
  int64_t* sums = pool.get<int64_t>(tiles);
  int64_t* base = pool.get<int64_t>(tiles + 1);
  if (!sums || !base) return SCAN_ENOMEM;
  k_tile_sums<T><<<(unsigned)tiles, SCAN_T, 0, s>>>(in, n, sums);
  GS_LAUNCH();
  GS_TRY(scan_impl<int64_t>(sums, base, tiles, pool, s));
  k_tile_scan<T><<<(unsigned)tiles, SCAN_T, 0, s>>>(in, n, base, out);
  GS_LAUNCH();
  pool.put(sums);
  pool.put(base);
  return SCAN_OK;
}

// deg[v], per-row checks, max degree. One warp per vertex row.
// Degrees and CSR checks, 32 rows per warp: lane j reads the bounds of row
// v0 + j, then the warp walks the group's arcs [off[v0], off[v0 + 32]) --
// contiguous -- 32 positions at a time, each lane finding its row among the
// group's by a five-step search over the lanes' row starts. (One warp per row
// would leave most lanes idle on the many short rows.) Rows longer than
// DEG_LONG are listed for k_degrees_long and jumped over (one warp would walk
// a hub's row alone, one dependent load at a time). A group with a bad row
// bound is not walked.
constexpr int DEG_LONG = 4096;

__global__ void k_degrees(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                          int64_t n, int64_t arcs, int32_t* __restrict__ deg, int32_t* maxdeg,
                          unsigned* status, int32_t* __restrict__ long_rows,
                          unsigned* __restrict__ n_long) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t local_max = 0;
  unsigned bad = 0;
  for (int64_t v0 = warp * 32; v0 < n; v0 += nwarps * 32) {
    const int cnt = (int)min((int64_t)32, n - v0);  // rows in this group
    const int64_t v = v0 + lane;
    int64_t b = 0, e = 0;
    if (lane < cnt) { b = off[v]; e = off[v + 1]; }
    // rows must lie inside [0, arcs] before adj is touched
    const bool row_bad = lane < cnt && (b < 0 || e > arcs || e - b < 0 || e - b > 0x7fffffff);
    const bool is_long = !row_bad && e - b > DEG_LONG;
    if (lane < cnt) {
      deg[v] = row_bad ? 0 : (int32_t)(e - b);
      if (!row_bad) local_max = max(local_max, (int32_t)(e - b));
      if (is_long) long_rows[atomicAdd(n_long, 1u)] = (int32_t)v;
    }
    if (__any_sync(FULL, row_bad)) {
      bad = 1;
      continue;
    }
    const int64_t gb = __shfl_sync(FULL, b, 0), ge = __shfl_sync(FULL, e, cnt - 1);
    int32_t carry = 0;  // adj[i - 1] for lane 0
    for (int64_t i0 = gb; i0 < ge;) {
      const int64_t i = i0 + lane;
      // row of position i: the last row of the group starting at or before it
      int j = 0;
#pragma unroll
      for (int step = 16; step; step >>= 1) {
        const int64_t bs = __shfl_sync(FULL, b, (j + step) & 31);
        if (j + step < cnt && bs <= i) j += step;
      }
      const bool row_long = __shfl_sync(FULL, is_long, j);
      const int j0 = __shfl_sync(FULL, j, 0);
      if (__shfl_sync(FULL, row_long, 0)) {  // the chunk starts inside a long row: skip it
        i0 = __shfl_sync(FULL, e, j0);
        continue;
      }
      const bool act = i < ge && !row_long;
      const int32_t x = act ? adj[i] : 0;
      const int64_t bj = __shfl_sync(FULL, b, j);
      int32_t prev = __shfl_up_sync(FULL, x, 1);
      if (lane == 0) prev = carry;
      carry = __shfl_sync(FULL, x, 31);
      if (act) {
        if (x < 0 || x >= n || x == v0 + j) bad = 1;
        if (i > bj && prev >= x) bad = 1;  // strictly ascending: sorted, no duplicates
      }
      i0 += 32;
    }
  }
  for (int o = 16; o; o >>= 1) local_max = max(local_max, __shfl_xor_sync(FULL, local_max, o));
  bad = __any_sync(FULL, bad);
  if (lane == 0) {
    if (local_max) atomicMax(maxdeg, local_max);
    if (bad) atomicOr(status, (unsigned)DEV_BADGRAPH);
  }
}

// The CSR checks of the listed long rows, one CTA per row.
__global__ void __launch_bounds__(1024)
k_degrees_long(const int64_t* __restrict__ off, const int32_t* __restrict__ adj, int64_t n,
               const int32_t* __restrict__ long_rows, const unsigned* __restrict__ n_long,
               unsigned* status) {
  const unsigned cnt = *n_long;
  unsigned bad = 0;
  for (unsigned r = blockIdx.x; r < cnt; r += gridDim.x) {
    const int32_t v = long_rows[r];
    const int64_t b = off[v], e = off[v + 1];
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
      const int32_t x = adj[i];
      if (x < 0 || x >= n || x == v) bad = 1;
      if (i > b && adj[i - 1] >= x) bad = 1;
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, (unsigned)DEV_BADGRAPH);
}

__device__ __forceinline__ bool lower(int32_t du, int32_t u, int32_t dv, int32_t v) {
  return du < dv || (du == dv && u < v);
}

// Orientation in place: the out-arcs of v (neighbours of larger (degree, id))
// are compacted, in id order, to the front of v's own CSR slot range, so
// out(v) = oadj[off[v] .. off[v] + od[v]) needs no separate offsets; the
// in-arcs fill the row from its end; opos holds each arc's position in the
// row. 32 rows per warp, as in k_degrees: lane j keeps row v0 + j's bounds
// and its running out- and in-arc counts, the warp walks the group's arcs 32
// positions at a time, and each lane finds its row by a five-step search and
// its place by ballots masked to its row's lanes. Rows longer than LONG_ROW
// are listed in long_rows for k_orient_long and jumped over.
constexpr int LONG_ROW = 4096;
constexpr int LONG_T = 1024;

__global__ void k_orient_inplace(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                                 const int32_t* __restrict__ deg, int64_t n,
                                 int32_t* __restrict__ od, int32_t* __restrict__ oadj,
                                 int32_t* __restrict__ opos, int32_t* max_od,
                                 unsigned long long* sum_od, int32_t* __restrict__ long_rows,
                                 unsigned* __restrict__ n_long) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;  // lanes below this one
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long local_sum = 0;
  int32_t local_max = 0;
  for (int64_t v0 = warp * 32; v0 < n; v0 += nwarps * 32) {
    const int cnt = (int)min((int64_t)32, n - v0);  // rows in this group
    const int64_t v = v0 + lane;
    int64_t b = 0, e = 0;
    int32_t d = 0;
    if (lane < cnt) { b = off[v]; e = off[v + 1]; d = deg[v]; }
    const bool is_long = d > LONG_ROW;
    if (is_long) long_rows[atomicAdd(n_long, 1u)] = (int32_t)v;
    int32_t w = 0, wi = 0;  // this lane's row: out-arcs placed from the front, in-arcs from the back
    const int64_t gb = __shfl_sync(FULL, b, 0), ge = __shfl_sync(FULL, e, cnt - 1);
    for (int64_t i0 = gb; i0 < ge;) {
      const int64_t i = i0 + lane;
      int j = 0;  // row of position i: the last row of the group starting at or before it
#pragma unroll
      for (int step = 16; step; step >>= 1) {
        const int64_t bs = __shfl_sync(FULL, b, (j + step) & 31);
        if (j + step < cnt && bs <= i) j += step;
      }
      const bool row_long = __shfl_sync(FULL, is_long, j);
      const int j0 = __shfl_sync(FULL, j, 0);
      if (__shfl_sync(FULL, row_long, 0)) {  // the chunk starts inside a long row: skip it
        i0 = __shfl_sync(FULL, e, j0);
        continue;
      }
      const int64_t bj = __shfl_sync(FULL, b, j), ej = __shfl_sync(FULL, e, j);
      const int32_t dj = __shfl_sync(FULL, d, j);
      const int32_t wj = __shfl_sync(FULL, w, j), wij = __shfl_sync(FULL, wi, j);
      const bool act = i < ge && !row_long;
      int32_t x = 0;
      bool up = false;
      if (act) { x = adj[i]; up = lower(dj, (int32_t)(v0 + j), deg[x], x); }
      const unsigned m = __ballot_sync(FULL, up), am = __ballot_sync(FULL, act);
      // lanes of row j in this chunk: [bj - i0, ej - i0) clipped to [0, 32)
      const int lo = (int)max((int64_t)0, bj - i0), hi = (int)min((int64_t)32, ej - i0);
      const unsigned rowm = (hi >= 32 ? FULL : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
      if (up) {
        const int64_t dst = bj + wj + __popc(m & rowm & lt);
        oadj[dst] = x;
        opos[dst] = (int32_t)(i - bj);
      } else if (act) {
        const int64_t dst = ej - 1 - (wij + __popc(~m & am & rowm & lt));
        oadj[dst] = x;
        opos[dst] = (int32_t)(i - bj);
      }
      // each row's owner lane adds its row's counts of this chunk
      const int mlo = (int)max((int64_t)0, b - i0), mhi = (int)min((int64_t)32, e - i0);
      if (lane < cnt && mlo < mhi) {
        const unsigned own = (mhi >= 32 ? FULL : ((1u << mhi) - 1u)) & ~((1u << mlo) - 1u);
        w += __popc(m & own);
        wi += __popc(~m & am & own);
      }
      i0 += 32;
    }
    if (lane < cnt && !is_long) {
      od[v] = w;
      local_sum += (unsigned long long)w;
      local_max = max(local_max, w);
    }
  }
  for (int o = 16; o; o >>= 1) {
    local_sum += __shfl_xor_sync(FULL, local_sum, o);
    local_max = max(local_max, __shfl_xor_sync(FULL, local_max, o));
  }
  if (lane == 0) {
    if (local_sum) atomicAdd(sum_od, local_sum);
    if (local_max) atomicMax(max_od, local_max);
  }
}

// One CTA per listed long row: chunks of LONG_T positions, the out-arcs of a
// chunk placed by a block-wide prefix count (ballots, then a scan of the 32
// warp counts), so the out-list stays in id order; the in-arcs fill the rest
// of the row from its end.
__global__ void __launch_bounds__(LONG_T)
k_orient_long(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
              const int32_t* __restrict__ deg, const int32_t* __restrict__ long_rows,
              const unsigned* __restrict__ n_long, int32_t* __restrict__ od,
              int32_t* __restrict__ oadj, int32_t* __restrict__ opos, int32_t* max_od,
              unsigned long long* sum_od) {
  __shared__ int s_cnt[LONG_T / 32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const unsigned cnt = *n_long;
  for (unsigned r = blockIdx.x; r < cnt; r += gridDim.x) {
    const int32_t v = long_rows[r];
    const int64_t b = off[v], e = off[v + 1];
    const int32_t dv = deg[v];
    int64_t w = b, wi = 0;  // out-arcs placed from the front, in-arcs from the back
    for (int64_t i0 = b; i0 < e; i0 += LONG_T) {
      const int64_t i = i0 + t;
      bool up = false;
      int32_t x = 0;
      if (i < e) { x = adj[i]; up = lower(dv, v, deg[x], x); }
      const unsigned m = __ballot_sync(0xffffffffu, up);
      if (lane == 0) s_cnt[wid] = __popc(m);
      __syncthreads();
      // warp prefix over the 32 warp counts, computed by every warp
      int c = s_cnt[lane];
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const int before = __shfl_sync(0xffffffffu, incl - c, wid);
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      const int up_before = before + __popc(m & ((1u << lane) - 1u));
      if (up) {
        const int64_t dst = w + up_before;
        oadj[dst] = x;
        opos[dst] = (int32_t)(i - b);
      } else if (i < e) {
        const int64_t dst = e - 1 - (wi + (t - up_before));
        oadj[dst] = x;
        opos[dst] = (int32_t)(i - b);
      }
      w += total;
      wi += min((int64_t)LONG_T, e - i0) - total;
      __syncthreads();  // s_cnt is rewritten by the next chunk
    }
    if (t == 0) {
      od[v] = (int32_t)(w - b);
      atomicAdd(sum_od, (unsigned long long)(w - b));
      atomicMax(max_od, (int32_t)(w - b));
    }
  }
}

inline unsigned grid_for(int64_t work, int per_block, int cap = sm_count() * 32) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

}  // namespace

int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, Pool& pool, cudaStream_t s) {
  return scan_impl<int64_t>(in, out, n, pool, s);
}

int exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, Pool& pool,
                              cudaStream_t s) {
  return scan_impl<int32_t>(in, out, n, pool, s);
}

int launch_degrees(const int64_t* off, const int32_t* adj, int64_t n, int64_t arcs, int32_t* deg,
                   int32_t* maxdeg_dev, unsigned* status, Pool& pool, cudaStream_t s) {
  if (n == 0) return SCAN_OK;
  const int64_t max_long = arcs / DEG_LONG + 1;
  int32_t* long_rows = pool.get<int32_t>(max_long);
  unsigned* n_long = pool.get<unsigned>(1);
  if (!long_rows || !n_long) return SCAN_ENOMEM;
  GS_CUDA(cudaMemsetAsync(n_long, 0, sizeof(unsigned), s));
  k_degrees<<<grid_for(n, 256), 256, 0, s>>>(off, adj, n, arcs, deg, maxdeg_dev, status, long_rows,
                                             n_long);
  GS_LAUNCH();
  k_degrees_long<<<(unsigned)std::min<int64_t>(max_long, sm_count() * 2), 1024, 0, s>>>(
      off, adj, n, long_rows, n_long, status);
  GS_LAUNCH();
  pool.put(long_rows);
  pool.put(n_long);
  return SCAN_OK;
}

int launch_orient(const int64_t* off, const int32_t* adj, const int32_t* deg, int64_t n,
                  int64_t arcs, Pool& pool, int32_t** od_out, int32_t** oadj_out,
                  int32_t** opos_out, int32_t* max_od_dev, unsigned long long* sum_od_dev,
                  cudaStream_t s) {
  int32_t* od = pool.get<int32_t>(n > 0 ? n : 1);
  int32_t* oadj = pool.get<int32_t>(arcs > 0 ? arcs : 1);
  int32_t* opos = pool.get<int32_t>(arcs > 0 ? arcs : 1);
  // rows longer than LONG_ROW: at most arcs / LONG_ROW of them
  const int64_t max_long = arcs / LONG_ROW + 1;
  int32_t* long_rows = pool.get<int32_t>(max_long);
  unsigned* n_long = pool.get<unsigned>(1);
  if (!od || !oadj || !opos || !long_rows || !n_long) return SCAN_ENOMEM;
  if (n > 0) {
    GS_CUDA(cudaMemsetAsync(n_long, 0, sizeof(unsigned), s));
    k_orient_inplace<<<grid_for(n, 256), 256, 0, s>>>(off, adj, deg, n, od, oadj, opos, max_od_dev,
                                                    sum_od_dev, long_rows, n_long);
    GS_LAUNCH();
    k_orient_long<<<(unsigned)std::min<int64_t>(max_long, sm_count() * 2), LONG_T, 0, s>>>(
        off, adj, deg, long_rows, n_long, od, oadj, opos, max_od_dev, sum_od_dev);
    GS_LAUNCH();
  }
  pool.put(long_rows);
  pool.put(n_long);
  *od_out = od;
  *oadj_out = oadj;
  *opos_out = opos;
  return SCAN_OK;
}

}  // namespace gscan
