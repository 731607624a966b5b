// Closed-neighbourhood counts c(u,v) = |N̄(u) ∩ N̄(v)| = t(u,v) + 2 for every
// edge, where t(u,v) is the number of triangles on the edge (Section 3.1), and
// the similarity of every arc computed from them (Section 3.1 cosine; Section
// 2.1.1 Jaccard).
//
// Counting follows the oriented triangle enumeration the paper implements
// (Section 6.1): edges point from the lower to the higher (degree, id)
// endpoint, so every out-list is short (at most sqrt(2m) long; 1,756 on R-MAT
// scale 24). Each triangle u < v < w is found exactly once, at its middle
// vertex v: the CTA that owns v keeps out(v) in a shared-memory hash table and
// streams out(u) for the in-neighbours u of v. A hit x = w adds one to
//   (u,v)  -- summed in registers, one atomic per (u,v) pair,
//   (v,w)  -- a shared-memory counter indexed by w's slot in out(v),
//   (u,w)  -- a global atomic at w's slot in out(u).
// This replaces the paper's merge (which reads sum(d+_u + d+_v)) by a hash
// probe of out(u) only (sum over u of d+_u squared), the scheme of the paper's
// Algorithm 1 applied to the oriented lists.
#include "scan_internal.cuh"

namespace gscan {

namespace {

#ifndef GS_TRI_FAST_ROUNDS
#define GS_TRI_FAST_ROUNDS 12  // 32-element rounds in flight for out-lists streamed one at a time
#endif

constexpr int TRI_THREADS = 512;
constexpr int TRI_WARPS = TRI_THREADS / 32;
constexpr int SMEM_OD_MAX = 4096;    // out(v) sizes handled by the shared-memory table

__device__ __forceinline__ bool lower(int32_t du, int32_t u, int32_t dv, int32_t v) {
  return du < dv || (du == dv && u < v);
}

// Key of vertex x in the degree order: descending keys = ascending (d_x, x).
__device__ __forceinline__ uint64_t rank_key(int32_t d, int32_t x) {
  return ~(((uint64_t)(uint32_t)d << 32) | (uint32_t)x);
}

// Position of key kv in the descending key list kb[0..len), or -1.
__device__ __forceinline__ int key_search(const uint64_t* __restrict__ kb, int len, uint64_t kv) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (kb[mid] > kv) lo = mid + 1; else hi = mid;
  }
  return (lo < len && kb[lo] == kv) ? lo : -1;
}

// A vertex whose row has at most cfg.warp_deg positions and whose out-list
// has at most SMALL_OD entries is handled by one warp with its own table;
// the rest by the CTA kernel (the strategy per degree bucket, a tuning
// parameter).
constexpr int SMALL_OD = 256;
constexpr int SW_SLOTS = 2 * SMALL_OD;  // 2^table_log2(SMALL_OD) slots per table

__host__ __device__ __forceinline__ bool warp_vertex(int64_t d, int64_t od, int warp_deg) {
  return d <= warp_deg && od <= SMALL_OD;
}
constexpr int SW_WARPS = 4;

// Work items of the CTA kernel: a vertex v not handled by a warp contributes
// ceil(in-degree/chunk) items when it has in-neighbours (every in-arc needs
// the position of its source in N(v), even when out(v) is empty and no
// triangle has v in the middle). items[v] -> prefix -> item index maps to
// (v, chunk).
// (v0, v1): only middle vertices in [v0, v1) get items (a rank's share of a
// sharded count; the whole graph otherwise).
__global__ void k_item_counts(const int32_t* __restrict__ odeg, const int32_t* __restrict__ deg,
                              int64_t n, int warp_deg, int chunk, int64_t v0, int64_t v1,
                              int32_t* __restrict__ items) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t od = odeg[v];
    const int32_t d = deg[v];
    int c = 0;
    if (v >= v0 && v < v1 && !warp_vertex(d, od, warp_deg) && d - od > 0)
      c = (int)((d - od + chunk - 1) / chunk);
    items[v] = c;
  }
}

// Order in which the CTA kernel takes its vertices: non-increasing degree.
// In-neighbours are shared far more among vertices of similar (high) degree
// than among vertices of consecutive ids, so their out-lists and counters
// are re-read from L2 instead of DRAM. bin(v) = maxdeg - d_v for vertices
// with items; equal degrees come in any order (the counts are sums).
__global__ void k_item_hist(const int32_t* __restrict__ items, const int32_t* __restrict__ deg,
                            int64_t n, int32_t maxdeg, unsigned long long* __restrict__ hist) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (items[v] > 0) atomicAdd(&hist[maxdeg - deg[v]], 1ull);
}

__global__ void k_item_place(const int32_t* __restrict__ items, const int32_t* __restrict__ deg,
                             int64_t n, int32_t maxdeg, const int64_t* __restrict__ start,
                             unsigned long long* __restrict__ fill, int32_t* __restrict__ order) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (items[v] > 0) {
      const int64_t b = maxdeg - deg[v];
      order[start[b] + (int64_t)atomicAdd(&fill[b], 1ull)] = (int32_t)v;
    }
}

// items of the i-th vertex of the order (0 past the placed vertices)
__global__ void k_item_gather(const int32_t* __restrict__ items, const int32_t* __restrict__ order,
                              const int64_t* __restrict__ start, int32_t maxdeg, int64_t n,
                              int32_t* __restrict__ items_sorted) {
  const int64_t placed = start[maxdeg + 1];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    items_sorted[i] = i < placed ? items[order[i]] : 0;
}

__device__ __forceinline__ int64_t find_item_vertex(const int64_t* item_off, int64_t n,
                                                     int64_t item) {
  // largest v with item_off[v] <= item
  int64_t lo = 0, hi = n;  // item_off[n] > item
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (item_off[mid] <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// Lookup of out(v): a two-table cuckoo hash in shared memory, or (BIG, and
// in the unlikely case that no cuckoo placement was found) binary search in
// the sorted global list.
//
// Each table has 2^L slots; out(v) has at most 2^(L-1) entries, so the load
// of the pair is at most 1/4. A key x hashes to h_i = x * C_i (mod 2^32, a
// bijection for odd C_i); its slot is the top L bits of h_i, and the slot
// stores h_i itself, so a probe is one load and one compare, with no probing
// loop. The position of x in out(v) sits in a parallel 16-bit array read on
// hits only. An empty slot of table i holds h_i(-1), which no vertex id
// produces; stream lanes past the end of a list carry NO_KEY = -2, which
// matches neither a key nor an empty slot.
constexpr int32_t NO_KEY = -2;
constexpr int CUCKOO_KICKS = 64;     // evictions before an insertion gives up
constexpr int CUCKOO_ATTEMPTS = 4;   // multiplier pairs tried before binary search

constexpr uint32_t mul_inverse(uint32_t c) {  // inverse of an odd c mod 2^32 (Newton)
  uint32_t y = c;
  for (int i = 0; i < 5; ++i) y *= 2u - c * y;
  return y;
}
// odd multipliers (from the golden ratio and common 32-bit hash primes)
__constant__ uint32_t CUCKOO_MUL[2 * CUCKOO_ATTEMPTS] = {
    0x9E3779B1u, 0x85EBCA77u, 0xC2B2AE3Du, 0x27D4EB2Fu,
    0x165667B1u, 0xD3A2646Du, 0xFD7046C5u, 0xB55A4F09u};

// Table memory: t0[hcap] | t1[hcap] (uint32 keys) | p0[hcap] | p1[hcap]
// (uint16 positions in out(v)), hcap a power of two >= 2^L.
struct OutTable {
  const uint32_t* t0;
  int hcap;
  int shift;              // 32 - L
  uint32_t c0, c1;        // multipliers of the two tables
  const uint64_t* gkey;   // rank keys of out(v) in global memory (binary search)
  const int32_t* deg;     // degrees, for the rank key of a probed vertex
  int32_t od;
  bool bsearch;           // no cuckoo placement: the item needs the binary-search path
};

template <bool BIG>
__device__ __forceinline__ int table_lookup(const OutTable& t, int32_t x) {
  if (BIG) return x < 0 ? -1 : key_search(t.gkey, t.od, rank_key(t.deg[x], x));
  const uint32_t h0 = (uint32_t)x * t.c0, h1 = (uint32_t)x * t.c1;
  const uint32_t s0 = h0 >> t.shift, s1 = (h1 >> t.shift) + t.hcap;  // slot in t0 / t1
  const bool m0 = t.t0[s0] == h0, m1 = t.t0[s1] == h1;
  const uint16_t* pos = reinterpret_cast<const uint16_t*>(t.t0 + 2 * t.hcap);
  return (m0 || m1) ? (int)pos[m0 ? s0 : s1] : -1;
}

// Cuckoo insertion of key x: place h_0(x) in table 0; an evicted key moves
// to its slot in the other table, and so on. Returns false if a key is still
// homeless after CUCKOO_KICKS moves (the table must then be rebuilt).
__device__ __forceinline__ bool cuckoo_insert(uint32_t* t0, uint32_t* t1, int shift, uint32_t c0,
                                              uint32_t c1, int32_t x) {
  const uint32_t e0 = 0u - c0, e1 = 0u - c1;  // h_i(-1): empty slots
  const uint32_t i0 = mul_inverse(c0), i1 = mul_inverse(c1);
  int which = 0;
  for (int kick = 0; kick < CUCKOO_KICKS; ++kick) {
    const uint32_t h = (uint32_t)x * (which ? c1 : c0);
    const uint32_t old = atomicExch(&(which ? t1 : t0)[h >> shift], h);
    if (old == (which ? e1 : e0)) return true;
    x = (int32_t)(old * (which ? i1 : i0));
    which ^= 1;
  }
  return false;
}

// log2 of the slots per table for an out-list of od entries (at least 32).
__device__ __forceinline__ int table_log2(int32_t od) {
  int L = 5;
  while ((1 << (L - 1)) < od) ++L;
  return L;
}

// Builds the table of out(v) = list[0..od) with `nthreads` threads (tid in
// [0, nthreads)); `sync` is the group barrier and `any` its OR-reduction.
// Keys are placed first, then every key's position is written next to the
// slot where it ended up. Returns the OutTable, with bsearch set if no
// attempt placed every key.
template <typename Sync, typename Any>
__device__ __forceinline__ OutTable table_build(uint32_t* t0, int hcap, uint32_t* vcnt,
                                                const int32_t* list, const uint64_t* gkey,
                                                const int32_t* deg, int32_t od, int tid,
                                                int nthreads, Sync sync, Any any) {
  uint32_t* t1 = t0 + hcap;
  uint16_t* p0 = reinterpret_cast<uint16_t*>(t0 + 2 * hcap);
  uint16_t* p1 = p0 + hcap;
  const int L = table_log2(od);
  const int H = 1 << L;
  const int shift = 32 - L;
  int attempt = 0;
  bool failed = true;
  uint32_t c0 = 0, c1 = 0;
  for (; attempt < CUCKOO_ATTEMPTS && failed; ++attempt) {
    c0 = CUCKOO_MUL[2 * attempt];
    c1 = CUCKOO_MUL[2 * attempt + 1];
    uint4* w0 = reinterpret_cast<uint4*>(t0);
    uint4* w1 = reinterpret_cast<uint4*>(t1);
    const uint32_t e0 = 0u - c0, e1 = 0u - c1;
    for (int i = tid; i < H / 4; i += nthreads) {
      w0[i] = make_uint4(e0, e0, e0, e0);
      w1[i] = make_uint4(e1, e1, e1, e1);
    }
    sync();
    bool ok = true;
    for (int j = tid; j < od; j += nthreads) ok &= cuckoo_insert(t0, t1, shift, c0, c1, list[j]);
    failed = any(!ok);
  }
  if (!failed)
    for (int j = tid; j < od; j += nthreads) {
      const uint32_t h0 = (uint32_t)list[j] * c0;
      if (t0[h0 >> shift] == h0) p0[h0 >> shift] = (uint16_t)j;
      else p1[((uint32_t)list[j] * c1) >> shift] = (uint16_t)j;
    }
  if (vcnt)
    for (int i = tid; i < od; i += nthreads) vcnt[i] = 0;
  sync();
  return OutTable{t0, hcap, shift, c0, c1, gkey, deg, od, failed};
}

// Per-warp scratch for one 32-position slice.
struct SliceSmem {
  int32_t* u;
  int32_t* p;
  uint32_t* acc;
};

// One probe of the stream element x at position j of out(u): a hit w = x
// adds one to (v,w) in vcnt (shared; global for BIG) and to (u,w) at j. The
// (u,w) count is at most d+(u) - 1 < sqrt(2m) < 2^16 whenever the graph has
// fewer than 2^31 arcs (IT = int32), so it is kept as a 16-bit half of a
// 32-bit word (tc16): half the footprint of the most scattered atomics.
template <bool BIG, typename IT>
__device__ __forceinline__ bool probe(const OutTable& tab, int32_t x, IT j, int64_t ob,
                                      uint32_t* vcnt, uint32_t* __restrict__ tcnt,
                                      uint32_t* __restrict__ tc16) {
  const int q = table_lookup<BIG>(tab, x);
  if (q < 0) return false;
  if (!BIG) atomicAdd(&vcnt[q], 1u);
  else atomicAdd(&tcnt[ob + q], 1u);
  if (sizeof(IT) == 4) atomicAdd(&tc16[j >> 1], 1u << ((j & 1) << 4));
  else atomicAdd(&tcnt[j], 1u);
  return true;
}

// Weighted cosine (Section 4.1.1, w(x,x) = 1): a triangle u < v < w adds
// w(u,w) w(v,w) to the numerator of (u,v), w(u,v) w(u,w) to that of (v,w)
// and w(u,v) w(v,w) to that of (u,w). ow[i] is the weight of out-arc i and
// tsum[i] its numerator sum. A hit is named by three out-arc slots: j
// (u->w), vq (v->w) and jo (u->v). FP64 instructions are issued for a whole
// warp at a time on a pipe of two lanes per clock, so hits are not summed
// where they are found: each warp appends them to a buffer in shared memory
// and applies 32 at a time, three products and three global double
// reductions per hit (executed in L2, off the FP64 pipe).
constexpr int WT_BUF = 64;  // entries per warp: 32 to apply + up to 31 waiting

struct Weights {
  const double* ow;  // weight of every out-arc, at its slot
  double* tsum;      // numerator sums of every out-arc (global)
  void* buf;         // this warp's hit buffer: IT j[WT_BUF], vq[WT_BUF], jo[WT_BUF]
};

template <typename IT>
__device__ __forceinline__ void wt_apply(IT j, IT vq, IT jo, const Weights& wt) {
  const double w_uw = wt.ow[j], w_vw = wt.ow[vq], w_uv = wt.ow[jo];
  atomicAdd(&wt.tsum[vq], w_uv * w_uw);
  atomicAdd(&wt.tsum[j], w_uv * w_vw);
  atomicAdd(&wt.tsum[jo], w_uw * w_vw);
}

// Warp-wide (all lanes): append this lane's hit, if any; apply the newest 32
// entries once the buffer holds at least 32.
template <typename IT>
__device__ __forceinline__ void wt_push(bool hit, IT j, IT vq, IT jo, int& cnt, const Weights& wt) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(FULL, hit);
  if (!m) return;
  IT* b = static_cast<IT*>(wt.buf);
  if (hit) {
    const int pos = cnt + __popc(m & ((1u << lane) - 1u));
    b[pos] = j;
    b[WT_BUF + pos] = vq;
    b[2 * WT_BUF + pos] = jo;
  }
  cnt += __popc(m);
  if (cnt >= 32) {
    __syncwarp();
    const int e = cnt - 32 + lane;
    wt_apply<IT>(b[e], b[WT_BUF + e], b[2 * WT_BUF + e], wt);
    cnt -= 32;
    __syncwarp();
  }
}

// Warp-wide: apply what is left in the buffer.
template <typename IT>
__device__ __forceinline__ void wt_drain(int cnt, const Weights& wt) {
  const int lane = threadIdx.x & 31;
  const IT* b = static_cast<const IT*>(wt.buf);
  __syncwarp();
  if (lane < cnt) wt_apply<IT>(b[lane], b[WT_BUF + lane], b[2 * WT_BUF + lane], wt);
  __syncwarp();
}

// One warp: triangles u < v < w for the in-neighbours u of v at positions
// [p0, min(p0+32, p_end)) of v's in-arc range (oadj[rb ..], packed by the
// orientation; in LSH mode the skipped ones are dropped). They are compacted
// to lanes 0..k-1, and each lane finds v in out(u) (ascending rank) by a
// binary search of its rank key: that gives the twin position of the arc
// u->v, and the possible third vertices w > v are the entries after it.
// Suffixes of at least long_list entries are streamed one at a time, lane l
// taking elements l, l+32, ... (RF rounds of loads in flight); the shorter
// ones are concatenated and walked 32 elements per round (R rounds in
// flight), the owner of an element coming from the suffix starts that fall
// in its round (ballot / or-reduce / popc). Hits on (u,v) are counted per
// list; weighted hits go to the warp's hit buffer.
template <bool BIG, typename IT, bool WT, int R>
__device__ __forceinline__ void process_slice(
    int64_t p0, int64_t p_end, int64_t rb, int32_t v, int32_t dv, int32_t od, int64_t ob,
    int long_list, const int32_t* __restrict__ opos,
    const int32_t* __restrict__ adj, const int32_t* __restrict__ deg,
    const int64_t* __restrict__ off, const int32_t* __restrict__ odeg,
    const int32_t* __restrict__ oadj, const uint64_t* __restrict__ okey,
    const int64_t* __restrict__ odp, int lsh_T, const OutTable& tab, uint32_t* vcnt,
    const SliceSmem& sm, uint32_t* __restrict__ tcnt, uint32_t* __restrict__ tc16,
    int32_t* __restrict__ twin_rel, unsigned& bad, const Weights& wt) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t p = p0 + lane;
  int32_t u = -1;
  bool is_in = false;
  if (p < p_end) {
    // v's in-neighbours are packed at the end of its slot range (orientation)
    u = oadj[rb + p];
    is_in = true;
    // LSH mode: if u and v are both above the threshold, every edge of
    // every triangle u < v < w is approximated, so the scan is not needed
    if (lsh_T >= 0 && deg[u] > lsh_T) is_in = false;
  }
  const unsigned m = __ballot_sync(FULL, is_in);
  if (!m) return;
  const int k = __popc(m);
  if (is_in) {
    const int r = __popc(m & ((1u << lane) - 1u));
    sm.u[r] = u;
    sm.p[r] = opos[rb + p];  // position of u in N(v), the twin of the arc u->v
  }
  __syncwarp();
  int32_t cp = 0, clen = 0;  // suffix length after v
  IT cub = 0, jv = 0;        // suffix start; position of v in out(u)
  bool found = false;
  if (lane < k) {
    const int32_t cu = sm.u[lane];
    cp = sm.p[lane];
    const IT ub = (IT)off[cu];
    const int32_t len = odeg[cu];
    const int pos = key_search(okey + odp[cu], len, rank_key(dv, v));
    found = pos >= 0;
    if (found) {
      jv = ub + (IT)pos;
      cub = jv + 1;
      clen = len - pos - 1;
    } else {
      bad = 1;  // v lists u but u does not list v
    }
  }
  if (od == 0) {
    // no triangle has v in the middle: only the twin positions
    if (found) twin_rel[jv] = cp;
    __syncwarp();
    return;
  }
  sm.acc[lane] = 0;
  int wcnt = 0;  // weighted mode: entries in this warp's hit buffer
  __syncwarp();

  // 1. long suffixes, one at a time
  constexpr int RF = GS_TRI_FAST_ROUNDS;
  unsigned lm = __ballot_sync(FULL, lane < k && clen >= long_list);
  while (lm) {
    const int i = __ffs(lm) - 1;
    lm &= lm - 1;
    const IT ub = __shfl_sync(FULL, cub, i);
    const int32_t len = __shfl_sync(FULL, clen, i);
    const IT jvi = WT ? __shfl_sync(FULL, jv, i) : (IT)0;  // the arc u->v of list i
    unsigned hits = 0;  // this lane's hits on the list
    for (int32_t t0 = 0; t0 < len; t0 += 32 * RF) {
      int32_t xs[RF];
#pragma unroll
      for (int rr = 0; rr < RF; ++rr) {
        const int32_t t = t0 + 32 * rr + lane;
        xs[rr] = t < len ? oadj[ub + (IT)t] : NO_KEY;
      }
#pragma unroll
      for (int rr = 0; rr < RF; ++rr) {
        if (t0 + 32 * rr >= len) break;
        const IT j = ub + (IT)(t0 + 32 * rr + lane);
        if (WT) {
          const int q = table_lookup<BIG>(tab, xs[rr]);
          wt_push<IT>(q >= 0, j, (IT)(ob + q), jvi, wcnt, wt);
        } else {
          hits += probe<BIG, IT>(tab, xs[rr], j, ob, vcnt, tcnt, tc16) ? 1u : 0u;
        }
      }
    }
    if (!WT) {
      hits = __reduce_add_sync(FULL, hits);
      if (lane == 0) sm.acc[i] += hits;
    }
  }

  // 2. short non-empty suffixes, concatenated: lane r takes the r-th of them
  const bool is_short = lane < k && clen > 0 && clen < long_list;
  const unsigned shm = __ballot_sync(FULL, is_short);
  if (shm) {
    const int k2 = __popc(shm);
    if (is_short) sm.u[__popc(shm & ((1u << lane) - 1u))] = lane;
    __syncwarp();
    const int orig = lane < k2 ? sm.u[lane] : 0;  // index of the list among the k
    const IT sub = __shfl_sync(FULL, cub, orig);
    const int32_t sl = __shfl_sync(FULL, clen, orig);
    const int32_t slen = lane < k2 ? sl : 0;
    int32_t incl = slen;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += y;
    }
    const int32_t cstart = incl - slen;
    const int32_t W = __shfl_sync(FULL, incl, 31);
    for (int32_t rbase = 0; rbase < W; rbase += 32 * R) {
      int32_t xs[R];
      IT js[R];
      int owns[R];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const int32_t r0 = rbase + 32 * rr;
        const int32_t t = r0 + lane;
        // the concatenated suffixes are non-empty, so their starts are distinct
        const bool starts_here = lane < k2 && cstart >= r0 && cstart < r0 + 32;
        const unsigned smask = __reduce_or_sync(FULL, starts_here ? (1u << (cstart - r0)) : 0u);
        const int before = __popc(__ballot_sync(FULL, lane < k2 && cstart < r0));
        const int owner = before + __popc(smask & ((2u << lane) - 1u)) - 1;
        const int own = owner < 0 ? 0 : owner;
        const IT ub_o = __shfl_sync(FULL, sub, own);
        const int32_t st_o = __shfl_sync(FULL, cstart, own);
        owns[rr] = __shfl_sync(FULL, orig, own);
        js[rr] = t < W ? ub_o + (IT)(t - st_o) : (IT)-1;
        xs[rr] = t < W ? oadj[js[rr]] : NO_KEY;
      }
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const int own = owns[rr];
        if (WT) {
          // the owner's arc u->v is held by lane `own`
          const IT jo = __shfl_sync(FULL, jv, own);
          const int q = table_lookup<BIG>(tab, xs[rr]);
          wt_push<IT>(q >= 0, js[rr], (IT)(ob + q), jo, wcnt, wt);
        } else {
          const bool hit = probe<BIG, IT>(tab, xs[rr], js[rr], ob, vcnt, tcnt, tc16);
          const unsigned hm = __ballot_sync(FULL, hit);
          if (hm) {
            // lanes of one owner are contiguous; its first lane adds
            const unsigned peers = __match_any_sync(FULL, own);
            if ((hm & peers) && lane == __ffs(peers) - 1) sm.acc[own] += __popc(hm & peers);
          }
        }
      }
    }
  }
  __syncwarp();
  if (WT) wt_drain<IT>(wcnt, wt);
  if (found) {
    if (!WT) {
      const uint32_t acc = sm.acc[lane];
      if (acc) atomicAdd(&tcnt[jv], acc);
    }
    twin_rel[jv] = cp;  // position of u in N(v)
  }
  __syncwarp();
}

// CTA kernel for the other rows: the CTA shares out(v)'s table and
// its warps pull 32-position slices of the item's range of in-arcs.
// BIG = out(v) too long for the shared table (binary search, global counters);
// the BIG kernel also takes the items listed in `deferred`, whose shared
// table could not be built (no cuckoo placement).
template <bool BIG, typename IT, bool WT, int R>
__global__ void __launch_bounds__(TRI_THREADS, 3)
k_triangles(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
            const int32_t* __restrict__ deg, const int32_t* __restrict__ odeg,
            const int32_t* __restrict__ oadj, const int32_t* __restrict__ opos,
            const uint64_t* __restrict__ okey,
            const int64_t* __restrict__ odp, int64_t n, const int64_t* __restrict__ item_off,
            const int32_t* __restrict__ order, unsigned long long* __restrict__ work, int lsh_T,
            int item_chunk, int long_list,
            int od_cap, int64_t* __restrict__ deferred, unsigned long long* __restrict__ n_deferred,
            bool deferred_only, uint32_t* __restrict__ tcnt, uint32_t* __restrict__ tc16,
            int32_t* __restrict__ twin_rel, unsigned* status, const double* __restrict__ ow,
            double* __restrict__ tsum) {
  // shared layout for od_cap (a power of two >= every od handled here) and
  // hcap = 2^table_log2(od_cap): the table (t0, t1, p0, p1; 12 bytes per
  // hcap), then vcnt[od_cap]
  extern __shared__ uint4 smem4[];
  __shared__ long long s_item;
  __shared__ int s_next;  // next 32-position slice of the item's CSR range
  __shared__ int32_t s_u[TRI_WARPS][32];
  __shared__ int32_t s_p[TRI_WARPS][32];
  __shared__ uint32_t s_acc[TRI_WARPS][32];
  __shared__ IT s_hb[WT ? TRI_WARPS : 1][WT ? 3 * WT_BUF : 1];  // weighted mode: hit buffers
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // BIG: first the items whose out-list is too long for the shared table
  // (unless deferred_only), then the deferred ones
  const int64_t total_items = (BIG && deferred_only) ? 0 : item_off[n];
  const int64_t total = BIG ? total_items + (int64_t)*n_deferred : total_items;
  const int hcap = 1 << table_log2(od_cap);
  uint32_t* t0 = reinterpret_cast<uint32_t*>(smem4);
  uint32_t* vcnt = t0 + 3 * hcap;  // (unweighted mode only)
  const Weights wt{ow, tsum, WT ? (void*)s_hb[wid] : nullptr};
  const SliceSmem sm{s_u[wid], s_p[wid], s_acc[wid]};
  unsigned bad = 0;

  for (;;) {
    if (threadIdx.x == 0) {
      s_item = (long long)atomicAdd(work, 1ull);
      s_next = 0;
    }
    __syncthreads();
    const int64_t w = s_item;
    if (w >= total) break;
    const bool was_deferred = BIG && w >= total_items;
    const int64_t item = was_deferred ? deferred[w - total_items] : w;
    const int64_t idx = find_item_vertex(item_off, n, item);
    const int64_t v = order[idx];
    const int64_t chunk = item - item_off[idx];
    const int32_t dv = deg[v];
    const int64_t ob = off[v];
    const int32_t od = odeg[v];
    const bool skip_item = BIG ? (od <= SMEM_OD_MAX && !was_deferred) : (od > SMEM_OD_MAX);
    if (skip_item) { __syncthreads(); continue; }
    OutTable tab{nullptr, 0, 27, 0u, 0u, okey + odp[v], deg, od, true};
    if (!BIG && od > 0) {
      tab = table_build(t0, hcap, WT ? nullptr : vcnt, oadj + ob, okey + odp[v], deg, od,
                        threadIdx.x, TRI_THREADS,
                        [] { __syncthreads(); }, [](bool b) { return __syncthreads_or(b) != 0; });
      if (tab.bsearch) {  // hand the item to the BIG kernel
        if (threadIdx.x == 0) deferred[atomicAdd(n_deferred, 1ull)] = item;
        __syncthreads();
        continue;
      }
    }
    const int64_t rb = off[v] + od;  // v's in-arcs
    const int64_t p_begin = chunk * item_chunk;
    const int64_t p_end = min((int64_t)(dv - od), p_begin + item_chunk);
    for (;;) {
      // warps pull 32-position slices until the item's range is exhausted
      int slice = 0;
      if (lane == 0) slice = atomicAdd(&s_next, 32);
      slice = __shfl_sync(FULL, slice, 0);
      const int64_t pos0 = p_begin + slice;
      if (pos0 >= p_end) break;
      process_slice<BIG, IT, WT, R>(pos0, p_end, rb, (int32_t)v, dv, od, ob, long_list, opos, adj, deg,
                                    off, odeg, oadj, okey, odp, lsh_T, tab, vcnt, sm, tcnt, tc16,
                                    twin_rel, bad, wt);
    }
    __syncthreads();
    if (!BIG && !WT)
      for (int j = threadIdx.x; j < od; j += TRI_THREADS) {
        const uint32_t c = vcnt[j];
        if (c) atomicAdd(&tcnt[ob + j], c);
      }
    __syncthreads();
  }
  if (bad) atomicOr(status, (unsigned)DEV_BADGRAPH);
}

// Warp kernel for rows of at most warp_deg positions with out-lists of at
// most SMALL_OD entries: each warp owns one
// vertex at a time, with its own table of out(v) (no CTA barrier). Warps take
// 32 vertices per atomic fetch.
template <typename IT, bool WT, int R>
__global__ void __launch_bounds__(SW_WARPS * 32, 8)
k_tri_small(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
            const int32_t* __restrict__ deg, const int32_t* __restrict__ odeg,
            const int32_t* __restrict__ oadj, const int32_t* __restrict__ opos,
            const uint64_t* __restrict__ okey,
            const int64_t* __restrict__ odp, int64_t n, unsigned long long* __restrict__ work,
            int lsh_T, int warp_deg, int long_list, uint32_t* __restrict__ tcnt,
            uint32_t* __restrict__ tc16,
            int32_t* __restrict__ twin_rel, unsigned* status, const double* __restrict__ ow,
            double* __restrict__ tsum) {
  __shared__ __align__(16) uint32_t s_tab[SW_WARPS][3 * SW_SLOTS];  // t0 | t1 | p0 p1
  __shared__ uint32_t s_cnt[WT ? 1 : SW_WARPS][SMALL_OD];
  __shared__ IT s_hb[WT ? SW_WARPS : 1][WT ? 3 * WT_BUF : 1];  // weighted mode: hit buffers
  __shared__ int32_t s_u[SW_WARPS][32];
  __shared__ int32_t s_p[SW_WARPS][32];
  __shared__ uint32_t s_acc[SW_WARPS][32];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* vcnt = WT ? nullptr : s_cnt[wid];
  const Weights wt{ow, tsum, WT ? (void*)s_hb[wid] : nullptr};
  const SliceSmem sm{s_u[wid], s_p[wid], s_acc[wid]};
  unsigned bad = 0;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(work, 32ull);
    base = __shfl_sync(FULL, base, 0);
    if ((int64_t)base >= n) break;
    // the lanes read the 32 vertices' degrees at once; the warp then visits
    // only its vertices with in-neighbours (most have none: their
    // neighbours all rank above them)
    const int64_t vl = (int64_t)base + lane;
    const int32_t dl = vl < n ? deg[vl] : 0;
    const int32_t ol = vl < n ? odeg[vl] : 0;
    const bool mine = dl > 0 && warp_vertex(dl, ol, warp_deg) && dl - ol > 0;
    const int64_t offl = mine ? off[vl] : 0, odpl = mine ? odp[vl] : 0;
    unsigned todo = __ballot_sync(FULL, mine);
    while (todo) {
      const int k = __ffs(todo) - 1;
      todo &= todo - 1;
      const int64_t vv = (int64_t)base + k;
      const int32_t dv = __shfl_sync(FULL, dl, k);
      const int32_t od = __shfl_sync(FULL, ol, k);
      const int64_t ob = __shfl_sync(FULL, offl, k);
      const uint64_t* okv = okey + __shfl_sync(FULL, odpl, k);
      OutTable tab{nullptr, 0, 27, 0u, 0u, okv, deg, od, true};
      if (od > 0) {
        tab = table_build(s_tab[wid], SW_SLOTS, vcnt, oadj + ob, okv, deg, od, lane, 32,
                          [] { __syncwarp(); },
                          [](bool b) { __syncwarp(); return __any_sync(0xffffffffu, b) != 0; });
      }
      const bool use_table = !tab.bsearch;
      const int64_t rb = ob + od;  // vv's in-arcs
      for (int64_t pos0 = 0; pos0 < dv - od; pos0 += 32) {
        if (use_table)
          process_slice<false, IT, WT, R>(pos0, dv - od, rb, (int32_t)vv, dv, od, ob, long_list, opos, adj,
                                          deg, off, odeg, oadj, okey, odp, lsh_T, tab, vcnt, sm,
                                          tcnt, tc16, twin_rel, bad, wt);
        else
          process_slice<true, IT, WT, R>(pos0, dv - od, rb, (int32_t)vv, dv, od, ob, long_list, opos, adj,
                                         deg, off, odeg, oadj, okey, odp, lsh_T, tab, vcnt, sm,
                                         tcnt, tc16, twin_rel, bad, wt);
      }
      __syncwarp();
      if (use_table && !WT)
        for (int j = lane; j < od; j += 32) {
          const uint32_t c = vcnt[j];
          if (c) atomicAdd(&tcnt[ob + j], c);
        }
      __syncwarp();
    }
  }
  if (bad) atomicOr(status, (unsigned)DEV_BADGRAPH);
}

// Cosine (Section 3.1) or Jaccard (Section 2.1.1) from the closed count.
__device__ __forceinline__ double sim_of(int kind, int64_t c, int64_t du, int64_t dv) {
  if (kind == SCAN_COSINE) {
    const int64_t prod = (du + 1) * (dv + 1);
    return __ddiv_rn((double)c, __dsqrt_rn((double)prod));
  }
  return __ddiv_rn((double)c, (double)(du + dv + 2 - c));
}

// Every oriented edge a->b writes sigma to both of its CSR arcs. Threads run
// over the oriented edges in order (odp = exclusive prefix of the
// out-degrees, so edge k is the (k - odp[a])-th out-arc of the vertex a with
// odp[a] <= k < odp[a+1]); a CTA's EXPAND_T * EXPAND_ITEMS edges span the
// vertices between two binary searches, and each edge finds its own vertex
// by a search inside that bracket.
constexpr int EXPAND_T = 256;
constexpr int EXPAND_ITEMS = 8;

__device__ __forceinline__ int64_t row_of(const int64_t* __restrict__ odp, int64_t lo, int64_t hi,
                                          int64_t k) {
  // largest a in [lo, hi) with odp[a] <= k (odp[lo] <= k)
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (odp[mid] <= k) lo = mid; else hi = mid;
  }
  return lo;
}

// Every out-arc in compact order (k = odp[a] + i, i < od[a], at CSR
// position j = off[a] + i), 32 rows per warp: lane l holds row v0 + l's odp
// and off, the warp walks the group's out-arcs [odp[v0], odp[v0 + 32]) --
// contiguous -- 32 at a time, and each lane finds its row by a five-step
// search over the lanes' odp values (no dependent global loads, unlike a
// binary search of odp). f(k, a, j) runs for every out-arc.
template <class F>
__device__ __forceinline__ void walk_out_arcs(const int64_t* __restrict__ off,
                                              const int64_t* __restrict__ odp, int64_t n, F f) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v0 = warp * 32; v0 < n; v0 += nwarps * 32) {
    const int cnt = (int)min((int64_t)32, n - v0);
    int64_t kb = 0, rb = 0;
    if (lane < cnt) { kb = odp[v0 + lane]; rb = off[v0 + lane]; }
    const int64_t g0 = __shfl_sync(FULL, kb, 0), g1 = odp[v0 + cnt];
    for (int64_t k0 = g0; k0 < g1; k0 += 32) {
      const int64_t k = k0 + lane;
      int r = 0;
#pragma unroll
      for (int step = 16; step; step >>= 1) {
        const int64_t bs = __shfl_sync(FULL, kb, (r + step) & 31);
        if (r + step < cnt && bs <= k) r += step;
      }
      const int64_t kbr = __shfl_sync(FULL, kb, r), rbr = __shfl_sync(FULL, rb, r);
      if (k < g1) f(k, v0 + r, rbr + (k - kbr));
    }
  }
}

__global__ void __launch_bounds__(EXPAND_T)
k_expand(int kind, const int64_t* __restrict__ off, const int32_t* __restrict__ deg,
         const int64_t* __restrict__ odp, const int32_t* __restrict__ oadj,
         const int32_t* __restrict__ opos, const uint32_t* __restrict__ tcnt,
         const uint32_t* __restrict__ tc16,
         const int32_t* __restrict__ twin_rel, int64_t n, int lsh_T,
         double* __restrict__ sim_csr, unsigned* status) {
  __shared__ int64_t s_bracket[2];
  const int64_t m = odp[n];
  constexpr int64_t CH = (int64_t)EXPAND_T * EXPAND_ITEMS;
  unsigned bad = 0;
  for (int64_t k0 = (int64_t)blockIdx.x * CH; k0 < m; k0 += (int64_t)gridDim.x * CH) {
    const int64_t k1 = min(m, k0 + CH);
    if (threadIdx.x == 0) s_bracket[0] = row_of(odp, 0, n + 1, k0);
    if (threadIdx.x == 1) s_bracket[1] = row_of(odp, 0, n + 1, k1 - 1) + 1;
    __syncthreads();
    const int64_t lo = s_bracket[0], hi = s_bracket[1];
    for (int64_t k = k0 + threadIdx.x; k < k1; k += EXPAND_T) {
      const int64_t a = row_of(odp, lo, hi, k);
      const int64_t ra = off[a];
      const int64_t j = ra + (k - odp[a]);
      const int32_t b = oadj[j];
      const int32_t da = deg[a], db = deg[b];
      // LSH mode: approximated edges are written by the estimate pass
      if (lsh_T >= 0 && da > lsh_T && db > lsh_T) continue;
      int64_t t = tcnt[j];
      if (tc16) t += (tc16[j >> 1] >> ((j & 1) << 4)) & 0xffffu;
      const double sv = sim_of(kind, t + 2, da, db);
      sim_csr[ra + opos[j]] = sv;
      const int32_t tr = twin_rel[j];
      if (tr < 0) bad = 1;
      else sim_csr[off[b] + tr] = sv;
    }
    __syncthreads();
  }
  if (bad) atomicOr(status, (unsigned)DEV_BADGRAPH);
}

// Out-lists in degree order. Each out(u) = oadj[off[u] .. off[u] + od[u])
// is re-ordered by the rank (d_x, x) ascending, with opos alongside; okey
// (compact: out-arc e of u at odp[u] + i) keeps the sorted rank keys, stored
// as ~(d_x << 32 | x) so that the descending segmented sort yields the
// ascending rank order. Then, for an in-neighbour u of a middle vertex v, the
// possible third vertices w > v of out(u) are exactly the entries after v:
// the streams read sum over u of d+(u)(d+(u)-1)/2 elements, half of
// sum d+(u)^2, and v's own position (its twin) comes from a binary search
// instead of a compare on every streamed element.

__global__ void __launch_bounds__(EXPAND_T)
k_rank_keys(const int64_t* __restrict__ off, const int32_t* __restrict__ deg,
            const int64_t* __restrict__ odp, const int32_t* __restrict__ oadj,
            const int32_t* __restrict__ opos, int64_t n, uint64_t* __restrict__ okey,
            int32_t* __restrict__ oval) {
  walk_out_arcs(off, odp, n, [&](int64_t k, int64_t, int64_t j) {
    const int32_t x = oadj[j];
    okey[k] = rank_key(deg[x], x);
    oval[k] = opos[j];
  });
}

__global__ void __launch_bounds__(EXPAND_T)
k_rank_scatter(const int64_t* __restrict__ off, const int64_t* __restrict__ odp, int64_t n,
               const uint64_t* __restrict__ okey, const int32_t* __restrict__ oval,
               int32_t* __restrict__ oadj, int32_t* __restrict__ opos) {
  walk_out_arcs(off, odp, n, [&](int64_t k, int64_t, int64_t j) {
    oadj[j] = (int32_t)(uint32_t)~okey[k];
    opos[j] = oval[k];
  });
}

// Count mode (a rank's share of a sharded count): the triangle count of every
// oriented edge, written to both of its arcs in CSR order; the second arc is
// found by a binary search of the tail in the head's id-sorted row.
__global__ void __launch_bounds__(EXPAND_T)
k_counts_out(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
             const int64_t* __restrict__ odp, const int32_t* __restrict__ oadj,
             const int32_t* __restrict__ opos, const uint32_t* __restrict__ tcnt,
             const uint32_t* __restrict__ tc16, int64_t n, uint32_t* __restrict__ out) {
  walk_out_arcs(off, odp, n, [&](int64_t, int64_t a, int64_t j) {
    const int32_t b = oadj[j];
    uint32_t t = tcnt[j];
    if (tc16) t += (tc16[j >> 1] >> ((j & 1) << 4)) & 0xffffu;
    out[off[a] + opos[j]] = t;
    int64_t lo = off[b], hi = off[b + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (adj[mid] < a) lo = mid + 1;
      else hi = mid;
    }
    if (lo < off[b + 1] && adj[lo] == (int32_t)a) out[lo] = t;
  });
}

// Weighted mode: ow[j] = weight of out-arc j (read at its row position);
// a weight that is negative or not finite marks the build DEV_BADWEIGHT.
__global__ void __launch_bounds__(EXPAND_T)
k_out_weights(const int64_t* __restrict__ off, const int64_t* __restrict__ odp, int64_t n,
              const int32_t* __restrict__ opos, const double* __restrict__ wcsr,
              double* __restrict__ ow, unsigned* status) {
  bool bad = false;
  walk_out_arcs(off, odp, n, [&](int64_t, int64_t a, int64_t j) {
    const double w = wcsr[off[a] + opos[j]];
    // integer tests (off the FP64 pipe): negative non-zero, or inf / NaN
    const long long bits = __double_as_longlong(w);
    if ((bits < 0 && bits != (long long)0x8000000000000000ull) || ((bits >> 52) & 0x7ff) == 0x7ff)
      bad = true;
    ow[j] = w;
  });
  if (bad) atomicOr(status, (unsigned)DEV_BADWEIGHT);
}

// norm[x] = sqrt(1 + sum of w(x,y)^2 over N(x)): the closed neighbourhood
// with w(x,x) = 1 (Section 4.1.1). FP64 instructions are issued for a whole
// warp at a time, so rows of at most 32 entries are summed by one thread each
// (32 vertices per instruction); longer rows by the whole warp.
__global__ void k_wnorm(const int64_t* __restrict__ off, const double* __restrict__ wcsr, int64_t n,
                        double* __restrict__ norm) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < n;
       base += stride) {
    const int64_t x = base + lane;
    int64_t b = 0, e = 0;
    if (x < n) {
      b = off[x];
      e = off[x + 1];
    }
    const bool long_row = e - b > 32;
    if (x < n && !long_row) {
      double s2 = 0.0;
      for (int64_t i = b; i < e; ++i) s2 += wcsr[i] * wcsr[i];
      norm[x] = sqrt(1.0 + s2);
    }
    unsigned lm = __ballot_sync(FULL, long_row);
    while (lm) {
      const int src = __ffs(lm) - 1;
      lm &= lm - 1;
      const int64_t bb = __shfl_sync(FULL, b, src), ee = __shfl_sync(FULL, e, src);
      double s2 = 0.0;
      for (int64_t i = bb + lane; i < ee; i += 32) s2 += wcsr[i] * wcsr[i];
      for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(FULL, s2, o);
      if (lane == 0) norm[base + src] = sqrt(1.0 + s2);
    }
  }
}

// Weighted cosine of every oriented edge a->b, written to both CSR arcs:
// (2 w(a,b) + triangle terms) / (norm[a] norm[b]) (Section 4.1.1); the weights
// of the two arcs must agree (else DEV_BADWEIGHT).
__global__ void __launch_bounds__(EXPAND_T)
k_expand_w(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
           const int64_t* __restrict__ odp, const int32_t* __restrict__ oadj,
           const int32_t* __restrict__ opos,
           const double* __restrict__ ow, const double* __restrict__ tsum,
           const int32_t* __restrict__ twin_rel, const double* __restrict__ wcsr,
           const double* __restrict__ norm, const int32_t* __restrict__ deg, int64_t n,
           int lsh_T, double* __restrict__ sim_csr, unsigned* status) {
  __shared__ int64_t s_bracket[2];
  const int64_t m = odp[n];
  constexpr int64_t CH = (int64_t)EXPAND_T * EXPAND_ITEMS;
  unsigned bad = 0;
  for (int64_t k0 = (int64_t)blockIdx.x * CH; k0 < m; k0 += (int64_t)gridDim.x * CH) {
    const int64_t k1 = min(m, k0 + CH);
    if (threadIdx.x == 0) s_bracket[0] = row_of(odp, 0, n + 1, k0);
    if (threadIdx.x == 1) s_bracket[1] = row_of(odp, 0, n + 1, k1 - 1) + 1;
    __syncthreads();
    const int64_t lo = s_bracket[0], hi = s_bracket[1];
    for (int64_t k = k0 + threadIdx.x; k < k1; k += EXPAND_T) {
      const int64_t a = row_of(odp, lo, hi, k);
      const int64_t ra = off[a];
      const int64_t j = ra + (k - odp[a]);
      const int32_t b = oadj[j];
      const double w = ow[j];
      if (lsh_T >= 0 && deg[a] > lsh_T && deg[b] > lsh_T) {
        // LSH mode: the estimate pass writes the similarity of an
        // approximated edge, and the counting kernels skipped its twin: find
        // a in N(b) to check the weights
        int64_t lo2 = off[b], hi2 = off[b + 1];
        while (lo2 < hi2) {
          const int64_t mid = (lo2 + hi2) >> 1;
          if (adj[mid] < a) lo2 = mid + 1;
          else hi2 = mid;
        }
        if (lo2 == off[b + 1] || adj[lo2] != a) bad |= DEV_BADGRAPH;
        else if (wcsr[lo2] != w) bad |= DEV_BADWEIGHT;
        continue;
      }
      const double sv = __ddiv_rn(__dadd_rn(2.0 * w, tsum[j]), __dmul_rn(norm[a], norm[b]));
      sim_csr[ra + opos[j]] = sv;
      const int32_t tr = twin_rel[j];
      if (tr < 0) {
        bad |= DEV_BADGRAPH;
      } else {
        if (wcsr[off[b] + tr] != w) bad |= DEV_BADWEIGHT;
        sim_csr[off[b] + tr] = sv;
      }
    }
    __syncthreads();
  }
  if (bad) atomicOr(status, bad);
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

}  // namespace

// The three counting kernels; IT indexes elements of the CSR (32-bit when the
// graph has fewer than 2^31 arcs, which halves the index arithmetic); WT
// accumulates weighted-cosine numerators (ow, tsum) instead of counts; R is
// the number of 32-element rounds of loads in flight for the concatenated
// short suffixes (a tuning parameter: 4 or 8).
template <typename IT, bool WT, int R>
int launch_counting(const int64_t* off, const int32_t* adj, const int32_t* deg, const int32_t* odeg,
                    const int32_t* oadj, const int32_t* opos, const uint64_t* okey,
                    const int64_t* odp, int64_t n,
                    const int64_t* item_off, const int32_t* order,
                    unsigned long long* work, int lsh_T, int32_t max_od, int64_t* deferred,
                    unsigned long long* n_deferred, uint32_t* tcnt, uint32_t* tc16, int32_t* twin,
                    unsigned* status, const double* ow, double* tsum, const CountCfg& cfg,
                    cudaStream_t s, cudaEvent_t k0, cudaEvent_t k1, int64_t small_end) {
  int od_cap = 16;
  while (od_cap < max_od && od_cap < SMEM_OD_MAX) od_cap <<= 1;
  // the table (12 bytes per slot, 2 * od_cap slots) and the counters (4 bytes)
  const size_t per_od = WT ? 24 : 28;  // weighted mode: no counters
  const size_t smem = per_od * od_cap;
  const size_t smem_max = per_od * SMEM_OD_MAX;
  GS_CUDA(cudaFuncSetAttribute(k_triangles<false, IT, WT, R>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
  const int sms = sm_count();
  int per_sm = 1;
  GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_triangles<false, IT, WT, R>,
                                                        TRI_THREADS, smem));
  if (per_sm < 1) per_sm = 1;
  if (k0) GS_CUDA(cudaEventRecord(k0, s));
  k_triangles<false, IT, WT, R><<<sms * per_sm, TRI_THREADS, smem, s>>>(
      off, adj, deg, odeg, oadj, opos, okey, odp, n, item_off, order, work, lsh_T, cfg.cta_chunk,
      cfg.long_list, od_cap, deferred, n_deferred, false, tcnt, tc16, twin, status, ow, tsum);
  GS_LAUNCH();
  if (k1) GS_CUDA(cudaEventRecord(k1, s));
  int small_per_sm = 1;
  GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&small_per_sm, k_tri_small<IT, WT, R>,
                                                        SW_WARPS * 32, 0));
  if (small_per_sm < 1) small_per_sm = 1;
  // the warp kernel takes its vertices from work[2] (set to the range's
  // first vertex) up to small_end
  k_tri_small<IT, WT, R><<<sms * small_per_sm, SW_WARPS * 32, 0, s>>>(
      off, adj, deg, odeg, oadj, opos, okey, odp, small_end, work + 2, lsh_T, cfg.warp_deg, cfg.long_list,
      tcnt,
      tc16, twin, status, ow, tsum);
  GS_LAUNCH();
  // items with out-lists too long for the shared table, and items deferred
  // by the CTA kernel (normally none: the launch then ends at once)
  const bool deferred_only = max_od <= SMEM_OD_MAX;
  k_triangles<true, IT, WT, R><<<deferred_only ? sms : sms * 4, TRI_THREADS, 0, s>>>(
      off, adj, deg, odeg, oadj, opos, okey, odp, n, item_off, order, work + 1, lsh_T, cfg.cta_chunk,
      cfg.long_list, 0, deferred, n_deferred, deferred_only, tcnt, tc16, twin, status, ow, tsum);
  GS_LAUNCH();
  return SCAN_OK;
}

// One set of counting kernels for the configuration: rounds 8 is compiled for
// the unweighted instances only.
template <typename IT, bool WT>
int launch_counting_cfg(const int64_t* off, const int32_t* adj, const int32_t* deg,
                        const int32_t* odeg, const int32_t* oadj, const int32_t* opos,
                        const uint64_t* okey,
                        const int64_t* odp, int64_t n, const int64_t* item_off,
                        const int32_t* order, unsigned long long* work, int lsh_T, int32_t max_od,
                        int64_t* deferred, unsigned long long* n_deferred, uint32_t* tcnt,
                        uint32_t* tc16, int32_t* twin, unsigned* status, const double* ow,
                        double* tsum, const CountCfg& cfg, cudaStream_t s, cudaEvent_t k0,
                        cudaEvent_t k1, int64_t small_end) {
  if (!WT && cfg.rounds == 8)
    return launch_counting<IT, WT, 8>(off, adj, deg, odeg, oadj, opos, okey, odp, n, item_off, order,
                                      work, lsh_T, max_od, deferred, n_deferred, tcnt, tc16, twin,
                                      status, ow, tsum, cfg, s, k0, k1, small_end);
  return launch_counting<IT, WT, 4>(off, adj, deg, odeg, oadj, opos, okey, odp, n, item_off, order,
                                    work, lsh_T, max_od, deferred, n_deferred, tcnt, tc16, twin,
                                    status, ow, tsum, cfg, s, k0, k1, small_end);
}

int launch_closed_counts_and_sims(int kind, const int64_t* off, const int32_t* adj,
                                  const int32_t* deg, int64_t n, int64_t arcs, const int32_t* odeg,
                                  int32_t* oadj, int32_t* opos, int32_t maxdeg,
                                  int32_t max_od, int lsh_T, const double* wcsr, double* sim_csr,
                                  unsigned* status, Pool& pool, cudaStream_t s, float* count_ms,
                                  const CountCfg& cfg, int64_t v0, int64_t v1,
                                  uint32_t* counts_out) {
  if (v1 < 0) v1 = n;
  const bool weighted = wcsr != nullptr;
  const int64_t m = arcs;  // out-lists live in CSR slots: counts and twins are indexed by arc
  const int64_t edges = m / 2;  // oriented edges (the orientation checked sum od = arcs / 2)
  int64_t* odp = pool.get<int64_t>(n + 1);
  uint64_t* okey = pool.get<uint64_t>(edges > 0 ? edges : 1);
  int32_t* oval = pool.get<int32_t>(edges > 0 ? edges : 1);
  if (!odp || !okey || !oval) return SCAN_ENOMEM;
  double* ow = weighted ? pool.get<double>(m) : nullptr;     // weight of every out-arc
  double* tsum = weighted ? pool.get<double>(m) : nullptr;   // numerator sums per out-arc
  double* norm = weighted ? pool.get<double>(n > 0 ? n : 1) : nullptr;
  if (weighted && (!ow || !tsum || !norm)) return SCAN_ENOMEM;
  if (weighted) GS_CUDA(cudaMemsetAsync(tsum, 0, m * sizeof(double), s));
  const int64_t nbins = (int64_t)maxdeg + 1;
  uint32_t* tcnt = pool.get<uint32_t>(m);
  // 16-bit (u,w) counters, two per word, when positions fit in 32 bits
  const bool narrow = m < ((int64_t)1 << 31) - 1 && !force_wide_index();
  uint32_t* tc16 = narrow ? pool.get<uint32_t>(m / 2 + 1) : nullptr;
  int32_t* twin = pool.get<int32_t>(m);
  int32_t* items = pool.get<int32_t>(n);
  int32_t* items_sorted = pool.get<int32_t>(n);
  int32_t* order = pool.get<int32_t>(n);
  int64_t* item_off = pool.get<int64_t>(n + 1);
  unsigned long long* hist = pool.get<unsigned long long>(2 * nbins);  // counts | fill cursors
  int64_t* start = pool.get<int64_t>(nbins + 1);
  unsigned long long* work = pool.get<unsigned long long>(4);  // 3 counters + deferred count
  // items: at most one per vertex plus one per cta_chunk arcs
  int64_t* deferred = pool.get<int64_t>(n + m / cfg.cta_chunk + 1);
  if (!tcnt || (narrow && !tc16) || !twin || !items || !items_sorted || !order || !item_off ||
      !hist || !start ||
      !work || !deferred)
    return SCAN_ENOMEM;
  GS_CUDA(cudaMemsetAsync(tcnt, 0, m * sizeof(uint32_t), s));
  if (narrow) GS_CUDA(cudaMemsetAsync(tc16, 0, (m / 2 + 1) * sizeof(uint32_t), s));
  GS_CUDA(cudaMemsetAsync(work, 0, 4 * sizeof(unsigned long long), s));
  if (v0 > 0) {  // the warp kernel's first vertex
    const unsigned long long first = (unsigned long long)v0;
    GS_CUDA(cudaMemcpyAsync(work + 2, &first, sizeof(first), cudaMemcpyHostToDevice, s));
    GS_CUDA(cudaStreamSynchronize(s));  // `first` lives on this stack frame
  }
  GS_CUDA(cudaMemsetAsync(hist, 0, 2 * nbins * sizeof(unsigned long long), s));
  if (m > 0) {
    k_fill_i32<<<1024, 256, 0, s>>>(twin, m, -1);
    GS_LAUNCH();
  }
  if (n > 0) {
    const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, sm_count() * 64);
    k_item_counts<<<g, 256, 0, s>>>(odeg, deg, n, cfg.warp_deg, cfg.cta_chunk, v0, v1, items);
    GS_LAUNCH();
    k_item_hist<<<g, 256, 0, s>>>(items, deg, n, maxdeg, hist);
    GS_LAUNCH();
    GS_TRY(exclusive_scan_i64(reinterpret_cast<const int64_t*>(hist), start, nbins, pool, s));
    k_item_place<<<g, 256, 0, s>>>(items, deg, n, maxdeg, start, hist + nbins, order);
    GS_LAUNCH();
    k_item_gather<<<g, 256, 0, s>>>(items, order, start, maxdeg, n, items_sorted);
    GS_LAUNCH();
  }
  GS_TRY(exclusive_scan_i32_to_i64(items_sorted, item_off, n, pool, s));
  cudaEvent_t e0, e1, k0 = nullptr, k1 = nullptr;
  GS_CUDA(cudaEventCreate(&e0));
  GS_CUDA(cudaEventCreate(&e1));
  if (count_ms) {  // the CTA counting kernel alone, for its roofline
    GS_CUDA(cudaEventCreate(&k0));
    GS_CUDA(cudaEventCreate(&k1));
  }
  GS_CUDA(cudaEventRecord(e0, s));
  // the rank and weight passes walk 32 rows per warp (EXPAND_T / 32 warps a
  // CTA); the similarity pass takes EXPAND_T * EXPAND_ITEMS edges per CTA
  const unsigned wgrid =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + EXPAND_T - 1) / EXPAND_T,
                                                       sm_count() * 32));
  const int64_t ch = (int64_t)EXPAND_T * EXPAND_ITEMS;
  const unsigned egrid =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>((edges + ch - 1) / ch, sm_count() * 32));
  if (n > 0 && m > 0) {
    // out-lists in ascending degree order, with their rank keys kept for the
    // searches of the counting kernels
    GS_TRY(exclusive_scan_i32_to_i64(odeg, odp, n, pool, s));
    k_rank_keys<<<wgrid, EXPAND_T, 0, s>>>(off, deg, odp, oadj, opos, n, okey, oval);
    GS_LAUNCH();
    GS_TRY(segmented_sort_desc(okey, oval, odp, n, edges, max_od, pool, s));
    k_rank_scatter<<<wgrid, EXPAND_T, 0, s>>>(off, odp, n, okey, oval, oadj, opos);
    GS_LAUNCH();
    if (weighted) {
      k_out_weights<<<wgrid, EXPAND_T, 0, s>>>(off, odp, n, opos, wcsr, ow, status);
      GS_LAUNCH();
      if (narrow) {
        GS_TRY((launch_counting_cfg<int32_t, true>(off, adj, deg, odeg, oadj, opos, okey, odp, n, item_off,
                                               order, work, lsh_T, max_od, deferred, work + 3,
                                               tcnt, tc16, twin, status, ow, tsum, cfg, s, k0, k1, v1)));
      } else {
        GS_TRY((launch_counting_cfg<int64_t, true>(off, adj, deg, odeg, oadj, opos, okey, odp, n, item_off,
                                               order, work, lsh_T, max_od, deferred, work + 3,
                                               tcnt, nullptr, twin, status, ow, tsum, cfg, s, k0, k1, v1)));
      }
    } else if (narrow) {
      GS_TRY((launch_counting_cfg<int32_t, false>(off, adj, deg, odeg, oadj, opos, okey, odp, n, item_off,
                                              order, work, lsh_T, max_od, deferred, work + 3, tcnt,
                                              tc16, twin, status, nullptr, nullptr, cfg, s, k0, k1, v1)));
    } else {
      GS_TRY((launch_counting_cfg<int64_t, false>(off, adj, deg, odeg, oadj, opos, okey, odp, n, item_off,
                                              order, work, lsh_T, max_od, deferred, work + 3, tcnt,
                                              nullptr, twin, status, nullptr, nullptr, cfg, s, k0, k1, v1)));
    }
  }
  GS_CUDA(cudaEventRecord(e1, s));
  if (n > 0 && m > 0 && counts_out) {
    k_counts_out<<<wgrid, EXPAND_T, 0, s>>>(off, adj, odp, oadj, opos, tcnt, tc16, n, counts_out);
    GS_LAUNCH();
  } else if (n > 0 && m > 0) {
    if (weighted) {
      k_wnorm<<<(unsigned)std::min<int64_t>((n + 255) / 256, sm_count() * 16), 256, 0, s>>>(off, wcsr, n,
                                                                                      norm);
      GS_LAUNCH();
      k_expand_w<<<egrid, EXPAND_T, 0, s>>>(off, adj, odp, oadj, opos, ow, tsum, twin, wcsr, norm,
                                            deg, n, lsh_T, sim_csr, status);
    } else {
      k_expand<<<egrid, EXPAND_T, 0, s>>>(kind, off, deg, odp, oadj, opos, tcnt, tc16, twin, n,
                                          lsh_T, sim_csr, status);
    }
    GS_LAUNCH();
  }
  if (count_ms) {
    GS_CUDA(cudaEventSynchronize(e1));
    GS_CUDA(cudaEventElapsedTime(count_ms, e0, e1));
    float kms = 0;
    if (n > 0 && m > 0 && cudaEventElapsedTime(&kms, k0, k1) == cudaSuccess)
      record_kernel_ms(kms);
    else
      record_kernel_ms(0);
    cudaGetLastError();
    cudaEventDestroy(k0);
    cudaEventDestroy(k1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pool.put(tcnt);
  if (tc16) pool.put(tc16);
  pool.put(twin);
  pool.put(deferred);
  pool.put(items);
  pool.put(items_sorted);
  pool.put(order);
  pool.put(hist);
  pool.put(start);
  pool.put(item_off);
  pool.put(work);
  pool.put(odp);
  pool.put(okey);
  pool.put(oval);
  if (ow) pool.put(ow);
  if (tsum) pool.put(tsum);
  if (norm) pool.put(norm);
  return SCAN_OK;
}

}  // namespace gscan
