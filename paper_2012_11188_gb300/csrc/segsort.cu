// Segmented sort of (key, val) pairs: key descending, then val ascending.
//
// Used for the neighbour order (each CSR row sorted by similarity, Algorithm
// 2 MakeNeighborOrder) and the core order (each CO[mu] sorted by threshold,
// Algorithm 2 MakeCoreOrder). Keys are the bit patterns of non-negative IEEE
// doubles, which order like the doubles. Within a segment the vals (vertex
// ids) are distinct, so (key, val) is a strict total order and the result
// does not depend on stability: equal similarities come out in ascending id,
// the tie rule of the paper's deterministic experiments.
//
// Segments are classed by length: <= 32 (one warp, one element per lane,
// bitonic network across lanes), <= 256, 512, 1024, 2048 and 4096 (one CTA
// of 32 to 512 threads: 8-element register sorts, then merge-path levels in
// shared memory), longer (split into buckets by sample sort, below; past
// three levels of splitting, 8192-element tiles sorted by one CTA the same
// way, then merge-path passes over global memory that double the run length,
// ping-ponging between the data and a scratch buffer).
#include "scan_internal.cuh"

namespace gscan {

namespace {

constexpr int WTILE = 256;   // rows up to this length are sorted by a one-warp CTA
constexpr int TILE = 8192;   // tiles of long segments (one CTA of 1024 threads each)
constexpr int NCLASS = 7;    // <=32, <=256, <=512, <=1024, <=2048, <=4096, >4096
constexpr int LONGC = NCLASS - 1;  // the long class

// Segments as begin/end arrays: segment i is [b[i], e[i]). A contiguous
// segmentation by offsets is {off, off + 1}; the buckets of long segments
// are listed on their own, without the short segments between them.
struct Segs {
  const int64_t* b;
  const int64_t* e;
};

// true iff a must come before b
__device__ __forceinline__ bool before(uint64_t ka, int32_t va, uint64_t kb, int32_t vb) {
  return ka > kb || (ka == kb && va < vb);
}

// before() on elements i and j of one (key, val) array pair, the vals read
// only when the keys tie: the searches are bound by shared-memory wavefronts,
// and most probes are decided by the keys alone
__device__ __forceinline__ bool before_at(const uint64_t* k, const int32_t* v, int64_t i,
                                          int64_t j) {
  const uint64_t ki = k[i], kj = k[j];
  if (ki != kj) return ki > kj;
  return v[i] < v[j];
}

constexpr int32_t SENT_V = 0x7fffffff;  // sorts after every real element (key 0, val max)

// The tile classes double in length and in CTA size (32 to 512 threads at 8
// elements each), so that a segment keeps at least half of its CTA busy.
__device__ __forceinline__ int seg_class(int64_t len) {
  return len <= 32 ? 0 : len <= WTILE ? 1 : len <= 512 ? 2 : len <= 1024 ? 3 : len <= 2048 ? 4
       : len <= 4096 ? 5 : LONGC;
}

// Count segments per class and number of tiles of long segments.
// counts[]: per class, tiles of the long class, the longest long segment,
// and a flag for offsets that are not non-decreasing within [0, total]
constexpr int NCNT = NCLASS + 3;

__global__ void k_classify_count(Segs S, int64_t nseg, int64_t total,
                                 unsigned long long* counts) {
  __shared__ unsigned long long c[NCLASS + 2];
  if (threadIdx.x < NCLASS + 2) c[threadIdx.x] = 0;
  __syncthreads();
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nseg;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = S.b[i], e = S.e[i];
    if (b < 0 || e < b || e > total) {
      bad = true;
      continue;
    }
    const int64_t len = e - b;
    if (len <= 1) continue;
    const int cl = seg_class(len);
    atomicAdd(&c[cl], 1ull);
    if (cl == LONGC) {
      atomicAdd(&c[NCLASS], (unsigned long long)((len + TILE - 1) / TILE));
      atomicMax(&c[NCLASS + 1], (unsigned long long)len);
    }
  }
  __syncthreads();
  if (threadIdx.x < NCLASS + 1 && c[threadIdx.x]) atomicAdd(&counts[threadIdx.x], c[threadIdx.x]);
  if (threadIdx.x == NCLASS + 1 && c[threadIdx.x]) atomicMax(&counts[threadIdx.x], c[threadIdx.x]);
  if (bad) atomicOr(&counts[NCLASS + 2], 1ull);
}

// Fill per-class segment lists (order irrelevant). The lanes of a warp that
// share a class take consecutive slots with one atomic.
__global__ void k_classify_fill(Segs S, int64_t nseg,
                                const int64_t* __restrict__ class_base,
                                unsigned long long* __restrict__ fill, int64_t* __restrict__ list) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < nseg;
       i0 += stride) {
    const int64_t i = i0 + lane;
    const int64_t len = i < nseg ? S.e[i] - S.b[i] : 0;
    const int cl = len <= 1 ? -1 : seg_class(len);
    const unsigned peers = __match_any_sync(0xffffffffu, cl);
    const int leader = __ffs(peers) - 1;
    unsigned long long pos = 0;
    if (cl >= 0 && lane == leader) pos = atomicAdd(&fill[cl], (unsigned long long)__popc(peers));
    pos = __shfl_sync(0xffffffffu, pos, leader);
    if (cl >= 0)
      list[class_base[cl] + (int64_t)pos + __popc(peers & ((1u << lane) - 1u))] = i;
  }
}

// <= 32 elements: one warp per segment, bitonic network across lanes; read
// from (ik, iv), written to (key, val) (the same arrays, or a copy).
__global__ void k_sort_warp(const uint64_t* ik, const int32_t* iv, uint64_t* key, int32_t* val,
                            Segs S, const int64_t* __restrict__ list,
                            const unsigned long long* __restrict__ count_ptr) {
  const int lane = threadIdx.x & 31;
  const int64_t cnt = (int64_t)*count_ptr;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = w0; w < cnt; w += nw) {
    const int64_t sg = list[w];
    const int64_t b = S.b[sg];
    const int len = (int)(S.e[sg] - b);
    uint64_t k = 0;
    int32_t v = SENT_V;
    if (lane < len) { k = ik[b + lane]; v = iv[b + lane]; }
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        const uint64_t ok = __shfl_xor_sync(0xffffffffu, k, stride);
        const int32_t ov = __shfl_xor_sync(0xffffffffu, v, stride);
        const bool lower_lane = (lane & stride) == 0;
        const bool ascending = (lane & size) == 0;  // "ascending" in the before() order
        // the lower lane of a pair keeps the element that comes first
        const bool other_first = before(ok, ov, k, v);
        const bool take = (lower_lane == ascending) ? other_first : !other_first;
        if (take) { k = ok; v = ov; }
      }
    }
    if (lane < len) { key[b + lane] = k; val[b + lane] = v; }
  }
}

// Passes a segment of length len takes part in: one per run length L = TILE,
// 2*TILE, ... below len.
__device__ __forceinline__ int passes_for(int64_t len) {
  int p = 0;
  for (int64_t L = TILE; L < len; L <<= 1) ++p;
  return p;
}

// Shared-memory slot of tile element i with one pad slot per R elements, so
// that a warp whose lanes hold R consecutive elements each (lane l: R*l ..
// R*l+R-1) touches distinct banks when it stores or loads them.
template <int R>
__device__ __forceinline__ int pslot(int i) { return i + i / R; }

// Merge path over padded shared runs: elements of A = [a0, a0+la) among the
// first d outputs of merge(A, B), B = [b0, b0+lb).
template <int R>
__device__ __forceinline__ int smem_merge_path_p(const uint64_t* k, const int32_t* v, int a0,
                                                 int la, int b0, int lb, int d) {
  int lo = max(0, d - lb), hi = min(d, la);
  while (lo < hi) {
    const int i = (lo + hi) >> 1;
    if (before_at(k, v, pslot<R>(b0 + d - 1 - i), pslot<R>(a0 + i))) hi = i;
    else lo = i + 1;
  }
  return lo;
}

// Compare-and-swap of a register pair: afterwards (ka, va) comes first.
__device__ __forceinline__ void cas(uint64_t& ka, int32_t& va, uint64_t& kb, int32_t& vb) {
  if (before(kb, vb, ka, va)) {
    const uint64_t tk = ka; ka = kb; kb = tk;
    const int32_t tv = va; va = vb; vb = tv;
  }
}

// Sorts 8 or 16 register elements with Batcher's odd-even merge network
// (19 or 63 compare-and-swaps).
#define GS_CAS(i, j) cas(K[i], V[i], K[j], V[j])
__device__ __forceinline__ void sort_regs(uint64_t (&K)[8], int32_t (&V)[8]) {
  GS_CAS(0, 1); GS_CAS(2, 3); GS_CAS(4, 5); GS_CAS(6, 7);
  GS_CAS(0, 2); GS_CAS(1, 3); GS_CAS(4, 6); GS_CAS(5, 7);
  GS_CAS(1, 2); GS_CAS(5, 6);
  GS_CAS(0, 4); GS_CAS(1, 5); GS_CAS(2, 6); GS_CAS(3, 7);
  GS_CAS(2, 4); GS_CAS(3, 5);
  GS_CAS(1, 2); GS_CAS(3, 4); GS_CAS(5, 6);
}
__device__ __forceinline__ void sort_regs(uint64_t (&K)[16], int32_t (&V)[16]) {
  // the two halves, then the odd-even merge of the halves
  GS_CAS(0, 1); GS_CAS(2, 3); GS_CAS(0, 2); GS_CAS(1, 3); GS_CAS(1, 2);
  GS_CAS(4, 5); GS_CAS(6, 7); GS_CAS(4, 6); GS_CAS(5, 7); GS_CAS(5, 6);
  GS_CAS(0, 4); GS_CAS(2, 6); GS_CAS(2, 4); GS_CAS(1, 5); GS_CAS(3, 7); GS_CAS(3, 5);
  GS_CAS(1, 2); GS_CAS(3, 4); GS_CAS(5, 6);
  GS_CAS(8, 9); GS_CAS(10, 11); GS_CAS(8, 10); GS_CAS(9, 11); GS_CAS(9, 10);
  GS_CAS(12, 13); GS_CAS(14, 15); GS_CAS(12, 14); GS_CAS(13, 15); GS_CAS(13, 14);
  GS_CAS(8, 12); GS_CAS(10, 14); GS_CAS(10, 12); GS_CAS(9, 13); GS_CAS(11, 15); GS_CAS(11, 13);
  GS_CAS(9, 10); GS_CAS(11, 12); GS_CAS(13, 14);
  GS_CAS(0, 8); GS_CAS(4, 12); GS_CAS(4, 8); GS_CAS(2, 10); GS_CAS(6, 14); GS_CAS(6, 10);
  GS_CAS(2, 4); GS_CAS(6, 8); GS_CAS(10, 12); GS_CAS(1, 9); GS_CAS(5, 13); GS_CAS(5, 9);
  GS_CAS(3, 11); GS_CAS(7, 15); GS_CAS(7, 11); GS_CAS(3, 5); GS_CAS(7, 9); GS_CAS(11, 13);
  GS_CAS(1, 2); GS_CAS(3, 4); GS_CAS(5, 6); GS_CAS(7, 8); GS_CAS(9, 10); GS_CAS(11, 12);
  GS_CAS(13, 14);
}
#undef GS_CAS

// Merges RI outputs starting at diagonal d of the runs A = src[a0, a0+la)
// and B = src[b0, b0+lb) (padded shared layout), writing dst slots o..o+RI-1.
// The current head of each run is kept in registers, so each output costs
// one dependent shared load.
template <int R, int RI>
__device__ __forceinline__ void merge_out(const uint64_t* ks, const int32_t* vs, int a0, int la,
                                          int b0, int lb, int d, uint64_t* kd, int32_t* vd, int o) {
  int ia = smem_merge_path_p<R>(ks, vs, a0, la, b0, lb, d);
  int ib = d - ia;
  uint64_t ka = 0, kb = 0;
  int32_t va = SENT_V, vb = SENT_V;
  if (ia < la) { const int p = pslot<R>(a0 + ia); ka = ks[p]; va = vs[p]; }
  if (ib < lb) { const int p = pslot<R>(b0 + ib); kb = ks[p]; vb = vs[p]; }
  // branch-free steps: every lane selects, advances and reloads the same way
#pragma unroll
  for (int q = 0; q < RI; ++q) {
    const bool take_a = ib >= lb || (ia < la && !before(kb, vb, ka, va));
    const int po = pslot<R>(o + q);
    kd[po] = take_a ? ka : kb;
    vd[po] = take_a ? va : vb;
    ia += take_a ? 1 : 0;
    ib += take_a ? 0 : 1;
    const int nxt = take_a ? a0 + ia : b0 + ib;
    const bool more = take_a ? ia < la : ib < lb;
    uint64_t kn = 0;
    int32_t vn = SENT_V;
    if (more) { const int p = pslot<R>(nxt); kn = ks[p]; vn = vs[p]; }
    ka = take_a ? kn : ka;
    va = take_a ? vn : va;
    kb = take_a ? kb : kn;
    vb = take_a ? vb : vn;
  }
}

// One CTA of TT threads sorts a tile of up to TT*RI elements (RI = 8 or 16):
// the tile is loaded into shared memory with coalesced reads (padded with
// sentinels that sort last up to a multiple of RI), each thread sorts RI
// consecutive elements in registers, then merge-path levels double the
// sorted runs (the last pair of a level may be short), each thread writing
// RI outputs per level. The tile is read from (ik, iv) and written to (key,
// val) (the same arrays, or a copy). Tiles are whole segments (TILED =
// false) or TILE-element pieces of longer segments (TILED = true, TT*RI =
// TILE, ik = key). A tiled segment that takes an odd number of merge passes
// has its tiles written to the scratch buffer (tk, tv), so that its last
// pass ends in (key, val).
template <int TT, int RI, bool TILED>
__global__ void __launch_bounds__(TT, TT * RI >= 8192 ? 1 : (TT >= 1024 ? 1 : 1024 / TT))
k_sort_tile(const uint64_t* ik, const int32_t* iv, uint64_t* key, int32_t* val, Segs S,
            const int64_t* __restrict__ list, const unsigned long long* __restrict__ count_ptr,
            const int64_t* __restrict__ tile_prefix, int64_t nlong, uint64_t* __restrict__ tk,
            int32_t* __restrict__ tv) {
  constexpr int CAP = TT * RI;
  constexpr int PCAP = CAP + CAP / RI;  // padded slots per buffer
  extern __shared__ uint64_t tsm[];
  uint64_t* k0 = tsm;
  uint64_t* k1 = tsm + PCAP;
  int32_t* v0 = (int32_t*)(tsm + 2 * PCAP);
  int32_t* v1 = v0 + PCAP;
  const int t = threadIdx.x;
  const int64_t cnt = (int64_t)*count_ptr;
  for (int64_t u = blockIdx.x; u < cnt; u += gridDim.x) {
    int64_t b, len;
    uint64_t* ok = key;
    int32_t* ov = val;
    if (!TILED) {
      const int64_t sg = list[u];
      b = S.b[sg];
      len = S.e[sg] - b;
    } else {
      int64_t lo = 0, hi = nlong;
      while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (tile_prefix[mid] <= u) lo = mid; else hi = mid;
      }
      const int64_t sg = list[lo];
      b = S.b[sg] + (u - tile_prefix[lo]) * CAP;
      len = min((int64_t)CAP, S.e[sg] - b);
      if (passes_for(S.e[sg] - S.b[sg]) & 1) { ok = tk; ov = tv; }
    }
    // the tile is worked up to len rounded up to RI (sentinels past len); the
    // merge levels clip their last run pair there, so the work follows len
    const int lr = len <= RI ? RI : (int)((len + RI - 1) / RI) * RI;
    // 1. coalesced load, sentinels past the end
    for (int i = t; i < lr; i += TT) {
      const int p = pslot<RI>(i);
      if (i < len) { k0[p] = ik[b + i]; v0[p] = iv[b + i]; }
      else { k0[p] = 0; v0[p] = SENT_V; }
    }
    __syncthreads();
    // 2. each thread sorts its RI consecutive elements in registers
    if (RI * t < lr) {
      uint64_t K[RI];
      int32_t V[RI];
#pragma unroll
      for (int r = 0; r < RI; ++r) { const int p = pslot<RI>(RI * t + r); K[r] = k0[p]; V[r] = v0[p]; }
      sort_regs(K, V);
#pragma unroll
      for (int r = 0; r < RI; ++r) { const int p = pslot<RI>(RI * t + r); k0[p] = K[r]; v0[p] = V[r]; }
    }
    __syncthreads();
    // 3. merge levels in shared memory: runs of w -> 2w, ping-pong k0/v0 <-> k1/v1
    uint64_t *ks = k0, *kd = k1;
    int32_t *vs = v0, *vd = v1;
    for (int w = RI; w < lr; w <<= 1) {
      const int o = RI * t;  // first output of this thread
      if (o < lr) {
        const int a0 = (o / (2 * w)) * (2 * w);
        const int la = min(w, lr - a0), lb = max(0, min(w, lr - a0 - w));
        merge_out<RI, RI>(ks, vs, a0, la, a0 + w, lb, o - a0, kd, vd, o);
      }
      __syncthreads();
      uint64_t* tk2 = ks; ks = kd; kd = tk2;
      int32_t* tv2 = vs; vs = vd; vd = tv2;
    }
    for (int i = t; i < len; i += TT) {
      const int pi = pslot<RI>(i);
      ok[b + i] = ks[pi];
      ov[b + i] = vs[pi];
    }
    __syncthreads();
  }
}

template <int TT, int RI>
constexpr size_t tile_smem_bytes() {
  return (size_t)(TT * RI + TT * RI / RI) * (2 * sizeof(uint64_t) + 2 * sizeof(int32_t));
}

#ifndef GS_SORT_LONG_RI
#define GS_SORT_LONG_RI 8  // elements per thread in the tiles of long segments (8 or 16)
#endif
// whole segments of 1025..4096 elements: 512 threads x 8; tiles of long
// segments: TILE elements, TILE / GS_SORT_LONG_RI threads (one CTA per SM)
constexpr int T4K_T = 512;
constexpr int TLONG_RI = GS_SORT_LONG_RI;
constexpr int TLONG_T = TILE / TLONG_RI;

// Tiles per long segment (prefix computed by the caller).
__global__ void k_long_tiles(Segs S, const int64_t* __restrict__ list,
                             const unsigned long long* __restrict__ count_ptr,
                             int64_t* __restrict__ tiles, int64_t* __restrict__ outchunks,
                             int chunk) {
  const int64_t cnt = (int64_t)*count_ptr;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sg = list[i];
    const int64_t len = S.e[sg] - S.b[sg];
    tiles[i] = (len + TILE - 1) / TILE;
    outchunks[i] = (len + chunk - 1) / chunk;
  }
}

#ifndef GS_MERGE_ITEMS
#define GS_MERGE_ITEMS 4  // outputs per thread of a merge pass
#endif
constexpr int MERGE_T = 256;
constexpr int MERGE_ITEMS = GS_MERGE_ITEMS;
constexpr int MERGE_CHUNK = MERGE_T * MERGE_ITEMS;  // output elements per CTA per pass
static_assert((2 * TILE) % MERGE_CHUNK == 0, "a chunk must not straddle two run pairs");
// shared memory of a merge pass: two input buffers and the padded output staging
constexpr size_t MERGE_SMEM = (size_t)2 * MERGE_CHUNK * 12 +
                              (size_t)(MERGE_CHUNK + MERGE_CHUNK / MERGE_ITEMS) * 12;

// Number of elements of A (length la) among the first d of merge(A, B).
__device__ __forceinline__ int64_t merge_path(const uint64_t* ka, const int32_t* va, int64_t la,
                                              const uint64_t* kb, const int32_t* vb, int64_t lb,
                                              int64_t d) {
  int64_t lo = max((int64_t)0, d - lb), hi = min(d, la);
  while (lo < hi) {
    const int64_t i = (lo + hi) >> 1;  // take i from A, d-i from B
    const uint64_t kbi = kb[d - 1 - i], kai = ka[i];
    if (kbi != kai ? kbi > kai : vb[d - 1 - i] < va[i]) hi = i;
    else lo = i + 1;
  }
  return lo;
}


__device__ __forceinline__ int64_t chunk_segment(const int64_t* chunk_prefix, int64_t nlong,
                                                 int64_t c) {
  int64_t lo = 0, hi = nlong;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (chunk_prefix[mid] <= c) lo = mid; else hi = mid;
  }
  return lo;
}

// Where one output chunk of a pass reads from and writes to: run A's part
// starts at element a0, run B's at b0, the chunk's outputs at out (absolute
// element indexes); na + nb outputs, 0 when the segment is already finished.
struct MergeDesc {
  int64_t a0, b0, out;
  int32_t na, nb;
  int32_t from_tmp;  // runs are read from the scratch buffer and written to (key, val)
};

// Merge-path splits of every output chunk of pass `pass` (run length L),
// all in parallel (one thread per chunk), written as chunk descriptors. A
// segment with P passes reads pass p from the scratch buffer when P - p is
// odd, so that its last pass writes (key, val).
__global__ void k_merge_partition(const uint64_t* __restrict__ key, const int32_t* __restrict__ val,
                                  const uint64_t* __restrict__ tk, const int32_t* __restrict__ tv,
                                  Segs S,
                                  const int64_t* __restrict__ list,
                                  const int64_t* __restrict__ chunk_prefix, int64_t nlong, int64_t L,
                                  int pass, MergeDesc* __restrict__ desc) {
  const int64_t total = chunk_prefix[nlong];
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t si = chunk_segment(chunk_prefix, nlong, c);
    const int64_t sg = list[si];
    const int64_t base = S.b[sg], len = S.e[sg] - base;
    MergeDesc d{0, 0, 0, 0, 0, 0};
    if (len > L) {
      d.from_tmp = (passes_for(len) - pass) & 1;
      const uint64_t* sk = d.from_tmp ? tk : key;
      const int32_t* sv = d.from_tmp ? tv : val;
      const int64_t o0 = (c - chunk_prefix[si]) * MERGE_CHUNK;
      const int64_t o1 = min(len, o0 + MERGE_CHUNK);
      // run pair containing [o0, o1): MERGE_CHUNK divides 2L
      const int64_t r0 = (o0 / (2 * L)) * (2 * L);
      const int64_t a1 = min(len, r0 + L), b1 = min(len, r0 + 2 * L);
      const uint64_t* KA = sk + base + r0;
      const int32_t* VA = sv + base + r0;
      const uint64_t* KB = sk + base + a1;
      const int32_t* VB = sv + base + a1;
      const int64_t i0 = merge_path(KA, VA, a1 - r0, KB, VB, b1 - a1, o0 - r0);
      const int64_t i1 = merge_path(KA, VA, a1 - r0, KB, VB, b1 - a1, o1 - r0);
      d.a0 = base + r0 + i0;
      d.b0 = base + a1 + (o0 - r0) - i0;
      d.out = base + o0;
      d.na = (int32_t)(i1 - i0);
      d.nb = (int32_t)((o1 - o0) - (i1 - i0));
    }
    desc[c] = d;
  }
}

// Asynchronous global -> shared copies (sm_80+ cp.async), so the next chunk's
// inputs are in flight while the current chunk is merged.
__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst_smem, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One merge pass: within every long segment still longer than L, runs of
// length L are merged in pairs from (sk, sv) into (dk, dv). Segments of length
// <= L are finished and stay where they are. Each CTA takes chunks of
// MERGE_CHUNK outputs; the inputs of its next chunk are copied into shared
// memory (cp.async) while it merges the current one, and outputs are staged
// in shared memory so the global stores are coalesced.
__global__ void __launch_bounds__(MERGE_T)
k_merge_pass(uint64_t* __restrict__ key, int32_t* __restrict__ val, uint64_t* __restrict__ tk,
             int32_t* __restrict__ tv, const int64_t* __restrict__ chunk_prefix, int64_t nlong,
             const MergeDesc* __restrict__ desc) {
  // two input buffers, then the output staging with one pad slot per
  // MERGE_ITEMS (a thread's consecutive outputs) so that the lanes of a warp
  // write distinct banks
  extern __shared__ uint64_t msm[];
  uint64_t (*ink)[MERGE_CHUNK] = reinterpret_cast<uint64_t (*)[MERGE_CHUNK]>(msm);
  uint64_t* ok_ = msm + 2 * MERGE_CHUNK;
  int32_t (*inv)[MERGE_CHUNK] =
      reinterpret_cast<int32_t (*)[MERGE_CHUNK]>(ok_ + MERGE_CHUNK + MERGE_CHUNK / MERGE_ITEMS);
  int32_t* ov_ = reinterpret_cast<int32_t*>(inv + 2);
  const int64_t total = chunk_prefix[nlong];
  const int t = threadIdx.x;
  auto po = [](int i) { return i + i / MERGE_ITEMS; };
  // issue the copies of chunk c into buffer b (an empty group when inactive)
  auto stage = [&](int64_t c, int b) -> MergeDesc {
    MergeDesc m{0, 0, 0, 0, 0, 0};
    if (c < total) m = desc[c];
    const uint64_t* sk = m.from_tmp ? tk : key;
    const int32_t* sv = m.from_tmp ? tv : val;
    for (int i = t; i < m.na; i += MERGE_T) {
      cp_async8(&ink[b][i], sk + m.a0 + i);
      cp_async4(&inv[b][i], sv + m.a0 + i);
    }
    for (int i = t; i < m.nb; i += MERGE_T) {
      cp_async8(&ink[b][m.na + i], sk + m.b0 + i);
      cp_async4(&inv[b][m.na + i], sv + m.b0 + i);
    }
    cp_async_commit();
    return m;
  };
  int64_t c = blockIdx.x;
  int b = 0;
  MergeDesc cur = stage(c, b);
  for (; c < total; c += gridDim.x) {
    const MergeDesc nxt = stage(c + gridDim.x, b ^ 1);
    cp_async_wait<1>();  // the current chunk's copies have landed
    __syncthreads();
    if (cur.na + cur.nb > 0) {
      const uint64_t* shk = ink[b];
      const int32_t* shv = inv[b];
      const int na = cur.na, nb = cur.nb, nout = na + nb;
      // each thread merges MERGE_ITEMS outputs from its own diagonal
      const int d = t * MERGE_ITEMS;
      if (d < nout) {
        int lo2 = max(0, d - nb), hi2 = min(d, na);
        while (lo2 < hi2) {
          const int i = (lo2 + hi2) >> 1;
          if (before_at(shk, shv, na + d - 1 - i, i)) hi2 = i;
          else lo2 = i + 1;
        }
        int ia = lo2, ib = d - lo2;
        // run heads in registers: one dependent shared load per output
        uint64_t ka = 0, kb = 0;
        int32_t va = SENT_V, vb = SENT_V;
        if (ia < na) { ka = shk[ia]; va = shv[ia]; }
        if (ib < nb) { kb = shk[na + ib]; vb = shv[na + ib]; }
#pragma unroll
        for (int q = 0; q < MERGE_ITEMS; ++q) {
          if (d + q >= nout) break;
          const bool take_a = ib >= nb || (ia < na && !before(kb, vb, ka, va));
          const int pq = po(d + q);
          ok_[pq] = take_a ? ka : kb;
          ov_[pq] = take_a ? va : vb;
          ia += take_a ? 1 : 0;
          ib += take_a ? 0 : 1;
          const int nxt = take_a ? ia : na + ib;
          const bool more = take_a ? ia < na : ib < nb;
          uint64_t kn = 0;
          int32_t vn = SENT_V;
          if (more) { kn = shk[nxt]; vn = shv[nxt]; }
          ka = take_a ? kn : ka;
          va = take_a ? vn : va;
          kb = take_a ? kb : kn;
          vb = take_a ? vb : vn;
        }
      }
      __syncthreads();
      const int64_t out = cur.out;
      uint64_t* dk = cur.from_tmp ? key : tk;
      int32_t* dv = cur.from_tmp ? val : tv;
      for (int i = t; i < nout; i += MERGE_T) {
        dk[out + i] = ok_[po(i)];
        dv[out + i] = ov_[po(i)];
      }
    }
    __syncthreads();  // buffer b and the staging area are free again
    cur = nxt;
    b ^= 1;
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------- buckets
// Long segments are split into buckets by sample sort before any tile is
// sorted: every long segment draws BKT_OS random samples per bucket (one per
// stratum of its positions, so each element is drawn with the same
// probability), the samples are sorted (the same segmented sort, one level
// down), and every BKT_OS-th sorted sample becomes a splitter. An element
// goes to the bucket numbered by the splitters that come strictly before it
// in the (key desc, val asc) order, so every element of bucket j comes
// before every element of bucket j + 1 and sorting the buckets sorts the
// segment. The buckets then take the place of their segment in one
// segmentation of the whole array, sorted one level down: by the short
// segment kernels, or, when still long, split again.
//
// A level splits a segment into at most BKT_FAN buckets, so that each
// 4096-element chunk, once sorted by bucket in shared memory, leaves for
// global memory in runs of about 4 or more elements per bucket (scattered
// single-element stores would be bound by L2 write transactions): a segment
// of up to BKT_FAN * BKT_TARGET elements gets buckets of about BKT_TARGET
// elements at once, a longer one buckets of BKT_TARGET * BKT_FAN^k first.
constexpr int BKT_TARGET = 896;   // expected final bucket length (swept on R-MAT s24: 448 to 2816)
constexpr int BKT_FAN = 1024;     // buckets per segment and level
constexpr int BKT_OS = 32;        // samples per bucket
constexpr int BKT_CH = 4096;      // elements of one segment per chunk (sorted by bucket as one)
constexpr int BKT_G = 8;          // chunks per group: a CTA's unit, one reservation per bucket
constexpr int BKT_T = 512;        // threads of the count and scatter CTAs
constexpr int BKT_E = BKT_CH / BKT_T;
constexpr int BKT_DEPTH = 3;      // levels of bucketing before the merge passes take over

__host__ __device__ __forceinline__ int64_t buckets_for(int64_t len) {
  int64_t unit = BKT_TARGET;
  while (unit * BKT_FAN < len) unit *= BKT_FAN;
  const int64_t b = (len + unit - 1) / unit;
  return b < 2 ? 2 : b;
}

// MurmurHash3's 64-bit finaliser (Appleby): sample positions within strata
__device__ __forceinline__ uint64_t fmix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdULL;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ULL;
  x ^= x >> 33;
  return x;
}

// Buckets, samples and count/scatter groups of every long segment.
__global__ void k_bucket_plan(Segs S, const int64_t* __restrict__ list,
                              int64_t nlong, int64_t* __restrict__ nb, int64_t* __restrict__ ns,
                              int64_t* __restrict__ nch) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nlong;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sg = list[x];
    const int64_t len = S.e[sg] - S.b[sg];
    const int64_t b = buckets_for(len);
    nb[x] = b;
    ns[x] = b * BKT_OS;
    nch[x] = (len + (int64_t)BKT_CH * BKT_G - 1) / ((int64_t)BKT_CH * BKT_G);  // groups
  }
}

// Sample j of long segment x: a random position of stratum j of its ns_x
// equal strata.
__global__ void k_take_samples(const uint64_t* __restrict__ key, const int32_t* __restrict__ val,
                               Segs S, const int64_t* __restrict__ list,
                               const int64_t* __restrict__ soff, int64_t nlong, int depth,
                               uint64_t* __restrict__ skey, int32_t* __restrict__ sval) {
  const int64_t nsamples = soff[nlong];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nsamples;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = chunk_segment(soff, nlong, i);
    const int64_t j = i - soff[x], nsx = soff[x + 1] - soff[x];
    const int64_t sg = list[x];
    const int64_t b = S.b[sg], len = S.e[sg] - b;
    const int64_t s0 = j * len / nsx, s1 = (j + 1) * len / nsx;
    const uint64_t h = fmix64(((uint64_t)x << 32) ^ (uint64_t)j ^ ((uint64_t)depth << 60));
    const int64_t p = s0 + (int64_t)(h % (uint64_t)(s1 - s0));
    skey[i] = key[b + p];
    sval[i] = val[b + p];
  }
}

// Exclusive block-wide scan of h[0 .. 2 * BKT_T) in place (two entries per
// thread).
__device__ __forceinline__ void block_exclusive_scan(unsigned* h, unsigned* wsum) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const unsigned h0 = h[2 * t], h1 = h[2 * t + 1];
  const unsigned own = h0 + h1;
  unsigned inc = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    const unsigned ws = lane < BKT_T / 32 ? wsum[lane] : 0u;
    unsigned wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < BKT_T / 32) wsum[lane] = wi - ws;
  }
  __syncthreads();
  const unsigned pre = inc - own + wsum[w];
  h[2 * t] = pre;
  h[2 * t + 1] = pre + h0;
}

// Bucket of every element of the long segments, written to bid, and the
// bucket sizes per group of BKT_G chunks (ghist) and per segment (one global
// atomic per bucket and group). The segment's splitters are held in shared
// memory as a complete binary search tree in breadth-first order (node i's
// children are 2i and 2i + 1; padded with entries that no element follows),
// so that every lane descends the same number of levels without branches.
__global__ void __launch_bounds__(BKT_T, 2)
k_bucket_count(const uint64_t* __restrict__ ck, const int32_t* __restrict__ cv, Segs S,
               const int64_t* __restrict__ list, int64_t nlong, const int64_t* __restrict__ soff,
               const int64_t* __restrict__ boff, const int64_t* __restrict__ gpre,
               const uint64_t* __restrict__ skey, const int32_t* __restrict__ sval,
               unsigned long long* __restrict__ bcount, unsigned* __restrict__ ghist,
               uint16_t* __restrict__ bid) {
  __shared__ uint64_t tkey[BKT_FAN];
  __shared__ int32_t tval[BKT_FAN];
  __shared__ unsigned hsum[BKT_FAN];
  constexpr int U = 8;  // elements per thread in flight
  const int t = threadIdx.x, lane = t & 31;
  const int64_t G = gpre[nlong];
  for (int64_t g = blockIdx.x; g < G; g += gridDim.x) {
    const int64_t x = chunk_segment(gpre, nlong, g);
    const int64_t sg = list[x];
    const int64_t b = S.b[sg], len = S.e[sg] - b;
    const int nbx = (int)(boff[x + 1] - boff[x]);
    const int nsp = nbx - 1;
    const int L = 32 - __clz(nsp);  // levels: 2^L - 1 >= nsp nodes
    const int64_t q0 = (g - gpre[x]) * BKT_CH * BKT_G;
    const int m = (int)(min(len, q0 + (int64_t)BKT_CH * BKT_G) - q0);
    for (int i = t + 1; i < (1 << L); i += BKT_T) {
      const int l = 31 - __clz(i), p = i - (1 << l);
      const int r = ((2 * p + 1) << (L - 1 - l)) - 1;  // in-order rank of node i
      if (r < nsp) {
        const int64_t q = soff[x] + (int64_t)(r + 1) * BKT_OS;
        tkey[i] = skey[q];
        tval[i] = sval[q];
      } else {
        tkey[i] = 0;  // sorts after every element
        tval[i] = SENT_V;
      }
    }
    for (int j = t; j < nbx; j += BKT_T) hsum[j] = 0;
    __syncthreads();
    const uint64_t* kc = ck + b + q0;
    const int32_t* vc = cv + b + q0;
    uint16_t* bc = bid + b + q0;
    for (int i0 = 0; i0 < m; i0 += BKT_T * U) {
      uint64_t K[U];
      int32_t V[U];
#pragma unroll
      for (int e = 0; e < U; ++e) {
        const int i = i0 + t + e * BKT_T;
        K[e] = i < m ? kc[i] : 0;
        V[e] = i < m ? vc[i] : 0;
      }
#pragma unroll
      for (int e = 0; e < U; ++e) {
        const int i = i0 + t + e * BKT_T;
        int j = 1;
        for (int l = 0; l < L; ++l) {
          const uint64_t tk = tkey[j];
          const bool right = tk > K[e] || (tk == K[e] && tval[j] < V[e]);
          j = 2 * j + (right ? 1 : 0);
        }
        const int bk = j - (1 << L);  // splitters before (K, V)
        const bool act = i < m;
        if (act) bc[i] = (uint16_t)bk;
        const unsigned peers = __match_any_sync(0xffffffffu, act ? bk : -1);
        if (act && lane == __ffs(peers) - 1) atomicAdd(&hsum[bk], (unsigned)__popc(peers));
      }
    }
    __syncthreads();
    for (int j = t; j < nbx; j += BKT_T) {
      const unsigned c = hsum[j];
      ghist[g * BKT_FAN + j] = c;
      if (c) atomicAdd(&bcount[boff[x] + j], (unsigned long long)c);
    }
    __syncthreads();
  }
}

// Every group of the long segments moves from (ck, cv) to its buckets in
// (ok, ov): one global reservation per bucket of the group (its size from
// ghist), then each chunk is sorted by bucket in shared memory (a counting
// sort; lanes of a warp that share a bucket take their ranks with one shared
// atomic) and leaves in runs, one run per bucket, at the bucket's next free
// positions. The order of the runs within a bucket is arbitrary; the bucket
// sort removes it.
__global__ void __launch_bounds__(BKT_T, 2)
k_bucket_scatter(const uint64_t* __restrict__ ck, const int32_t* __restrict__ cv,
                 const uint16_t* __restrict__ bid, const unsigned* __restrict__ ghist, Segs S,
                 const int64_t* __restrict__ list, int64_t nlong, const int64_t* __restrict__ boff,
                 const int64_t* __restrict__ gpre, const int64_t* __restrict__ bscan,
                 unsigned long long* __restrict__ bfill, uint64_t* __restrict__ ok,
                 int32_t* __restrict__ ov) {
  extern __shared__ uint64_t bsm[];
  uint64_t* stk = bsm;                                            // staged keys [BKT_CH]
  unsigned long long* gpos = reinterpret_cast<unsigned long long*>(stk + BKT_CH);  // [BKT_FAN]
  int32_t* stv = reinterpret_cast<int32_t*>(gpos + BKT_FAN);      // staged vals [BKT_CH]
  unsigned* hist = reinterpret_cast<unsigned*>(stv + BKT_CH);     // chunk sizes, then starts
  uint16_t* stb = reinterpret_cast<uint16_t*>(hist + BKT_FAN);    // staged buckets [BKT_CH]
  __shared__ unsigned wsum[32];
  const int t = threadIdx.x, lane = t & 31;
  const int64_t G = gpre[nlong];
  for (int64_t g = blockIdx.x; g < G; g += gridDim.x) {
    const int64_t x = chunk_segment(gpre, nlong, g);
    const int64_t sg = list[x];
    const int64_t b = S.b[sg], len = S.e[sg] - b;
    const int nbx = (int)(boff[x + 1] - boff[x]);
    const int64_t q0 = (g - gpre[x]) * BKT_CH * BKT_G;
    const int64_t q1 = min(len, q0 + (int64_t)BKT_CH * BKT_G);
    const int64_t bb0 = boff[x];
    const int64_t base = b - bscan[bb0];  // bucket j starts at base + bscan[bb0 + j]
    for (int j = t; j < nbx; j += BKT_T) {
      const unsigned c = ghist[g * BKT_FAN + j];
      gpos[j] = (unsigned long long)(base + bscan[bb0 + j]) +
                (c ? atomicAdd(&bfill[bb0 + j], (unsigned long long)c) : 0ull);
    }
    for (int64_t p0 = q0; p0 < q1; p0 += BKT_CH) {
      const int n = (int)min((int64_t)BKT_CH, q1 - p0);
      const uint64_t* kc = ck + b + p0;
      const int32_t* vc = cv + b + p0;
      const uint16_t* bc = bid + b + p0;
      hist[2 * t] = 0;
      hist[2 * t + 1] = 0;
      uint64_t K[BKT_E];
      int32_t V[BKT_E];
      unsigned B[BKT_E], R[BKT_E];
#pragma unroll
      for (int e = 0; e < BKT_E; ++e) {
        const int i = t + e * BKT_T;
        K[e] = i < n ? kc[i] : 0;
        V[e] = i < n ? vc[i] : 0;
        B[e] = i < n ? bc[i] : 0u;
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < BKT_E; ++e) {
        const bool act = t + e * BKT_T < n;
        const unsigned peers = __match_any_sync(0xffffffffu, act ? (int)B[e] : -1);
        const int leader = __ffs(peers) - 1;
        unsigned r0 = 0;
        if (act && lane == leader) r0 = atomicAdd(&hist[B[e]], (unsigned)__popc(peers));
        r0 = __shfl_sync(0xffffffffu, r0, leader);
        R[e] = r0 + __popc(peers & ((1u << lane) - 1u));
      }
      __syncthreads();
      block_exclusive_scan(hist, wsum);  // hist[j] = first slot of bucket j in the chunk
      __syncthreads();
#pragma unroll
      for (int e = 0; e < BKT_E; ++e) {
        if (t + e * BKT_T < n) {
          const unsigned q = hist[B[e]] + R[e];
          stk[q] = K[e];
          stv[q] = V[e];
          stb[q] = (uint16_t)B[e];
        }
      }
      __syncthreads();
      for (int i = t; i < n; i += BKT_T) {
        const int j = stb[i];
        const int64_t q = (int64_t)gpos[j] + (i - (int)hist[j]);
        ok[q] = stk[i];
        ov[q] = stv[i];
      }
      __syncthreads();
      for (int i = t; i < n; i += BKT_T) {
        const int j = stb[i];
        if (i == n - 1 || stb[i + 1] != j) gpos[j] += (unsigned long long)(i + 1 - (int)hist[j]);
      }
      __syncthreads();
    }
  }
}

// Copies the listed segments from (sk, sv) to (dk, dv), one CTA per segment.
__global__ void k_copy_segments(const uint64_t* __restrict__ sk, const int32_t* __restrict__ sv,
                                uint64_t* __restrict__ dk, int32_t* __restrict__ dv, Segs S,
                                const int64_t* __restrict__ list, int64_t nlist) {
  for (int64_t x = blockIdx.x; x < nlist; x += gridDim.x) {
    const int64_t sg = list[x];
    for (int64_t i = S.b[sg] + threadIdx.x; i < S.e[sg]; i += blockDim.x) {
      dk[i] = sk[i];
      dv[i] = sv[i];
    }
  }
}

// Begin and end of every bucket in (key, val); the entries past the real
// buckets are empty segments.
__global__ void k_bucket_bounds(Segs S, const int64_t* __restrict__ list, int64_t nlong,
                                const int64_t* __restrict__ boff, const int64_t* __restrict__ bscan,
                                int64_t nb_ub, int64_t* __restrict__ bb, int64_t* __restrict__ be) {
  const int64_t B = boff[nlong];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nb_ub;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (k >= B) {
      bb[k] = be[k] = 0;
      continue;
    }
    const int64_t x = chunk_segment(boff, nlong, k);
    const int64_t start = S.b[list[x]] + bscan[k] - bscan[boff[x]];
    bb[k] = start;
    be[k] = start + (bscan[k + 1] - bscan[k]);
  }
}

}  // namespace

namespace {

unsigned grid_of(int64_t units, int per) {
  int64_t g = (units + per - 1) / per;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, sm_count() * 32));
}

// Sorts every segment of S into (key, val). The data is in (key, val), or
// in the copy (alt_k, alt_v) when in_alt; alt_k may be null until a level
// needs it (it then holds total elements).
int sort_level(uint64_t* key, int32_t* val, uint64_t* alt_k, int32_t* alt_v, Segs S, int64_t nseg,
               int64_t total, bool in_alt, Pool& pool, cudaStream_t s, int depth);

// Moves the elements of the nlong long segments (device list llist) into
// their buckets in the other array pair and sorts the buckets, as segments of
// their own, one level down. total bounds every position of the array.
int bucket_level(uint64_t* key, int32_t* val, uint64_t* alt_k, int32_t* alt_v, Segs S,
                 int64_t total, const int64_t* llist, int64_t nlong, bool in_alt, Pool& pool,
                 cudaStream_t s, int depth) {
  const bool own_alt = alt_k == nullptr;
  if (own_alt) {
    alt_k = pool.get<uint64_t>(total);
    alt_v = pool.get<int32_t>(total);
    if (!alt_k || !alt_v) return SCAN_ENOMEM;
  }
  const uint64_t* ck = in_alt ? alt_k : key;  // where the data is
  const int32_t* cv = in_alt ? alt_v : val;
  uint64_t* ok = in_alt ? key : alt_k;        // where the buckets go
  int32_t* ov = in_alt ? val : alt_v;
  // bounds known on the host: every long segment has at most len / BKT_TARGET
  // + 1 buckets and len / (BKT_CH * BKT_G) + 1 groups
  const int64_t B_ub = std::min<int64_t>(total / BKT_TARGET + 2 * nlong, nlong * BKT_FAN);
  const int64_t S_ub = B_ub * BKT_OS;
  const int64_t G_ub = total / ((int64_t)BKT_CH * BKT_G) + nlong;
  int64_t* nb = pool.get<int64_t>(nlong);
  int64_t* ns = pool.get<int64_t>(nlong);
  int64_t* ngr = pool.get<int64_t>(nlong);
  int64_t* boff = pool.get<int64_t>(nlong + 1);
  int64_t* soff = pool.get<int64_t>(nlong + 1);
  int64_t* gpre = pool.get<int64_t>(nlong + 1);
  uint64_t* skey = pool.get<uint64_t>(S_ub);
  int32_t* sval = pool.get<int32_t>(S_ub);
  if (!nb || !ns || !ngr || !boff || !soff || !gpre || !skey || !sval) return SCAN_ENOMEM;
  k_bucket_plan<<<grid_of(nlong, 256), 256, 0, s>>>(S, llist, nlong, nb, ns, ngr);
  GS_LAUNCH();
  GS_TRY(exclusive_scan_i64(nb, boff, nlong, pool, s));
  GS_TRY(exclusive_scan_i64(ns, soff, nlong, pool, s));
  GS_TRY(exclusive_scan_i64(ngr, gpre, nlong, pool, s));
  k_take_samples<<<grid_of(S_ub, 256), 256, 0, s>>>(ck, cv, S, llist, soff, nlong, depth, skey,
                                                    sval);
  GS_LAUNCH();
  GS_TRY(sort_level(skey, sval, nullptr, nullptr, Segs{soff, soff + 1}, nlong, S_ub, false, pool, s,
                    depth + 1));
  unsigned long long* bcount = pool.get<unsigned long long>(B_ub);
  unsigned long long* bfill = pool.get<unsigned long long>(B_ub);
  int64_t* bscan = pool.get<int64_t>(B_ub + 1);
  uint16_t* bid = pool.get<uint16_t>(total);
  unsigned* ghist = pool.get<unsigned>((size_t)G_ub * BKT_FAN);
  if (!bcount || !bfill || !bscan || !bid || !ghist) return SCAN_ENOMEM;
  GS_CUDA(cudaMemsetAsync(bcount, 0, B_ub * sizeof(unsigned long long), s));
  GS_CUDA(cudaMemsetAsync(bfill, 0, B_ub * sizeof(unsigned long long), s));
  constexpr size_t scatter_smem = (size_t)BKT_FAN * 12 + (size_t)BKT_CH * 14;
  GS_CUDA(cudaFuncSetAttribute(k_bucket_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)scatter_smem));
  const unsigned g_groups =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>(G_ub, sm_count() * 2));
  k_bucket_count<<<g_groups, BKT_T, 0, s>>>(ck, cv, S, llist, nlong, soff, boff, gpre, skey, sval,
                                            bcount, ghist, bid);
  GS_LAUNCH();
  GS_TRY(exclusive_scan_i64(reinterpret_cast<const int64_t*>(bcount), bscan, B_ub, pool, s));
  k_bucket_scatter<<<g_groups, BKT_T, scatter_smem, s>>>(ck, cv, bid, ghist, S, llist, nlong, boff,
                                                         gpre, bscan, bfill, ok, ov);
  GS_LAUNCH();
  pool.put(bid);
  pool.put(ghist);
  pool.put(skey);
  pool.put(sval);
  pool.put(bcount);
  pool.put(bfill);
  // the buckets as segments of their own
  int64_t* bb = pool.get<int64_t>(B_ub);
  int64_t* be = pool.get<int64_t>(B_ub);
  if (!bb || !be) return SCAN_ENOMEM;
  k_bucket_bounds<<<grid_of(B_ub, 256), 256, 0, s>>>(S, llist, nlong, boff, bscan, B_ub, bb, be);
  GS_LAUNCH();
  pool.put(bscan);
  pool.put(nb);
  pool.put(ns);
  pool.put(ngr);
  pool.put(boff);
  pool.put(soff);
  pool.put(gpre);
  GS_TRY(sort_level(key, val, alt_k, alt_v, Segs{bb, be}, B_ub, total, !in_alt, pool, s,
                    depth + 1));
  pool.put(bb);
  pool.put(be);
  if (own_alt) {
    pool.put(alt_k);
    pool.put(alt_v);
  }
  return SCAN_OK;
}

int sort_level(uint64_t* key, int32_t* val, uint64_t* alt_k, int32_t* alt_v, Segs S, int64_t nseg,
               int64_t total, bool in_alt, Pool& pool, cudaStream_t s, int depth) {
  if (nseg <= 0 || total <= 1) return SCAN_OK;
  unsigned long long* counts = pool.get<unsigned long long>(2 * NCNT);
  if (!counts) return SCAN_ENOMEM;
  GS_CUDA(cudaMemsetAsync(counts, 0, 2 * NCNT * sizeof(unsigned long long), s));
  const unsigned g_seg = (unsigned)std::min<int64_t>((nseg + 255) / 256, sm_count() * 16);
  k_classify_count<<<g_seg, 256, 0, s>>>(S, nseg, total, counts);
  GS_LAUNCH();
  unsigned long long hc[NCNT];
  GS_CUDA(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (hc[NCLASS + 2]) return SCAN_EINVAL;  // before any element is touched
  int64_t base[NCLASS + 1];
  base[0] = 0;
  for (int c = 0; c < NCLASS; ++c) base[c + 1] = base[c] + (int64_t)hc[c];
  int64_t* list = pool.get<int64_t>(base[NCLASS] > 0 ? base[NCLASS] : 1);
  int64_t* base_dev = pool.get<int64_t>(NCLASS + 1);
  if (!list || !base_dev) return SCAN_ENOMEM;
  GS_CUDA(cudaMemcpyAsync(base_dev, base, sizeof(base), cudaMemcpyHostToDevice, s));
  const uint64_t* ik = in_alt ? alt_k : key;  // where the data is
  const int32_t* iv = in_alt ? alt_v : val;
  unsigned long long* fill = counts + NCNT;
  k_classify_fill<<<g_seg, 256, 0, s>>>(S, nseg, base_dev, fill, list);
  GS_LAUNCH();
  const int64_t nlong = (int64_t)hc[LONGC];
  const int64_t max_long = (int64_t)hc[NCLASS + 1];
  // long segments are split into buckets, sorted one level down; below
  // BKT_DEPTH levels they take the tiles and merge passes
  const bool bucketed = nlong && depth < BKT_DEPTH;
  if (bucketed)
    GS_TRY(bucket_level(key, val, alt_k, alt_v, S, total, list + base[LONGC], nlong, in_alt, pool,
                        s, depth));
  // per-class counts on the device for the grid-stride kernels: counts[c]
  if (hc[0]) {
    k_sort_warp<<<grid_of((int64_t)hc[0], 8), 256, 0, s>>>(ik, iv, key, val, S, list + base[0],
                                                           counts + 0);
    GS_LAUNCH();
  }
  if (hc[1]) {
    // 33..256 elements: one 32-thread CTA per row (8-element register
    // networks and merge levels: compact code, unlike fully unrolled bitonic
    // networks, whose instruction footprint stalls the warp on fetches)
    k_sort_tile<32, 8, false><<<grid_of((int64_t)hc[1], 1), 32, tile_smem_bytes<32, 8>(), s>>>(
        ik, iv, key, val, S, list + base[1], counts + 1, nullptr, 0, nullptr, nullptr);
    GS_LAUNCH();
  }
  GS_CUDA(cudaFuncSetAttribute(k_merge_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)MERGE_SMEM));
  GS_CUDA(cudaFuncSetAttribute(k_sort_tile<TLONG_T, TLONG_RI, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tile_smem_bytes<TLONG_T, TLONG_RI>()));
  GS_CUDA(cudaFuncSetAttribute(k_sort_tile<256, 8, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tile_smem_bytes<256, 8>()));
  GS_CUDA(cudaFuncSetAttribute(k_sort_tile<T4K_T, 8, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tile_smem_bytes<T4K_T, 8>()));
  if (hc[2]) {
    k_sort_tile<64, 8, false><<<grid_of((int64_t)hc[2], 1), 64, tile_smem_bytes<64, 8>(), s>>>(
        ik, iv, key, val, S, list + base[2], counts + 2, nullptr, 0, nullptr, nullptr);
    GS_LAUNCH();
  }
  if (hc[3]) {
    k_sort_tile<128, 8, false><<<grid_of((int64_t)hc[3], 1), 128, tile_smem_bytes<128, 8>(), s>>>(
        ik, iv, key, val, S, list + base[3], counts + 3, nullptr, 0, nullptr, nullptr);
    GS_LAUNCH();
  }
  if (hc[4]) {
    k_sort_tile<256, 8, false><<<grid_of((int64_t)hc[4], 1), 256, tile_smem_bytes<256, 8>(), s>>>(
        ik, iv, key, val, S, list + base[4], counts + 4, nullptr, 0, nullptr, nullptr);
    GS_LAUNCH();
  }
  if (hc[5]) {
    k_sort_tile<T4K_T, 8, false><<<grid_of((int64_t)hc[5], 1), T4K_T, tile_smem_bytes<T4K_T, 8>(),
                                 s>>>(
        ik, iv, key, val, S, list + base[5], counts + 5, nullptr, 0, nullptr, nullptr);
    GS_LAUNCH();
  }
  if (nlong && !bucketed) {
    const int64_t* llist = list + base[LONGC];
    if (in_alt) {  // the tiles and merge passes work in (key, val)
      k_copy_segments<<<grid_of(nlong, 1), 256, 0, s>>>(alt_k, alt_v, key, val, S, llist, nlong);
      GS_LAUNCH();
    }
    int64_t* tiles = pool.get<int64_t>(nlong);
    int64_t* tile_prefix = pool.get<int64_t>(nlong + 1);
    int64_t* chunks = pool.get<int64_t>(nlong);
    int64_t* chunk_prefix = pool.get<int64_t>(nlong + 1);
    uint64_t* tk = pool.get<uint64_t>(total);
    int32_t* tv = pool.get<int32_t>(total);
    if (!tiles || !tile_prefix || !chunks || !chunk_prefix || !tk || !tv) return SCAN_ENOMEM;
    k_long_tiles<<<grid_of(nlong, 256), 256, 0, s>>>(S, llist, counts + LONGC, tiles, chunks,
                                                     MERGE_CHUNK);
    GS_LAUNCH();
    GS_TRY(exclusive_scan_i64(tiles, tile_prefix, nlong, pool, s));
    GS_TRY(exclusive_scan_i64(chunks, chunk_prefix, nlong, pool, s));
    const int64_t ntiles = (int64_t)hc[NCLASS];
    // tile sort (count = ntiles, read from counts[NCLASS])
    k_sort_tile<TLONG_T, TLONG_RI, true><<<grid_of(ntiles, 1), TLONG_T,
                                          tile_smem_bytes<TLONG_T, TLONG_RI>(), s>>>(
        key, val, key, val, S, llist, counts + NCLASS, tile_prefix, nlong, tk, tv);
    GS_LAUNCH();
    const int64_t total_chunks_ub = (total + MERGE_CHUNK - 1) / MERGE_CHUNK + nlong;
    MergeDesc* desc = pool.get<MergeDesc>((size_t)total_chunks_ub);
    if (!desc) return SCAN_ENOMEM;
    // every pass reads each segment from the buffer its parity says and
    // writes the other; the last pass of every segment writes (key, val)
    int pass = 0;
    for (int64_t L = TILE; L < max_long; L <<= 1, ++pass) {
      k_merge_partition<<<grid_of(total_chunks_ub, 256), 256, 0, s>>>(
          key, val, tk, tv, S, llist, chunk_prefix, nlong, L, pass, desc);
      GS_LAUNCH();
      k_merge_pass<<<grid_of(total_chunks_ub, 1), MERGE_T, MERGE_SMEM, s>>>(key, val, tk, tv,
                                                                           chunk_prefix, nlong,
                                                                           desc);
      GS_LAUNCH();
    }
    pool.put(desc);
    pool.put(tk);
    pool.put(tv);
    pool.put(tiles);
    pool.put(tile_prefix);
    pool.put(chunks);
    pool.put(chunk_prefix);
  }
  pool.put(list);
  pool.put(base_dev);
  pool.put(counts);
  return SCAN_OK;
}

}  // namespace

int segmented_sort_desc(uint64_t* key, int32_t* val, const int64_t* seg_off, int64_t nseg,
                        int64_t total, int64_t max_len, Pool& pool, cudaStream_t s) {
  if (nseg <= 0 || total <= 1 || max_len <= 1) return SCAN_OK;
  return sort_level(key, val, nullptr, nullptr, Segs{seg_off, seg_off + 1}, nseg, total, false, pool,
                    s, 0);
}

}  // namespace gscan
