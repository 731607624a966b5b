// Closed counts of a dense graph by one matrix product (Section 4.1.1): with
// A the adjacency matrix and I the identity, ((A+I)^2)[u][v] = |N̄(u) ∩ N̄(v)|
// for every pair, in particular for every edge. (A+I) holds only 0 and 1, so
// it is exact in bf16; every entry of the product is an integer of at most
// n+1 < 2^24, so it is exact in an fp32 accumulator.
//
// The product is a hand-written tcgen05 GEMM (sm_100 family): TMA loads 128-
// byte-swizzled K-slices of (A+I) into a 4-stage shared-memory ring, one
// thread issues tcgen05.mma (bf16 x bf16 -> fp32, 128 x 256 tiles) into one
// of two TMEM accumulators, and four epilogue warps read the other with
// tcgen05.ld while the next tile is being multiplied (two groups of four
// epilogue warps, one per accumulator buffer). (A+I) is symmetric, so
// the product is too, and only the tiles that hold some pair u < v are
// computed. The epilogue never writes the n x n product: it reads, for the
// arcs that fall in the tile, their counts and writes the similarity of both
// arcs of every edge u < v once (cosine, Section 3.1; Jaccard, Section 2.1.1).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "scan_internal.cuh"

namespace gscan {

namespace {

constexpr int BM = 128;          // rows of a tile (TMEM lanes)
constexpr int BN = 256;          // columns of a tile (TMEM columns per accumulator)
constexpr int BK = 64;           // bf16 elements of K per stage: one 128-byte swizzle row
constexpr int KSTEP = 16;        // K of one tcgen05.mma of kind f16
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;              // 16 KB
constexpr int B_BYTES = BN * BK * 2;              // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;    // 48 KB
constexpr int CHUNK = 8;                          // accumulator columns per epilogue step
constexpr int EPI_WARPS = 4;                      // warps of one epilogue group (4 lane quadrants)
constexpr int EPI_GROUPS = 2;                     // group g drains TMEM buffer g (tiles it % 2 == g)
constexpr int THREADS = 64 + 32 * EPI_WARPS * EPI_GROUPS;  // producer, MMA, epilogue groups
constexpr int CNT_PITCH = CHUNK + 1;              // padded row of the count staging
constexpr size_t EPI_SMEM = (size_t)BM * CNT_PITCH * 4 + (size_t)BM * CHUNK * 8;  // per group
constexpr size_t SMEM_BYTES = 1024 /* alignment slack */ + (size_t)STAGES * STAGE_BYTES +
                              EPI_GROUPS * EPI_SMEM + 256;
// The matrices are np x np with np = n rounded up to DENSE_PAD: zero rows
// and columns leave the n x n block of the product unchanged.
constexpr int64_t DENSE_PAD = 256;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // a wait longer than 2 s gives up

// tcgen05 instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A and B
// bf16 (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bit 17, M >> 4 at bit 24.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `parity` to complete, for at most WAIT_NS or until
// another role has given up (*abort). Returns false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  for (;;) {
    if (mbar_test(bar, parity)) return true;
    if (*abort || now_ns() - t0 > WAIT_NS) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle
// layout written by TMA: rows of 128 bytes, 8-row groups 1024 bytes apart
// (stride byte offset), descriptor version 1, layout SWIZZLE_128B (2).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 8 consecutive 32-bit accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Named barrier of one epilogue group (non-aligned form: the threads arrive
// from divergent loops); group g uses barriers 1 + 2g (sync) and 2 + 2g (vote).
__device__ __forceinline__ void epi_barrier(int id) {
  asm volatile("barrier.sync %0, %1;" ::"r"(id), "n"(32 * EPI_WARPS) : "memory");
}

__device__ __forceinline__ double sim_from(int kind, int64_t c, int64_t du, int64_t dv) {
  if (kind == SCAN_COSINE) return __ddiv_rn((double)c, __dsqrt_rn((double)((du + 1) * (dv + 1))));
  return __ddiv_rn((double)c, (double)(du + dv + 2 - c));
}

// (A+I) as a dense row-major np x np bf16 matrix (zeroed by the caller), and
// for every vertex u the first position of N(u) at or after column 128*b,
// b = 0..nb (bpos[u * (nb+1) + b]); the rows are id-sorted.
__global__ void k_dense_fill(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                             int64_t n, int64_t np, int64_t nb, __nv_bfloat16* __restrict__ M,
                             int64_t* __restrict__ bpos) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const __nv_bfloat16 one = __float2bfloat16(1.0f);
  for (int64_t u = warp; u < n; u += nwarps) {
    __nv_bfloat16* row = M + u * np;
    int64_t* bp = bpos + u * (nb + 1);
    const int64_t b0 = off[u], b1 = off[u + 1];
    if (lane == 0) row[u] = one;
    if (lane == 0 && b0 == b1)
      for (int64_t b = 0; b <= nb; ++b) bp[b] = b0;
    for (int64_t i = b0 + lane; i < b1; i += 32) {
      const int32_t x = adj[i];
      row[x] = one;
      // blocks (previous entry's block, this entry's block] start here
      const int64_t bprev = i > b0 ? (int64_t)(adj[i - 1] >> 7) : -1;
      for (int64_t b = bprev + 1; b <= (x >> 7); ++b) bp[b] = i;
      if (i == b1 - 1)
        for (int64_t b = (x >> 7) + 1; b <= nb; ++b) bp[b] = b1;
    }
  }
}

// Every arc (u,v) needs its reverse (v,u): M[v][u] must be 1.
__global__ void k_dense_check(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                              int64_t n, int64_t np, const __nv_bfloat16* __restrict__ M,
                              unsigned* status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned short* Mb = reinterpret_cast<const unsigned short*>(M);
  bool bad = false;
  for (int64_t u = warp; u < n; u += nwarps)
    for (int64_t i = off[u] + lane; i < off[u + 1]; i += 32)
      if (Mb[(int64_t)adj[i] * np + u] == 0) bad = true;
  if (bad) atomicOr(status, (unsigned)DEV_BADGRAPH);
}

struct DenseArgs {
  const int64_t* off;
  const int32_t* adj;
  const int32_t* deg;
  const int64_t* bpos;      // n x (nb+1)
  const uint32_t* tiles;    // (bi << 16) | bj, in schedule order
  int64_t n, nb, ntiles;
  int kind, lsh_T, nk;      // nk = np / BK
  double* sim;
  unsigned* status;
};

// Persistent GEMM + similarity epilogue. Warp 0 loads (TMA), warp 1 issues
// the MMAs (one elected thread) and owns the TMEM allocation, warps 2-5 and
// 6-9 are two epilogue groups, each draining one of the two accumulator
// buffers; warp w reads TMEM lanes 32*(w%4) .. +31 (tile rows).
__global__ void __launch_bounds__(THREADS, 1)
k_dense_mma(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
            const DenseArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* stage_a = smem;                                  // STAGES x A_BYTES
  uint8_t* stage_b = smem + (size_t)STAGES * A_BYTES;       // STAGES x B_BYTES
  uint8_t* epi_smem = smem + (size_t)STAGES * STAGE_BYTES;   // EPI_GROUPS x EPI_SMEM
  uint64_t* bars = reinterpret_cast<uint64_t*>(epi_smem + EPI_GROUPS * EPI_SMEM);
  uint64_t* full = bars;                 // STAGES
  uint64_t* empty = bars + STAGES;       // STAGES
  uint64_t* acc_full = bars + 2 * STAGES;      // 2
  uint64_t* acc_empty = bars + 2 * STAGES + 2;  // 2
  uint64_t* drain = bars + 2 * STAGES + 4;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], EPI_WARPS);
    }
    mbar_init(drain, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(s_tmem)),
                 "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  if (warp == 0) {
    // ---- producer: one elected lane issues the TMA loads
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        const uint32_t tl = a.tiles[t];
        const int y_a = (int)(tl >> 16) * BM, y_b = (int)(tl & 0xFFFFu) * BN;
        for (int kb = 0; kb < a.nk; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, s_abort)) { ok = false; break; }
          mbar_expect_tx(&full[stage], STAGE_BYTES);
          tma_load_2d(stage_a + (size_t)stage * A_BYTES, &map_a, &full[stage], kb * BK, y_a);
          tma_load_2d(stage_b + (size_t)stage * B_BYTES, &map_b, &full[stage], kb * BK, y_b);
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) *s_abort = 1;
      // every load in flight lands before the CTA may exit: wait for the
      // stages not yet consumed (bounded)
      for (int s = 0; s < STAGES; ++s) {
        if (!mbar_wait(&empty[stage], phase ^ 1u, s_abort)) {
          const unsigned long long t0 = now_ns();
          while (!mbar_test(&full[stage], phase) && now_ns() - t0 < WAIT_NS) {
          }
        }
        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++it) {
        const int buf = it & 1;
        const uint32_t use = (uint32_t)(it >> 1);  // this buffer's use count
        if (!mbar_wait(&acc_empty[buf], (use & 1u) ^ 1u, s_abort)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * BN);
        for (int kb = 0; kb < a.nk; ++kb) {
          if (!mbar_wait(&full[stage], phase, s_abort)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(stage_a + (size_t)stage * A_BYTES);
          const uint32_t sb = smem_u32(stage_b + (size_t)stage * B_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / KSTEP; ++kk)  // 32 bytes of K per MMA
            mma_bf16(d, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32),
                     (kb | kk) != 0 ? 1u : 0u);
          mma_commit(&empty[stage]);  // the stage is free once these MMAs are done
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit(&acc_full[buf]);
      }
      if (!ok) *s_abort = 1;
      // every MMA issued has completed before TMEM is released
      mma_commit(drain);
      const unsigned long long t0 = now_ns();
      while (!mbar_test(drain, 0) && now_ns() - t0 < WAIT_NS) {
      }
    }
  } else {
    // ---- epilogue: group g = (w-2)/4 drains TMEM buffer g, i.e. the tiles
    // of odd or even iteration; warp w owns TMEM lanes 32*(w%4) .. +31
    const int grp = (warp - 2) / EPI_WARPS;
    const int q = warp & 3;
    const int r_loc = 32 * q + lane;                          // row of the tile
    const int et = threadIdx.x - 64 - 32 * EPI_WARPS * grp;   // 0..127 in the group
    const int bar_sync = 1 + 2 * grp, bar_vote = 2 + 2 * grp;
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(epi_smem + grp * EPI_SMEM);
    int64_t* s_pos = reinterpret_cast<int64_t*>(s_cnt + BM * CNT_PITCH);
    int it = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++it) {
      const int buf = it & 1;
      if (buf != grp) continue;
      const uint32_t use = (uint32_t)(it >> 1);
      const uint32_t tl = a.tiles[t];
      const int64_t bi = tl >> 16, bj = tl & 0xFFFFu;
      const int64_t i0 = bi * BM, j0 = bj * BN;
      const int64_t i = i0 + r_loc;
      // this row's arcs with columns in the tile (the rows are id-sorted)
      int64_t cur = 0, cend = 0;
      if (i < a.n) {
        const int64_t* bp = a.bpos + i * (a.nb + 1);
        cur = bp[2 * bj];
        cend = bp[min(2 * bj + 2, a.nb)];
      }
      // one decision for all epilogue threads (a named barrier with an AND
      // vote), so that no warp leaves the loop while others wait at a barrier
      const uint32_t w_ok = mbar_wait(&acc_full[buf], use & 1u, s_abort) ? 1u : 0u;
      uint32_t all_ok;
      asm volatile(
          "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n"
          " barrier.red.and.pred po, %2, %3, pi;\n selp.u32 %0, 1, 0, po;\n}\n"
          : "=r"(all_ok)
          : "r"(w_ok), "r"(bar_vote), "n"(32 * EPI_WARPS)
          : "memory");
      if (!all_ok) { ok = false; break; }
      tc_fence_after();
      const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * BN);
      for (int c = 0; c < BN / CHUNK; ++c) {
        const int64_t c0 = j0 + (int64_t)c * CHUNK;
        uint32_t r[CHUNK];
        __syncwarp();
        tmem_ld8(tbase + (uint32_t)(c * CHUNK), r);
#pragma unroll
        for (int x = 0; x < CHUNK; ++x)
          s_cnt[r_loc * CNT_PITCH + x] = (uint32_t)__uint_as_float(r[x]);
        // row pass: positions of the arcs (i, j), i < j, j in this chunk
        while (cur < cend) {
          const int32_t j = a.adj[cur];
          if (j >= c0 + CHUNK) break;
          if (j > i) s_pos[r_loc * CHUNK + (j - c0)] = cur;
          ++cur;
        }
        epi_barrier(bar_sync);
        // column pass: for column j, the arcs (j, x) with x in the tile's rows
        // and x < j; each edge x < j gets its similarity once, written to both
        // arcs. 16 threads per column.
        {
          const int jc = et >> 4, sub = et & 15;
          const int64_t j = c0 + jc;
          if (j < a.n && j > i0) {
            const int64_t* bp = a.bpos + j * (a.nb + 1);
            const int64_t p0 = bp[bi], p1 = bp[bi + 1];
            const int64_t dj = a.deg[j];
            for (int64_t p = p0 + sub; p < p1; p += 16) {
              const int32_t x = a.adj[p];
              if (x >= j) break;
              const int xl = (int)(x - i0);
              const int64_t pos_x = s_pos[xl * CHUNK + jc];
              const int64_t cnt = (int64_t)s_cnt[xl * CNT_PITCH + jc];
              const int64_t dx = a.deg[x];
              // LSH mode: approximated edges are written by the estimate pass
              if (a.lsh_T >= 0 && dx > a.lsh_T && dj > a.lsh_T) continue;
              const double sv = sim_from(a.kind, cnt, dx, dj);
              a.sim[pos_x] = sv;
              a.sim[p] = sv;
            }
          }
        }
        epi_barrier(bar_sync);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
    if (!ok) *s_abort = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x == 0 && *s_abort) atomicOr(a.status, (unsigned)DEV_LIMIT);
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

int encode_map(CUtensorMap* map, const void* base, int64_t np, int box_rows) {
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return SCAN_ECUDA;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)np, (cuuint64_t)np};
  const cuuint64_t strides[1] = {(cuuint64_t)np * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
                              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SCAN_OK : SCAN_ECUDA;
}

// Tiles that hold some pair i < j (rows [128 bi, +128), columns [256 bj,
// +256): bi <= 2 bj + 1), in groups of 8 column blocks so that the tiles in
// flight at one time share their K-slices in L2.
std::vector<uint32_t> upper_tiles(int64_t np) {
  const int64_t nbi = np / BM, nbj = np / BN;
  constexpr int64_t G = 8;
  std::vector<uint32_t> t;
  for (int64_t g0 = 0; g0 < nbj; g0 += G)
    for (int64_t bi = 0; bi < nbi; ++bi)
      for (int64_t bj = g0; bj < std::min(nbj, g0 + G); ++bj)
        if (bi <= 2 * bj + 1) t.push_back((uint32_t)(bi << 16) | (uint32_t)bj);
  return t;
}

}  // namespace

bool dense_counts_pay(int64_t n, int64_t arcs, const CountCfg& cfg) {
  // the product costs ~n^3 flops (half of the tiles); the sparse enumeration
  // ~ n (d/2)^2 probes at about 1000 flop-times each: dense wins from an
  // average degree of about n/16 on (dense_div = 16), for graphs large
  // enough that a GEMM beats the enumeration's launch and table costs
  return cfg.dense_div > 0 && n >= cfg.dense_min_n && n <= DENSE_MAX_N &&
         (int64_t)cfg.dense_div * arcs >= n * n;
}

int dense_counts_and_sims(int kind, const int64_t* off, const int32_t* adj, const int32_t* deg,
                          int64_t n, int lsh_T, double* sim_csr, unsigned* status, Pool& pool,
                          cudaStream_t s, float* count_ms) {
  if (n > DENSE_MAX_N) return SCAN_EINVAL;
  if (n == 0) return SCAN_OK;
  const int64_t np = (n + DENSE_PAD - 1) / DENSE_PAD * DENSE_PAD;
  const int64_t nb = np / 128;
  const size_t nn = (size_t)np * (size_t)np;
  const std::vector<uint32_t> tiles = upper_tiles(np);
  __nv_bfloat16* M = pool.get<__nv_bfloat16>(nn);
  int64_t* bpos = pool.get<int64_t>((size_t)n * (size_t)(nb + 1));
  uint32_t* tiles_d = pool.get<uint32_t>(tiles.size());
  if (!M || !bpos || !tiles_d) return SCAN_ENOMEM;
  CUtensorMap map_a, map_b;
  GS_TRY(encode_map(&map_a, M, np, BM));
  GS_TRY(encode_map(&map_b, M, np, BN));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (count_ms) {
    GS_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      return SCAN_ECUDA;
    }
  }
  // events are released on every return path
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } guard{e0, e1};
  if (e0) GS_CUDA(cudaEventRecord(e0, s));
  GS_CUDA(cudaMemcpyAsync(tiles_d, tiles.data(), tiles.size() * sizeof(uint32_t),
                          cudaMemcpyHostToDevice, s));
  GS_CUDA(cudaMemsetAsync(M, 0, nn * sizeof(__nv_bfloat16), s));
  const unsigned grid =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, (int64_t)sm_count() * 16));
  k_dense_fill<<<grid, 256, 0, s>>>(off, adj, n, np, nb, M, bpos);
  GS_LAUNCH();
  k_dense_check<<<grid, 256, 0, s>>>(off, adj, n, np, M, status);
  GS_LAUNCH();
  // the epilogue pairs every arc with its reverse: check symmetry first
  unsigned hst = 0;
  GS_CUDA(cudaMemcpyAsync(&hst, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (hst & DEV_BADGRAPH) return SCAN_EBADGRAPH;
  GS_CUDA(cudaFuncSetAttribute(k_dense_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)SMEM_BYTES));
  DenseArgs da{off, adj, deg, bpos, tiles_d, n, nb, (int64_t)tiles.size(), kind, lsh_T,
               (int)(np / BK), sim_csr, status};
  const unsigned mgrid = (unsigned)std::min<int64_t>((int64_t)tiles.size(), sm_count());
  k_dense_mma<<<mgrid, THREADS, SMEM_BYTES, s>>>(map_a, map_b, da);
  GS_LAUNCH();
  if (e1) {
    GS_CUDA(cudaEventRecord(e1, s));
    GS_CUDA(cudaEventSynchronize(e1));
    GS_CUDA(cudaEventElapsedTime(count_ms, e0, e1));
  }
  pool.put(M);
  pool.put(bpos);
  pool.put(tiles_d);
  return SCAN_OK;
}

}  // namespace gscan
