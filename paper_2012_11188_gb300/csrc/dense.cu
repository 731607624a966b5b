// Closed counts of a dense graph by one matrix product (Section 4.1.1): with
// A the adjacency matrix and I the identity, ((A+I)^2)[u][v] = |N̄(u) ∩ N̄(v)|
// for every pair, in particular for every edge. (A+I) holds only 0 and 1, so
// it is exact in bf16; every entry of the product is an integer of at most
// n+1 < 2^24, so it is exact in an fp32 accumulator. The product is one
// bf16 x bf16 -> fp32 GEMM (cuBLAS, tensor cores), the similarities are then
// read off at the arcs, so no orientation or triangle enumeration runs.
// For n = 25,825 and average degree 5,400 (shaped like the paper's blood
// vessel graph) the product is 3.4e13 flops, tens of milliseconds, against
// ~2e11 probes of the sparse enumeration.
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "scan_internal.cuh"

namespace gscan {

namespace {

// The matrices are np x np with np = n rounded up to DENSE_PAD: zero rows
// and columns leave the n x n block of the product unchanged, and aligned
// leading dimensions let the GEMM use its tensor-core tiles.
constexpr int64_t DENSE_PAD = 128;

// (A+I) as a dense row-major np x np bf16 matrix (zeroed by the caller).
__global__ void k_dense_fill(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                             int64_t n, int64_t np, __nv_bfloat16* __restrict__ M) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const __nv_bfloat16 one = __float2bfloat16(1.0f);
  for (int64_t u = warp; u < n; u += nwarps) {
    __nv_bfloat16* row = M + u * np;
    if (lane == 0) row[u] = one;
    for (int64_t i = off[u] + lane; i < off[u + 1]; i += 32) row[adj[i]] = one;
  }
}

__device__ __forceinline__ double sim_from(int kind, int64_t c, int64_t du, int64_t dv) {
  if (kind == SCAN_COSINE) return __ddiv_rn((double)c, __dsqrt_rn((double)((du + 1) * (dv + 1))));
  return __ddiv_rn((double)c, (double)(du + dv + 2 - c));
}

// sigma of every arc (u,v) from C[u][v] (C symmetric, fp32 integers). The
// graph must be undirected: an arc (u,v) without (v,u), i.e. M[v][u] = 0,
// marks the build SCAN_EBADGRAPH (the sparse path finds it in orientation).
__global__ void k_dense_sims(int kind, const int64_t* __restrict__ off,
                             const int32_t* __restrict__ adj, const int32_t* __restrict__ deg,
                             int64_t n, int64_t np, const __nv_bfloat16* __restrict__ M,
                             const float* __restrict__ C, int lsh_T, double* __restrict__ sim_csr,
                             unsigned* status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned short* Mb = reinterpret_cast<const unsigned short*>(M);
  bool bad = false;
  for (int64_t u = warp; u < n; u += nwarps) {
    const int32_t du = deg[u];
    const float* row = C + u * np;
    for (int64_t i = off[u] + lane; i < off[u + 1]; i += 32) {
      const int32_t v = adj[i];
      if (Mb[(int64_t)v * np + u] == 0) bad = true;
      const int32_t dv = deg[v];
      // LSH mode: approximated edges are written by the estimate pass
      if (lsh_T >= 0 && du > lsh_T && dv > lsh_T) continue;
      sim_csr[i] = sim_from(kind, (int64_t)row[v], du, dv);
    }
  }
  if (bad) atomicOr(status, (unsigned)DEV_BADGRAPH);
}

std::mutex g_cublas_mu;
cublasHandle_t g_cublas[64] = {};

}  // namespace

bool dense_counts_pay(int64_t n, int64_t arcs) {
  // the product costs 2 n^3 flops; the sparse enumeration ~ n (d/2)^2 probes
  // at about 1000 flop-times each: dense wins from an average degree of
  // about n/16 on, and n^2 bf16 + fp32 entries must stay modest
  return n >= 2 && n <= DENSE_MAX_N && 16 * arcs >= n * n;
}

int dense_counts_and_sims(int kind, const int64_t* off, const int32_t* adj, const int32_t* deg,
                          int64_t n, int lsh_T, double* sim_csr, unsigned* status, Pool& pool,
                          cudaStream_t s, float* count_ms) {
  if (n > DENSE_MAX_N) return SCAN_EINVAL;
  const int64_t np = (n + DENSE_PAD - 1) / DENSE_PAD * DENSE_PAD;
  const size_t nn = (size_t)np * (size_t)np;
  __nv_bfloat16* M = pool.get<__nv_bfloat16>(nn);
  float* C = pool.get<float>(nn);
  if (!M || !C) return SCAN_ENOMEM;
  cudaEvent_t e0, e1;
  GS_CUDA(cudaEventCreate(&e0));
  GS_CUDA(cudaEventCreate(&e1));
  GS_CUDA(cudaEventRecord(e0, s));
  GS_CUDA(cudaMemsetAsync(M, 0, nn * sizeof(__nv_bfloat16), s));
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, 152 * 16));
  k_dense_fill<<<grid, 256, 0, s>>>(off, adj, n, np, M);
  GS_LAUNCH();
  {
    std::lock_guard<std::mutex> lock(g_cublas_mu);
    int dev = 0;
    GS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SCAN_ECUDA;
    if (!g_cublas[dev] && cublasCreate(&g_cublas[dev]) != CUBLAS_STATUS_SUCCESS) return SCAN_ECUDA;
    cublasHandle_t h = g_cublas[dev];
    if (cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) return SCAN_ECUDA;
    const float one = 1.0f, zero = 0.0f;
    const int ni = (int)np;
    // (A+I) is symmetric, so row- and column-major agree: C = (A+I)(A+I)
    if (cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, ni, ni, ni, &one, M, CUDA_R_16BF, ni, M,
                     CUDA_R_16BF, ni, &zero, C, CUDA_R_32F, ni, CUBLAS_COMPUTE_32F,
                     CUBLAS_GEMM_DEFAULT) != CUBLAS_STATUS_SUCCESS)
      return SCAN_ECUDA;
  }
  GS_CUDA(cudaEventRecord(e1, s));
  k_dense_sims<<<grid, 256, 0, s>>>(kind, off, adj, deg, n, np, M, C, lsh_T, sim_csr, status);
  GS_LAUNCH();
  if (count_ms) {
    GS_CUDA(cudaEventSynchronize(e1));
    GS_CUDA(cudaEventElapsedTime(count_ms, e0, e1));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pool.put(M);
  pool.put(C);
  return SCAN_OK;
}

}  // namespace gscan
