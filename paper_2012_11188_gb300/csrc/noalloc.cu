// scan_query_noalloc: the (mu, eps) query of scan_query without any device
// allocation. The paper has no counterpart; this exists for callers that must
// not allocate device memory while answering a query (see include/scan.h).
//
// All per-call scratch -- the union-find parents of every vertex, the core
// count, the query's mu and eps and a status word -- lives in one array
// compiled into the library. Host code cannot use the array's name as a
// device address (it is a host-side stand-in), so the first call on each
// device looks the address up with cudaGetSymbolAddress while that device is
// current, and caches it.
#include <mutex>

#include "scan_internal.cuh"

namespace {

// scratch layout, in int32 words:
//   [0, NOALLOC_MAX_N)            parents
//   NOALLOC_MAX_N + 0 .. +5       core count and its prefix sums (3 x int64)
//   NOALLOC_MAX_N + 6             mu (int32)
//   NOALLOC_MAX_N + 8 .. +9       eps (double)
//   NOALLOC_MAX_N + 10            status word
constexpr int64_t NOALLOC_MAX_N = (int64_t)1 << 22;
constexpr int64_t NOALLOC_WORDS = NOALLOC_MAX_N + 64;

static __device__ __align__(256) int32_t g_query_scratch[NOALLOC_WORDS];

std::mutex g_addr_mu;
int32_t* g_addr[64] = {nullptr};

int scratch_address(int32_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SCAN_ECUDA;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_query_scratch) != cudaSuccess) {
      cudaGetLastError();
      return SCAN_ECUDA;
    }
    g_addr[dev] = (int32_t*)p;
  }
  *out = g_addr[dev];
  return SCAN_OK;
}

}  // namespace

extern "C" int scan_query_noalloc(scan_index* index, int mu, double eps, int32_t* labels,
                                  int flags, uintptr_t stream) {
  if (!index) return SCAN_EINVAL;
  if (mu < 2 || !(eps >= 0.0 && eps <= 1.0) || (flags & ~SCAN_Q_HUBS)) return SCAN_EINVAL;
  const gscan::IndexData& ix = index->d;
  if (ix.n > NOALLOC_MAX_N) return SCAN_EINVAL;  // beyond the compiled-in scratch
  if (ix.n == 0) return SCAN_OK;
  if (!labels || !gscan::is_device_ptr(labels)) return SCAN_EINVAL;
  int32_t* base = nullptr;
  GS_TRY(scratch_address(&base));
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* parent = base;
  int64_t* ncores = (int64_t*)(base + NOALLOC_MAX_N);
  int* mu_dev = (int*)(base + NOALLOC_MAX_N + 6);
  double* eps_dev = (double*)(base + NOALLOC_MAX_N + 8);
  unsigned* status = (unsigned*)(base + NOALLOC_MAX_N + 10);
  // the scratch keeps the previous call's contents: reset what must start clear
  GS_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), s));
  GS_CUDA(cudaMemcpyAsync(mu_dev, &mu, sizeof(int), cudaMemcpyHostToDevice, s));
  GS_CUDA(cudaMemcpyAsync(eps_dev, &eps, sizeof(double), cudaMemcpyHostToDevice, s));
  GS_TRY(gscan::run_queries_prealloc(ix, 1, mu_dev, eps_dev, ncores, parent, labels, flags, s,
                                     status));
  unsigned st = 0;
  GS_CUDA(cudaMemcpyAsync(&st, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (st & gscan::DEV_LIMIT) return SCAN_ETIMEOUT;
  return SCAN_OK;
}
