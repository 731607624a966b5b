// Internal declarations shared by the translation units of libscan.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <memory>
#include <vector>

#include "../../include/scan.h"

namespace gscan {

// Kernels launched by this library (every launch site is followed by GS_LAUNCH).
extern std::atomic<unsigned long long> g_kernel_launches;

// ------------------------------------------------------------ error plumbing
struct Err {
  int code = SCAN_OK;
  bool ok() const { return code == SCAN_OK; }
};

#define GS_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return (int)SCAN_ECUDA;      \
  } while (0)

#define GS_LAUNCH()                                     \
  do {                                                  \
    ::gscan::g_kernel_launches.fetch_add(1, std::memory_order_relaxed); \
    cudaError_t e_ = cudaGetLastError();                \
    if (e_ != cudaSuccess) return (int)SCAN_ECUDA;      \
  } while (0)

#define GS_TRY(expr)                                    \
  do {                                                  \
    int r_ = (expr);                                    \
    if (r_ != SCAN_OK) return r_;                       \
  } while (0)

// Device status word bits (written by kernels, read by the host).
enum : unsigned {
  DEV_BADGRAPH = 1u,   // unsorted / duplicate / self-loop / out-of-range / asymmetric
  DEV_LIMIT = 2u,      // a bounded loop gave up
  DEV_OVERFLOW = 4u,   // a fixed-capacity structure would overflow
  DEV_BADWEIGHT = 8u,  // a weight negative, not finite, or not symmetric
};

// ------------------------------------------------------------ device memory
// All device allocations go through the installed hooks (or the stream-ordered
// CUDA allocator). A Pool remembers what it handed out so a failed build can
// release everything.
void* dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void* p, size_t bytes, cudaStream_t s);

struct Pool {
  cudaStream_t s;
  struct Blk { void* p; size_t b; };
  std::vector<Blk> blocks;
  explicit Pool(cudaStream_t st) : s(st) {}
  ~Pool() { release_all(); }
  template <class T>
  T* get(size_t count) {
    size_t b = count * sizeof(T);
    if (b == 0) b = 16;
    void* p = dev_alloc(b, s);
    if (p) blocks.push_back({p, b});
    return (T*)p;
  }
  void put(void* p) {
    for (size_t i = 0; i < blocks.size(); ++i)
      if (blocks[i].p == p) {
        dev_free(p, blocks[i].b, s);
        blocks[i] = blocks.back();
        blocks.pop_back();
        return;
      }
  }
  void release_all() {
    for (auto& b : blocks) dev_free(b.p, b.b, s);
    blocks.clear();
  }
  // hand ownership of every block to the caller (the index)
  std::vector<Blk> detach() {
    std::vector<Blk> out;
    out.swap(blocks);
    return out;
  }
};

// ------------------------------------------------------------ the index
struct IndexData {
  int64_t n = 0, arcs = 0;
  int32_t maxdeg = 0;
  int kind = SCAN_COSINE;
  int lsh = 0;
  // device arrays
  int64_t* off = nullptr;    // n+1
  int32_t* deg = nullptr;    // n
  int32_t* adj = nullptr;    // arcs (id-sorted lists)
  int32_t* no_id = nullptr;  // arcs
  double* no_sim = nullptr;  // arcs
  int64_t* co_off = nullptr; // maxdeg+1
  int32_t* co_id = nullptr;  // arcs
  double* co_thr = nullptr;  // arcs
  unsigned* status = nullptr;  // one device status word
  std::vector<Pool::Blk> blocks;
  std::shared_ptr<void> arena;  // batched builds: the arena shared by all graphs' views
  size_t bytes = 0;
  cudaStream_t home = 0;
};

// ------------------------------------------------------------ kernels' host launchers
// Each returns a scan_status; all work is enqueued on `s`.

// Degrees, CSR checks (sorted, in range, no self-loops), max degree.
int launch_degrees(const int64_t* off, const int32_t* adj, int64_t n, int64_t arcs, int32_t* deg,
                   int32_t* maxdeg_dev, unsigned* status, Pool& pool, cudaStream_t s);

// Orientation by (degree, id), in place: out(v) = oadj[off[v] .. off[v]+od[v]),
// in id order; the in-neighbours of v fill the rest of its slot range,
// oadj[off[v]+od[v] .. off[v+1]), in descending id order; opos = position of
// each arc inside v's CSR row.
// max_od_dev receives the largest out-degree, sum_od_dev the number of out-arcs.
int launch_orient(const int64_t* off, const int32_t* adj, const int32_t* deg, int64_t n,
                  int64_t arcs, Pool& pool, int32_t** od, int32_t** oadj, int32_t** opos,
                  int32_t* max_od_dev, unsigned long long* sum_od_dev, cudaStream_t s);

// Counting strategy per degree bucket (a tuning point): a graph of at least
// dense_min_n vertices with dense_div * arcs >= n^2 takes the dense GEMM
// path (dense_div = 0: never); otherwise, rows of at most warp_deg positions
// with out-lists of at most 256 entries go to the warp kernel, the others to
// the CTA kernel in items of cta_chunk CSR positions; suffixes of at least
// long_list entries are streamed one at a time; rounds (4 or 8) of 32-element
// loads stay in flight for the short ones.
constexpr int64_t DENSE_MIN_N = 4096;
struct CountCfg {
  int warp_deg = 512;
  int cta_chunk = 32768;
  int long_list = 64;
  int rounds = 4;
  int dense_div = 16;
  int dense_min_n = (int)DENSE_MIN_N;
};
// The configuration of a build (a batch: its largest graph has n_max
// vertices, all of them n_total vertices and arcs arcs): a process or thread
// override, else the tuning table's entry for its class, else the defaults.
CountCfg count_config_for(int64_t n_max, int64_t n_total, int64_t arcs);

// Closed counts of every edge by oriented triangle enumeration, then the
// similarity of every CSR arc written to sim_csr (the unsorted NO). With
// lsh_T >= 0, edges whose endpoints both have degree > lsh_T are left for the
// LSH estimate (their sim_csr entries are overwritten later). Only the
// triangles whose middle vertex lies in [v0, v1) are counted (v1 < 0: n);
// with counts_out, the triangle count of every arc is written there (CSR
// order, zeroed by the caller) instead of the similarities.
int launch_closed_counts_and_sims(int kind, const int64_t* off, const int32_t* adj,
                                  const int32_t* deg, int64_t n, int64_t arcs, const int32_t* od,
                                  int32_t* oadj, int32_t* opos, int32_t maxdeg,
                                  int32_t max_od, int lsh_T, const double* wcsr, double* sim_csr,
                                  unsigned* status, Pool& pool, cudaStream_t s, float* count_ms,
                                  const CountCfg& cfg, int64_t v0 = 0, int64_t v1 = -1,
                                  uint32_t* counts_out = nullptr);

// Sort every segment [seg_off[i], seg_off[i+1]) of (key, val) pairs by key
// descending, then val ascending. Keys are non-negative doubles viewed as
// uint64. max_len bounds every segment length.
int segmented_sort_desc(uint64_t* key, int32_t* val, const int64_t* seg_off, int64_t nseg,
                        int64_t total, int64_t max_len, Pool& pool, cudaStream_t s);

// Core order from the neighbour order (Algorithm 2, MakeCoreOrder).
int build_core_order(IndexData& ix, Pool& pool, cudaStream_t s);
// The same for G graphs packed in one vertex range: vb[G+1] vertex bases,
// maxdeg[G]; co_off_all[sum maxdeg + 1] absolute offsets; co_id local ids.
int build_core_order_multi(int64_t N, int64_t A, const int64_t* off, const int32_t* deg,
                           const uint64_t* no_key, const std::vector<int64_t>& vb,
                           const std::vector<int32_t>& maxdeg, int64_t* co_off_all,
                           int32_t* co_id, uint64_t* co_key, Pool& pool, cudaStream_t s);

// Dense path (dense.cu): closed counts of every arc as ((A+I)^2)[u][v] by one
// hand-written tcgen05 bf16 GEMM with fp32 accumulation, the similarities
// written by its epilogue; for graphs of at most DENSE_MAX_N vertices, and
// chosen automatically by the rule of the counting configuration.
constexpr int64_t DENSE_MAX_N = 65536;
bool dense_counts_pay(int64_t n, int64_t arcs, const CountCfg& cfg);
int dense_counts_and_sims(int kind, const int64_t* off, const int32_t* adj, const int32_t* deg,
                          int64_t n, int lsh_T, double* sim_csr, unsigned* status, Pool& pool,
                          cudaStream_t s, float* count_ms);

// Queries (Algorithms 3-5). status_dev: a zeroed device word that receives
// DEV_LIMIT if a bounded union-find loop gave up.
int run_queries(const IndexData& ix, int q, const int* mu, const double* eps, int32_t* labels_dev,
                int flags, Pool& pool, cudaStream_t s, unsigned* status_dev);

// Launch sequence of a batch of Q queries on device arrays: mu/eps hold Q
// entries, nc 2Q+1 (core counts and their prefix sums), parent Q*n; labels either Q*n contiguous (lab_ptrs null) or Q
// device destinations listed in lab_ptrs.
int launch_query_batch(const IndexData& ix, int Q, const int* mu, const double* eps, int64_t* nc,
                       int32_t* parent, int32_t* labels, int32_t* const* lab_ptrs, int flags,
                       cudaStream_t s, unsigned* status_dev);

// run_queries with caller-supplied device scratch: mu_dev/eps_dev hold Q
// entries, nc_dev 2Q+1, parent Q*n; nothing is allocated.
int run_queries_prealloc(const IndexData& ix, int Q, const int* mu_dev, const double* eps_dev,
                         int64_t* nc_dev, int32_t* parent, int32_t* labels_dev, int flags,
                         cudaStream_t s, unsigned* status_dev);

// Whole index build into ix (scan_api.cu); on error every block is released.
int build_index(const scan_csr* csr, int kind, const scan_lsh_params* lsh, cudaStream_t s,
                IndexData* ix);
// Release an index's device memory.
void free_index_data(IndexData* ix);
// Device footprint estimate of a build (temporaries included), bytes.
size_t build_footprint(int64_t n, int64_t arcs);
// Host or device pointer?
bool is_device_ptr(const void* p);

// LSH mode: overwrite the similarities of approximated arcs.
int lsh_apply(const scan_lsh_params& p, int kind, const int64_t* off, const int32_t* adj,
              const int32_t* deg, int64_t n, int64_t arcs, const int32_t* row, int64_t nH,
              double* no_sim, Pool& pool, cudaStream_t s,
              const double* wcsr = nullptr);
int lsh_select(const int64_t* off, const int32_t* adj, const int32_t* deg, int64_t n,
               int threshold, int32_t* row, int64_t* nH_host, Pool& pool, cudaStream_t s);

// Device-wide exclusive scan of int64 counts (n entries -> n+1 offsets).
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, Pool& pool, cudaStream_t s);
int exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, Pool& pool,
                              cudaStream_t s);

// Streaming multiprocessors of the current device (looked up once per
// device); grids are sized in multiples of it.
int sm_count();

// Per-thread record of the last build's phase timings, and of the duration
// of its CTA counting kernel (k_triangles over the shared-table rows).
void record_timings(const double* ms7);
void record_kernel_ms(double ms);

// scan_set_wide_index: counting with 64-bit element indices at any size.
bool force_wide_index();

}  // namespace gscan

struct scan_index {
  gscan::IndexData d;
};
