/*
 * scan.h -- C ABI of the GB300 index-based SCAN library (libscan.so).
 *
 * The library builds the SCAN index of Tseng, Dhulipala and Shun, "Parallel
 * Index-Based Structural Graph Clustering and Its Approximation" (SIGMOD
 * 2021), on one NVIDIA GPU, and answers (mu, eps) clustering queries from it.
 *
 *   index = per-edge similarity sigma over closed neighbourhoods (Section 3.1),
 *           the neighbour order NO and the core order CO (Section 3.2,
 *           Algorithm 2), optionally with LSH-approximated similarities
 *           (Sections 5 and 6.3);
 *   query = GetCores / Cluster / AssignNonCores (Algorithms 3-5), with the
 *           union-find of Section 6.2 and the hub/outlier pass of Section 4.3.
 *
 * Conventions shared by every entry point
 *  - Every function returns a scan_status (0 = SCAN_OK, negative = error) and
 *    never aborts the process. scan_strerror() names a status.
 *  - Graphs are simple and undirected (Section 2.2): CSR with ascending
 *    adjacency lists, no self-loops, no duplicates, every arc u->v matched by
 *    v->u. Vertex ids are 0-based int32 (the paper numbers them 1..n).
 *  - Pointers passed in are borrowed for the duration of the call only, unless
 *    stated otherwise. Output buffers belong to the caller. "host or device"
 *    buffers are classified with cudaPointerGetAttributes: device (or managed)
 *    memory is written by kernels, anything else is treated as host memory and
 *    filled by a copy.
 *  - `stream` is a cudaStream_t cast to uintptr_t (0 = the legacy default
 *    stream). Work is enqueued on it; functions that return data to host
 *    memory synchronise it before returning.
 *  - Device memory is obtained from the allocator installed with
 *    scan_set_allocator (default: cudaMallocAsync/cudaFreeAsync on the
 *    stream). An allocation failure returns SCAN_ENOMEM and leaves no partial
 *    index behind.
 *  - Similarities are IEEE double. Cosine is c / sqrt((d_u+1)(d_v+1)) with
 *    one correctly rounded square root of the exact integer product and one
 *    correctly rounded division; Jaccard is c / (d_u + d_v + 2 - c); c is
 *    |N̄(u) ∩ N̄(v)|. The results are therefore bit-reproducible (weighted
 *    similarities are sums of products: see scan_index_build_weighted).
 */
#ifndef GB300_SCAN_H
#define GB300_SCAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SCAN_OK = 0,
  SCAN_EINVAL = -1,    /* bad argument (mu < 2, eps outside [0,1] or NaN, ...) */
  SCAN_ENOMEM = -2,    /* the allocator returned NULL */
  SCAN_EBADGRAPH = -3, /* CSR is not a simple undirected graph (Section 2.2) */
  SCAN_ECUDA = -4,     /* a CUDA runtime call failed */
  SCAN_ETIMEOUT = -5,  /* a bounded wait expired */
  SCAN_EBUSY = -6      /* serving: admission refused (memory or slots) */
} scan_status;

typedef enum { SCAN_COSINE = 0, SCAN_JACCARD = 1 } scan_sim_kind;

/* Query flags. */
enum { SCAN_Q_HUBS = 1 /* label unclustered vertices -2 (hub) or -1 (outlier), Section 4.3 */ };

/* Compressed sparse rows of a simple undirected graph (Section 2.2).
 * offsets: n+1 entries, int32 (offsets_64 = 0) or int64 (offsets_64 = 1);
 * adj: num_arcs int32 vertex ids, each list strictly ascending.
 * on_device = 1: both arrays are in device memory; 0: host memory (copied in). */
typedef struct scan_csr {
  int64_t n;
  int64_t num_arcs;
  const void* offsets;
  int offsets_64;
  const int32_t* adj;
  int on_device;
} scan_csr;

/* LSH index mode (Sections 5 and 6.3). With enabled = 0 the index is exact.
 * An edge is approximated iff both endpoints have degree > degree_threshold;
 * every other edge keeps its exact similarity.
 *  cosine  -> SimHash with simhash_bits (a multiple of 64, <= 4096) Rademacher
 *             hyperplanes; estimate max(0, cos(pi * hamming / bits)).
 *  Jaccard -> MinHash with minhash_k (power of two when minhash_kpartition = 1,
 *             <= 1024); k-partition (one-permutation) by default, estimate =
 *             equal non-empty bins / (k - bins empty in both); standard
 *             k-hash MinHash when minhash_kpartition = 0, estimate = equal / k.
 * Random signs and hashes are SplitMix64 outputs of `seed`. */
typedef struct scan_lsh_params {
  int enabled;
  int simhash_bits;
  int minhash_k;
  int minhash_kpartition;
  int degree_threshold;
  uint64_t seed;
} scan_lsh_params;

typedef struct scan_index scan_index; /* opaque, owned by the library */

/* Device memory hooks. alloc returns NULL on failure. Passing NULL for both
 * restores the default (cudaMallocAsync / cudaFreeAsync on the stream). The
 * hooks are process-wide; install them before any other call. */
typedef void* (*scan_alloc_fn)(size_t bytes, uintptr_t stream, void* ctx);
typedef void (*scan_free_fn)(void* ptr, size_t bytes, uintptr_t stream, void* ctx);
int scan_set_allocator(scan_alloc_fn alloc, scan_free_fn release, void* ctx);

/* Build the index (Algorithms 1-2; Section 6.1 for the oriented counting).
 * csr: borrowed; kind: similarity; lsh: NULL or enabled = 0 for the exact
 * index; *out receives a new handle (NULL on error). The CSR is checked: a
 * graph that is not simple and undirected returns SCAN_EBADGRAPH. Returns
 * after the build has completed on the stream. */
int scan_index_build(const scan_csr* csr, scan_sim_kind kind, const scan_lsh_params* lsh,
                     uintptr_t stream, scan_index** out);

/* scan_index_build with a choice of how the closed counts are obtained:
 *  SCAN_COUNTS_AUTO   - dense when n <= 65536 and the average degree is at
 *                       least n/16, else sparse (what scan_index_build does);
 *  SCAN_COUNTS_SPARSE - oriented triangle enumeration (Section 6.1);
 *  SCAN_COUNTS_DENSE  - ((A+I)^2)[u][v] = |N̄(u) ∩ N̄(v)| (Section 4.1.1) from
 *                       one bf16 GEMM with fp32 accumulation (exact: 0/1
 *                       operands, sums below 2^24); needs n <= 65536 (else
 *                       SCAN_EINVAL) and about 6 n^2 bytes of device memory.
 * Every choice gives the same index, bit for bit. */
#define SCAN_COUNTS_AUTO 0
#define SCAN_COUNTS_SPARSE 1
#define SCAN_COUNTS_DENSE 2
int scan_index_build_ex(const scan_csr* csr, scan_sim_kind kind, const scan_lsh_params* lsh,
                        int counts, uintptr_t stream, scan_index** out);

/* Build the index of a weighted graph with the weighted cosine similarity
 * (Section 4.1.1; WeightedCosineSim of Section 2.1.1): with w(x,x) = 1 and N̄
 * the closed neighbourhood,
 *   sigma(u,v) = sum over x in N̄(u) ∩ N̄(v) of w(u,x) w(v,x)
 *                / ( sqrt(sum over N̄(u) of w(u,x)^2) sqrt(sum over N̄(v) of w(v,x)^2) ),
 * i.e. (2 w(u,v) + sum over common neighbours x of w(u,x) w(v,x)) divided by
 * sqrt(1 + sum of w(u,x)^2) sqrt(1 + sum of w(v,x)^2) for an edge (u,v).
 * weights: num_arcs doubles aligned with csr->adj (weights[i] belongs to the
 * arc stored at adj[i]), on the device when csr->on_device, else on the
 * host; borrowed. Every weight must be finite and >= 0 and the two arcs of an
 * edge must carry the same weight, else SCAN_EINVAL (a graph that is not
 * simple and undirected returns SCAN_EBADGRAPH). The result is a cosine
 * index: queries, exports, modularity and the sweep work on it unchanged.
 * Counts are always sparse. lsh: NULL or disabled for the exact index, else
 * SimHash (simhash_bits, degree_threshold, seed as for scan_index_build) of
 * the weighted closed neighbourhoods: hyperplane j sums +-w(v,x) over N̄(v)
 * in double precision, v first, then N(v) in id order, and bit j is
 * [sum >= 0] (Sections 2.1.2 and 5).
 * Exact similarities are sums of floating-point products in an unspecified
 * order: each lies within (2 (d_u + d_v) + 16) units of 2^-53, relative,
 * of the value summed in id order without fused multiply-adds (and is not
 * bit-identical run to run for edges on many triangles); with integer
 * weights every sum is exact and so is the result. */
int scan_index_build_weighted(const scan_csr* csr, const double* weights,
                              const scan_lsh_params* lsh, uintptr_t stream, scan_index** out);

/* Build `count` independent indexes (one per graph) in one batched pass:
 * the graphs are packed into one device arena and every step runs once over
 * all of them; each handle then behaves exactly like one from
 * scan_index_build. out: array of `count` handles. */
int scan_index_build_batch(const scan_csr* graphs, int count, scan_sim_kind kind,
                           const scan_lsh_params* lsh, uintptr_t stream, scan_index** out);

/* Answer one (mu, eps) query (Algorithms 3-5). labels: n int32, host or
 * device. Label = smallest core id of the vertex's cluster; -1 unclustered;
 * with SCAN_Q_HUBS, -2 marks hubs. Borders join the most similar adjacent
 * eps-similar core, the smallest id on ties (Section 7.3.4). mu < 2 or eps
 * outside [0,1] returns SCAN_EINVAL; mu > maxdeg+1 gives no cores. */
int scan_query(scan_index* index, int mu, double eps, int32_t* labels, int flags,
               uintptr_t stream);

/* Answer q queries in one batched pass over the index. mu, eps: q entries
 * (host memory). labels: q*n int32 (row i = query i), host or device. */
int scan_query_batch(scan_index* index, int q, const int* mu, const double* eps,
                     int32_t* labels, int flags, uintptr_t stream);

/* The same query as scan_query, for callers that must not allocate device
 * memory while they answer it -- for example a service that has handed all
 * device memory to its own pool up front, or a latency-critical loop that
 * cannot afford an allocation stalling it. No counterpart exists in the
 * paper.
 *
 * Nothing is allocated: the per-call scratch (union-find parents for every
 * vertex plus a few words) is one array compiled into the library, so every
 * GPU that loads the library holds about 16 MiB for it until the process
 * exits. Limits and rules:
 *  - the index may have at most SCAN_NOALLOC_MAX_VERTICES vertices; a larger
 *    index returns SCAN_EINVAL;
 *  - labels must be device memory (n int32); host memory returns SCAN_EINVAL;
 *  - the first call on a device looks up the scratch address for that device
 *    (cudaGetSymbolAddress, with the device current) and keeps it for the
 *    life of the process; make that first call before any stream capture.
 *    Do not reset the device (cudaDeviceReset) while the library is loaded:
 *    a new context may place the array elsewhere, and the kept address would
 *    then be stale;
 *  - each call copies mu and eps from host memory to the scratch and
 *    synchronises `stream` before it returns;
 *  - every call on a device shares the same scratch, and the scratch keeps
 *    the last call's contents: calls whose work overlaps on the GPU race and
 *    give wrong labels, so issue them one after another.
 * Other arguments and results are those of scan_query. */
#define SCAN_NOALLOC_MAX_VERTICES 4194304
int scan_query_noalloc(scan_index* index, int mu, double eps, int32_t* labels, int flags,
                       uintptr_t stream);

/* Modularity (Section 7.2) of a clustering of the index's graph, with every
 * vertex of negative label (outlier, hub, unclustered) as a cluster of its
 * own:  Q = (arcs inside clusters) / 2m - sum over clusters of (sum of the
 * degrees in it)^2 / (2m)^2. labels: n int32, host or device, any cluster ids
 * in [0, n) (the labels of scan_query qualify); a label >= n returns
 * SCAN_EINVAL. The sums are exact 64-bit integers; *q receives the double
 * result. Synchronises `stream`. */
int scan_modularity(scan_index* index, const int32_t* labels, double* q, uintptr_t stream);

/* Parameter sweep (Section 7.3.4): for each of `count` pairs (mu[i], eps[i])
 * (host arrays, each pair valid for scan_query), the clustering without hub
 * marks and its modularity, written to q[i] (host). The paper's set Sigma is
 * mu in {2, 4, ..., 2^18} x eps in {.01, ..., .99}; the pair of highest
 * modularity is its choice of parameters. Queries run 32 at a time on the
 * GPU, each followed by its modularity passes. Synchronises `stream`. */
int scan_sweep(scan_index* index, int count, const int* mu, const double* eps, double* q,
               uintptr_t stream);

/* Copy the index out (test hook; any pointer may be NULL, each host or
 * device): sim[num_arcs] in CSR arc order, no_id/no_sim[num_arcs] (NO[v]
 * occupies the slots of v's CSR row), co_off[max_deg+1], co_id/co_thr
 * [num_arcs] (CO[mu] = entries co_off[mu-2] .. co_off[mu-1]). */
int scan_index_export(scan_index* index, double* sim, int32_t* no_id, double* no_sim,
                      int64_t* co_off, int32_t* co_id, double* co_thr);

/* Sizes of an index; any pointer may be NULL. */
int scan_index_info(scan_index* index, int64_t* n, int64_t* num_arcs, int32_t* max_deg,
                    size_t* device_bytes);

/* Release an index (NULL is ignored). */
void scan_index_free(scan_index* index);

/* Human-readable name of a status. */
const char* scan_strerror(int status);

/* Timings of the last build on this thread, milliseconds per phase measured
 * with CUDA events: [0] orientation, [1] counting, [2] similarity/keys,
 * [3] neighbour order, [4] core order, [5] LSH sketch+estimate, [6] total.
 * Also the duration of the dominant (counting) kernel. */
int scan_last_build_timings(double* ms7);

/* Duration (ms, CUDA events on the build's stream) of the last exact build's
 * CTA counting kernel on this thread: the oriented triangle enumeration over
 * the rows whose out-lists sit in a shared-memory table (Section 6.1 and the
 * hash intersection of Algorithm 1), the bulk of the counting step; 0 if the
 * last build did not run it. */
int scan_last_count_kernel_ms(double* ms);

/* Test hook for the index width of the counting kernels. Graphs with at
 * least 2^31 arcs are counted with 64-bit element indices and 32-bit (u,w)
 * counters; smaller ones with 32-bit indices and 16-bit counters. With
 * on != 0, every later build (process-wide) takes the 64-bit path, so that
 * path can be checked against the oracle on small graphs; the results are
 * identical either way. Returns SCAN_OK. */
int scan_set_wide_index(int on);

/* Number of CUDA kernels this library has launched in this process so far
 * (all threads); a benchmark reads it before and after a timed region. */
int scan_kernel_launches(uint64_t* count);

/* ---- Counting strategy per degree bucket, and its autotuner ----
 * No counterpart in the paper, which runs one merge-based intersection on a
 * multicore host (Section 6.1). Here the closed counts of every edge
 * (Section 3.1) come either from one tcgen05 matrix product for a dense
 * graph ((A+I)^2, Section 4.1.1) or from oriented triangle enumeration with
 * a hash table of the middle vertex's out-list, and how each graph and each
 * vertex is handled depends on its degree bucket:
 *   dense_div, dense_min_n  a graph of at least dense_min_n vertices with
 *              dense_div * arcs >= n^2 takes the dense path under the
 *              automatic choice (dense_div = 0: never; 0..1024,
 *              dense_min_n 2..65536);
 *   warp_deg   rows of at most this many positions whose out-list has at
 *              most 256 entries are handled by one warp with its own table;
 *              the others by a CTA sharing one table (32..4096);
 *   cta_chunk  CSR positions of a row per CTA work item (256..65536, a
 *              multiple of 32);
 *   long_list  suffixes of an out-list at least this long are streamed one
 *              at a time by a whole warp, shorter ones are concatenated
 *              (1..2^20);
 *   rounds     32-element rounds of loads in flight for the concatenated
 *              suffixes (4 or 8).
 * Every configuration gives bit-identical results; only the speed differs.
 * A build uses, in this order: the configuration set by
 * scan_set_count_config, the tuning table's entry for its class (the bit
 * length of the vertex count of its largest graph and of its average
 * degree, both known before any device work), or the defaults
 * {512, 32768, 64, 4, 16, 4096}. In a batched build the members that the
 * dense rule selects are built one by one on the dense path, the others
 * together. */
typedef struct scan_count_config {
  int warp_deg;
  int cta_chunk;
  int long_list;
  int rounds;
  int dense_div;
  int dense_min_n;
} scan_count_config;

/* Set (cfg) or clear (NULL) a process-wide configuration for every later
 * build; SCAN_EINVAL if a field is out of range. */
int scan_set_count_config(const scan_count_config* cfg);

/* Autotuner of the batched build: builds the `count` graphs with
 * scan_index_build_batch repeatedly (each configuration `reps` times, the
 * fastest counted), timing the whole build with CUDA events on `stream`,
 * and searches the configurations one parameter at a time (dense_div in
 * {0, 8, 16, 32, 64}, dense_min_n in {2048, 4096, 8192}, warp_deg in
 * {128, 256, 512, 1024, 2048}, cta_chunk in {1024, 2048, 4096, 8192},
 * long_list in {32, 64, 128, 256}, rounds in {4, 8}), keeping each change
 * that is faster. The winner is stored in the in-process tuning table under
 * the class of the batch, so later builds of that class use it. *best
 * receives it, *best_ms its build time, *default_ms that of the defaults
 * (any of the three may be NULL). Builds run on the calling thread; the
 * graphs follow the rules of scan_index_build_batch. */
int scan_autotune_batch(const scan_csr* graphs, int count, scan_sim_kind kind, int reps,
                        uintptr_t stream, scan_count_config* best, double* best_ms,
                        double* default_ms);

/* The configuration a build would use (see above): a single graph has
 * max_n = total_n = its vertex count; SCAN_EINVAL if total_n < max_n or a
 * size is negative. */
int scan_count_config_for(int64_t max_n, int64_t total_n, int64_t num_arcs,
                          scan_count_config* cfg);

/* Persist the tuning table as text (one line per class: vertex-count bits,
 * average-degree bits, warp_deg, cta_chunk, long_list, rounds, dense_div,
 * dense_min_n), load such a file (entries are added or replaced; a
 * malformed file changes nothing and returns SCAN_EINVAL), or empty the
 * table. */
int scan_tuning_save(const char* path);
int scan_tuning_load(const char* path);
int scan_tuning_clear(void);

/* The counting step of a sharded build (Section 3.1, closed counts; Section
 * 6.1, the degree orientation): every triangle u < v < w of the orientation
 * (order by degree, then id) has one middle vertex v, and this call counts
 * only the triangles whose middle vertex lies in [v_begin, v_end). For every
 * arc (x, y), counts[arc] receives the number of such triangles through the
 * edge {x, y} (both arcs of an edge get the same value). Ranks whose ranges
 * partition [0, n) and add their counts (one sum all-reduce) obtain
 * t(x, y) = |N(x) ∩ N(y)| for every arc; the closed count is t + 2.
 * csr: as for scan_index_build (host or device, checked the same way:
 * SCAN_EBADGRAPH). counts: num_arcs uint32 in CSR order, host or device,
 * written whole. 0 <= v_begin <= v_end <= n, else SCAN_EINVAL. Synchronises
 * `stream`. */
int scan_closed_counts_range(const scan_csr* csr, int64_t v_begin, int64_t v_end,
                             uint32_t* counts, uintptr_t stream);

/* The segmented sort of the neighbour and core orders (Algorithm 2), for
 * callers that assemble orders themselves, such as the sharded build, whose
 * ranks sort their runs of CO[mu] and merge the runs they receive. Every
 * segment [seg_off[i], seg_off[i+1]) of (keys, ids) is sorted in place by key
 * descending, then id ascending. keys: non-negative doubles (similarities);
 * ids: int32; seg_off: nseg+1 int64 offsets, non-decreasing within [0, total]
 * (checked on the device before any element is read or written: otherwise
 * SCAN_EINVAL and the arrays are unchanged); max_len: an upper bound of every
 * segment's length. All three arrays device memory (host pointers:
 * SCAN_EINVAL). Synchronises `stream`. Segments longer than 4096 are split
 * into buckets by a sample sort (sorted random samples give the splitters,
 * one scatter places every element in its bucket), then the buckets are
 * sorted in shared memory. */
int scan_sort_segments_desc(double* keys, int32_t* ids, const int64_t* seg_off, int64_t nseg,
                            int64_t total, int64_t max_len, uintptr_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GB300_SCAN_H */
