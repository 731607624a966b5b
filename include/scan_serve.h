/*
 * scan_serve.h -- continuous-batching request loop over resident SCAN indexes.
 *
 * No counterpart in the paper: the paper answers one (mu, eps) query at a time
 * on a multicore host (Algorithms 3-5). This runtime keeps indexes resident on
 * one GPU and serves a stream of (mu, eps) queries and whole index builds:
 *
 *  - queries that arrive while a batch is on the GPU are admitted into the
 *    next batch as soon as the previous one completes (continuous batching);
 *    each batch is one scan_query_batch-style pass (one launch per phase for
 *    all of its queries, sharing the CO/NO reads) on the server's query stream;
 *  - build requests run on a separate build stream, so their kernels overlap
 *    with query batches; a build is admitted only when its estimated device
 *    footprint fits the memory budget next to the indexes already built;
 *  - every request gets a ticket; scan_serve_wait blocks (with a time limit)
 *    until it completes. Results are identical to the same request made alone:
 *    the server's builds are unweighted (exact mode is deterministic bit for
 *    bit), and a query's labels depend only on its index, so queries on a
 *    weighted index (built outside the server, whose similarities may differ
 *    in the last bits from one build to the next) are identical alone and in
 *    the mix as well.
 *
 * Ownership: the CSR arrays of a build request and the label buffer of a query
 * must stay valid until the ticket completes. Indexes built by the server
 * belong to the caller once scan_serve_wait returns them. All functions return
 * a scan_status (include/scan.h).
 */
#ifndef GB300_SCAN_SERVE_H
#define GB300_SCAN_SERVE_H

#include "scan.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scan_server scan_server;

typedef struct scan_serve_params {
  size_t memory_budget_bytes; /* device bytes builds may use (0 = no limit) */
  int max_batch;              /* queries per batch (1 = one launch per query; 0 = 64) */
  int max_pending;            /* queued requests before submit returns SCAN_EBUSY (0 = 1<<20) */
  int device;                 /* CUDA device ordinal */
} scan_serve_params;

/* Start the server threads and streams. */
int scan_serve_create(const scan_serve_params* params, scan_server** out);

/* Queue one query on `index` (which must stay alive until the ticket
 * completes). labels: n int32, host or device; flags: SCAN_Q_HUBS or 0. */
int scan_serve_submit_query(scan_server* srv, scan_index* index, int mu, double eps,
                            int32_t* labels, int flags, uint64_t* ticket);

/* Queue one index build. Returns SCAN_EBUSY when the request alone exceeds
 * the memory budget; otherwise it waits in the queue until it fits. */
int scan_serve_submit_build(scan_server* srv, const scan_csr* csr, scan_sim_kind kind,
                            const scan_lsh_params* lsh, uint64_t* ticket);

/* Wait up to timeout_ms (< 0: no limit) for a ticket. Returns the request's
 * own status, or SCAN_ETIMEOUT if it has not completed (the ticket stays
 * valid). For a build, *built receives the new index (may be NULL to free
 * it immediately). A completed ticket can be waited on once. */
int scan_serve_wait(scan_server* srv, uint64_t ticket, int timeout_ms, scan_index** built);

/* Latency percentiles (submit -> completion, milliseconds) and throughput of
 * the queries completed since creation or the last reset. */
int scan_serve_stats(scan_server* srv, double* p50_ms, double* p99_ms, double* qps,
                     int64_t* completed);
int scan_serve_reset_stats(scan_server* srv);

/* Open-loop replay of a request trace, driven by a C++ thread so the arrival
 * times do not depend on the caller's language runtime. Query i is submitted
 * at q_arrival_s[i] seconds after the start, build j at b_arrival_s[j].
 *
 * Label rows (each n int32): query i writes row i % R of `labels`, host or
 * device. A row is handed to a new query only after the query that used it
 * before has completed, so every query in flight owns its row; when the row
 * of the next arrival is still busy, the replay waits for it, and that wait
 * counts in the query's latency.
 *   labels != NULL, label_rows = R > 0: a caller-owned ring of R rows;
 *   labels != NULL, label_rows = 0: nq rows, one per query;
 *   labels == NULL: the library allocates a device ring of label_rows rows
 *     (0 = max(2 * max_batch, 128), capped at nq) for the call and releases
 *     it before returning.
 * latency_ms[i] receives the time from query i's scheduled arrival to its
 * completion (-1 if it did not complete). Returns after every request
 * completed or after timeout_ms (SCAN_ETIMEOUT). label_rows < 0: SCAN_EINVAL.
 * (No counterpart in the paper: a serving harness for the query path of
 * Algorithms 3-5.) */
int scan_serve_replay(scan_server* srv, scan_index* index, int64_t nq, const double* q_arrival_s,
                      const int* q_mu, const double* q_eps, int flags, int32_t* labels,
                      int64_t label_rows, double* latency_ms, int64_t nb,
                      const double* b_arrival_s, const scan_csr* b_graphs, scan_sim_kind b_kind,
                      int timeout_ms);

/* Stop the threads, finish queued work and release the server. */
void scan_serve_destroy(scan_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* GB300_SCAN_SERVE_H */
