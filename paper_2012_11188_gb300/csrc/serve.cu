// Continuous-batching request loop over resident SCAN indexes (include/scan_serve.h).
//
// Two worker threads own the CUDA streams:
//  - the query worker takes every query queued for one (index, flags) pair, up
//    to max_batch (default 64), and answers them with one batched pass (one
//    launch per phase for the whole batch, labels written straight into device
//    destinations; host destinations go through staging rows, copied out on a
//    third stream while the next batch's kernels run; a host function on that
//    stream completes the batch). At most two batches are in flight; queries
//    that arrive meanwhile wait in the queue and join the next batch.
//  - the build worker admits build requests in arrival order when their
//    footprint fits the memory budget and the device's free memory, and builds
//    them on its own stream, overlapping with the query batches.
// Latencies are measured on the host from submit to completion (the trace
// replay measures from each query's scheduled arrival instead).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/scan_serve.h"
#include "scan_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  bool is_build = false;
  // query
  scan_index* ix = nullptr;
  int mu = 0;
  double eps = 0;
  int32_t* labels = nullptr;
  int flags = 0;
  // build
  scan_csr csr{};
  int kind = 0;
  bool has_lsh = false;
  scan_lsh_params lsh{};
  size_t est = 0;
  // completion
  int status = SCAN_OK;
  bool done = false;
  scan_index* built = nullptr;
  Clock::time_point t_submit, t_done;
};

}  // namespace

struct scan_server {
  scan_serve_params p{};
  int device = 0;
  cudaStream_t qs = nullptr, bs = nullptr;
  cudaStream_t cs = nullptr;  // copies of host-bound labels, and batch completions
  std::mutex mu;
  std::condition_variable cv_q, cv_b, cv_done, cv_slot;
  int batches_in_flight = 0;  // query batches launched and not yet completed (at most 2)
  std::deque<Request*> qq, bq;
  std::unordered_map<uint64_t, Request*> reqs;
  uint64_t next_ticket = 1;
  size_t inflight_build_bytes = 0;
  bool stop = false;
  std::thread qt, bt;
  // stats
  std::vector<double> lat_ms;
  Clock::time_point stats_t0;
  bool stats_started = false;
  Clock::time_point stats_last;
};

namespace {

void finish(scan_server* s, Request* r, int status) {
  std::lock_guard<std::mutex> lk(s->mu);
  r->status = status;
  r->done = true;
  r->t_done = Clock::now();
  if (!r->is_build) {
    s->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    s->stats_last = r->t_done;
  }
  s->cv_done.notify_all();
}

// Scratch of the query worker, kept across batches and grown on demand:
// parents (cap x n), mu/eps/core counts and the table of label destinations,
// and two sets of what a batch in flight owns until its copies are done:
// staging rows for host destinations, a device status word, its pinned host
// copy and the event that marks its kernels done.
struct QueryScratch {
  int cap = 0;
  int64_t n = 0;
  int32_t* parent = nullptr;
  int32_t** ptrs = nullptr;
  int* mu = nullptr;
  double* eps = nullptr;
  int64_t* nc = nullptr;
  unsigned* status[2] = {nullptr, nullptr};
  unsigned* status_host = nullptr;  // pinned, 2 words
  int32_t* staging[2] = {nullptr, nullptr};
  int staging_rows[2] = {0, 0};
  cudaEvent_t kern_done[2] = {nullptr, nullptr};
  std::vector<std::pair<void*, size_t>> held;  // every device block, for release
  template <class T>
  T* get(size_t count, cudaStream_t s) {
    const size_t b = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
    void* p = gscan::dev_alloc(b, s);
    if (p) held.emplace_back(p, b);
    return (T*)p;
  }
  void release(cudaStream_t s) {
    for (auto& h : held) gscan::dev_free(h.first, h.second, s);
    if (status_host) cudaFreeHost(status_host);
    for (auto& e : kern_done)
      if (e) cudaEventDestroy(e);
    *this = QueryScratch();
  }
  int ensure(int c, int64_t nn, cudaStream_t s, cudaStream_t cs) {
    if (c <= cap && nn <= n) return SCAN_OK;
    if (cap > 0) {
      // a batch may still be in flight on the old scratch: drain both streams
      cudaStreamSynchronize(s);
      cudaStreamSynchronize(cs);
    }
    release(s);
    cap = c;
    n = nn;
    parent = get<int32_t>((size_t)c * (size_t)nn, s);
    ptrs = get<int32_t*>(c, s);
    mu = get<int>(c, s);
    eps = get<double>(c, s);
    nc = get<int64_t>(2 * (size_t)c + 1, s);
    status[0] = get<unsigned>(1, s);
    status[1] = get<unsigned>(1, s);
    if (cudaHostAlloc((void**)&status_host, 2 * sizeof(unsigned), cudaHostAllocDefault) !=
        cudaSuccess)
      status_host = nullptr;
    bool ev_ok = true;
    for (auto& e : kern_done)
      ev_ok &= cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!parent || !ptrs || !mu || !eps || !nc || !status[0] || !status[1] || !status_host ||
        !ev_ok) {
      release(s);
      return SCAN_ENOMEM;
    }
    return SCAN_OK;
  }
  int ensure_staging(int set, int rows, cudaStream_t s) {
    if (rows <= staging_rows[set]) return SCAN_OK;
    staging[set] = get<int32_t>((size_t)rows * (size_t)n, s);  // the smaller one is released with the rest
    if (!staging[set]) return SCAN_ENOMEM;
    staging_rows[set] = rows;
    return SCAN_OK;
  }
};

// A launched batch, completed by a host function on the copy stream once its
// kernels and its label copies are done.
struct BatchDone {
  scan_server* s;
  std::vector<Request*> batch;
  const unsigned* status_host;
};

void finish_batch(scan_server* s, const std::vector<Request*>& batch, int rc) {
  for (Request* r : batch) finish(s, r, rc);
  std::lock_guard<std::mutex> lk(s->mu);
  --s->batches_in_flight;
  s->cv_slot.notify_all();
}

// Host function (no CUDA calls): the batch's status word has landed.
void CUDART_CB on_batch_done(void* p) {
  BatchDone* d = static_cast<BatchDone*>(p);
  const int rc = (*d->status_host & gscan::DEV_LIMIT) ? SCAN_ETIMEOUT : SCAN_OK;
  finish_batch(d->s, d->batch, rc);
  delete d;
}

// Launch one batch: kernels on the query stream, writing device destinations
// directly and host destinations into the staging rows of set `set`; then,
// on the copy stream, once the kernels are done, the staging rows go to the
// host buffers, the status word to pinned memory, and a host function
// completes the requests. The next batch's kernels overlap these copies; a
// set is reused two batches later, when the copy stream has drained it.
int launch_batch(scan_server* s, QueryScratch& qs, const std::vector<Request*>& batch, int set) {
  const gscan::IndexData& d = batch[0]->ix->d;
  const int Q = (int)batch.size();
  GS_TRY(qs.ensure(std::max(Q, s->p.max_batch > 0 ? s->p.max_batch : 64), d.n, s->qs, s->cs));
  std::vector<int> mus(Q);
  std::vector<double> epss(Q);
  std::vector<int32_t*> dst(Q);
  std::vector<int> host_rows;
  for (int i = 0; i < Q; ++i) {
    mus[i] = batch[i]->mu;
    epss[i] = batch[i]->eps;
    if (gscan::is_device_ptr(batch[i]->labels)) {
      dst[i] = batch[i]->labels;
    } else {
      host_rows.push_back(i);
      dst[i] = nullptr;
    }
  }
  // the staging rows of this set belonged to the batch before the previous
  // one, which has completed (at most two batches are in flight)
  if (!host_rows.empty()) {
    GS_TRY(qs.ensure_staging(set, (int)host_rows.size(), s->qs));
    for (size_t r = 0; r < host_rows.size(); ++r)
      dst[host_rows[r]] = qs.staging[set] + r * (size_t)d.n;
  }
  GS_CUDA(cudaMemcpyAsync(qs.mu, mus.data(), sizeof(int) * Q, cudaMemcpyHostToDevice, s->qs));
  GS_CUDA(cudaMemcpyAsync(qs.eps, epss.data(), sizeof(double) * Q, cudaMemcpyHostToDevice, s->qs));
  GS_CUDA(cudaMemcpyAsync(qs.ptrs, dst.data(), sizeof(int32_t*) * Q, cudaMemcpyHostToDevice, s->qs));
  GS_CUDA(cudaMemsetAsync(qs.status[set], 0, sizeof(unsigned), s->qs));
  GS_TRY(gscan::launch_query_batch(d, Q, qs.mu, qs.eps, qs.nc, qs.parent, nullptr, qs.ptrs,
                                   batch[0]->flags, s->qs, qs.status[set]));
  GS_CUDA(cudaEventRecord(qs.kern_done[set], s->qs));
  GS_CUDA(cudaStreamWaitEvent(s->cs, qs.kern_done[set], 0));
  for (size_t r = 0; r < host_rows.size(); ++r)
    GS_CUDA(cudaMemcpyAsync(batch[host_rows[r]]->labels, qs.staging[set] + r * (size_t)d.n,
                            sizeof(int32_t) * (size_t)d.n, cudaMemcpyDeviceToHost, s->cs));
  GS_CUDA(cudaMemcpyAsync(qs.status_host + set, qs.status[set], sizeof(unsigned),
                          cudaMemcpyDeviceToHost, s->cs));
  BatchDone* done = new (std::nothrow) BatchDone{s, batch, qs.status_host + set};
  if (!done) return SCAN_ENOMEM;
  if (cudaLaunchHostFunc(s->cs, on_batch_done, done) != cudaSuccess) {
    delete done;
    return SCAN_ECUDA;
  }
  return SCAN_OK;
}

void query_worker(scan_server* s) {
  cudaSetDevice(s->device);
  const int max_batch = s->p.max_batch > 0 ? s->p.max_batch : 64;
  QueryScratch qs;
  std::vector<Request*> batch;
  int set = 0;
  for (;;) {
    batch.clear();
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_q.wait(lk, [&] { return s->stop || !s->qq.empty(); });
      if (s->qq.empty() && s->stop) break;
      // at most two batches in flight: the next one may overlap the copies
      // of the previous one, and queries arriving meanwhile join it
      s->cv_slot.wait(lk, [&] { return s->batches_in_flight < 2; });
      // everything queued for the front request's (index, flags), up to max_batch
      scan_index* ix = s->qq.front()->ix;
      const int flags = s->qq.front()->flags;
      for (auto it = s->qq.begin(); it != s->qq.end() && (int)batch.size() < max_batch;) {
        if ((*it)->ix == ix && (*it)->flags == flags) {
          batch.push_back(*it);
          it = s->qq.erase(it);
        } else {
          ++it;
        }
      }
      ++s->batches_in_flight;
    }
    if (batch[0]->ix->d.n == 0) {
      finish_batch(s, batch, SCAN_OK);
      continue;
    }
    const int rc = launch_batch(s, qs, batch, set);
    if (rc != SCAN_OK) {
      // nothing was handed to the copy stream for this batch: complete it now
      cudaStreamSynchronize(s->qs);
      cudaStreamSynchronize(s->cs);
      finish_batch(s, batch, rc);
    }
    set ^= 1;
  }
  cudaStreamSynchronize(s->qs);
  cudaStreamSynchronize(s->cs);  // the last batches' host functions have run
  qs.release(s->qs);
  cudaStreamSynchronize(s->qs);
}

size_t free_device_bytes() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 0;
  return fr;
}

void build_worker(scan_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_b.wait(lk, [&] { return s->stop || !s->bq.empty(); });
      if (s->bq.empty() && s->stop) return;
      r = s->bq.front();
      s->bq.pop_front();
      s->inflight_build_bytes += r->est;
    }
    // admission by device memory: wait (bounded) for room next to resident data
    int rc = SCAN_OK;
    for (int tries = 0; r->est > free_device_bytes(); ++tries) {
      if (tries > 2000) { rc = SCAN_EBUSY; break; }  // ~10 s
      std::this_thread::sleep_for(std::chrono::milliseconds(5));
    }
    scan_index* h = nullptr;
    if (rc == SCAN_OK) {
      h = new (std::nothrow) scan_index();
      if (!h) rc = SCAN_ENOMEM;
    }
    if (rc == SCAN_OK) {
      rc = gscan::build_index(&r->csr, r->kind, r->has_lsh ? &r->lsh : nullptr, s->bs, &h->d);
      if (rc != SCAN_OK) { delete h; h = nullptr; }
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->inflight_build_bytes -= r->est;
      r->built = h;
    }
    finish(s, r, rc);
  }
}

int submit(scan_server* s, Request* r, uint64_t* ticket) {
  std::lock_guard<std::mutex> lk(s->mu);
  const int max_pending = s->p.max_pending > 0 ? s->p.max_pending : (1 << 20);
  if ((int)(s->qq.size() + s->bq.size()) >= max_pending) return SCAN_EBUSY;
  r->ticket = s->next_ticket++;
  r->t_submit = Clock::now();
  if (!r->is_build && !s->stats_started) {
    s->stats_started = true;
    s->stats_t0 = r->t_submit;
  }
  s->reqs[r->ticket] = r;
  if (r->is_build) {
    s->bq.push_back(r);
    s->cv_b.notify_one();
  } else {
    s->qq.push_back(r);
    s->cv_q.notify_one();
  }
  *ticket = r->ticket;
  return SCAN_OK;
}

}  // namespace

extern "C" {

int scan_serve_create(const scan_serve_params* params, scan_server** out) {
  if (!out) return SCAN_EINVAL;
  *out = nullptr;
  scan_server* s = new (std::nothrow) scan_server();
  if (!s) return SCAN_ENOMEM;
  if (params) s->p = *params;
  if (s->p.max_batch < 0 || s->p.max_pending < 0) { delete s; return SCAN_EINVAL; }
  s->device = s->p.device;
  if (cudaSetDevice(s->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->qs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->bs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking) != cudaSuccess) {
    if (s->qs) cudaStreamDestroy(s->qs);
    if (s->bs) cudaStreamDestroy(s->bs);
    delete s;
    return SCAN_ECUDA;
  }
  s->qt = std::thread(query_worker, s);
  s->bt = std::thread(build_worker, s);
  *out = s;
  return SCAN_OK;
}

int scan_serve_submit_query(scan_server* s, scan_index* index, int mu, double eps, int32_t* labels,
                            int flags, uint64_t* ticket) {
  if (!s || !index || !ticket || (!labels && index->d.n > 0)) return SCAN_EINVAL;
  if (mu < 2 || !(eps >= 0.0 && eps <= 1.0) || (flags & ~SCAN_Q_HUBS)) return SCAN_EINVAL;
  Request* r = new (std::nothrow) Request();
  if (!r) return SCAN_ENOMEM;
  r->ix = index;
  r->mu = mu;
  r->eps = eps;
  r->labels = labels;
  r->flags = flags;
  const int rc = submit(s, r, ticket);
  if (rc != SCAN_OK) delete r;
  return rc;
}

int scan_serve_submit_build(scan_server* s, const scan_csr* csr, scan_sim_kind kind,
                            const scan_lsh_params* lsh, uint64_t* ticket) {
  if (!s || !csr || !ticket) return SCAN_EINVAL;
  if (csr->n < 0 || csr->num_arcs < 0) return SCAN_EINVAL;
  Request* r = new (std::nothrow) Request();
  if (!r) return SCAN_ENOMEM;
  r->is_build = true;
  r->csr = *csr;
  r->kind = (int)kind;
  if (lsh) { r->has_lsh = true; r->lsh = *lsh; }
  r->est = gscan::build_footprint(csr->n, csr->num_arcs);
  if (s->p.memory_budget_bytes && r->est > s->p.memory_budget_bytes) {
    delete r;
    return SCAN_EBUSY;  // would never fit
  }
  const int rc = submit(s, r, ticket);
  if (rc != SCAN_OK) delete r;
  return rc;
}

int scan_serve_wait(scan_server* s, uint64_t ticket, int timeout_ms, scan_index** built) {
  if (!s) return SCAN_EINVAL;
  if (built) *built = nullptr;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return SCAN_EINVAL;
  Request* r = it->second;
  auto pred = [&] { return r->done; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, pred);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
    return SCAN_ETIMEOUT;
  }
  const int rc = r->status;
  scan_index* h = r->built;
  s->reqs.erase(it);
  lk.unlock();
  if (built) *built = h;
  else if (h) scan_index_free(h);
  delete r;
  return rc;
}

int scan_serve_stats(scan_server* s, double* p50_ms, double* p99_ms, double* qps, int64_t* completed) {
  if (!s) return SCAN_EINVAL;
  std::vector<double> v;
  double span = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    v = s->lat_ms;
    if (s->stats_started && !v.empty())
      span = std::chrono::duration<double>(s->stats_last - s->stats_t0).count();
  }
  auto pct = [&](double q) {
    if (v.empty()) return 0.0;
    size_t k = (size_t)(q * (double)(v.size() - 1) + 0.5);
    std::nth_element(v.begin(), v.begin() + k, v.end());
    return v[k];
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (qps) *qps = span > 0 ? (double)v.size() / span : 0.0;
  if (completed) *completed = (int64_t)v.size();
  return SCAN_OK;
}

int scan_serve_reset_stats(scan_server* s) {
  if (!s) return SCAN_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat_ms.clear();
  s->stats_started = false;
  return SCAN_OK;
}

int scan_serve_replay(scan_server* s, scan_index* index, int64_t nq, const double* q_arrival_s,
                      const int* q_mu, const double* q_eps, int flags, int32_t* labels,
                      int64_t label_rows, double* latency_ms, int64_t nb,
                      const double* b_arrival_s, const scan_csr* b_graphs, scan_sim_kind b_kind,
                      int timeout_ms) {
  if (!s || !index || nq < 0 || nb < 0 || label_rows < 0) return SCAN_EINVAL;
  if (nq > 0 && (!q_arrival_s || !q_mu || !q_eps)) return SCAN_EINVAL;
  if (nb > 0 && (!b_arrival_s || !b_graphs)) return SCAN_EINVAL;
  const int64_t n = index->d.n;
  const int max_batch = s->p.max_batch > 0 ? s->p.max_batch : 64;
  // Label rows: query i writes row i % rows. A row is handed to a new query
  // only after the query that used it before has completed, so every query in
  // flight has a row of its own.
  int64_t rows = label_rows;
  if (labels && rows == 0) rows = std::max<int64_t>(nq, 1);  // one row per query
  if (!labels && rows == 0) rows = std::max<int64_t>(2 * (int64_t)max_batch, 128);
  gscan::Pool pool(s->qs);
  int32_t* ring = labels;
  if (!labels && n > 0 && nq > 0) {
    rows = std::min(rows, nq);
    ring = pool.get<int32_t>((size_t)rows * (size_t)n);
    if (!ring) return SCAN_ENOMEM;
    GS_CUDA(cudaStreamSynchronize(s->qs));
  }
  std::vector<uint64_t> qt((size_t)nq, 0), bt((size_t)nb, 0);
  std::vector<Request*> qr((size_t)nq, nullptr);
  std::vector<Clock::time_point> q_sched((size_t)nq);
  int rc_all = SCAN_OK;
  const auto t0 = Clock::now();
  const auto deadline = t0 + std::chrono::milliseconds(timeout_ms < 0 ? 1LL << 40 : timeout_ms);
  auto at_time = [&](double sec) {
    return t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(sec));
  };
  int64_t i = 0, j = 0;
  while (i < nq || j < nb) {
    const bool take_q = j >= nb || (i < nq && q_arrival_s[i] <= b_arrival_s[j]);
    const auto when = at_time(take_q ? q_arrival_s[i] : b_arrival_s[j]);
    // sleep until shortly before the arrival, then spin
    auto now = Clock::now();
    if (when - now > std::chrono::microseconds(300))
      std::this_thread::sleep_until(when - std::chrono::microseconds(200));
    while (Clock::now() < when) {
    }
    int rc;
    if (take_q) {
      q_sched[i] = when;
      const int64_t slot = i % rows;
      if (i >= rows && qr[i - rows]) {
        // the row's previous query must have completed (bounded by the deadline)
        Request* prev = qr[i - rows];
        std::unique_lock<std::mutex> lk(s->mu);
        if (!s->cv_done.wait_until(lk, deadline, [&] { return prev->done; })) {
          lk.unlock();
          if (rc_all == SCAN_OK) rc_all = SCAN_ETIMEOUT;
          break;
        }
      }
      rc = scan_serve_submit_query(s, index, q_mu[i], q_eps[i], ring ? ring + (size_t)slot * n : nullptr,
                                   flags, &qt[i]);
      if (rc == SCAN_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(qt[i]);
        qr[i] = it != s->reqs.end() ? it->second : nullptr;
      }
      ++i;
    } else {
      rc = scan_serve_submit_build(s, &b_graphs[j], b_kind, nullptr, &bt[j]);
      ++j;
    }
    if (rc != SCAN_OK && rc_all == SCAN_OK) rc_all = rc;
  }
  // collect: latency runs from the scheduled arrival to the completion, so a
  // submission delayed by a busy row still counts its wait
  for (int64_t k = 0; k < nq; ++k) {
    if (latency_ms) latency_ms[k] = -1;
    if (!qt[k]) continue;
    Request* r = qr[k];
    double lat = -1;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (r && s->cv_done.wait_until(lk, deadline, [&] { return r->done; }))
        lat = std::chrono::duration<double, std::milli>(r->t_done - q_sched[k]).count();
    }
    const int rc = lat >= 0 ? scan_serve_wait(s, qt[k], 0, nullptr) : SCAN_ETIMEOUT;
    if (latency_ms) latency_ms[k] = lat;
    if (rc != SCAN_OK && rc_all == SCAN_OK) rc_all = rc;
  }
  for (int64_t k = 0; k < nb; ++k) {
    if (!bt[k]) continue;
    const int left = (int)std::max<int64_t>(
        0, std::chrono::duration_cast<std::chrono::milliseconds>(deadline - Clock::now()).count());
    const int rc = scan_serve_wait(s, bt[k], left, nullptr);
    if (rc != SCAN_OK && rc_all == SCAN_OK) rc_all = rc;
  }
  if (rc_all == SCAN_ETIMEOUT && ring != labels) {
    // queries still queued may write the internal ring: wait (bounded) for
    // them; if some are still pending, leave the ring allocated
    const auto grace = Clock::now() + std::chrono::seconds(60);
    bool all_done = true;
    for (int64_t k = 0; k < nq && all_done; ++k) {
      if (!qt[k] || !qr[k]) continue;
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->reqs.count(qt[k]) && !s->cv_done.wait_until(lk, grace, [&] { return qr[k]->done; }))
        all_done = false;
    }
    if (!all_done) pool.detach();
  }
  cudaStreamSynchronize(s->qs);
  return rc_all;
}

void scan_serve_destroy(scan_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_q.notify_all();
  s->cv_b.notify_all();
  if (s->qt.joinable()) s->qt.join();
  if (s->bt.joinable()) s->bt.join();
  for (auto& kv : s->reqs) {
    if (kv.second->built) scan_index_free(kv.second->built);
    delete kv.second;
  }
  cudaStreamDestroy(s->qs);
  cudaStreamDestroy(s->bs);
  cudaStreamDestroy(s->cs);
  delete s;
}

}  // extern "C"
