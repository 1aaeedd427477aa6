// Serving engine: continuous batching of k-NN requests over a resident index.
//
// The paper evaluates the Random Ball Cover as a batch primitive (Section 7:
// all queries of a data set searched at once).  A deployment receives queries
// as a stream of requests of different sizes; this engine turns that stream
// into merged batches for rbc_search, keeps the index and per-worker device
// buffers resident, and runs several batches at once on separate CUDA
// streams so that one batch's copies, host synchronisation and small kernels
// overlap another batch's tensor-core pass.
//
//   * Arrival: rbc_server_submit queues a request (host buffers) and returns
//     a ticket immediately.
//   * Batching: a worker that is free takes requests from the head of the
//     queue in arrival order, as many as fit within max_batch queries (the
//     requests that arrived while the previous batches were on the GPU).
//   * Admission by memory: a batch is admitted only if its workspace bound
//     (rbc_search_workspace) fits the HBM budget left by the batches already
//     in flight; otherwise it is shrunk, or waits until memory is released.
//   * Execution: host-to-device copies of the requests' queries into the
//     worker's resident batch buffer, one rbc_search over the merged batch
//     with k = the batch's largest k, device-to-host copies of each
//     request's first k columns straight into its own host buffers.
//
// Every query's result depends only on that query (the search is exact and
// ordered by (rho, id)), so a request's answer is the same alone and in any
// mix; the tests check exactly that.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t ticket = 0;
  const float* Q = nullptr;
  int64_t m = 0;
  int32_t k = 0;
  int64_t* ids = nullptr;
  float* dist = nullptr;
  rbc_request_info info{};
  bool done = false;
  std::string err;
};

// Requests taken from the head of the queue: as many as keep the batch within
// max_batch queries, then fewer until bound(queries, largest k) fits mem_left.
// Returns the count (0: nothing fits, wait for memory).
template <class Bound>
int plan_batch(const int64_t* m, const int32_t* k, int n, int64_t max_batch, int64_t mem_left,
               Bound bound) {
  int c = 0;
  int64_t tot = 0;
  while (c < n && tot + m[c] <= max_batch) tot += m[c++];
  while (c > 0) {
    int32_t kb = 1;
    for (int i = 0; i < c; ++i) kb = std::max(kb, k[i]);
    if (bound(tot, kb) <= mem_left) return c;
    tot -= m[--c];
  }
  return 0;
}

struct Worker {
  cudaStream_t st = nullptr;
  float* Qd = nullptr;
  int64_t* ids_d = nullptr;
  float* dist_d = nullptr;
  std::thread th;
};

struct Done {
  int64_t t_submit, t_start, t_done, m;
};

double pct_ms(std::vector<int64_t>& v, double p) {
  if (v.empty()) return 0.0;
  const size_t i = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
  std::nth_element(v.begin(), v.begin() + i, v.end());
  return (double)v[i] * 1e-6;
}

}  // namespace

struct rbc_server {
  const rbc_index* ix = nullptr;
  rbc_index_desc desc{};
  rbc_server_opts o{};
  std::mutex mu;
  std::condition_variable cv_work;  // queue or memory changed
  std::condition_variable cv_done;  // a request completed
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> live;  // submitted, not yet collected
  uint64_t next_ticket = 1;
  int64_t next_batch = 0;
  int64_t reserved = 0;  // workspace bound of the batches in flight
  int inflight = 0;
  bool stop = false;
  // statistics since creation / the last reset
  std::vector<Done> done;
  int64_t batches = 0, batch_queries = 0, peak_reserved = 0;
  int max_inflight = 0;
  std::vector<Worker> workers;

  int64_t bound(int64_t m, int32_t k) const {
    int64_t b = 0;
    rbc_search_workspace(ix, m, k, &b);
    return b;
  }
  void run(Worker* w);
};

void rbc_server::run(Worker* w) {
  cudaSetDevice(desc.device);
  const int d = desc.d;
  std::vector<Request*> batch;
  std::vector<int64_t> qm;
  std::vector<int32_t> qk;
  for (;;) {
    int64_t total = 0, reserve = 0, bid = 0;
    int32_t kb = 1;
    {
      std::unique_lock<std::mutex> lk(mu);
      int take = 0;
      cv_work.wait(lk, [&] {
        if (queue.empty()) return stop;
        const int n = (int)std::min<size_t>(queue.size(), (size_t)o.max_batch);
        qm.resize(n);
        qk.resize(n);
        for (int i = 0; i < n; ++i) {
          qm[i] = queue[i]->m;
          qk[i] = queue[i]->k;
        }
        take = plan_batch(qm.data(), qk.data(), n, o.max_batch, o.hbm_budget - reserved,
                          [this](int64_t mm, int32_t kk) { return bound(mm, kk); });
        // a request alone always fits the whole budget (checked at submit)
        if (take == 0 && inflight == 0) take = 1;
        return take > 0;
      });
      if (queue.empty()) return;  // stopping and drained
      batch.assign(queue.begin(), queue.begin() + take);
      queue.erase(queue.begin(), queue.begin() + take);
      for (Request* r : batch) {
        total += r->m;
        kb = std::max(kb, r->k);
      }
      reserve = bound(total, kb);
      reserved += reserve;
      peak_reserved = std::max(peak_reserved, reserved);
      max_inflight = std::max(max_inflight, ++inflight);
      bid = next_batch++;
    }
    const int64_t t_start = now_ns();
    int rc = RBC_OK;
    std::string msg;
    int64_t off = 0;
    for (Request* r : batch) {
      if (rc == RBC_OK && r->m > 0) {
        cudaError_t e = cudaMemcpyAsync(w->Qd + off * d, r->Q, (size_t)r->m * d * sizeof(float),
                                        cudaMemcpyDefault, w->st);
        if (e != cudaSuccess) rc = rbc::cuda_fail(e, "cudaMemcpyAsync (queries)", __FILE__, __LINE__);
      }
      off += r->m;
    }
    if (rc == RBC_OK) rc = rbc_search(ix, w->Qd, total, kb, w->ids_d, w->dist_d, w->st);
    off = 0;
    for (Request* r : batch) {
      if (rc == RBC_OK && r->m > 0) {
        cudaError_t e = cudaMemcpy2DAsync(r->ids, r->k * sizeof(int64_t), w->ids_d + off * kb,
                                          kb * sizeof(int64_t), r->k * sizeof(int64_t), r->m,
                                          cudaMemcpyDefault, w->st);
        if (e == cudaSuccess)
          e = cudaMemcpy2DAsync(r->dist, r->k * sizeof(float), w->dist_d + off * kb,
                                kb * sizeof(float), r->k * sizeof(float), r->m, cudaMemcpyDefault,
                                w->st);
        if (e != cudaSuccess) rc = rbc::cuda_fail(e, "cudaMemcpy2DAsync (results)", __FILE__, __LINE__);
      }
      off += r->m;
    }
    cudaError_t e = cudaStreamSynchronize(w->st);
    if (rc == RBC_OK && e != cudaSuccess)
      rc = rbc::cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
    if (rc != RBC_OK) msg = rbc_last_error();
    const int64_t t_done = now_ns();
    {
      std::lock_guard<std::mutex> lk(mu);
      reserved -= reserve;
      --inflight;
      ++batches;
      batch_queries += total;
      for (Request* r : batch) {
        r->info.t_start_ns = t_start;
        r->info.t_done_ns = t_done;
        r->info.batch = bid;
        r->info.batch_queries = total;
        r->info.batch_requests = (int32_t)batch.size();
        r->info.status = rc;
        r->err = msg;
        r->done = true;
        done.push_back(Done{r->info.t_submit_ns, t_start, t_done, r->m});
      }
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

using rbc::set_error;

extern "C" {

int rbc_plan_batch(const int64_t* m, const int32_t* k, int32_t n, int64_t max_batch,
                   int64_t mem_left, int64_t fixed_bytes, int64_t bytes_per_query,
                   int64_t bytes_per_query_k) {
  if (n < 0 || (n > 0 && (!m || !k)) || max_batch < 1) {
    set_error("rbc_plan_batch: bad arguments");
    return RBC_ERR_ARG;
  }
  return plan_batch(m, k, n, max_batch, mem_left, [&](int64_t mm, int32_t kk) {
    return fixed_bytes + mm * (bytes_per_query + kk * bytes_per_query_k);
  });
}

int rbc_server_create(const rbc_index* idx, const rbc_server_opts* opts, rbc_server** out) {
  if (!idx || !out) {
    set_error("rbc_server_create: NULL index or out");
    return RBC_ERR_ARG;
  }
  *out = nullptr;
  std::unique_ptr<rbc_server> S(new (std::nothrow) rbc_server());
  if (!S) {
    set_error("rbc_server_create: host allocation failed");
    return RBC_ERR_OOM;
  }
  S->ix = idx;
  const int irc = rbc_index_info(idx, &S->desc);
  if (irc != RBC_OK) return irc;
  if (opts) S->o = *opts;
  if (S->o.workers <= 0) S->o.workers = 2;
  if (S->o.max_batch <= 0) S->o.max_batch = 16384;
  if (S->o.k_max <= 0) S->o.k_max = 10;
  if (S->o.workers > 16 || S->o.max_batch > (1 << 24) || S->o.k_max > 31 ||
      S->o.k_max > S->desc.n || (S->desc.mode == RBC_ONESHOT && S->o.k_max > S->desc.s)) {
    set_error("rbc_server_create: workers %d (1..16), max_batch %d (<= 2^24), k_max %d "
              "(<= 31, <= n, one-shot <= s)",
              S->o.workers, S->o.max_batch, S->o.k_max);
    return RBC_ERR_ARG;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  RBC_CUDA(cudaSetDevice(S->desc.device));
  const int64_t mb = S->o.max_batch;
  S->workers.resize(S->o.workers);
  int rc = RBC_OK;
  for (Worker& w : S->workers) {
    cudaError_t e = cudaStreamCreateWithFlags(&w.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&w.Qd, (size_t)mb * S->desc.d * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&w.ids_d, (size_t)mb * S->o.k_max * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&w.dist_d, (size_t)mb * S->o.k_max * sizeof(float));
    if (e != cudaSuccess) {
      rc = rbc::cuda_fail(e, "rbc_server_create (worker buffers)", __FILE__, __LINE__);
      break;
    }
  }
  if (rc == RBC_OK && S->o.hbm_budget <= 0) {
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) rc = rbc::cuda_fail(e, "cudaMemGetInfo", __FILE__, __LINE__);
    S->o.hbm_budget = (int64_t)(fr / 2);
  }
  if (rc != RBC_OK) {
    for (Worker& w : S->workers) {
      cudaFree(w.Qd);
      cudaFree(w.ids_d);
      cudaFree(w.dist_d);
      if (w.st) cudaStreamDestroy(w.st);
    }
    cudaSetDevice(prev);
    return rc;
  }
  rbc_server* raw = S.get();
  for (Worker& w : raw->workers) w.th = std::thread([raw, &w] { raw->run(&w); });
  cudaSetDevice(prev);
  *out = S.release();
  return RBC_OK;
}

int rbc_server_submit(rbc_server* S, const float* Q, int64_t m, int32_t k, int64_t* out_ids,
                      float* out_dist, uint64_t* ticket) {
  if (!S || !ticket || (m > 0 && (!Q || !out_ids || !out_dist))) {
    set_error("rbc_server_submit: NULL pointer");
    return RBC_ERR_ARG;
  }
  if (m < 0 || m > S->o.max_batch || k < 1 || k > S->o.k_max) {
    set_error("rbc_server_submit: m=%lld must be in [0, max_batch=%d] and k=%d in [1, k_max=%d]",
              (long long)m, S->o.max_batch, k, S->o.k_max);
    return RBC_ERR_ARG;
  }
  const int64_t need = S->bound(m, k);
  if (need > S->o.hbm_budget) {
    set_error("rbc_server_submit: a batch of %lld queries needs up to %lld workspace bytes, "
              "over the budget of %lld",
              (long long)m, (long long)need, (long long)S->o.hbm_budget);
    return RBC_ERR_OOM;
  }
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) {
    set_error("rbc_server_submit: host allocation failed");
    return RBC_ERR_OOM;
  }
  r->Q = Q;
  r->m = m;
  r->k = k;
  r->ids = out_ids;
  r->dist = out_dist;
  r->info.t_submit_ns = now_ns();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      set_error("rbc_server_submit: the server is shutting down");
      return RBC_ERR_ARG;
    }
    r->ticket = S->next_ticket++;
    *ticket = r->ticket;
    if (m == 0) {  // nothing to search
      r->info.t_start_ns = r->info.t_done_ns = r->info.t_submit_ns;
      r->info.batch = -1;
      r->done = true;
    } else {
      S->queue.push_back(r.get());
    }
    S->live.emplace(r->ticket, std::move(r));
  }
  S->cv_work.notify_one();
  return RBC_OK;
}

int rbc_server_wait(rbc_server* S, uint64_t ticket, int64_t timeout_us, rbc_request_info* info) {
  if (!S) {
    set_error("rbc_server_wait: NULL server");
    return RBC_ERR_ARG;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->live.find(ticket);
  if (it == S->live.end()) {
    set_error("rbc_server_wait: unknown or already collected ticket %llu",
              (unsigned long long)ticket);
    return RBC_ERR_ARG;
  }
  Request* r = it->second.get();
  auto ready = [r] { return r->done; };
  if (timeout_us < 0)
    S->cv_done.wait(lk, ready);
  else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
    set_error("rbc_server_wait: request %llu still running", (unsigned long long)ticket);
    return RBC_ERR_TIMEOUT;
  }
  if (info) *info = r->info;
  const int rc = r->info.status;
  if (rc != RBC_OK) set_error("%s", r->err.c_str());
  S->live.erase(it);
  return rc;
}

int rbc_server_stats(rbc_server* S, int32_t reset, rbc_serving_stats* out) {
  if (!S || !out) {
    set_error("rbc_server_stats: NULL");
    return RBC_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  memset(out, 0, sizeof(*out));
  const std::vector<Done>& v = S->done;
  out->requests = (int64_t)v.size();
  out->batches = S->batches;
  out->workers = S->o.workers;
  out->max_in_flight = S->max_inflight;
  out->peak_reserved_bytes = S->peak_reserved;
  out->hbm_budget = S->o.hbm_budget;
  out->mean_batch_queries = S->batches ? (double)S->batch_queries / (double)S->batches : 0.0;
  if (!v.empty()) {
    std::vector<int64_t> lat(v.size()), qw(v.size());
    int64_t first = v[0].t_submit, last = v[0].t_done;
    double sum = 0;
    for (size_t i = 0; i < v.size(); ++i) {
      lat[i] = v[i].t_done - v[i].t_submit;
      qw[i] = v[i].t_start - v[i].t_submit;
      first = std::min(first, v[i].t_submit);
      last = std::max(last, v[i].t_done);
      out->queries += v[i].m;
      sum += (double)lat[i];
    }
    out->mean_ms = sum / (double)v.size() * 1e-6;
    out->max_ms = (double)*std::max_element(lat.begin(), lat.end()) * 1e-6;
    out->p50_ms = pct_ms(lat, 0.50);
    out->p99_ms = pct_ms(lat, 0.99);
    out->queue_p50_ms = pct_ms(qw, 0.50);
    out->queue_p99_ms = pct_ms(qw, 0.99);
    out->wall_s = (double)(last - first) * 1e-9;
    out->queries_per_s = out->wall_s > 0 ? (double)out->queries / out->wall_s : 0.0;
  }
  if (reset) {
    S->done.clear();
    S->batches = 0;
    S->batch_queries = 0;
    S->peak_reserved = S->reserved;
    S->max_inflight = S->inflight;
  }
  return RBC_OK;
}

void rbc_server_destroy(rbc_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (Worker& w : S->workers)
    if (w.th.joinable()) w.th.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->desc.device);
  for (Worker& w : S->workers) {
    cudaFree(w.Qd);
    cudaFree(w.ids_d);
    cudaFree(w.dist_d);
    if (w.st) cudaStreamDestroy(w.st);
  }
  cudaSetDevice(prev);
  delete S;
}

}  // extern "C"
