// server.cpp -- continuous-batching serving loop around the query path
// (Sec. 3.1 probe, Sec. 6 rerank) with the data and index resident on the GPU.
//
// Requests (batches of host queries) enter a FIFO.  A scheduler thread admits
// the head request as soon as a slot is free and the device bytes held by the
// batches in flight plus the request's own footprint stay within the memory
// budget; requests that arrive while others run are admitted the same way,
// so several batches overlap on the device, each on its slot's stream.  A
// slot owns a stream, device buffers sized for the largest batch, pinned host
// staging and, per power-of-two batch bucket, a captured CUDA graph of
//   H2D(queries) -> hash (all L tables) -> probe/dedup/rerank -> D2H(results)
// that later batches of that bucket replay (rows beyond the batch are padding:
// the live row count is copied into the graph from a pinned word, and the
// query CTAs of padding rows return at once).  A host callback on the stream
// marks the batch done; latency runs from submit to results on the host.
// Every query is answered from its own row by its own CTAs, whose merged list
// does not depend on how many CTAs share it, so a result does not depend on
// which requests share its batch or run beside it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace lsh {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket = 0;
  int64_t q = 0;
  int32_t dtype = 0;
  std::vector<unsigned char> data;  // the queries, copied at submit
  Clock::time_point t_submit, t_done;
  bool done = false;
  lsh_status status = LSH_OK;
  std::vector<int32_t> ids;
  std::vector<float> dist;
};

struct Slot {
  cudaStream_t stream = nullptr;
  unsigned char *Qd = nullptr;   // device queries [max_batch][d] (<= 4-byte elements)
  uint64_t *qkeys = nullptr;     // [L][max_batch]
  int32_t *ids_d = nullptr;      // [max_batch][k]
  float *dist_d = nullptr;
  void *qscratch = nullptr;      // split-query lists (query_scratch_bytes(max_batch, k))
  int64_t *qlive_d = nullptr;    // live rows of the batch in flight (device word) ...
  int64_t *qlive_h = nullptr;    // ... copied from this pinned word inside the batch's graph
  unsigned char *Qh = nullptr;   // pinned staging
  int32_t *ids_h = nullptr;
  float *dist_h = nullptr;
  std::map<std::pair<int64_t, int32_t>, cudaGraphExec_t> graphs;  // (bucket, dtype)
  std::shared_ptr<Request> req;  // in flight
  int64_t bytes = 0;             // footprint charged to the budget
  bool busy = false;
  bool finished = false;         // set by the stream callback
};

}  // namespace
}  // namespace lsh

struct lsh_server_s {
  lsh_index_t idx = nullptr;
  lsh_server_config cfg{};
  std::vector<lsh::Slot> slots;
  std::deque<std::shared_ptr<lsh::Request>> queue;
  std::unordered_map<int64_t, std::shared_ptr<lsh::Request>> live;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::thread sched;
  bool stop = false;
  int64_t next_ticket = 1;
  int64_t in_flight_bytes = 0;
  int device = 0;
  // stats
  std::vector<double> lat_ms;
  int64_t completed_requests = 0, completed_queries = 0, admitted_peak = 0, replays = 0, captures = 0;
  bool have_first = false;
  lsh::Clock::time_point first_submit, last_done;
};

namespace lsh {
namespace {

struct CallbackArg {
  lsh_server_s *srv;
  int slot;
};

void CUDART_CB on_batch_done(void *p) {
  CallbackArg *a = static_cast<CallbackArg *>(p);
  {
    std::lock_guard<std::mutex> lock(a->srv->mu);
    a->srv->slots[a->slot].finished = true;
  }
  a->srv->cv_sched.notify_one();
}

int64_t bucket_of(int64_t q, int64_t max_batch) {
  int64_t b = 16;
  while (b < q) b <<= 1;
  return std::min(b, max_batch);
}

int64_t footprint(const lsh_server_s *s, int64_t rows) {
  const lsh_family_desc &d = s->idx->fam->host.desc;
  return rows * (int64_t(d.d) * 4 + int64_t(d.L) * 8 + int64_t(s->cfg.k) * 8);
}

size_t esize(int32_t dt) { return dt == LSH_F32 ? 4 : 2; }

// The device work of one batch of `rows` rows on the slot's stream.
lsh_status enqueue_batch(lsh_server_s *s, Slot &sl, int64_t rows, int32_t dtype) {
  const lsh_family_desc &d = s->idx->fam->host.desc;
  const size_t rb = size_t(d.d) * esize(dtype);
  LSH_CUDA_TRY(cudaMemcpyAsync(sl.Qd, sl.Qh, rb * rows, cudaMemcpyHostToDevice, sl.stream));
  lsh_matrix Q{};
  Q.dtype = dtype;
  Q.n = rows;
  Q.d = d.d;
  Q.ld = d.d;
  Q.values = sl.Qd;
  lsh_status st = hash_impl(s->idx->fam, &Q, nullptr, sl.qkeys, rows, nullptr, nullptr, sl.stream);
  if (st != LSH_OK) return st;
  LSH_CUDA_TRY(cudaMemcpyAsync(sl.qlive_d, sl.qlive_h, sizeof(int64_t), cudaMemcpyHostToDevice, sl.stream));
  LSH_CUDA_TRY(launch_query(sl.qkeys, rows, d.L, s->cfg.k, kind_is_srp(d.kind) ? 1 : 0, d.d, sl.Qd, dtype, d.d,
                            s->idx, sl.ids_d, sl.dist_d, nullptr, sl.qscratch, s->cfg.max_batch, sl.qlive_d,
                            sl.stream));
  if (!s->cfg.use_graphs) count_launches(1);
  LSH_CUDA_TRY(cudaMemcpyAsync(sl.ids_h, sl.ids_d, size_t(rows) * s->cfg.k * 4, cudaMemcpyDeviceToHost, sl.stream));
  LSH_CUDA_TRY(cudaMemcpyAsync(sl.dist_h, sl.dist_d, size_t(rows) * s->cfg.k * 4, cudaMemcpyDeviceToHost,
                               sl.stream));
  return LSH_OK;
}

// Launch a batch: replay (or capture, then replay) the bucket's graph, or
// launch directly.  Called by the scheduler with the lock released.
lsh_status launch_batch(lsh_server_s *s, int si, CallbackArg *cb) {
  Slot &sl = s->slots[si];
  Request &r = *sl.req;
  const lsh_family_desc &d = s->idx->fam->host.desc;
  std::memcpy(sl.Qh, r.data.data(), r.data.size());
  *sl.qlive_h = r.q;  // rows beyond it (bucket padding) skip the query work
  lsh_status st = LSH_OK;
  if (s->cfg.use_graphs) {
    const int64_t b = bucket_of(r.q, s->cfg.max_batch);
    if (b > r.q) std::memset(sl.Qh + r.data.size(), 0, size_t(b - r.q) * d.d * esize(r.dtype));
    auto key = std::make_pair(b, r.dtype);
    auto it = sl.graphs.find(key);
    if (it == sl.graphs.end()) {
      cudaGraph_t g = nullptr;
      LSH_CUDA_TRY(cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal));
      st = enqueue_batch(s, sl, b, r.dtype);
      cudaError_t e = cudaStreamEndCapture(sl.stream, &g);
      if (st != LSH_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(e, "server graph capture");
      cudaGraphExec_t ex = nullptr;
      e = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "server graph instantiate");
      it = sl.graphs.emplace(key, ex).first;
      std::lock_guard<std::mutex> lock(s->mu);
      ++s->captures;
    }
    LSH_CUDA_TRY(cudaGraphLaunch(it->second, sl.stream));
    count_launches(2);  // the hashing and query kernels of the replayed graph
    std::lock_guard<std::mutex> lock(s->mu);
    ++s->replays;
  } else {
    st = enqueue_batch(s, sl, r.q, r.dtype);
    if (st != LSH_OK) return st;
  }
  LSH_CUDA_TRY(cudaLaunchHostFunc(sl.stream, on_batch_done, cb));
  return LSH_OK;
}

void scheduler(lsh_server_s *s) {
  cudaSetDevice(s->device);
  std::vector<CallbackArg> cbs(s->slots.size());
  for (size_t i = 0; i < cbs.size(); ++i) cbs[i] = CallbackArg{s, int(i)};
  std::unique_lock<std::mutex> lock(s->mu);
  while (true) {
    // 1. retire finished batches
    for (size_t i = 0; i < s->slots.size(); ++i) {
      Slot &sl = s->slots[i];
      if (!sl.busy || !sl.finished) continue;
      Request &r = *sl.req;
      r.ids.assign(sl.ids_h, sl.ids_h + r.q * s->cfg.k);
      r.dist.assign(sl.dist_h, sl.dist_h + r.q * s->cfg.k);
      r.t_done = Clock::now();
      r.done = true;
      const double ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
      s->lat_ms.push_back(ms);
      ++s->completed_requests;
      s->completed_queries += r.q;
      s->last_done = r.t_done;
      s->in_flight_bytes -= sl.bytes;
      sl.req.reset();
      sl.busy = false;
      sl.finished = false;
      s->cv_done.notify_all();
    }
    if (s->stop && s->queue.empty()) {
      bool any = false;
      for (auto &sl : s->slots) any = any || sl.busy;
      if (!any) break;
    }
    // 2. admit from the head of the queue while a slot and memory are free
    bool launched = false;
    while (!s->queue.empty()) {
      int free_slot = -1;
      for (size_t i = 0; i < s->slots.size(); ++i)
        if (!s->slots[i].busy) {
          free_slot = int(i);
          break;
        }
      if (free_slot < 0) break;
      std::shared_ptr<Request> r = s->queue.front();
      const int64_t need = footprint(s, s->cfg.use_graphs ? bucket_of(r->q, s->cfg.max_batch) : r->q);
      if (s->cfg.mem_budget > 0 && s->in_flight_bytes > 0 && s->in_flight_bytes + need > s->cfg.mem_budget) break;
      s->queue.pop_front();
      Slot &sl = s->slots[free_slot];
      sl.req = r;
      sl.busy = true;
      sl.finished = false;
      sl.bytes = need;
      s->in_flight_bytes += need;
      int64_t inflight = 0;
      for (auto &x : s->slots) inflight += x.busy ? 1 : 0;
      s->admitted_peak = std::max(s->admitted_peak, inflight);
      lock.unlock();
      const lsh_status st = launch_batch(s, free_slot, &cbs[free_slot]);
      lock.lock();
      if (st != LSH_OK) {  // the batch never reached the device: fail it
        r->status = st;
        r->done = true;
        r->t_done = Clock::now();
        s->in_flight_bytes -= sl.bytes;
        sl.req.reset();
        sl.busy = false;
        s->cv_done.notify_all();
      }
      launched = true;
    }
    if (launched) continue;
    s->cv_sched.wait(lock);
  }
}

void free_server(lsh_server_s *s) {
  for (auto &sl : s->slots) {
    for (auto &g : sl.graphs) cudaGraphExecDestroy(g.second);
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    cudaFree(sl.Qd);
    cudaFree(sl.qkeys);
    cudaFree(sl.ids_d);
    cudaFree(sl.dist_d);
    cudaFree(sl.qscratch);
    cudaFree(sl.qlive_d);
    cudaFreeHost(sl.qlive_h);
    cudaFreeHost(sl.Qh);
    cudaFreeHost(sl.ids_h);
    cudaFreeHost(sl.dist_h);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete s;
}

}  // namespace
}  // namespace lsh

using namespace lsh;

extern "C" {

lsh_status lsh_server_create(lsh_index_t idx, const lsh_server_config *cfg, lsh_server_t *out) {
  if (!idx || !cfg || !out) return fail(LSH_EINVAL, "NULL argument");
  *out = nullptr;
  if (!idx->d_data && idx->n > 0) return fail(LSH_EINVAL, "the index was built without keep_data");
  if (cfg->max_batch < 1 || cfg->max_batch > 65536) return fail(LSH_EINVAL, "max_batch must be in [1, 65536]");
  if (cfg->slots < 1 || cfg->slots > 64) return fail(LSH_EINVAL, "slots must be in [1, 64]");
  if (cfg->k < 1 || cfg->k > 256) return fail(LSH_EINVAL, "k must be in [1, 256]");
  if (cfg->mem_budget < 0) return fail(LSH_EINVAL, "mem_budget must be >= 0");
  const lsh_family_desc &d = idx->fam->host.desc;
  if (d.L > 128) return fail(LSH_EUNSUPPORTED, "serving supports L <= 128");
  lsh_server_s *s = new (std::nothrow) lsh_server_s();
  if (!s) return fail(LSH_ENOMEM, "host allocation");
  s->idx = idx;
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  const int64_t one = footprint(s, cfg->max_batch);
  if (cfg->mem_budget > 0 && one > cfg->mem_budget) {
    delete s;
    return fail(LSH_EINVAL, "mem_budget is below the footprint of one largest batch");
  }
  s->slots.resize(cfg->slots);
  const size_t mb = size_t(cfg->max_batch);
  cudaError_t e = cudaSuccess;
  for (auto &sl : s->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&sl.Qd, mb * d.d * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sl.qkeys, mb * d.L * 8);
    if (e == cudaSuccess) e = cudaMalloc(&sl.ids_d, mb * cfg->k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sl.dist_d, mb * cfg->k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sl.qscratch, query_scratch_bytes(cfg->max_batch, cfg->k));
    if (e == cudaSuccess) e = cudaMemset(sl.qscratch, 0, mb * 4);  // the per-query counters start at zero
    if (e == cudaSuccess) e = cudaMalloc(&sl.qlive_d, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMallocHost(&sl.qlive_h, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMallocHost(&sl.Qh, mb * d.d * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.ids_h, mb * cfg->k * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.dist_h, mb * cfg->k * 4);
  }
  if (e != cudaSuccess) {
    free_server(s);
    return cuda_fail(e, "lsh_server_create");
  }
  s->sched = std::thread(scheduler, s);
  *out = s;
  return LSH_OK;
}

lsh_status lsh_server_submit(lsh_server_t s, const void *queries, int32_t dtype, int64_t q, int64_t *ticket) {
  if (!s || !ticket || (q > 0 && !queries)) return fail(LSH_EINVAL, "NULL argument");
  if (q < 1 || q > s->cfg.max_batch) return fail(LSH_EINVAL, "batch size must be in [1, max_batch]");
  if (dtype != LSH_F32 && dtype != LSH_BF16 && dtype != LSH_F16) return fail(LSH_EINVAL, "unsupported dtype");
  auto r = std::make_shared<Request>();
  const size_t bytes = size_t(q) * s->idx->fam->host.desc.d * esize(dtype);
  r->q = q;
  r->dtype = dtype;
  r->data.assign(static_cast<const unsigned char *>(queries), static_cast<const unsigned char *>(queries) + bytes);
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return fail(LSH_EINVAL, "server is stopping");
    r->ticket = s->next_ticket++;
    if (!s->have_first) {
      s->have_first = true;
      s->first_submit = r->t_submit;
    }
    s->queue.push_back(r);
    s->live[r->ticket] = r;
    *ticket = r->ticket;
  }
  s->cv_sched.notify_one();
  return LSH_OK;
}

lsh_status lsh_server_wait(lsh_server_t s, int64_t ticket, int32_t *ids, float *dist, double *latency_ms) {
  if (!s) return fail(LSH_EINVAL, "NULL server");
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->live.find(ticket);
    if (it == s->live.end()) return fail(LSH_EINVAL, "unknown ticket");
    r = it->second;
    s->cv_done.wait(lock, [&] { return r->done; });
    s->live.erase(it);
  }
  if (r->status != LSH_OK) return r->status;
  if (ids) std::memcpy(ids, r->ids.data(), r->ids.size() * 4);
  if (dist) std::memcpy(dist, r->dist.data(), r->dist.size() * 4);
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  return LSH_OK;
}

lsh_status lsh_server_stats_get(lsh_server_t s, lsh_server_stats *st, int32_t reset) {
  if (!s || !st) return fail(LSH_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  std::memset(st, 0, sizeof(*st));
  st->completed_requests = s->completed_requests;
  st->completed_queries = s->completed_queries;
  st->admitted_peak = s->admitted_peak;
  st->graph_replays = s->replays;
  st->graph_captures = s->captures;
  if (!s->lat_ms.empty()) {
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[std::min(v.size() - 1, size_t(p * (v.size() - 1) + 0.5))]; };
    double sum = 0;
    for (double x : v) sum += x;
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    st->mean_ms = sum / v.size();
    st->max_ms = v.back();
  }
  if (s->have_first && s->completed_requests > 0)
    st->busy_s = std::chrono::duration<double>(s->last_done - s->first_submit).count();
  if (reset) {
    s->lat_ms.clear();
    s->completed_requests = s->completed_queries = 0;
    s->admitted_peak = 0;
    s->have_first = false;
  }
  return LSH_OK;
}

void lsh_server_destroy(lsh_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_all();
  if (s->sched.joinable()) s->sched.join();
  free_server(s);
}

}  // extern "C"
