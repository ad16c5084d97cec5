// Continuous-batching serving loop over one index.
//
// Requests (q, k, mode) are submitted from any host thread and queued.  Each worker
// owns a CUDA stream, a call context (workspace) and pinned staging buffers; whenever it
// is free it takes every queued request up to its batch limit (a "tick"), runs the
// batched query path (Alg. 5 for all of them in one pass) on its stream, and publishes
// each request's ids with its latency.  Requests that arrive while a batch is on the GPU
// are taken by the next free worker, so batches of different ticks overlap on the
// device.  A tick is admitted only if its workspace fits in the server's device-memory
// budget and in the device's free memory; otherwise it is split.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "sah_internal.cuh"

struct sah_index;   // defined in api.cu as { sah::Index impl; }
namespace sah {
Index* index_impl(sah_index* h);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket;
  std::vector<float> q;
  int32_t k, mode;
  Clock::time_point t0;
};

struct Done {
  sah_status status;
  std::vector<int32_t> ids;
  double latency_s;
  std::string error;   // the worker's error message when the batch failed
};

struct Worker {
  std::thread th;
  cudaStream_t stream = nullptr;
  sah::CallCtx ctx;
  float* q_h = nullptr;
  int32_t* km_h = nullptr;       // ks then modes
  float* q_d = nullptr;
  int32_t* km_d = nullptr;
  int32_t* ids_h = nullptr;
  size_t ids_cap = 0;
};

}  // namespace

struct sah_server {
  sah::Index* ix = nullptr;
  int device = 0;
  int32_t max_slots = 0, max_batch = 0;
  int64_t budget = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request> pending;
  std::unordered_set<uint64_t> inflight;
  std::unordered_map<uint64_t, Done> done;
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::vector<Worker*> workers;
  int64_t batches = 0, batched_requests = 0, max_seen_batch = 0, split_ticks = 0;
};

namespace {

void worker_loop(sah_server* s, Worker* w) {
  cudaSetDevice(s->device);
  sah::Index* ix = s->ix;
  const int d = ix->d;
  const int64_t per_worker_budget = s->budget / (int64_t)s->workers.size();
  for (;;) {
    std::vector<Request> batch;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stopping || !s->pending.empty(); });
      if (s->pending.empty()) return;   // stopping and drained
      // admission: the tick's workspace must fit the budget and the free device memory
      int32_t B = std::min<int32_t>((int32_t)s->pending.size(), s->max_batch);
      size_t free_b = 0, total_b = 0;
      cudaMemGetInfo(&free_b, &total_b);
      while (B > 1) {
        const size_t need = sah::batch_workspace_bytes(ix, B);
        const size_t grow = need > w->ctx.ws.bytes ? need - w->ctx.ws.bytes : 0;
        // the part of the workspace that grows with the batch; the survivor lists and the
        // result buffer are sized by the counts of earlier batches and do not shrink with B
        if ((int64_t)need <= per_worker_budget && grow <= free_b / 2)
          break;
        B /= 2;
        ++s->split_ticks;
      }
      for (int32_t i = 0; i < B; ++i) {
        batch.push_back(std::move(s->pending.front()));
        s->pending.pop_front();
        s->inflight.insert(batch.back().ticket);
      }
      ++s->batches;
      s->batched_requests += B;
      s->max_seen_batch = std::max<int64_t>(s->max_seen_batch, B);
    }
    const int32_t B = (int32_t)batch.size();
    for (int32_t i = 0; i < B; ++i) {
      std::memcpy(w->q_h + (size_t)i * d, batch[i].q.data(), sizeof(float) * d);
      w->km_h[i] = batch[i].k;
      w->km_h[s->max_batch + i] = batch[i].mode;
    }
    bool any_sa = false;
    for (auto& r : batch) any_sa |= r.mode == SAH_SAALSH;
    std::vector<int64_t> offs(B + 1, 0);
    sah_status st = SAH_OK;
    if (cudaMemcpyAsync(w->q_d, w->q_h, sizeof(float) * (size_t)B * d, cudaMemcpyHostToDevice, w->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(w->km_d, w->km_h, sizeof(int32_t) * 2 * s->max_batch, cudaMemcpyHostToDevice, w->stream) !=
            cudaSuccess) {
      st = SAH_ERR_CUDA;
    }
    bool wrote = false;
    if (st == SAH_OK)
      st = sah::run_batch(ix, &w->ctx, w->q_d, B, w->km_d, any_sa ? w->km_d + s->max_batch : nullptr, nullptr, 0,
                          nullptr, offs.data(), &wrote, w->stream);
    const int64_t total = st == SAH_OK ? offs[B] : 0;
    if (st == SAH_OK && total > 0) {
      if ((size_t)total > w->ids_cap) {
        if (w->ids_h) cudaFreeHost(w->ids_h);
        w->ids_cap = (size_t)total * 2;
        if (cudaMallocHost((void**)&w->ids_h, sizeof(int32_t) * w->ids_cap) != cudaSuccess) {
          w->ids_h = nullptr;
          w->ids_cap = 0;
          st = SAH_ERR_OOM;
        }
      }
      if (st == SAH_OK &&
          (cudaMemcpyAsync(w->ids_h, w->ctx.res.base, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, w->stream) !=
               cudaSuccess ||
           cudaStreamSynchronize(w->stream) != cudaSuccess))
        st = SAH_ERR_CUDA;
    }
    const auto t1 = Clock::now();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (int32_t i = 0; i < B; ++i) {
        Done dn;
        dn.status = st;
        if (st == SAH_OK) dn.ids.assign(w->ids_h + offs[i], w->ids_h + offs[i + 1]);
        dn.latency_s = std::chrono::duration<double>(t1 - batch[i].t0).count();
        if (st != SAH_OK) dn.error = sah_last_error();
        s->done.emplace(batch[i].ticket, std::move(dn));
        s->inflight.erase(batch[i].ticket);
      }
    }
    s->cv.notify_all();
  }
}

}  // namespace

extern "C" {

sah_status sah_server_start(sah_index* index, int32_t max_slots, int32_t max_batch, int32_t workers,
                            int64_t hbm_budget_bytes, sah_server** out) {
  if (!index || !out || max_slots < 1 || max_batch < 1 || workers < 1 || workers > 8 || hbm_budget_bytes < 0) {
    sah::set_error("sah_server_start: invalid argument");
    return SAH_ERR_ARG;
  }
  *out = nullptr;
  sah::Index* ix = sah::index_impl(index);
  auto* s = new sah_server();
  s->ix = ix;
  s->device = ix->device;
  s->max_slots = max_slots;
  s->max_batch = max_batch;
  s->budget = hbm_budget_bytes > 0 ? hbm_budget_bytes : (int64_t(8) << 30);
  cudaSetDevice(s->device);
  for (int i = 0; i < workers; ++i) {
    auto* w = new Worker();
    w->ctx.graphs_allowed = true;   // a repeated batch shape replays its captured graph
    bool ok = cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMallocHost((void**)&w->q_h, sizeof(float) * (size_t)max_batch * ix->d) == cudaSuccess &&
              cudaMallocHost((void**)&w->km_h, sizeof(int32_t) * 2 * (size_t)max_batch) == cudaSuccess &&
              cudaMalloc((void**)&w->q_d, sizeof(float) * (size_t)max_batch * ix->d) == cudaSuccess &&
              cudaMalloc((void**)&w->km_d, sizeof(int32_t) * 2 * (size_t)max_batch) == cudaSuccess;
    s->workers.push_back(w);
    if (!ok) {
      cudaGetLastError();
      sah_server_stop(s);
      sah::set_error("sah_server_start: could not allocate a worker's buffers");
      return SAH_ERR_OOM;
    }
  }
  for (Worker* w : s->workers) w->th = std::thread(worker_loop, s, w);
  *out = s;
  return SAH_OK;
}

sah_status sah_server_submit(sah_server* s, const float* q, int32_t k, int32_t mode, uint64_t* ticket) {
  if (!s || !q || !ticket || k < 1 || (mode != SAH_EXACT && mode != SAH_SAALSH)) {
    sah::set_error("sah_server_submit: invalid argument");
    return SAH_ERR_ARG;
  }
  for (int i = 0; i < s->ix->d; ++i)
    if (!std::isfinite(q[i])) {
      sah::set_error("sah_server_submit: the query holds a non-finite value");
      return SAH_ERR_ARG;
    }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) {
      sah::set_error("sah_server_submit: the server is stopping");
      return SAH_ERR_ARG;
    }
    if ((int64_t)(s->pending.size() + s->inflight.size() + s->done.size()) >= s->max_slots) {
      sah::set_error("sah_server_submit: every request slot is taken; poll finished requests first");
      return SAH_ERR_BUSY;
    }
    Request r;
    r.ticket = s->next_ticket++;
    r.q.assign(q, q + s->ix->d);
    r.k = k;
    r.mode = mode;
    r.t0 = Clock::now();
    *ticket = r.ticket;
    s->pending.push_back(std::move(r));
  }
  s->cv.notify_one();
  return SAH_OK;
}

sah_status sah_server_poll(sah_server* s, uint64_t ticket, int32_t* out_ids, int64_t cap, int64_t* out_count,
                           double* latency_s) {
  if (!s || !out_count || cap < 0 || (cap > 0 && !out_ids)) {
    sah::set_error("sah_server_poll: invalid argument");
    return SAH_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) {
    bool queued = s->inflight.count(ticket) != 0;
    for (const auto& r : s->pending) queued |= r.ticket == ticket;
    if (queued) return SAH_ERR_BUSY;
    sah::set_error("sah_server_poll: unknown ticket");
    return SAH_ERR_ARG;
  }
  Done& dn = it->second;
  *out_count = (int64_t)dn.ids.size();
  if (latency_s) *latency_s = dn.latency_s;
  if (dn.status != SAH_OK) {
    const sah_status st = dn.status;
    const std::string why = dn.error;
    s->done.erase(it);
    sah::set_error("sah_server_poll: the request's batch failed: " + why);
    return st;
  }
  if ((int64_t)dn.ids.size() > cap) return SAH_ERR_BUFFER_TOO_SMALL;
  if (!dn.ids.empty()) std::memcpy(out_ids, dn.ids.data(), sizeof(int32_t) * dn.ids.size());
  s->done.erase(it);
  return SAH_OK;
}

sah_status sah_server_info(sah_server* s, int64_t* batches, int64_t* batched_requests, int64_t* max_batch_seen,
                           int64_t* split_ticks) {
  if (!s) {
    sah::set_error("sah_server_info: server is NULL");
    return SAH_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (batches) *batches = s->batches;
  if (batched_requests) *batched_requests = s->batched_requests;
  if (max_batch_seen) *max_batch_seen = s->max_seen_batch;
  if (split_ticks) *split_ticks = s->split_ticks;
  return SAH_OK;
}

sah_status sah_server_stop(sah_server* s) {
  if (!s) return SAH_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv.notify_all();
  for (Worker* w : s->workers)
    if (w->th.joinable()) w->th.join();
  cudaSetDevice(s->device);
  for (Worker* w : s->workers) {
    if (w->stream) cudaStreamSynchronize(w->stream);
    sah::free_ctx(&w->ctx);
    if (w->q_h) cudaFreeHost(w->q_h);
    if (w->km_h) cudaFreeHost(w->km_h);
    if (w->ids_h) cudaFreeHost(w->ids_h);
    if (w->q_d) cudaFree(w->q_d);
    if (w->km_d) cudaFree(w->km_d);
    if (w->stream) cudaStreamDestroy(w->stream);
    delete w;
  }
  delete s;
  return SAH_OK;
}

}  // extern "C"
