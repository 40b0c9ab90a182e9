// Continuous-batching least-squares server (host code; the GPU work is the persistent
// batched TSQR kernel).
//
// Requests (tsqr_batch_item, device buffers owned by the caller) are queued by
// tsqr_server_submit. A worker thread keeps up to `streams` batches in flight: whenever
// a stream is free it admits the oldest pending requests, as many as fit the device
// memory free at that moment (and the caller's budget, if set), up to max_batch, and
// launches them as
// one persistent kernel on that stream. Completion is observed with an event per batch;
// the request's latency runs from its submission to that observation. Requests that
// arrive while others are on the GPU join the next batch as soon as a stream and memory
// free up, so their work overlaps with the running batch on the device.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/tsqr.h"
#include "tsqr_internal.h"

using Clock = std::chrono::steady_clock;

namespace {

struct SrvReq {
  tsqr_batch_item item;
  int64_t ticket;
  Clock::time_point t0;
  size_t bytes;
};

struct SrvSlot {
  cudaStream_t stream = nullptr;
  cudaEvent_t event = nullptr;
  int32_t *hstatus = nullptr;  // pinned, max_batch entries
  std::vector<SrvReq> reqs;
  size_t bytes = 0;
  bool busy = false;
};

}  // namespace

struct tsqr_server {
  int device = 0;
  size_t budget = 0, used = 0;  // budget 0: admission by the live free device memory only
  size_t last_free = 0;         // free device memory seen at the last admission
  int32_t max_batch = 256, chain_tiles = 0, ctas_per_sm = 0;
  std::vector<SrvSlot> slots;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::deque<SrvReq> pending;
  std::deque<std::tuple<int64_t, double, int32_t>> done;
  int64_t next_ticket = 0, submitted = 0, completed = 0, batches = 0, max_batch_seen = 0;
  bool stop = false;
  std::thread worker;
};

static void server_loop(tsqr_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool progress = false;
    for (SrvSlot &sl : S->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.event);
      if (q == cudaErrorNotReady) continue;
      const Clock::time_point now = Clock::now();
      for (size_t i = 0; i < sl.reqs.size(); ++i) {
        const double lat = std::chrono::duration<double>(now - sl.reqs[i].t0).count();
        const int32_t st = (q == cudaSuccess) ? sl.hstatus[i] : (int32_t)TSQR_ERR_CUDA;
        S->done.emplace_back(sl.reqs[i].ticket, lat, st);
      }
      S->completed += (int64_t)sl.reqs.size();
      S->used -= sl.bytes;
      sl.reqs.clear();
      sl.bytes = 0;
      sl.busy = false;
      progress = true;
      S->cv_done.notify_all();
    }
    for (SrvSlot &sl : S->slots) {
      if (sl.busy || S->pending.empty()) continue;
      // admit the oldest requests that fit the device memory free now (less a 5% margin;
      // the in-flight batches' workspaces are already taken from it) and the budget, if
      // one was set; a request larger than either runs alone once nothing else is in flight
      const size_t live = tsqr::live_free_bytes();
      S->last_free = live;
      const size_t room = live - live / 20;
      std::vector<SrvReq> batch;
      size_t bytes = 0;
      while (!S->pending.empty() && (int32_t)batch.size() < S->max_batch) {
        const SrvReq &r = S->pending.front();
        const bool fits = bytes + r.bytes <= room && (S->budget == 0 || S->used + bytes + r.bytes <= S->budget);
        if (!fits && !(batch.empty() && S->used == 0)) break;
        bytes += r.bytes;
        batch.push_back(r);
        S->pending.pop_front();
      }
      if (batch.empty()) break;
      sl.reqs = batch;
      sl.bytes = bytes;
      sl.busy = true;
      S->used += bytes;
      S->batches += 1;
      if ((int64_t)batch.size() > S->max_batch_seen) S->max_batch_seen = (int64_t)batch.size();
      std::vector<tsqr_batch_item> items(batch.size());
      for (size_t i = 0; i < batch.size(); ++i) items[i] = batch[i].item;
      lk.unlock();
      tsqr_status st = tsqr::batch_solve_internal(items.data(), (int32_t)items.size(), S->chain_tiles, 0, sl.stream,
                                                  nullptr, sl.hstatus, nullptr, S->ctas_per_sm);
      if (st != TSQR_OK)
        for (size_t i = 0; i < items.size(); ++i) sl.hstatus[i] = (int32_t)st;
      cudaEventRecord(sl.event, sl.stream);
      lk.lock();
      progress = true;
    }
    bool idle = S->pending.empty();
    for (const SrvSlot &sl : S->slots) idle = idle && !sl.busy;
    if (S->stop && idle) break;
    if (!progress) {
      bool any_busy = false;
      for (const SrvSlot &sl : S->slots) any_busy = any_busy || sl.busy;
      if (any_busy)
        S->cv.wait_for(lk, std::chrono::microseconds(10));  // poll the in-flight batches
      else
        S->cv.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

extern "C" {

tsqr_status tsqr_server_create(int64_t max_bytes, int32_t max_batch, int32_t streams, int32_t chain_tiles,
                               int32_t ctas_per_sm, tsqr_server **out) {
  if (!out || max_batch < 1 || streams < 1 || streams > 16 || chain_tiles < 0 || ctas_per_sm < 0 || ctas_per_sm > 2)
    return TSQR_ERR_ARG;
  *out = nullptr;
  tsqr_server *S = new (std::nothrow) tsqr_server();
  if (!S) return TSQR_ERR_OOM;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return TSQR_ERR_CUDA;
  }
  S->budget = max_bytes > 0 ? (size_t)max_bytes : 0;
  S->last_free = tsqr::live_free_bytes();
  S->max_batch = max_batch;
  S->chain_tiles = chain_tiles;
  S->ctas_per_sm = ctas_per_sm;
  S->slots.resize(streams);
  for (SrvSlot &sl : S->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.event, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&sl.hstatus, sizeof(int32_t) * (size_t)max_batch) != cudaSuccess) {
      tsqr_server_destroy(S);
      return TSQR_ERR_CUDA;
    }
  }
  S->worker = std::thread(server_loop, S);
  *out = S;
  return TSQR_OK;
}

tsqr_status tsqr_server_submit(tsqr_server *S, const tsqr_batch_item *item, int64_t *ticket) {
  if (!S || !item) return TSQR_ERR_ARG;
  tsqr_status st = tsqr::check_batch_item(*item, 0);
  if (st != TSQR_OK) return st;
  SrvReq r{*item, 0, Clock::now(), tsqr::batch_item_bytes(*item)};
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r.ticket = S->next_ticket++;
    S->submitted += 1;
    S->pending.push_back(r);
  }
  S->cv.notify_one();
  if (ticket) *ticket = r.ticket;
  return TSQR_OK;
}

tsqr_status tsqr_server_poll(tsqr_server *S, int32_t max, int64_t *tickets, double *latency_s, int32_t *status,
                             int32_t *count) {
  if (!S || !count || max < 0) return TSQR_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  int32_t c = 0;
  while (c < max && !S->done.empty()) {
    const auto &d = S->done.front();
    if (tickets) tickets[c] = std::get<0>(d);
    if (latency_s) latency_s[c] = std::get<1>(d);
    if (status) status[c] = std::get<2>(d);
    S->done.pop_front();
    ++c;
  }
  *count = c;
  return TSQR_OK;
}

tsqr_status tsqr_server_drain(tsqr_server *S) {
  if (!S) return TSQR_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  S->cv_done.wait(lk, [&] { return S->completed == S->submitted; });
  return TSQR_OK;
}

tsqr_status tsqr_server_stats(tsqr_server *S, int64_t *out) {
  if (!S || !out) return TSQR_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  out[0] = S->submitted;
  out[1] = S->completed;
  out[2] = S->batches;
  out[3] = S->max_batch_seen;
  out[4] = (int64_t)(S->budget ? S->budget : S->last_free);
  out[5] = (int64_t)S->used;
  return TSQR_OK;
}

tsqr_status tsqr_server_destroy(tsqr_server *S) {
  if (!S) return TSQR_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (SrvSlot &sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.event) cudaEventDestroy(sl.event);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.hstatus) cudaFreeHost(sl.hstatus);
  }
  delete S;
  return TSQR_OK;
}

}  // extern "C"
