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
//
// The resident server (tsqr_server_create_resident) admits requests into a kernel that
// is already running instead: one persistent kernel (resident.cu) stays on the GPU and
// claims work from a ring in device memory, and the worker appends each admitted request
// to the ring while the kernel runs. Each request gets a block of a device arena carved
// out at creation (first fit), a slot in the kernel's request table and a completion
// word in mapped host memory; the kernel is launched again whenever requests are in
// flight and the previous launch has ended (it ends once idle).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/tsqr.h"
#include "tsqr_internal.h"

using Clock = std::chrono::steady_clock;

namespace {

struct PlanFree {
  void operator()(tsqr::ResidentPlan *p) const {
    tsqr::resident_plan_free(*p);
    delete p;
  }
};
using PlanPtr = std::shared_ptr<tsqr::ResidentPlan>;

struct SrvReq {
  tsqr_batch_item item;
  int64_t ticket;
  Clock::time_point t0;
  size_t bytes;
  PlanPtr plan;  // resident server: the request's plan, made at submission
};

// First-fit allocator over the resident server's arena (offsets, 256-byte granules).
class Arena {
 public:
  void reset(size_t bytes) {
    free_.clear();
    if (bytes >= 256) free_[0] = bytes & ~(size_t)255;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t &off) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      off = it->first;
      const size_t rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[off + bytes] = rest;
      used_ += bytes;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    used_ -= bytes;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;  // offset -> bytes
  size_t used_ = 0;
};

constexpr int32_t kResSlots = 4096;
constexpr unsigned long long kRingCap = 1ull << 20;   // host ring entries (chain jobs)
constexpr unsigned long long kDringCap = 1ull << 20;  // device ring entries (refinement tasks)
// Test hook (tsqr_debug_resident_ring_entries): both rings of resident servers created
// afterwards get this many entries (0: the defaults above), so that tests wrap them.
std::atomic<unsigned long long> g_ring_entries{0};

struct ResLive {
  SrvReq req;
  size_t off = 0, bytes = 0;
  int32_t seq = 0;
  bool active = false;
  int cls = 0;                   // its host ring (0: at most kResSmallChains chain jobs)
  unsigned long long first = 0;  // its first entry in that ring
  int64_t dtasks = 0;            // device-ring entries it can hold at once
};

struct ResState {
  char *arena = nullptr;
  size_t arena_bytes = 0;
  Arena alloc;
  tsqr::ResCtl *ctl = nullptr;
  tsqr::ResEntry *ring = nullptr;
  tsqr::ResTask *dring = nullptr;
  tsqr::ResItemDev *items = nullptr;
  int32_t *hdone = nullptr, *hstatus = nullptr;  // mapped pinned host memory
  int32_t *ddone = nullptr, *dstatus = nullptr;  // their device addresses
  int32_t *err = nullptr;
  cudaStream_t up = nullptr, ks = nullptr;
  cudaEvent_t kev = nullptr;
  bool running = false, stop_sent = false;
  size_t smem = 0;
  int grid = 0;
  int64_t idle_polls = 64;
  unsigned long long ring_cap = kRingCap, dring_cap = kDringCap;  // powers of two
  unsigned long long tail[2] = {0, 0};
  bool published[2] = {false, false};  // a ring's tail moved since its last copy
  int64_t dtasks = 0, nlive = 0, max_live = 0, launches = 0;
  int32_t next_seq = 0;
  std::vector<ResLive> live;
  std::vector<int32_t> free_slots;
  std::vector<int32_t> active;  // slots of the requests in flight (any order)
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
  std::unique_ptr<ResState> res;  // set for a resident server
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

// Completes a resident request (the worker holds the lock).
static void res_finish(tsqr_server *S, ResState &R, int32_t slot, int32_t status) {
  ResLive &L = R.live[slot];
  const double lat = std::chrono::duration<double>(Clock::now() - L.req.t0).count();
  S->done.emplace_back(L.req.ticket, lat, status);
  S->completed += 1;
  R.alloc.release(L.off, L.bytes);
  R.dtasks -= L.dtasks;
  R.nlive -= 1;
  L.active = false;
  L.req.plan.reset();
  R.free_slots.push_back(slot);
  for (size_t a = 0; a < R.active.size(); ++a)
    if (R.active[a] == slot) {
      R.active[a] = R.active.back();
      R.active.pop_back();
      break;
    }
  S->cv_done.notify_all();
}

// A request that never reached the kernel (the library refused it) completes at once.
static void res_reject(tsqr_server *S, const SrvReq &r, int32_t status) {
  const double lat = std::chrono::duration<double>(Clock::now() - r.t0).count();
  S->done.emplace_back(r.ticket, lat, status);
  S->completed += 1;
  S->cv_done.notify_all();
}

static cudaError_t res_copy(void *dst, const void *src, size_t bytes, cudaStream_t s) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
}

// Admits the oldest pending request into the running (or next) launch of the resident
// kernel; false when it has to wait for room.
static bool res_admit(tsqr_server *S, ResState &R) {
  SrvReq r = S->pending.front();
  const tsqr::ResidentPlan &p = *r.plan;
  const int cls = p.nchains <= tsqr::kResSmallChains ? 0 : 1;
  unsigned long long oldest = R.tail[cls];  // entries before it belong to completed requests
  for (const int32_t q : R.active)
    if (R.live[q].cls == cls) oldest = std::min(oldest, R.live[q].first);
  const int64_t need_d = (int64_t)p.ngroups * p.nt;
  if (R.free_slots.empty() || R.tail[cls] + (unsigned long long)p.nchains - oldest > R.ring_cap ||
      R.dtasks + need_d > (int64_t)R.dring_cap)
    return false;
  size_t off = 0;
  if (!R.alloc.alloc(p.bytes, off)) {
    if (R.nlive > 0) return false;  // wait for memory to come back
    S->pending.pop_front();
    res_reject(S, r, (int32_t)TSQR_ERR_OOM);
    return true;
  }
  if (tsqr::debug_take_allocation_failure()) {  // failure injection: the block "failed"
    R.alloc.release(off, p.bytes);
    S->pending.pop_front();
    res_reject(S, r, (int32_t)TSQR_ERR_OOM);
    return true;
  }
  S->pending.pop_front();
  const int32_t slot = R.free_slots.back();
  R.free_slots.pop_back();
  const int32_t seq = ++R.next_seq == 0 ? ++R.next_seq : R.next_seq;
  tsqr::ResItemDev dev{};
  tsqr_status st = tsqr::resident_upload(p, R.arena + off, R.up, dev);
  cudaError_t e = cudaSuccess;
  if (st == TSQR_OK) {
    dev.seq = seq;
    R.hdone[slot] = 0;
    e = res_copy(R.items + slot, &dev, sizeof(dev), R.up);
    // the request's chain jobs into the host ring (two pieces where it wraps)
    std::vector<tsqr::ResEntry> ent((size_t)p.nchains);
    for (int32_t j = 0; j < p.nchains; ++j) ent[(size_t)j] = {slot, j};
    tsqr::ResEntry *ring = R.ring + (size_t)cls * R.ring_cap;
    size_t done = 0;
    while (e == cudaSuccess && done < ent.size()) {
      const unsigned long long pos = (R.tail[cls] + done) & (R.ring_cap - 1);
      const size_t cnt = std::min(ent.size() - done, (size_t)(R.ring_cap - pos));
      e = res_copy(ring + pos, ent.data() + done, sizeof(tsqr::ResEntry) * cnt, R.up);
      done += cnt;
    }
  }
  ResLive &L = R.live[slot];
  L.req = r;
  L.off = off;
  L.bytes = p.bytes;
  L.seq = seq;
  L.cls = cls;
  L.first = R.tail[cls];
  L.dtasks = need_d;
  L.active = true;
  R.active.push_back(slot);
  R.dtasks += need_d;
  R.nlive += 1;
  R.max_live = std::max(R.max_live, R.nlive);
  if (st != TSQR_OK || e != cudaSuccess) {  // nothing of it was published
    res_finish(S, R, slot, (int32_t)(st != TSQR_OK ? st : TSQR_ERR_CUDA));
    return true;
  }
  R.tail[cls] += (unsigned long long)p.nchains;
  R.published[cls] = true;
  return true;
}

// Every request in flight fails (the kernel reported a lost work entry, or a launch or an
// upload failed); the rings start over empty once no launch is running (a running one ends
// by itself within its bounded polls: nothing new is published for it).
static void res_fail_all(tsqr_server *S, ResState &R, int32_t status) {
  if (R.running) {
    cudaEventSynchronize(R.kev);
    R.running = false;
  }
  cudaStreamSynchronize(R.up);
  while (!R.active.empty()) res_finish(S, R, R.active.back(), status);
  cudaMemsetAsync(R.ctl, 0, sizeof(tsqr::ResCtl), R.ks);
  const int32_t zero = 0;
  cudaMemcpyAsync(R.err, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, R.ks);
  cudaStreamSynchronize(R.ks);
  R.tail[0] = R.tail[1] = 0;
  R.published[0] = R.published[1] = false;
}

static void resident_loop(tsqr_server *S) {
  cudaSetDevice(S->device);
  ResState &R = *S->res;
  tsqr::ResParams kp{};
  kp.ctl = R.ctl;
  kp.ring = R.ring;
  kp.dring = R.dring;
  kp.items = R.items;
  kp.hstatus = R.dstatus;
  kp.hdone = R.ddone;
  kp.err = R.err;
  kp.ring_mask = R.ring_cap - 1;
  kp.dring_mask = R.dring_cap - 1;
  kp.idle_polls = R.idle_polls;
  kp.refine_rows = tsqr::refine_rows_per_task();
  kp.max_steps = tsqr::refine_max_steps();
  kp.tol = tsqr::refine_tolerance();
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool progress = false;
    // completions: the kernel writes the status, then the request's sequence number
    for (size_t a = 0; a < R.active.size();) {
      const int32_t q = R.active[a];
      if (__atomic_load_n(R.hdone + q, __ATOMIC_ACQUIRE) != R.live[q].seq) {
        ++a;
        continue;
      }
      res_finish(S, R, q, __atomic_load_n(R.hstatus + q, __ATOMIC_ACQUIRE));  // moves the last slot here
      progress = true;
    }
    // the launch ended (idle, or a lost entry: the error word says which)
    if (R.running && cudaEventQuery(R.kev) != cudaErrorNotReady) {
      R.running = false;
      int32_t word = 0;
      cudaError_t e = cudaMemcpyAsync(&word, R.err, sizeof(int32_t), cudaMemcpyDeviceToHost, R.ks);
      if (e == cudaSuccess) e = cudaStreamSynchronize(R.ks);
      if (e != cudaSuccess || (word & tsqr::kErrTimeout))
        res_fail_all(S, R, (int32_t)(e != cudaSuccess ? TSQR_ERR_CUDA : TSQR_ERR_TIMEOUT));
      progress = true;
    }
    // admission into the running kernel
    while (!S->pending.empty() && res_admit(S, R)) progress = true;
    for (int c = 0; c < 2; ++c) {
      if (!R.published[c]) continue;
      R.published[c] = false;
      const unsigned long long t = R.tail[c];  // staged by the copy before the call returns
      if (res_copy(&R.ctl->tail[c], &t, sizeof(t), R.up) != cudaSuccess) res_fail_all(S, R, (int32_t)TSQR_ERR_CUDA);
    }
    // a launch whenever requests are in flight and none is running
    if (!R.running && R.nlive > 0) {
      cudaError_t e = cudaMemsetAsync(&R.ctl->quit, 0, sizeof(int32_t), R.ks);
      if (e == cudaSuccess) e = tsqr::launch_resident(kp, R.grid, R.smem, R.ks);
      if (e == cudaSuccess) e = cudaEventRecord(R.kev, R.ks);
      if (e == cudaSuccess) {
        R.running = true;
        R.launches += 1;
        S->batches += 1;
      } else {
        res_fail_all(S, R, (int32_t)TSQR_ERR_CUDA);
      }
      progress = true;
    }
    if (S->stop && S->pending.empty() && R.nlive == 0) {
      if (!R.running) break;
      if (!R.stop_sent) {  // the kernel ends as soon as it finds nothing to claim
        const int32_t one = 1;
        res_copy(&R.ctl->stop, &one, sizeof(one), R.up);
        R.stop_sent = true;
      }
    }
    if (!progress) S->cv.wait_for(lk, R.running ? std::chrono::microseconds(20) : std::chrono::milliseconds(5));
  }
}

// Frees the resident server's device and host memory (the kernel has ended).
static void res_release(ResState &R) {
  if (R.ks) cudaStreamSynchronize(R.ks);
  if (R.up) cudaStreamSynchronize(R.up);
  if (R.kev) cudaEventDestroy(R.kev);
  if (R.ks) cudaStreamDestroy(R.ks);
  if (R.up) cudaStreamDestroy(R.up);
  for (void *p : {(void *)R.arena, (void *)R.ctl, (void *)R.ring, (void *)R.dring, (void *)R.items})
    if (p) cudaFree(p);
  if (R.hdone) cudaFreeHost(R.hdone);
  if (R.hstatus) cudaFreeHost(R.hstatus);
  R = ResState{};
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

tsqr_status tsqr_server_create_resident(int64_t max_bytes, int32_t chain_tiles, int32_t ctas_per_sm, int32_t idle_us,
                                        tsqr_server **out) {
  tsqr::clear_last_error();
  if (!out || chain_tiles < 0 || ctas_per_sm < 0 || ctas_per_sm > 2 || idle_us < 0)
    return tsqr::set_last_error(TSQR_ERR_ARG, "bad chain_tiles, ctas_per_sm or idle_us");
  *out = nullptr;
  tsqr_server *S = new (std::nothrow) tsqr_server();
  if (!S) return TSQR_ERR_OOM;
  S->res.reset(new (std::nothrow) ResState());
  if (!S->res) {
    delete S;
    return TSQR_ERR_OOM;
  }
  ResState &R = *S->res;
  S->chain_tiles = chain_tiles;
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDevice(&S->device);
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, S->device);
  if (e != cudaSuccess) {
    delete S;
    return tsqr::set_last_error(TSQR_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
  }
  const int cps = ctas_per_sm == 0 ? 2 : ctas_per_sm;
  R.smem = tsqr::resident_smem_bytes(cps);
  R.grid = prop.multiProcessorCount * cps;
  R.idle_polls = std::max<int64_t>(8, (int64_t)idle_us / 32);
  size_t arena = max_bytes > 0 ? (size_t)max_bytes : tsqr::live_free_bytes() / 4;
  arena &= ~(size_t)255;
  R.arena_bytes = arena;
  R.live.resize(kResSlots);
  for (int32_t q = kResSlots - 1; q >= 0; --q) R.free_slots.push_back(q);
  e = cudaMalloc(&R.arena, arena);
  if (e == cudaSuccess) e = cudaMalloc(&R.ctl, sizeof(tsqr::ResCtl));
  if (const unsigned long long cap = g_ring_entries.load()) R.ring_cap = R.dring_cap = cap;
  if (e == cudaSuccess) e = cudaMalloc(&R.ring, sizeof(tsqr::ResEntry) * 2 * R.ring_cap);
  if (e == cudaSuccess) e = cudaMalloc(&R.dring, sizeof(tsqr::ResTask) * R.dring_cap);
  if (e == cudaSuccess) e = cudaMalloc(&R.items, sizeof(tsqr::ResItemDev) * kResSlots);
  if (e == cudaSuccess) e = cudaHostAlloc(&R.hdone, sizeof(int32_t) * kResSlots, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostAlloc(&R.hstatus, sizeof(int32_t) * kResSlots, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&R.ddone, R.hdone, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&R.dstatus, R.hstatus, 0);
  if (e == cudaSuccess) e = tsqr::device_error_word(&R.err);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&R.up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&R.ks, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R.kev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(R.ctl, 0, sizeof(tsqr::ResCtl), R.up);
  if (e == cudaSuccess) e = cudaMemsetAsync(R.dring, 0, sizeof(tsqr::ResTask) * R.dring_cap, R.up);
  if (e == cudaSuccess) e = cudaStreamSynchronize(R.up);  // before any launch
  if (e != cudaSuccess) {
    const tsqr_status st = tsqr::set_last_error(e == cudaErrorMemoryAllocation ? TSQR_ERR_OOM : TSQR_ERR_CUDA,
                                                "resident server set-up: %s", cudaGetErrorString(e));
    res_release(R);
    delete S;
    return st;
  }
  memset(R.hdone, 0, sizeof(int32_t) * kResSlots);
  memset(R.hstatus, 0, sizeof(int32_t) * kResSlots);
  R.alloc.reset(arena);
  S->worker = std::thread(resident_loop, S);
  *out = S;
  return TSQR_OK;
}

tsqr_status tsqr_debug_resident_ring_entries(int64_t entries) {
  if (entries != 0 && (entries < 16 || (entries & (entries - 1)) != 0)) return TSQR_ERR_ARG;
  g_ring_entries.store((unsigned long long)entries);
  return TSQR_OK;
}

tsqr_status tsqr_server_submit(tsqr_server *S, const tsqr_batch_item *item, int64_t *ticket) {
  if (!S || !item) return TSQR_ERR_ARG;
  tsqr_status st = tsqr::check_batch_item(*item, 0);
  if (st != TSQR_OK) return st;
  SrvReq r{*item, 0, Clock::now(), tsqr::batch_item_bytes(*item), nullptr};
  if (S->res) {  // plan now: a request the resident kernel cannot run is refused here
    PlanPtr p(new (std::nothrow) tsqr::ResidentPlan(), PlanFree());
    if (!p) return TSQR_ERR_OOM;
    st = tsqr::resident_plan(*item, S->chain_tiles, *p);
    if (st != TSQR_OK) return st;
    if (p->smem > S->res->smem)
      return tsqr::set_last_error(TSQR_ERR_UNSUPPORTED,
                                  "request needs %zu bytes of shared memory per CTA, the resident kernel has %zu",
                                  p->smem, S->res->smem);
    if (p->bytes > S->res->arena_bytes)
      return tsqr::set_last_error(TSQR_ERR_UNSUPPORTED, "request needs %zu bytes of the %zu-byte arena", p->bytes,
                                  S->res->arena_bytes);
    if ((unsigned long long)p->nchains > S->res->ring_cap ||
        (unsigned long long)p->ngroups * (unsigned long long)p->nt > S->res->dring_cap)
      return tsqr::set_last_error(TSQR_ERR_UNSUPPORTED, "request has more jobs (%d chains, %d tasks) than a ring holds",
                                  p->nchains, p->ngroups * p->nt);
    r.bytes = p->bytes;
    r.plan = p;
  }
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
  if (S->res) {
    out[3] = S->res->max_live;
    out[4] = (int64_t)S->res->arena_bytes;
    out[5] = (int64_t)S->res->alloc.used();
    return TSQR_OK;
  }
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
  if (S->res) res_release(*S->res);
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
