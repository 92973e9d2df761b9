// serve.cpp -- the serving loop of hd.h (hd_serve_*): decode requests against
// resident fields, admitted by a device-memory budget and batched as they
// arrive (continuous batching).
//
// One worker thread owns the GPU side.  It keeps up to `slots` batches in
// flight, each on its own stream with its own decode context (workspace and
// captured graphs), so a batch admitted while others run overlaps them on the
// device.  Whenever a slot is free it takes the oldest pending requests (up to
// max_batch) whose outputs fit the budget -- outputs are carved from one
// device allocation of budget bytes -- and queues them as one hd_decode_batch
// call.  Completion is observed with an event per slot; latency is measured
// from submission to that observation.  A watchdog (watch.h) bounds the wait:
// a batch still running after cfg.watchdog_us has its requests completed with
// HD_ERR_TIMEOUT, while its slot and their output memory stay held until the
// device work really ends.  The paper decodes one field per launch; this loop
// is the serving counterpart of its batched decoder.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arena.h"
#include "hd.h"
#include "watch.h"

namespace {

using Clock = std::chrono::steady_clock;

double us_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::micro>(b - a).count();
}

enum class State { kPending, kInFlight, kDone };

struct Request {
  uint32_t field = 0;
  State state = State::kPending;
  int32_t status = HD_PENDING;
  size_t out_off = hd::Arena::kNone;
  Clock::time_point t_submit, t_launch, t_done;
};

// Worker-owned: one batch in flight at most.
struct Slot {
  hd_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  hd::SlotWatch watch;
  std::vector<uint64_t> tickets;
};

constexpr uint64_t kDefaultWatchdogUs = 10000000;  // 10 s

uint64_t now_us() {
  return static_cast<uint64_t>(
      std::chrono::duration_cast<std::chrono::microseconds>(Clock::now().time_since_epoch())
          .count());
}

}  // namespace

struct hd_server {
  int device = 0;
  hd_serve_config cfg{};
  char* base = nullptr;  // device allocation of cfg.budget_bytes
  std::vector<Slot> slots;
  std::thread worker;

  std::mutex mu;  // guards everything below
  std::condition_variable cv_work, cv_done;
  hd::Arena arena;
  std::vector<hd_field> fields;
  std::deque<uint64_t> pending;
  std::deque<uint64_t> finished;  // completed tickets not yet handed out
  std::unordered_map<uint64_t, Request> reqs;
  uint64_t next_ticket = 1;
  std::atomic<uint64_t> wake{0};  // bumped by submit / release / stop
  size_t inflight = 0;
  bool stop = false;
  uint64_t submitted = 0, completed = 0, batches = 0;
  uint64_t watchdog_us = 0;  // per-batch limit (0: none)
  uint64_t retired = 0;      // timed-out batches whose work ended later
  uint64_t stop_us = 0;      // when shutdown found only timed-out batches left
};

namespace {

int check_resident(const hd_field* f) {
  if (!f || !f->lengths) return HD_ERR_ARG;
  if (f->subseq_bits != 64 && f->subseq_bits != 128 && f->subseq_bits != 256) return HD_ERR_ARG;
  if (f->alphabet < 2 || f->alphabet > 65536) return HD_ERR_ARG;
  if (f->n == 0 && f->nbits == 0) return HD_OK;
  if (!f->words || (reinterpret_cast<uintptr_t>(f->words) & 15u)) return HD_ERR_ARG;
  if (f->nwords * 32 < f->nbits) return HD_ERR_ARG;
  return HD_OK;
}

// Marks the requests of a finished (or failed) slot done.  With `hold` (the
// batch timed out and may still be running) their output blocks move to the
// slot's watch instead of staying with the requests, so releasing a request
// cannot hand memory the GPU may still write to another one.
void finish_requests(hd_server* s, Slot& sl, const std::vector<int32_t>& st, bool hold) {
  const auto now = Clock::now();
  for (size_t j = 0; j < sl.tickets.size(); ++j) {
    auto it = s->reqs.find(sl.tickets[j]);
    if (it == s->reqs.end()) continue;
    Request& r = it->second;
    r.status = st[j];
    r.t_done = now;
    r.state = State::kDone;
    if (hold && r.out_off != hd::Arena::kNone) {
      sl.watch.hold(r.out_off);
      r.out_off = hd::Arena::kNone;
    }
    s->finished.push_back(sl.tickets[j]);
  }
  s->inflight -= sl.tickets.size();
  s->completed += sl.tickets.size();
  sl.tickets.clear();
  s->cv_done.notify_all();
}

bool any_busy(const hd_server* s) {
  for (const auto& sl : s->slots)
    if (sl.watch.busy()) return true;
  return false;
}

void serve_loop(hd_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    bool progressed = false;
    // completions, time-outs and retirements
    for (auto& sl : s->slots) {
      if (!sl.watch.busy()) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      const auto v = sl.watch.poll(q != cudaErrorNotReady, now_us());
      if (v == hd::SlotWatch::Verdict::kWaiting) continue;
      progressed = true;
      if (v == hd::SlotWatch::Verdict::kTimedOut) {
        finish_requests(s, sl, std::vector<int32_t>(sl.tickets.size(), HD_ERR_TIMEOUT), true);
        continue;
      }
      if (q != cudaSuccess && q != cudaErrorNotReady) cudaGetLastError();
      if (v == hd::SlotWatch::Verdict::kRetired) {
        // the late batch's statuses were reported as time-outs already
        for (size_t off : sl.watch.take_held()) s->arena.release(off);
        ++s->retired;
        continue;
      }
      std::vector<int32_t> st(sl.tickets.size(), HD_ERR_CUDA);
      if (q == cudaSuccess) {
        lk.unlock();
        if (s->cfg.direct) {
          st[0] = hd_status(sl.ctx, sl.stream);
        } else {
          hd_batch_status(sl.ctx, st.data(), static_cast<uint32_t>(st.size()), sl.stream);
        }
        lk.lock();
      }
      finish_requests(s, sl, st, false);
    }
    // admissions: oldest requests first, while their outputs fit the budget
    for (auto& sl : s->slots) {
      if (sl.watch.busy() || s->pending.empty()) continue;
      std::vector<uint64_t> take;
      while (!s->pending.empty() && take.size() < s->cfg.max_batch) {
        Request& r = s->reqs[s->pending.front()];
        const size_t off = s->arena.alloc(2 * s->fields[r.field].n);
        if (off == hd::Arena::kNone) break;
        r.out_off = off;
        take.push_back(s->pending.front());
        s->pending.pop_front();
      }
      if (take.empty()) break;  // the oldest request waits for memory
      std::vector<hd_field> fs;
      std::vector<uint16_t*> outs;
      const auto now = Clock::now();
      for (uint64_t t : take) {
        Request& r = s->reqs[t];
        r.state = State::kInFlight;
        r.t_launch = now;
        fs.push_back(s->fields[r.field]);
        outs.push_back(reinterpret_cast<uint16_t*>(s->base + r.out_off));
      }
      sl.tickets = take;
      sl.watch.launch(now_us(), s->watchdog_us);
      s->inflight += take.size();
      s->batches += 1;
      lk.unlock();
      int rc;
      if (s->cfg.direct) {
        rc = hd_decode(sl.ctx, &fs[0], outs[0], sl.stream);
      } else {
        rc = hd_decode_batch(sl.ctx, fs.data(), static_cast<uint32_t>(fs.size()), outs.data(),
                             sl.stream);
      }
      if (rc == HD_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) rc = HD_ERR_CUDA;
      lk.lock();
      if (rc != HD_OK) {
        finish_requests(s, sl, std::vector<int32_t>(take.size(), rc), false);
        sl.watch.poll(true, now_us());  // nothing was queued: the slot is free again
      }
      progressed = true;
    }
    if (s->stop && !s->pending.empty()) {
      // shutting down: requests not yet admitted are dropped
      const auto now = Clock::now();
      for (uint64_t t : s->pending) {
        Request& r = s->reqs[t];
        r.status = HD_ERR_BUSY;
        r.t_launch = r.t_done = now;
        r.state = State::kDone;
        s->finished.push_back(t);
      }
      s->pending.clear();
      s->cv_done.notify_all();
    }
    if (s->stop && s->inflight == 0) {
      // timed-out batches still on the GPU keep their slots until they end,
      // for one more watchdog period; after that they are abandoned
      if (!any_busy(s)) break;
      if (!s->stop_us) s->stop_us = now_us();
      if (now_us() - s->stop_us > s->watchdog_us) break;
    }
    if (progressed) continue;
    const uint64_t w = s->wake.load();
    if (s->inflight) {
      // batches on the GPU: poll their events briefly, then look again
      lk.unlock();
      for (int k = 0; k < 64 && s->wake.load() == w; ++k) {
        bool ready = false;
        for (auto& sl : s->slots)
          ready |= sl.watch.busy() && cudaEventQuery(sl.done) != cudaErrorNotReady;
        if (ready) break;
        std::this_thread::yield();
      }
      lk.lock();
    } else if (any_busy(s)) {
      // only timed-out batches are left on the GPU: look again later
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(200));
      lk.lock();
    } else {
      s->cv_work.wait(lk, [&] { return s->wake.load() != w; });
    }
  }
}

}  // namespace

extern "C" {

int hd_serve_create(int device, const hd_serve_config* cfg, const hd_config* shape,
                    hd_server** out) {
  if (!out || !cfg) return HD_ERR_ARG;
  *out = nullptr;
  if (cfg->slots < 1 || cfg->slots > 8 || cfg->max_batch < 1 || cfg->max_batch > 4096 ||
      cfg->budget_bytes < hd::Arena::kAlign || (cfg->direct && cfg->max_batch != 1))
    return HD_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return HD_ERR_CUDA;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  hd_server* s = new (std::nothrow) hd_server();
  if (!s) return HD_ERR_NOMEM;
  s->device = device;
  s->cfg = *cfg;
  if (!s->cfg.queue_cap) s->cfg.queue_cap = 1u << 20;
  s->watchdog_us = cfg->watchdog_us ? cfg->watchdog_us : kDefaultWatchdogUs;
  int rc = HD_OK;
  if (cudaMalloc(&s->base, cfg->budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    rc = HD_ERR_NOMEM;
  }
  s->arena.reset(cfg->budget_bytes);
  s->slots.resize(cfg->slots);
  for (auto& sl : s->slots) {
    if (rc) break;
    rc = hd_ctx_create(device, &sl.ctx);
    if (!rc && shape) rc = hd_set_config(sl.ctx, shape);
    if (!rc && (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      rc = HD_ERR_CUDA;
    }
  }
  if (rc) {
    for (auto& sl : s->slots) {
      if (sl.ctx) hd_ctx_destroy(sl.ctx);
      if (sl.stream) cudaStreamDestroy(sl.stream);
      if (sl.done) cudaEventDestroy(sl.done);
    }
    if (s->base) cudaFree(s->base);
    delete s;
    cudaSetDevice(prev);
    return rc;
  }
  s->worker = std::thread(serve_loop, s);
  cudaSetDevice(prev);
  *out = s;
  return HD_OK;
}

int hd_serve_destroy(hd_server* s) {
  if (!s) return HD_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    ++s->wake;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  bool abandoned = false;
  for (auto& sl : s->slots) {
    if (sl.watch.busy()) {
      // a timed-out batch that never ended: its context, stream and the
      // output memory stay allocated rather than freed under running work
      abandoned = true;
      continue;
    }
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.ctx) hd_ctx_destroy(sl.ctx);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
  }
  if (s->base && !abandoned) cudaFree(s->base);
  cudaSetDevice(prev);
  delete s;
  return HD_OK;
}

int hd_serve_register(hd_server* s, const hd_field* f, uint32_t* field_id) {
  if (!s || !field_id) return HD_ERR_ARG;
  const int rc = check_resident(f);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(s->mu);
  *field_id = static_cast<uint32_t>(s->fields.size());
  s->fields.push_back(*f);
  return HD_OK;
}

int hd_serve_submit(hd_server* s, uint32_t field_id, uint64_t* ticket) {
  if (!s || !ticket) return HD_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (field_id >= s->fields.size()) return HD_ERR_ARG;
    if (s->stop || s->pending.size() >= s->cfg.queue_cap) return HD_ERR_BUSY;
    if (hd::Arena::round(2 * s->fields[field_id].n) > s->arena.capacity()) return HD_ERR_NOMEM;
    const uint64_t t = s->next_ticket++;
    Request& r = s->reqs[t];
    r.field = field_id;
    r.t_submit = Clock::now();
    s->pending.push_back(t);
    s->submitted += 1;
    ++s->wake;
    *ticket = t;
  }
  s->cv_work.notify_one();
  return HD_OK;
}

int hd_serve_poll(hd_server* s, uint64_t ticket, hd_result* res) {
  if (!s || !res) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return HD_ERR_ARG;
  const Request& r = it->second;
  if (r.state != State::kDone) return HD_PENDING;
  res->status = r.status;
  res->d_out = r.out_off == hd::Arena::kNone
                   ? nullptr
                   : reinterpret_cast<const uint16_t*>(s->base + r.out_off);
  res->n = s->fields[r.field].n;
  res->queue_us = us_between(r.t_submit, r.t_launch);
  res->latency_us = us_between(r.t_submit, r.t_done);
  return HD_OK;
}

int hd_serve_release(hd_server* s, uint64_t ticket) {
  if (!s) return HD_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return HD_ERR_ARG;
    if (it->second.state != State::kDone) return HD_ERR_BUSY;
    if (it->second.out_off != hd::Arena::kNone) s->arena.release(it->second.out_off);
    s->reqs.erase(it);
    ++s->wake;
  }
  s->cv_work.notify_one();
  return HD_OK;
}

int hd_serve_completed(hd_server* s, uint64_t* tickets, uint32_t cap, uint32_t* count) {
  if (!s || !count || (cap && !tickets)) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  uint32_t k = 0;
  while (k < cap && !s->finished.empty()) {
    tickets[k++] = s->finished.front();
    s->finished.pop_front();
  }
  *count = k;
  return HD_OK;
}

int hd_serve_drain(hd_server* s) {
  if (!s) return HD_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] { return s->pending.empty() && s->inflight == 0; });
  return HD_OK;
}

int hd_serve_stats(hd_server* s, hd_serve_stats_t* out) {
  if (!s || !out) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->batches = s->batches;
  out->pending = s->pending.size();
  out->in_flight = s->inflight;
  out->budget_bytes = s->arena.capacity();
  out->used_bytes = s->arena.used();
  out->peak_bytes = s->arena.peak();
  uint64_t held = 0;
  for (const auto& sl : s->slots) held += sl.watch.timed_out() ? 1 : 0;
  out->timed_out_batches = held;
  out->retired_batches = s->retired;
  return HD_OK;
}

}  // extern "C"
