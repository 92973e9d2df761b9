// watch.h -- the serving loop's watchdog over one slot's batch in flight
// (host logic only; no CUDA).
//
// A batch is launched on a slot with a time limit.  Each poll passes whether
// the device work has finished (the slot's completion event) and the current
// time, and the watch says what the loop must do:
//   kDone      the batch finished in time: read its statuses, free the slot;
//   kTimedOut  the limit passed first: report its requests failed now; the
//              slot stays held, and so does every output block of those
//              requests, because the GPU may still be writing them;
//   kRetired   a timed-out batch's work finally finished: only now may its
//              output blocks go back to the budget and the slot take new work;
//   kWaiting / kIdle  nothing to do.
// A batch that never finishes therefore never hands its memory or its slot to
// another request, and its requests still complete (with an error) on time.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace hd {

class SlotWatch {
 public:
  enum class Verdict { kIdle, kWaiting, kDone, kTimedOut, kRetired };

  // A batch was queued at `now_us`; limit_us = 0 waits without limit.
  void launch(uint64_t now_us, uint64_t limit_us) {
    busy_ = true;
    timed_out_ = false;
    t0_ = now_us;
    limit_ = limit_us;
    held_.clear();
  }

  Verdict poll(bool finished, uint64_t now_us) {
    if (!busy_) return Verdict::kIdle;
    if (finished) {
      busy_ = false;
      if (timed_out_) {
        timed_out_ = false;
        return Verdict::kRetired;
      }
      return Verdict::kDone;
    }
    if (!timed_out_ && limit_ && now_us - t0_ > limit_) {
      timed_out_ = true;
      return Verdict::kTimedOut;
    }
    return Verdict::kWaiting;
  }

  // Output blocks of timed-out requests, kept until the batch retires.
  void hold(size_t block) { held_.push_back(block); }
  std::vector<size_t> take_held() {
    std::vector<size_t> h;
    h.swap(held_);
    return h;
  }

  bool busy() const { return busy_; }
  bool timed_out() const { return timed_out_; }
  size_t held() const { return held_.size(); }

 private:
  bool busy_ = false, timed_out_ = false;
  uint64_t t0_ = 0, limit_ = 0;
  std::vector<size_t> held_;
};

}  // namespace hd
