// arena.h -- first-fit sub-allocator over one fixed byte range (host logic
// only; no CUDA).  The serving loop carves request outputs out of one device
// allocation sized by its admission budget with it, so admitting a request
// never calls cudaMalloc and the budget is a hard limit.
#pragma once

#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

namespace hd {

class Arena {
 public:
  static constexpr size_t kAlign = 256;
  static constexpr size_t kNone = ~static_cast<size_t>(0);

  void reset(size_t capacity) {
    cap_ = capacity / kAlign * kAlign;
    used_ = 0;
    peak_ = 0;
    free_.clear();
    live_.clear();
    if (cap_) free_[0] = cap_;
  }

  // Offset of a new block of at least `bytes` (kAlign-aligned), or kNone when
  // no free range is large enough.  Zero-byte requests get a kAlign block.
  size_t alloc(size_t bytes) {
    const size_t need = round(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      const size_t off = it->first;
      const size_t rest = it->second - need;
      free_.erase(it);
      if (rest) free_[off + need] = rest;
      live_[off] = need;
      used_ += need;
      if (used_ > peak_) peak_ = used_;
      return off;
    }
    return kNone;
  }

  // Returns a block; false for an offset that is not a live block.
  bool release(size_t off) {
    auto lit = live_.find(off);
    if (lit == live_.end()) return false;
    size_t start = off, len = lit->second;
    used_ -= len;
    live_.erase(lit);
    auto next = free_.lower_bound(start);
    if (next != free_.end() && next->first == start + len) {  // merge with the right
      len += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {  // merge with the left
      auto prev = std::prev(next);
      if (prev->first + prev->second == start) {
        start = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    free_[start] = len;
    return true;
  }

  size_t capacity() const { return cap_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }
  size_t live_blocks() const { return live_.size(); }
  size_t free_ranges() const { return free_.size(); }
  // Largest block alloc() could return now.
  size_t largest_free() const {
    size_t m = 0;
    for (const auto& kv : free_) m = kv.second > m ? kv.second : m;
    return m;
  }
  static size_t round(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

 private:
  size_t cap_ = 0, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length, disjoint, coalesced
  std::map<size_t, size_t> live_;  // offset -> length
};

}  // namespace hd
