// Randomised check of the serving loop's output sub-allocator (host logic,
// no GPU): blocks are aligned, inside the range and disjoint; freed space
// coalesces back into one range; `used` and `peak` track the live bytes; a
// request larger than every free range fails instead of overlapping.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "arena.h"

static int fail(const char* what, unsigned long long a, unsigned long long b) {
  std::printf("FAIL %s %llu %llu\n", what, a, b);
  return 1;
}

int main(int argc, char** argv) {
  const unsigned seed = argc > 1 ? static_cast<unsigned>(std::atoi(argv[1])) : 1u;
  std::mt19937_64 rng(seed);
  const size_t cap = (1u << 20) + 77;  // not a multiple of the alignment
  hd::Arena a;
  a.reset(cap);
  if (a.capacity() != (cap / hd::Arena::kAlign) * hd::Arena::kAlign)
    return fail("capacity", a.capacity(), cap);
  std::vector<char> owner(a.capacity(), 0);  // byte map of live blocks
  struct Blk { size_t off, len; };
  std::vector<Blk> live;
  size_t used = 0, peak = 0;
  for (int step = 0; step < 20000; ++step) {
    const bool do_alloc = live.empty() || (rng() % 100) < 55;
    if (do_alloc) {
      const size_t want = rng() % 3 == 0 ? rng() % 64 : rng() % 40000;
      const size_t off = a.alloc(want);
      const size_t len = hd::Arena::round(want ? want : 1);
      if (off == hd::Arena::kNone) {
        if (a.largest_free() >= len) return fail("spurious failure", want, a.largest_free());
        continue;
      }
      if (off % hd::Arena::kAlign) return fail("alignment", off, want);
      if (off + len > a.capacity()) return fail("range", off, len);
      for (size_t i = off; i < off + len; ++i)
        if (owner[i]) return fail("overlap", off, i);
      for (size_t i = off; i < off + len; ++i) owner[i] = 1;
      live.push_back({off, len});
      used += len;
      if (used > peak) peak = used;
    } else {
      const size_t k = rng() % live.size();
      const Blk b = live[k];
      live[k] = live.back();
      live.pop_back();
      if (!a.release(b.off)) return fail("release", b.off, b.len);
      if (a.release(b.off)) return fail("double release accepted", b.off, b.len);
      for (size_t i = b.off; i < b.off + b.len; ++i) owner[i] = 0;
      used -= b.len;
    }
    if (a.used() != used) return fail("used", a.used(), used);
    if (a.peak() != peak) return fail("peak", a.peak(), peak);
    if (a.live_blocks() != live.size()) return fail("live", a.live_blocks(), live.size());
  }
  for (const Blk& b : live) a.release(b.off);
  if (a.used() != 0 || a.free_ranges() != 1 || a.largest_free() != a.capacity())
    return fail("coalesce", a.free_ranges(), a.largest_free());
  if (a.alloc(a.capacity() + 1) != hd::Arena::kNone) return fail("oversize", a.capacity(), 0);
  if (a.alloc(a.capacity()) != 0) return fail("whole range", a.capacity(), 0);
  std::printf("ok\n");
  return 0;
}
