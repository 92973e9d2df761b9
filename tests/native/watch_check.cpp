// Check of the serving loop's watchdog state machine (host logic, no GPU):
// a batch whose completion never comes times out exactly once, after its
// limit and not before; its output blocks stay held (never handed back) until
// the work finishes, and then come back exactly once; a batch that finishes in
// time is done without holding anything; a zero limit never times out.
// Randomised sequences drive a fake clock and a fake completion event.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "watch.h"

using V = hd::SlotWatch::Verdict;

static int fail(const char* what, long long a, long long b) {
  std::printf("FAIL %s %lld %lld\n", what, a, b);
  return 1;
}

int main(int argc, char** argv) {
  const unsigned seed = argc > 1 ? static_cast<unsigned>(std::atoi(argv[1])) : 1u;
  std::mt19937_64 rng(seed);

  // an event that never completes: times out once, then waits forever
  {
    hd::SlotWatch w;
    if (w.poll(false, 0) != V::kIdle) return fail("idle", 0, 0);
    w.launch(1000, 50);
    for (uint64_t t = 1000; t <= 1050; ++t)
      if (w.poll(false, t) != V::kWaiting) return fail("early timeout", static_cast<long long>(t), 0);
    if (w.poll(false, 1051) != V::kTimedOut) return fail("no timeout", 1051, 0);
    w.hold(256);
    w.hold(512);
    for (uint64_t t = 1052; t < 100000; t += 997)
      if (w.poll(false, t) != V::kWaiting) return fail("second verdict", static_cast<long long>(t), 0);
    if (!w.busy() || !w.timed_out() || w.held() != 2) return fail("state", w.busy(), w.held());
  }
  // zero limit: never times out
  {
    hd::SlotWatch w;
    w.launch(0, 0);
    for (uint64_t t = 0; t < (1ull << 40); t += (1ull << 33))
      if (w.poll(false, t) != V::kWaiting) return fail("zero limit", static_cast<long long>(t), 0);
    if (w.poll(true, 5) != V::kDone) return fail("zero limit done", 0, 0);
  }
  // randomised: model of when the work ends against when the limit passes
  for (int it = 0; it < 20000; ++it) {
    hd::SlotWatch w;
    const uint64_t t0 = rng() % 1000000, limit = 1 + rng() % 500;
    const bool never = (rng() % 4) == 0;
    const uint64_t end = t0 + rng() % 1200;  // when the device work finishes
    const int nblk = static_cast<int>(rng() % 5);
    w.launch(t0, limit);
    bool timed = false, done = false, retired = false;
    size_t returned = 0;
    for (uint64_t t = t0; t < t0 + 2000 && !done && !retired; t += 1 + rng() % 7) {
      const bool fin = !never && t >= end;
      const V v = w.poll(fin, t);
      if (v == V::kTimedOut) {
        if (timed) return fail("timed out twice", it, 0);
        if (t - t0 <= limit) return fail("timed out early", static_cast<long long>(t - t0), limit);
        if (fin) return fail("timed out a finished batch", it, 0);
        timed = true;
        for (int b = 0; b < nblk; ++b) w.hold(256u * (b + 1));
      } else if (v == V::kDone) {
        if (timed) return fail("done after timeout", it, 0);
        if (!fin) return fail("done before finish", it, 0);
        if (w.held()) return fail("done with held blocks", it, w.held());
        done = true;
      } else if (v == V::kRetired) {
        if (!timed || !fin) return fail("retired", timed, fin);
        returned = w.take_held().size();
        if (returned != static_cast<size_t>(nblk)) return fail("held blocks", returned, nblk);
        retired = true;
      } else if (v == V::kWaiting) {
        if (fin) return fail("waiting after finish", it, 0);
        if (!timed && t - t0 > limit) return fail("missed timeout", static_cast<long long>(t - t0), limit);
      } else {
        return fail("idle while busy", it, 0);
      }
    }
    if (never && (done || retired)) return fail("finished a batch that never ends", it, 0);
    if (never && !timed) return fail("never-ending batch not timed out", it, 0);
    if ((done || retired) && w.busy()) return fail("busy after finish", it, 0);
    if (never && !w.busy()) return fail("slot freed under running work", it, 0);
  }
  std::printf("ok\n");
  return 0;
}
