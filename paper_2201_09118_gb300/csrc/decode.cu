// decode.cu -- the persistent Huffman decode kernel (gap-array and
// self-synchronising variants), single pass over the bitstream.
//
// Geometry.  A subsequence is S bits (one thread); a tile is B subsequences
// (one block pass).  Tiles are handed out in order through an atomic ticket;
// a tile's output offset comes from a decoupled look-back over tiles whose
// warp reads 256 predecessor states per round trip, so one launch decodes a
// whole field (or many fields) at full rate.
//
// Per tile:
//   1. stage the tile's units in shared memory (one vector load per thread,
//      stored transposed so a warp's lanes always hit distinct banks);
//   2. find each subsequence's first codeword:
//        - gap array (Sec. III-C): start = i*S + gap[i];
//        - self-synchronisation (Sec. III-B, IV-A): every thread starts at its
//          nominal position i*S; a thread whose start differs from its
//          predecessor's stop position walks its new and old paths side by
//          side until they meet at a common codeword boundary, after which the
//          old stop position, count and symbols hold.  Rounds end when no
//          start changes (block vote).  The tile's first start comes from a
//          few lanes that re-synchronise the subsequences before the tile;
//   3. decode each subsequence once, into a per-thread column of a
//      shared-memory scratch (threads with more codewords than the column
//      holds decode again at step 6);
//   4. block scan of the codeword counts (Sec. III-B2 step 3);
//   5. look-back across tiles for the tile's first output index; the
//      self-synchronising variant also checks that the tile's start equals
//      its predecessor's verified stop, and re-runs step 2 if not;
//   6. copy the symbols into the shared-memory window in output order and
//      write it out with coalesced 16-byte stores (Algorithm 1, Sec. IV-B).
#include <cuda_runtime.h>

#include "common.cuh"
#include "decode_common.cuh"
#include "kernels.h"

namespace hd {
namespace {

using namespace dev;

// Look-back state word of the self-synchronising variant:
// flag (2) | start offset a (6) | stop offset e (6) | count (50).
constexpr uint64_t kValMask50 = (1ull << 50) - 1;
__device__ __forceinline__ uint64_t pack_state(uint64_t flag, uint32_t a, uint32_t e, uint64_t v) {
  return flag | (static_cast<uint64_t>(a & 63u) << 56) | (static_cast<uint64_t>(e & 63u) << 50) |
         (v & kValMask50);
}

constexpr int kLbPerLane = 8;                 // states each look-back lane reads
constexpr int kLbSpan = 32 * kLbPerLane;      // tiles per look-back round trip

// Decodes `count` codewords from position p into scr[j * B] (j < count).
template <int B>
__device__ __forceinline__ uint32_t decode_into(const Tables& T, const uint32_t* col,
                                                uint32_t p, uint32_t count, uint16_t* scr,
                                                bool& bad) {
  for (uint32_t j = 0; j < count; ++j) {
    uint32_t sym;
    p += code_sym(T, peek<B>(col, p), sym, bad);
    scr[j * B] = static_cast<uint16_t>(sym);
  }
  return p;
}

// One pass from `p` to `end`: symbols into the scratch column while they fit
// (cmax slots), codewords counted to the end.  Returns the stop position.
template <int B>
__device__ __forceinline__ uint32_t decode_pass(const Tables& T, const uint32_t* col, uint32_t p,
                                                uint32_t end, uint32_t cmax, uint16_t* scr,
                                                uint32_t& c, bool& bad) {
  uint32_t j = 0;
  while (p < end && j < cmax) {
    uint32_t sym;
    p += code_sym(T, peek<B>(col, p), sym, bad);
    scr[j * B] = static_cast<uint16_t>(sym);
    ++j;
  }
  while (p < end) {
    p += code_len(T, peek<B>(col, p), bad);
    ++j;
  }
  c = j;
  return p;
}

// Self-synchronisation step for one thread: replace the path from `s` (stop
// e, count c, symbols in the scratch column when c <= cmax) by the path from
// ns.  The two paths are walked side by side until they share a codeword
// boundary; from there on they coincide, so only the new prefix is decoded
// and the old tail is shifted into place.
template <int STRIDE, bool SCRATCH>
__device__ __forceinline__ void repath(const Tables& T, const uint32_t* col, uint32_t end,
                                       uint32_t ns, uint32_t& s, uint32_t& e, uint32_t& c,
                                       bool& scr_ok, uint32_t cmax, uint16_t* scr) {
  uint32_t a = ns, b = s, ca = 0, cb = 0;
  bool met = false, bad = false;
  for (;;) {
    if (a == b) {
      met = true;
      break;
    }
    if (a >= end && b >= end) break;
    if (a < b) {
      a += code_len(T, peek<STRIDE>(col, a), bad);
      ++ca;
    } else {
      b += code_len(T, peek<STRIDE>(col, b), bad);
      ++cb;
    }
  }
  const uint32_t c_old = c;
  if (met) {
    c = ca + (c_old - cb);
  } else {
    c = ca;
    e = a;
  }
  if (SCRATCH) {
    if (c > cmax || (met && !scr_ok)) {
      scr_ok = false;
    } else {
      if (met) {
        // old symbols [cb, c_old) move to [ca, c)
        if (ca > cb) {
          for (uint32_t k = c_old; k-- > cb;) scr[(k + ca - cb) * STRIDE] = scr[k * STRIDE];
        } else if (ca < cb) {
          for (uint32_t k = cb; k < c_old; ++k) scr[(k - (cb - ca)) * STRIDE] = scr[k * STRIDE];
        }
        decode_into<STRIDE>(T, col, ns, ca, scr, bad);
      } else {
        decode_into<STRIDE>(T, col, ns, c, scr, bad);
      }
      scr_ok = true;
    }
  }
  s = ns;
}

// Intra-sequence synchronisation over one tile (all threads call it).
// Thread 0's predecessor stopped at e_pred (thread 0 starts at e_pred - S).
// Returns false if the round cap was hit.
template <int S, int B>
__device__ __forceinline__ bool sync_rounds(const Tables& T, const uint32_t* col, bool valid,
                                            uint32_t end, uint32_t e_pred, uint32_t& s,
                                            uint32_t& e, uint32_t& c, bool& scr_ok,
                                            uint32_t cmax, uint16_t* scr, uint32_t* s_e_last) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (uint32_t round = 0;; ++round) {
    uint32_t e_prev = __shfl_up_sync(0xffffffffu, e, 1);
    if (lane == 31) s_e_last[warp] = e;
    __syncthreads();
    if (lane == 0) e_prev = warp ? s_e_last[warp - 1] : e_pred;
    bool changed = false;
    uint32_t ns = s;
    if (valid) {
      ns = e_prev - S;
      changed = ns != s;
    }
    if (!__syncthreads_or(changed)) return true;
    if (round > B + 1) return false;
    if (changed) repath<B, true>(T, col, end, ns, s, e, c, scr_ok, cmax, scr);
  }
}

// Lanes 0..PRE-1 of warp 0: where does the tile whose first subsequence is i0
// begin?  They self-synchronise the PRE subsequences before it (lane 0 starts
// at its nominal position) and return the first boundary at or after i0*S.
template <int S, int PRE>
__device__ __forceinline__ uint32_t presync_guess(const Tables& T, uint32_t* s_pre,
                                                  const FieldDesc& F, uint64_t i0) {
  const int lane = threadIdx.x & 31;
  const bool on = lane < PRE;
  uint32_t* col = s_pre + lane;
  if (on) stage_units<S>(col, F, i0 - PRE + lane, PRE);
  __syncwarp();
  bool bad = false;
  uint32_t s = 0, e = 0, c = 0;
  bool scr_ok = false;
  if (on) {
    uint32_t p = 0;
    while (p < S) p += code_len(T, peek<PRE>(col, p), bad);
    e = p;
  }
  for (int round = 0; round < PRE + 2; ++round) {
    const uint32_t e_prev = __shfl_up_sync(0xffffffffu, e, 1);
    const uint32_t ns = (on && lane) ? e_prev - S : s;
    const bool changed = ns != s;
    if (!__any_sync(0xffffffffu, changed)) break;
    if (changed) repath<PRE, false>(T, col, S, ns, s, e, c, scr_ok, 0, nullptr);
  }
  return __shfl_sync(0xffffffffu, e, PRE - 1) - S;
}

__device__ __forceinline__ void lb_load(const uint64_t* st, int64_t j, int64_t lo, int lane,
                                        uint64_t (&s)[kLbPerLane]) {
#pragma unroll
  for (int k = 0; k < kLbPerLane; ++k) {
    const int64_t idx = j - kLbPerLane * lane - k;
    s[k] = idx >= lo ? ld_relaxed(st + idx) : kStateInc;
  }
}

// Look-back over tiles for the count prefix (warp 0).  Publishes the tile's
// aggregate, sums predecessors back to the nearest inclusive prefix, then
// publishes its own inclusive prefix.  Returns the exclusive prefix.
__device__ __forceinline__ uint64_t lookback_counts(const DecodeParams& P, uint64_t g,
                                                    uint64_t first, uint64_t C, uint32_t* err) {
  const int lane = threadIdx.x & 31;
  uint64_t* st = P.unit_state;
  if (g == first) {
    if (lane == 0) st_relaxed(st + g, kStateInc | C);
    return 0;
  }
  if (lane == 0) st_relaxed(st + g, kStateAgg | C);
  uint64_t excl = 0;
  int64_t j = static_cast<int64_t>(g) - 1;
  const int64_t lo = static_cast<int64_t>(first);
  const uint64_t t0 = static_cast<uint64_t>(clock64());
  for (;;) {
    uint64_t s[kLbPerLane];
    lb_load(st, j, lo, lane, s);
    bool has_inc = false, notready = false;
    uint64_t sum = 0;
#pragma unroll
    for (int k = 0; k < kLbPerLane; ++k) {
      if (!has_inc) {
        const uint32_t flag = static_cast<uint32_t>(s[k] >> 62);
        notready |= flag == 0u;
        sum += s[k] & kStateValMask;
        has_inc = flag == 2u;
      }
    }
    const uint32_t inc = __ballot_sync(0xffffffffu, has_inc);
    const uint32_t need = inc ? (((inc & (0u - inc)) << 1) - 1u) : 0xffffffffu;
    if (__ballot_sync(0xffffffffu, notready) & need) {
      bool go = true;
      if (lane == 0) go = backoff_wait(P, t0);
      if (!__shfl_sync(0xffffffffu, go, 0)) {
        if (lane == 0) atomicOr(err, kErrTimeout);
        break;
      }
      continue;
    }
    excl += warp_sum_u64((need >> lane) & 1u ? sum : 0ull);
    if (inc) break;
    j -= kLbSpan;
  }
  if (lane == 0) st_relaxed(st + g, kStateInc | ((excl + C) & kStateValMask));
  return excl;
}

// Look-back of the self-synchronising variant (warp 0): also checks that
// every tile's assumed start offset (a) equals its predecessor's stop offset
// (e).  Returns 0 when this tile's start is verified (its inclusive state is
// then published), or 1 when the immediate predecessor is verified and ends
// elsewhere: *true_start then holds that stop offset and *excl_out the
// predecessor's inclusive count.
__device__ __forceinline__ uint32_t lookback_sync(const DecodeParams& P, uint64_t g,
                                                  uint64_t first, uint32_t a_self,
                                                  uint32_t e_self, uint64_t C, uint32_t* err,
                                                  uint64_t* excl_out, uint32_t* true_start) {
  const int lane = threadIdx.x & 31;
  uint64_t* st = P.unit_state;
  if (g == first) {
    if (lane == 0) st_relaxed(st + g, pack_state(kStateInc, a_self, e_self, C));
    *excl_out = 0;
    return 0;
  }
  if (lane == 0) st_relaxed(st + g, pack_state(kStateAgg, a_self, e_self, C));
  uint64_t excl = 0;
  int64_t j = static_cast<int64_t>(g) - 1;
  const int64_t lo = static_cast<int64_t>(first);
  uint32_t carry_a = a_self;
  const uint64_t t0 = static_cast<uint64_t>(clock64());
  for (;;) {
    uint64_t s[kLbPerLane];
    lb_load(st, j, lo, lane, s);
    // successor of this lane's nearest tile = previous lane's farthest tile
    uint32_t succ_a = __shfl_up_sync(
        0xffffffffu, static_cast<uint32_t>(s[kLbPerLane - 1] >> 56) & 63u, 1);
    if (lane == 0) succ_a = carry_a;
    bool has_inc = false, notready = false, broken = false, broken_near = false;
    uint64_t sum = 0;
    uint64_t near_state = s[0];
#pragma unroll
    for (int k = 0; k < kLbPerLane; ++k) {
      if (!has_inc) {
        const int64_t idx = j - kLbPerLane * lane - k;
        const uint32_t flag = static_cast<uint32_t>(s[k] >> 62);
        const uint32_t a_k = static_cast<uint32_t>(s[k] >> 56) & 63u;
        const uint32_t e_k = static_cast<uint32_t>(s[k] >> 50) & 63u;
        if (flag == 0u) {
          notready = true;
        } else if (idx >= lo && e_k != succ_a) {
          broken = true;
          if (k == 0) broken_near = true;
        }
        sum += s[k] & kValMask50;
        has_inc = flag == 2u;
        succ_a = a_k;
      }
    }
    const uint32_t inc = __ballot_sync(0xffffffffu, has_inc);
    const uint32_t need = inc ? (((inc & (0u - inc)) << 1) - 1u) : 0xffffffffu;
    bool wait = (__ballot_sync(0xffffffffu, notready) & need) != 0;
    bool restart = false;
    const uint32_t brk = __ballot_sync(0xffffffffu, broken) & need;
    if (!wait && brk) {
      const bool near0 = __shfl_sync(0xffffffffu, broken_near, 0);
      const uint64_t s0 = __shfl_sync(0xffffffffu, near_state, 0);
      if (near0 && (s0 >> 62) == 2u && j == static_cast<int64_t>(g) - 1) {
        *true_start = static_cast<uint32_t>(s0 >> 50) & 63u;
        *excl_out = s0 & kValMask50;
        return 1;
      }
      // an earlier tile's start is wrong; it will publish a fix, and the
      // tiles after it may change too, so the walk starts over
      wait = true;
      restart = true;
    }
    if (wait) {
      bool go = true;
      if (lane == 0) go = backoff_wait(P, t0);
      if (!__shfl_sync(0xffffffffu, go, 0)) {
        if (lane == 0) atomicOr(err, kErrTimeout);
        break;
      }
      if (restart) {
        excl = 0;
        j = static_cast<int64_t>(g) - 1;
        carry_a = a_self;
      }
      continue;
    }
    excl += warp_sum_u64((need >> lane) & 1u ? sum : 0ull);
    if (inc) break;
    carry_a = __shfl_sync(0xffffffffu, static_cast<uint32_t>(s[kLbPerLane - 1] >> 56) & 63u, 31);
    j -= kLbSpan;
  }
  if (lane == 0) st_relaxed(st + g, pack_state(kStateInc, a_self, e_self, excl + C));
  *excl_out = excl;
  return 0;
}

template <int S>
__host__ __device__ constexpr int presync_lanes() {
  return 1024 / S < 32 ? 1024 / S : 32;
}

template <int S, int B, bool SS>
__global__ void __launch_bounds__(B) k_decode(const __grid_constant__ DecodeParams P) {
  constexpr int W = S / 32 + 1;
  constexpr int NW = B / 32;
  constexpr int PRE = SS ? presync_lanes<S>() : 0;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_lut = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_bits = s_lut + (1u << P.K);
  uint32_t* s_pre = s_bits + W * B;
  uint16_t* s_out = reinterpret_cast<uint16_t*>(s_pre + W * PRE);  // window + 16
  uint16_t* s_scr = s_out + P.window + 16;                           // [cmax][B]
  uint16_t* s_long = s_scr + P.cmax * B;                             // [long_cap]

  __shared__ uint64_t s_end[34];
  __shared__ uint32_t s_base[34];
  __shared__ uint32_t s_meta[3];
  __shared__ uint32_t s_warp[NW];
  __shared__ uint32_t s_e_last[NW];
  __shared__ uint64_t s_tile_base;
  __shared__ uint32_t s_ticket;
  __shared__ uint32_t s_field;
  __shared__ uint32_t s_a, s_e, s_resync, s_true_start;

  const int t = threadIdx.x;
  const int lane = t & 31;
  const int warp = t >> 5;
  const uint32_t cmax = P.cmax;
  uint32_t cur_field = 0xffffffffu;
  uint32_t* col = s_bits + t;
  uint16_t* scr = s_scr + t;

  for (;;) {
    if (t == 0) {
      const uint32_t g = atomicAdd(P.ticket, 1u);
      s_ticket = g;
      s_field = g < P.total_units ? find_field(P, g) : 0u;
    }
    __syncthreads();
    const uint64_t g = s_ticket;
    if (g >= P.total_units) break;
    const uint32_t fi = s_field;
    const FieldDesc& F = field_of(P, fi);
    if (fi != cur_field) {
      load_table(F.table, P.K, s_lut, s_end, s_base, s_meta, B, s_long, P.long_cap);
      cur_field = fi;
      __syncthreads();
    }
    const Tables T{s_lut,
                   s_end,
                   s_base,
                   reinterpret_cast<const uint16_t*>(reinterpret_cast<const char*>(F.table) +
                                                     kTableHeaderBytes + (4u << P.K)),
                   s_long,
                   s_meta[2],
                   P.long_cap,
                   s_meta[0],
                   32u - P.K};
    const bool table_ok = s_meta[1] == 0;

    const uint64_t tl = g - F.unit_begin;
    const uint64_t i = tl * B + t;
    const bool valid = table_ok && i < F.nsub;
    uint32_t end = 0;
    if (valid) {
      stage_units<S>(col, F, i, B);
      const uint64_t rem = F.nbits - i * S;
      end = rem < S ? static_cast<uint32_t>(rem) : S;
    }

    // ---- starts, counts, symbols into the scratch ---------------------------
    uint32_t s = 0, c = 0;
    bool scr_ok = false;
    uint32_t err = 0;
    if constexpr (!SS) {
      if (valid) {
        uint32_t gp = F.gap[i * F.gap_stride];
        const uint32_t expect = (i + 1 < F.nsub) ? S + F.gap[(i + 1) * F.gap_stride]
                                                 : static_cast<uint32_t>(F.nbits - i * S);
        if (gp > end || gp >= S) {
          err |= kErrGap;
          gp = end;
        }
        bool bad = false;
        const uint32_t p = decode_pass<B>(T, col, gp, end, cmax, scr, c, bad);
        scr_ok = c <= cmax;
        if (bad) err |= kErrCode;
        else if (p != expect) err |= kErrGap;
        s = gp;
      }
      if (err) atomicOr(F.err, err);
    } else {
      uint32_t a0 = 0;
      if (warp == 0) {
        const uint32_t guess =
            (tl > 0 && table_ok) ? presync_guess<S, PRE>(T, s_pre, F, i - t) : 0u;
        if (lane == 0) s_a = guess;
      }
      uint32_t e = 0;
      if (valid) {
        bool bad = false;
        e = decode_pass<B>(T, col, 0, end, cmax, scr, c, bad);
        scr_ok = c <= cmax;
      }
      __syncthreads();
      a0 = s_a;
      if (!sync_rounds<S, B>(T, col, valid, end, S + a0, s, e, c, scr_ok, cmax, s_scr + t,
                             s_e_last))
        err |= kErrNoSync;
      if (t == B - 1) s_e = e - S;
      uint32_t C;
      block_excl_scan<B>(c, s_warp, &C);
      if (warp == 0) {
        uint64_t excl = 0;
        uint32_t ts = 0;
        const uint32_t r = lookback_sync(P, g, F.unit_begin, a0, s_e, C, F.err, &excl, &ts);
        if (t == 0) {
          s_resync = r;
          s_true_start = ts;
          s_tile_base = excl;
        }
      }
      __syncthreads();
      if (s_resync) {
        // the assumed start was wrong: restart thread 0 at the verified start
        if (!sync_rounds<S, B>(T, col, valid, end, S + s_true_start, s, e, c, scr_ok, cmax,
                               s_scr + t, s_e_last))
          err |= kErrNoSync;
        if (t == B - 1) s_e = e - S;
        block_excl_scan<B>(c, s_warp, &C);
        if (t == 0)
          st_relaxed(P.unit_state + g, pack_state(kStateInc, s_true_start, s_e, s_tile_base + C));
      }
      if (valid && i + 1 == F.nsub && e != end) err |= kErrCode;
      if (err) atomicOr(F.err, err);
      if (P.sync_only) {
        if (valid) F.gap_out[i] = static_cast<uint8_t>(s);
        if (t == 0 && !table_ok && tl == 0) atomicOr(F.err, kErrTable);
        __syncthreads();
        continue;
      }
    }

    // ---- output offsets ----------------------------------------------------
    uint32_t C;
    const uint32_t o = block_excl_scan<B>(c, s_warp, &C);
    if constexpr (!SS) {
      if (warp == 0) {
        const uint64_t excl = lookback_counts(P, g, F.unit_begin, C, F.err);
        if (t == 0) s_tile_base = excl;
      }
      __syncthreads();
    }
    const uint64_t base = s_tile_base;
    if (t == 0) {
      if (tl + 1 == F.nunits && base + C != F.n) atomicOr(F.err, kErrCount);
      if (!table_ok && tl == 0) atomicOr(F.err, kErrTable);
    }

    // ---- copy into the window in output order, coalesced stores ------------
    const uint32_t off0 = static_cast<uint32_t>((reinterpret_cast<uintptr_t>(F.out) >> 1) & 7u);
    uint16_t* out_al = F.out - off0;  // 16-byte aligned; virtual index X = x + off0
    const uint64_t Xn = F.n + off0;
    bool bad_any = false;
    for (uint32_t ws = 0; ws < C; ws += P.window) {
      const uint32_t we = min(C, ws + P.window);
      const uint64_t X0 = base + ws + off0;
      const uint32_t pad = static_cast<uint32_t>(X0 & 7u);
      const uint32_t lo = max(o, ws), hi = min(o + c, we);
      if (lo < hi) {
        uint16_t* dst = s_out + pad + (lo - ws);
        if (scr_ok) {
          for (uint32_t x = lo; x < hi; ++x) dst[x - lo] = scr[(x - o) * B];
        } else {
          // decode again from the start, keeping the part inside the window
          uint32_t p = s;
          bool bad = false;
          for (uint32_t j = 0; j < hi - o; ++j) {
            uint32_t sym;
            p += code_sym(T, peek<B>(col, p), sym, bad);
            if (o + j >= lo) dst[o + j - lo] = static_cast<uint16_t>(sym);
          }
          bad_any |= bad;
        }
      }
      __syncthreads();
      const uint64_t a0 = X0 & ~7ull;
      const uint64_t Xe = base + we + off0;
      const uint64_t q0 = a0 >> 3, q1 = (Xe + 7) >> 3;
      for (uint64_t q = q0 + t; q < q1; q += B) {
        const uint64_t Xq = q << 3;
        if (Xq >= X0 && Xq + 8 <= Xe && Xq + 8 <= Xn) {
          *reinterpret_cast<uint4*>(out_al + Xq) =
              *reinterpret_cast<const uint4*>(s_out + (Xq - a0));
        } else {
          const uint64_t xlo = Xq > X0 ? Xq : X0;
          uint64_t xhi = Xq + 8 < Xe ? Xq + 8 : Xe;
          xhi = xhi < Xn ? xhi : Xn;
          for (uint64_t X = xlo; X < xhi; ++X) out_al[X] = s_out[X - a0];
        }
      }
      __syncthreads();
    }
    if (bad_any) atomicOr(F.err, kErrCode);
  }
}

template <int S, int B, bool SS>
cudaError_t launch_t(const DecodeParams& p, const LaunchShape& s, int num_sms,
                     cudaStream_t stream) {
  const size_t smem = decode_smem_bytes(s, SS);
  auto kern = k_decode<S, B, SS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, B, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  uint64_t grid = static_cast<uint64_t>(per_sm) * num_sms;
  if (s.grid && s.grid < grid) grid = s.grid;
  if (grid > p.total_units) grid = p.total_units;
  if (grid == 0) return cudaSuccess;
  kern<<<static_cast<unsigned>(grid), B, smem, stream>>>(p);
  return cudaGetLastError();
}

template <int S, bool SS>
cudaError_t launch_s(const DecodeParams& p, const LaunchShape& s, int num_sms,
                     cudaStream_t stream) {
  switch (s.threads) {
    case 128: return launch_t<S, 128, SS>(p, s, num_sms, stream);
    case 256: return launch_t<S, 256, SS>(p, s, num_sms, stream);
    case 512: return launch_t<S, 512, SS>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <bool SS>
cudaError_t launch_v(const DecodeParams& p, const LaunchShape& s, int num_sms,
                     cudaStream_t stream) {
  switch (s.S) {
    case 64: return launch_s<64, SS>(p, s, num_sms, stream);
    case 128: return launch_s<128, SS>(p, s, num_sms, stream);
    case 256: return launch_s<256, SS>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t decode_smem_bytes(const LaunchShape& s, bool self_sync) {
  const size_t W = s.S / 32 + 1;
  const size_t pre = self_sync ? (1024 / s.S < 32 ? 1024 / s.S : 32) : 0;
  size_t b = (static_cast<size_t>(1) << s.K) * 4 + W * s.threads * 4 + W * pre * 4;
  b += (static_cast<size_t>(s.window) + 16) * 2;
  b += static_cast<size_t>(s.cmax) * s.threads * 2;
  b += static_cast<size_t>(s.long_cap) * 2;
  return (b + 15) & ~static_cast<size_t>(15);
}

cudaError_t launch_decode(const DecodeParams& p, const LaunchShape& s, bool self_sync,
                          int num_sms, cudaStream_t stream) {
  if (p.cmax != s.cmax || s.cmax > s.S || p.long_cap != s.long_cap) return cudaErrorInvalidValue;
  return self_sync ? launch_v<true>(p, s, num_sms, stream)
                   : launch_v<false>(p, s, num_sms, stream);
}

}  // namespace hd
