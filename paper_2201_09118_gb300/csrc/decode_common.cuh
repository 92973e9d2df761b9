// decode_common.cuh -- device building blocks of the decode kernels:
// bitstream staging, decode-table lookups, block scans, bounded waits and the
// shared-memory staged output window.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "common.cuh"

namespace hd {
namespace dev {

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bulk stores of a staged output window by the TMA engine (cp.async.bulk,
// shared to global).  The shared-memory writes that filled the window must be
// made visible to that engine first: every writing thread runs
// fence_async_smem() before the barrier after which one thread issues the
// copy.  The issuing thread's groups are waited for with bulk_wait_read()
// before the window is written again, and with bulk_wait_all() before the
// thread exits.
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Copies `bytes` from shared address `src` to global `dst` as one bulk group.
// Both addresses and the size must be multiples of 16; a request that is not
// is refused (returns false, nothing issued) and the caller stores plainly.
__device__ __forceinline__ bool bulk_store(void* dst, uint32_t src, uint32_t bytes) {
  if (((reinterpret_cast<uintptr_t>(dst) | src | bytes) & 15u) != 0 || bytes == 0) return false;
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
               ::"l"(dst), "r"(src), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  return true;
}
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ uint4 ldg_v4(const uint32_t* p) {
  return __ldg(reinterpret_cast<const uint4*>(p));
}
__device__ __forceinline__ uint2 ldg_v2(const uint32_t* p) {
  return __ldg(reinterpret_cast<const uint2*>(p));
}

// Decode tables as seen by one block: one first-level table in shared memory
// (32-bit, 16-bit or length entries, see common.cuh), the per-length limits in
// shared memory, the sorted symbols in global memory (only codes longer than
// K bits read them) with the first long_cap long-code symbols in shared memory.
struct Tables {
  const void* lut;
  const uint64_t* end;
  const uint32_t* base;
  const uint16_t* sorted;    // all symbols by (length, symbol), global memory
  const uint16_t* long_syms; // shared-memory copy of sorted[long0 ..], long_cap entries
  uint32_t long0;
  uint32_t long_cap;
  uint32_t maxlen;
  uint32_t shift;  // 32 - K
};

// Bits [p, p + 32) of a staged subsequence.  Column `col` holds the
// subsequence's units at stride B (unit k at col[k * B]), so the 32 lanes of a
// warp always read 32 distinct banks whatever their positions.
template <int B>
__device__ __forceinline__ uint32_t peek(const uint32_t* col, uint32_t p) {
  const uint32_t k = p >> 5;
  return __funnelshift_l(col[(k + 1) * B], col[k * B], p);
}

// The length of the code at window w when the first-level entry only gave a
// lower bound L: walk the canonical limits.  An invalid bit pattern sets `bad`
// and counts as one bit, so a decoder that started at a wrong position still
// advances.
__device__ __forceinline__ uint32_t walk_len(const Tables& T, uint32_t w, uint32_t L, bool& bad) {
  while (L <= T.maxlen && static_cast<uint64_t>(w) >= T.end[L]) ++L;
  if (L > T.maxlen) {
    bad = true;
    return 0;
  }
  return L;
}

// Symbol of a code longer than the first-level table.
__device__ __forceinline__ uint32_t long_sym(const Tables& T, uint32_t w, uint32_t L) {
  const uint32_t rank = (w >> (32 - L)) + T.base[L];
  const uint32_t li = rank - T.long0;
  return li < T.long_cap ? T.long_syms[li] : __ldg(T.sorted + rank);
}

// Length of the codeword at window w from the 32-bit table.
__device__ __forceinline__ uint32_t code_len(const Tables& T, uint32_t w, bool& bad) {
  const uint32_t e = static_cast<const uint32_t*>(T.lut)[w >> T.shift];
  if (!(e & kLongFlag)) return e >> 16;
  const uint32_t L = e & 0xFFu;
  if (L == ((e >> 8) & 0xFFu)) return L;  // one length under this prefix
  const uint32_t Lw = walk_len(T, w, L, bad);
  return Lw ? Lw : 1u;
}

// Length of the codeword at window w from the length table.
__device__ __forceinline__ uint32_t code_len8(const Tables& T, uint32_t w, bool& bad) {
  const uint32_t e = static_cast<const uint8_t*>(T.lut)[w >> T.shift];
  if (!(e & kLen8Walk)) return e;
  const uint32_t Lw = walk_len(T, w, e & 0x7Fu, bad);
  return Lw ? Lw : 1u;
}

// Length and symbol of the codeword at window w from the 32-bit table.
__device__ __forceinline__ uint32_t code_sym(const Tables& T, uint32_t w, uint32_t& sym,
                                             bool& bad) {
  const uint32_t e = static_cast<const uint32_t*>(T.lut)[w >> T.shift];
  if (!(e & kLongFlag)) {
    sym = e & 0xFFFFu;
    return e >> 16;
  }
  uint32_t L = e & 0xFFu;
  if (L != ((e >> 8) & 0xFFu)) {
    L = walk_len(T, w, L, bad);
    if (!L) {
      sym = 0;
      return 1;
    }
  }
  sym = long_sym(T, w, L);
  return L;
}

// Length and symbol of the codeword at window w from the 16-bit table.
__device__ __forceinline__ uint32_t code_sym16(const Tables& T, uint32_t w, uint32_t& sym,
                                               bool& bad) {
  const uint32_t e = static_cast<const uint16_t*>(T.lut)[w >> T.shift];
  uint32_t L = e >> 12;
  if (L) {
    sym = e & 0xFFFu;
    return L;
  }
  L = e & 0xFFu;
  if (e & kLut16Mixed) {
    L = walk_len(T, w, L, bad);
    if (!L) {
      sym = 0;
      return 1;
    }
  }
  sym = long_sym(T, w, L);
  return L;
}

// Entry type of the two-code table (see table_pair_off).
struct PairEntry {};

// Length and symbol of the first codeword at window w from the two-code
// table (entry e = the table's entry for w).
__device__ __forceinline__ uint32_t code_sym_pair(const Tables& T, uint32_t w, uint32_t e,
                                                  uint32_t& sym, bool& bad) {
  const uint32_t m = e >> 30;
  if (m) {
    sym = m == 1 ? (e & 0xFFFu) : (e & 0x3FFu);
    return (e >> 26) & 15u;
  }
  uint32_t L = e & 0xFFu;
  if (e & kLut16Mixed) {
    L = walk_len(T, w, L, bad);
    if (!L) {
      sym = 0;
      return 1;
    }
  }
  sym = long_sym(T, w, L);
  return L;
}

// Entry type of the symbol table: E = uint32_t, uint16_t or PairEntry.
template <class E>
__device__ __forceinline__ uint32_t code_sym_t(const Tables& T, uint32_t w, uint32_t& sym,
                                               bool& bad) {
  if constexpr (std::is_same_v<E, PairEntry>) {
    return code_sym_pair(T, w, static_cast<const uint32_t*>(T.lut)[w >> T.shift], sym, bad);
  } else if constexpr (sizeof(E) == 2) {
    return code_sym16(T, w, sym, bad);
  } else {
    return code_sym(T, w, sym, bad);
  }
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive block scan of per-thread counts; returns the exclusive prefix and
// writes the block total to *total.  Uses s_warp[B/32]; ends with a barrier.
template <int B>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t c, uint32_t* s_warp,
                                                    uint32_t* total) {
  constexpr int NW = B / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t incl = warp_incl_scan(c, lane);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < NW ? s_warp[lane] : 0u;
    v = warp_incl_scan(v, lane);
    if (lane < NW) s_warp[lane] = v;
  }
  __syncthreads();
  *total = s_warp[NW - 1];
  return (warp ? s_warp[warp - 1] : 0u) + incl - c;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One more round of a spin-wait that began at t0 (an SM cycle count).  The
// caller re-reads global state between rounds, which paces the spin; this
// returns false once the launch was aborted or the wait exceeded its limit
// (the caller then records a timeout and stops waiting).
__device__ __forceinline__ bool backoff_wait(const DecodeParams& P, uint64_t t0) {
  if (ld_relaxed32(P.abort_flag)) return false;
  if (static_cast<uint64_t>(clock64()) - t0 > P.timeout_cycles) {
    atomicExch(P.abort_flag, 1u);
    return false;
  }
  return true;
}

// Decoupled look-back over per-tile states (the output-index prefix of
// Sec. III-B2 step 3 across tiles): each lane reads kLbPerLane states, so one
// round trip through L2 covers kLbSpan predecessor tiles.
constexpr int kLbPerLane = 8;
constexpr int kLbSpan = 32 * kLbPerLane;

__device__ __forceinline__ void lb_load(const uint64_t* st, int64_t j, int64_t lo, int lane,
                                        uint64_t (&s)[kLbPerLane]) {
#pragma unroll
  for (int k = 0; k < kLbPerLane; ++k) {
    const int64_t idx = j - kLbPerLane * lane - k;
    s[k] = idx >= lo ? ld_relaxed(st + idx) : kStateInc;
  }
}

// Look-back over tiles for the count prefix (one whole warp).  Publishes the tile's
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
  uint32_t nap = 32;  // ns between re-reads of predecessors not yet counted
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
      // leave the issue slots to the warps that are decoding
      __nanosleep(nap);
      nap = nap < 1024 ? 2 * nap : nap;
      continue;
    }
    excl += warp_sum_u64((need >> lane) & 1u ? sum : 0ull);
    if (inc) break;
    j -= kLbSpan;
  }
  if (lane == 0) st_relaxed(st + g, kStateInc | ((excl + C) & kStateValMask));
  return excl;
}


// Writes window symbols [lo, end) of a block's window (16-byte aligned,
// shared) to dst[lo .. end) (dst 16-byte aligned): the 16-byte aligned middle
// as one bulk copy by the TMA engine, issued by thread 16 and read before it
// returns, the at most 7 symbols on either side by threads 0-15.  The threads
// that wrote the window ran fence_async_smem() before the barrier preceding
// this; the caller's next barrier follows the read.
template <int B>
__device__ __forceinline__ void flush_block(const uint16_t* s_out, uint16_t* dst, uint32_t lo,
                                            uint32_t end) {
  static_assert(B >= 32, "threads 0-16 take part");
  const int t = threadIdx.x;
  const uint32_t ra = (lo + 7) & ~7u, rb = end & ~7u;
  if (rb > ra) {
    if (t < 8) {
      const uint32_t r = lo + t;
      if (r < ra) dst[r] = s_out[r];
    } else if (t < 16) {
      const uint32_t r = rb + (t - 8);
      if (r < end) dst[r] = s_out[r];
    } else if (t == 16) {
      const uint32_t src = static_cast<uint32_t>(__cvta_generic_to_shared(s_out + ra));
      if (bulk_store(dst + ra, src, 2 * (rb - ra))) {
        bulk_wait_read();
      } else {
        for (uint32_t r = ra; r < rb; ++r) dst[r] = s_out[r];
      }
    }
  } else {
    for (uint32_t r = lo + t; r < end; r += B) dst[r] = s_out[r];
  }
}

// Algorithm 1 (Sec. IV-B): the block's output [0, C) is produced through a
// shared-memory window of `window` symbols.  A thread decodes its whole range
// [o, o + c) into the window only when it fits; the first thread that does
// not fit ends the window, the window is written to global memory with
// coalesced 16-byte stores, and the next window starts at that thread.  When
// the whole tile fits (the usual case, the window being sized for it) one
// pass with two barriers does it.
// `decode(dst)` writes the thread's c symbols to dst[0 .. c).
// Requires window >= max c (c <= S).  Global writes are clipped to [0, n).
// With `prefill` every window pass is first filled with the symbol pair
// `fill2` by all threads (16-byte stores, one barrier), so that `decode`
// may leave the positions of that symbol unwritten: runs of a field's
// 1-bit code then cost no shared stores.  (Written by their own threads,
// such runs put every thread of a warp on one bank when the subsequences
// hold equal counts, as they do when almost every code is that 1-bit code.)
template <int B, class DecodeFn>
__device__ __forceinline__ void window_write(uint16_t* s_out, uint32_t* s_flush_end,
                                             uint32_t window, uint32_t o, uint32_t c,
                                             uint32_t C, uint64_t base, uint16_t* out,
                                             uint64_t n, DecodeFn&& decode,
                                             bool prefill = false, uint32_t fill2 = 0) {
  const int t = threadIdx.x;
  const uint32_t off0 = static_cast<uint32_t>((reinterpret_cast<uintptr_t>(out) >> 1) & 7u);
  // out - off0 is 16-byte aligned; virtual index X = x + off0
  uint16_t* out_al = out - off0;
  // fills window symbols [0, 8 * ceil(m / 8)) with fill2 (s_out is 16-byte
  // aligned and holds window + 16 symbols)
  auto fill_window = [&](uint32_t m) {
    const uint4 v = make_uint4(fill2, fill2, fill2, fill2);
    for (uint32_t k = t; k < (m + 7) >> 3; k += B) reinterpret_cast<uint4*>(s_out)[k] = v;
    __syncthreads();
  };
  if (C <= window) {
    const uint64_t X0 = base + off0;
    const uint32_t pad = static_cast<uint32_t>(X0 & 7u);
    if (prefill) fill_window(pad + C);
    if (c) decode(s_out + pad + o);
    fence_async_smem();
    __syncthreads();
    const uint64_t a0 = X0 - pad;
    uint16_t* dst = out_al + a0;
    const uint32_t end_r = pad + C;
    const uint64_t Xn = n + off0;  // first virtual index past the output
    const uint32_t end_ok =
        a0 >= Xn ? 0u : (Xn - a0 < end_r ? static_cast<uint32_t>(Xn - a0) : end_r);
    if (end_ok > pad) flush_block<B>(s_out, dst, pad, end_ok);
    __syncthreads();
    return;
  }
  bool done = c == 0;
  uint32_t ws = 0;
  while (ws < C) {
    const uint32_t we = ws + window;
    if (t == 0) *s_flush_end = C < we ? C : we;
    __syncthreads();
    if (!done && o < we && o + c > we) atomicMin(s_flush_end, o);
    __syncthreads();
    const uint32_t fe = *s_flush_end;
    const uint64_t X0 = base + ws + off0;
    const uint32_t pad = static_cast<uint32_t>(X0 & 7u);
    if (prefill) fill_window(pad + (fe - ws));
    if (!done && o + c <= fe) {
      decode(s_out + pad + (o - ws));
      done = true;
    }
    fence_async_smem();
    __syncthreads();
    // store virtual range [X0, Xe), clipped to Xn, from s_out[X - a0]
    const uint64_t a0 = X0 & ~7ull;
    const uint64_t Xe = base + fe + off0;
    const uint64_t Xn = n + off0;  // first virtual index past the output
    const uint64_t Xend = Xe < Xn ? Xe : Xn;
    if (Xend > X0) flush_block<B>(s_out, out_al + a0, pad, static_cast<uint32_t>(Xend - a0));
    __syncthreads();
    ws = fe;
  }
}

// True when a 32-bit word may hold a zero half-word (exact for the high half;
// a zero low half's borrow can make it fire for the high one too).
__device__ __forceinline__ bool has_zero_half(uint32_t w) {
  return ((w - 0x00010001u) & ~w & 0x80008000u) != 0;
}

// Decode + 1D Lorenzo reconstruction: the residue of code c at output G (code
// 0: the outlier stored for G, searched in the tile's outliers [olo, ohi)).
__device__ __forceinline__ int32_t value_residue(const DecodeParams& P, uint32_t c, uint64_t G,
                                                 uint64_t olo, uint64_t ohi) {
  if (c) return static_cast<int32_t>(c) - P.radius;
  uint64_t lo = olo, hi = ohi;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (P.out_idx[mid] < G)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo < ohi && P.out_idx[lo] == G) return P.out_val[lo];
  atomicOr(P.verr, kErrOutlier);
  return 0;
}

// Writes the values of outputs [G0, G1): q is `carry` plus the inclusive
// prefix of the residues; value = float32(q) * float32(2 eb).  Positions are
// taken relative to A = G0 rounded down to a multiple of 4; the code of
// position x sits at s_pos[x] (s_pos 16-byte aligned, x from G0 - A), so a
// thread's 8 consecutive positions are one 16-byte shared load and two
// 16-byte global stores.  B * 8 positions per row, one barrier per row (warp
// totals double-buffered in s_vw[2][32], scanned with shuffles).  carry
// leaves with q at G1 - 1.
template <int B>
__device__ __forceinline__ void flush_values(const uint16_t* s_pos, uint64_t G0, uint64_t G1,
                                             uint64_t n, int32_t& carry, const DecodeParams& P,
                                             uint64_t olo, uint64_t ohi, int32_t* s_vw) {
  constexpr int NW = B / 32;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint64_t A = G0 & ~3ull;
  const uint32_t lo = static_cast<uint32_t>(G0 - A);       // first valid position
  const uint32_t hi = lo + static_cast<uint32_t>(G1 - G0);  // end of the valid positions
  const uint64_t room = n > A ? n - A : 0ull;
  const uint32_t hn = room < hi ? static_cast<uint32_t>(room) : hi;  // end of the stored ones
  int buf = 0;
  for (uint32_t x0 = 0; x0 < hi; x0 += 8u * B, buf ^= 1) {
    const uint32_t x = x0 + 8u * t;
    int32_t r[8];
    if (x >= lo && x + 8 <= hi) {
      const uint4 u = *reinterpret_cast<const uint4*>(s_pos + x);
      const uint32_t w[4] = {u.x, u.y, u.z, u.w};
      if (has_zero_half(u.x) | has_zero_half(u.y) | has_zero_half(u.z) | has_zero_half(u.w)) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
          r[k] = value_residue(P, (w[k >> 1] >> (16 * (k & 1))) & 0xffffu, A + x + k, olo, ohi);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k)
          r[k] = static_cast<int32_t>((w[k >> 1] >> (16 * (k & 1))) & 0xffffu) - P.radius;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t xk = x + k;
        r[k] = xk >= lo && xk < hi ? value_residue(P, s_pos[xk], A + xk, olo, ohi) : 0;
      }
    }
#pragma unroll
    for (int k = 1; k < 8; ++k) r[k] += r[k - 1];
    int32_t incl = r[7];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    int32_t* sw = s_vw + buf * 32;
    if (lane == 31) sw[warp] = incl;
    __syncthreads();
    // warp totals of the row, scanned by every warp with shuffles
    const int32_t wt = lane < NW ? sw[lane] : 0;
    int32_t wi = wt;
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    const int32_t before = __shfl_sync(0xffffffffu, wi - wt, warp);
    const int32_t row = __shfl_sync(0xffffffffu, wi, NW - 1);
    const int32_t e = carry + before + incl - r[7];
    carry += row;
    if (x < hi) {
      float f[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) f[k] = __fmul_rn(__int2float_rn(e + r[k]), P.ebx2);
      float* dst = P.vout + A + x;
      if (x >= lo && x + 8 <= hn) {
        __stcs(reinterpret_cast<float4*>(dst), make_float4(f[0], f[1], f[2], f[3]));
        __stcs(reinterpret_cast<float4*>(dst) + 1, make_float4(f[4], f[5], f[6], f[7]));
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (x + k >= lo && x + k < hn) dst[k] = f[k];
      }
    }
  }
}

// Algorithm 1's window (as window_write) with float32 values out: each pass's
// codes are decoded into s_out[G & 3 ..) (the window holds window + 16 codes)
// and written by flush_values, q running on from the tile's prefix q0 across
// passes.  s_out is 16-byte aligned.
template <int B, class DecodeFn>
__device__ __forceinline__ void window_write_values(uint16_t* s_out, uint32_t* s_flush_end,
                                                    uint32_t window, uint32_t o, uint32_t c,
                                                    uint32_t C, uint64_t base, uint64_t n,
                                                    const DecodeParams& P, int32_t q0,
                                                    uint64_t olo, uint64_t ohi, int32_t* s_vw,
                                                    DecodeFn&& decode) {
  const int t = threadIdx.x;
  int32_t carry = q0;
  if (C <= window) {
    if (c) decode(s_out + (base & 3u) + o);
    __syncthreads();
    flush_values<B>(s_out, base, base + C, n, carry, P, olo, ohi, s_vw);
    __syncthreads();
    return;
  }
  bool done = c == 0;
  uint32_t ws = 0;
  while (ws < C) {
    const uint32_t we = ws + window;
    if (t == 0) *s_flush_end = C < we ? C : we;
    __syncthreads();
    if (!done && o < we && o + c > we) atomicMin(s_flush_end, o);
    __syncthreads();
    const uint32_t fe = *s_flush_end;
    if (!done && o + c <= fe) {
      decode(s_out + ((base + ws) & 3u) + (o - ws));
      done = true;
    }
    __syncthreads();
    flush_values<B>(s_out, base + ws, base + fe, n, carry, P, olo, ohi, s_vw);
    __syncthreads();
    ws = fe;
  }
}

// Which first-level table a kernel keeps in shared memory.
// k8r: the length table followed by the run table (2 x 2^K bytes).
enum class Lut { k32, k16, k8, k8r, kPair };

__host__ __device__ constexpr uint32_t lut_bytes(Lut kind, uint32_t K) {
  return kind == Lut::k32 || kind == Lut::kPair ? (4u << K)
         : kind == Lut::k16 ? (2u << K)
         : kind == Lut::k8r ? (2u << K)
                            : (1u << K);
}

// Loads the decode table of a field into shared memory (threads [0, nthreads)):
// the chosen first-level table (s_lut, 16-byte aligned), the per-length limits
// and the first long_cap symbols of codes longer than K.
// s_meta = {maxlen, status, long0}.
__device__ __forceinline__ void load_table(const TableHeader* H, uint32_t K, uint32_t alphabet,
                                           Lut kind, void* s_lut, uint64_t* s_end,
                                           uint32_t* s_base, uint32_t* s_meta, int nthreads,
                                           uint16_t* s_long = nullptr, uint32_t long_cap = 0) {
  const int t = threadIdx.x;
  const char* tb = reinterpret_cast<const char*>(H);
  const uint64_t off = kind == Lut::k32     ? kTableHeaderBytes
                       : kind == Lut::k16   ? table_lut16_off(K, alphabet)
                       : kind == Lut::kPair ? table_pair_off(K, alphabet)
                                            : table_len8_off(K, alphabet);
  const uint4* src = reinterpret_cast<const uint4*>(tb + off);
  uint4* dst = reinterpret_cast<uint4*>(s_lut);
  const uint32_t nv = lut_bytes(kind, K) / 16;
  for (uint32_t k = t; k < nv; k += nthreads) dst[k] = __ldg(src + k);
  if (t < 34) {
    s_end[t] = H->end[t];
    s_base[t] = H->base[t];
  }
  if (t == 0) {
    s_meta[0] = H->maxlen;
    s_meta[1] = H->status;
    s_meta[2] = H->long0;
  }
  if (long_cap) {
    const uint16_t* sorted = reinterpret_cast<const uint16_t*>(tb + table_sorted_off(K));
    const uint32_t nused = H->nused, l0 = H->long0;
    const uint32_t nl = nused > l0 ? nused - l0 : 0u;
    for (uint32_t k = t; k < long_cap; k += nthreads) s_long[k] = k < nl ? sorted[l0 + k] : 0;
  }
}

// The Tables view of a loaded table.
__device__ __forceinline__ Tables make_tables(const FieldDesc& F, uint32_t K, const void* s_lut,
                                              const uint64_t* s_end, const uint32_t* s_base,
                                              const uint32_t* s_meta, const uint16_t* s_long,
                                              uint32_t long_cap) {
  return Tables{s_lut,
                s_end,
                s_base,
                reinterpret_cast<const uint16_t*>(reinterpret_cast<const char*>(F.table) +
                                                  table_sorted_off(K)),
                s_long,
                s_meta[2],
                long_cap,
                s_meta[0],
                32u - K};
}

// Field and tile counts of this launch (kernel parameters, or the device-side
// header of a graph launch).
struct LaunchSize {
  uint64_t units;  // end of the tile range
  uint32_t nfields;
  bool single;     // the one field is the kernel parameter f0
  uint64_t lo;     // start of the tile range
};

__device__ __forceinline__ LaunchSize launch_size(const DecodeParams& P) {
  if (P.hdr) return {P.hdr->total_units, P.hdr->nfields, false, 0};
  return {P.unit_hi ? P.unit_hi : P.total_units, P.nfields, P.nfields == 1, P.unit_lo};
}

__device__ __forceinline__ const FieldDesc& field_of(const DecodeParams& P, const LaunchSize& L,
                                                     uint32_t f) {
  return L.single ? P.f0 : P.fields[f];
}

// Index of the field whose work units contain unit g (fields are in order).
__device__ __forceinline__ uint32_t find_field(const DecodeParams& P, const LaunchSize& L,
                                               uint64_t g) {
  if (L.nfields <= 1) return 0;
  uint32_t lo = 0, hi = L.nfields - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (P.fields[mid].unit_begin <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Copies subsequence i (S bits, plus the following unit that a codeword
// starting near its end may reach) into a shared-memory column with stride
// `stride`.  Units past the readable stream read as zero.
template <int S>
__device__ __forceinline__ void stage_units(uint32_t* col, const FieldDesc& F, uint64_t i,
                                            int stride) {
  constexpr int U = S / 32;
  const uint64_t w0 = i * U;
  const uint32_t* src = F.words + w0;
  if (w0 + U <= F.nwords) {
    if constexpr (U == 2) {
      const uint2 v = ldg_v2(src);
      col[0] = v.x;
      col[stride] = v.y;
    } else {
#pragma unroll
      for (int h = 0; h < U / 4; ++h) {
        const uint4 v = ldg_v4(src + 4 * h);
        col[(4 * h + 0) * stride] = v.x;
        col[(4 * h + 1) * stride] = v.y;
        col[(4 * h + 2) * stride] = v.z;
        col[(4 * h + 3) * stride] = v.w;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < U; ++k) col[k * stride] = (w0 + k < F.nwords) ? __ldg(src + k) : 0u;
  }
  col[U * stride] = (w0 + U < F.nwords) ? __ldg(src + U) : 0u;
}

// Exclusive scan of 32-bit totals into 64-bit bases by one block of
// kScanThreads: base[j] = base[lo] + sum of total[k] for lo <= k < j, for j in
// [lo, hi], where base[lo] is read as 0 when lo == 0 (a later range continues
// the previous one).  end_out (may be NULL) also receives base[hi].  The
// totals are taken in passes of kScanPer rows of kScanThreads; thread t loads
// and stores entry t of every row (coalesced), the rows' warp scans run
// together, warp k scans the warp totals of row k, and each thread adds the
// rows before its own.  A warp's 32 totals must sum below 2^32 (tile totals
// are at most 2^18) or be meant modulo 2^32.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 16;

__device__ __forceinline__ void scan_totals(const uint32_t* total, uint64_t* base, uint64_t lo,
                                            uint64_t hi, uint64_t* end_out) {
  constexpr int NW = kScanThreads / 32;
  static_assert(kScanPer <= NW, "one warp per row");
  __shared__ uint64_t s_off[kScanPer][NW];  // per row: exclusive warp offsets
  __shared__ uint64_t s_row[kScanPer];      // per row: its total
  __shared__ uint64_t s_carry;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) s_carry = lo ? base[lo] : 0ull;
  __syncthreads();
  for (uint64_t p0 = lo; p0 < hi; p0 += static_cast<uint64_t>(kScanThreads) * kScanPer) {
    uint32_t v[kScanPer], incl[kScanPer];
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      const uint64_t i = p0 + static_cast<uint64_t>(k) * kScanThreads + t;
      v[k] = i < hi ? total[i] : 0u;
      incl[k] = v[k];
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
      for (int k = 0; k < kScanPer; ++k) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl[k], o);
        if (lane >= o) incl[k] += u;
      }
    }
    if (lane == 31) {
#pragma unroll
      for (int k = 0; k < kScanPer; ++k) s_off[k][warp] = incl[k];
    }
    __syncthreads();
    if (warp < kScanPer) {
      const uint64_t x = s_off[warp][lane];
      uint64_t xi = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t u = __shfl_up_sync(0xffffffffu, xi, o);
        if (lane >= o) xi += u;
      }
      s_off[warp][lane] = xi - x;
      if (lane == 31) s_row[warp] = xi;
    }
    __syncthreads();
    uint64_t run = s_carry;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      const uint64_t i = p0 + static_cast<uint64_t>(k) * kScanThreads + t;
      if (i < hi) base[i] = run + s_off[k][warp] + (incl[k] - v[k]);
      run += s_row[k];
    }
    __syncthreads();
    if (t == 0) s_carry = run;
    __syncthreads();
  }
  if (t == 0) {
    base[hi] = s_carry;
    if (end_out) *end_out = s_carry;
  }
}

// The units of one subsequence held in registers, so that a tile's loads can
// be issued while the previous tile is still being decoded.
template <int S>
struct UnitRegs {
  uint32_t u[S / 32 + 1];
};

// Loads subsequence i (its S/32 units and the following one) of field F;
// units past the readable stream read as zero.
template <int S>
__device__ __forceinline__ void fetch_units(UnitRegs<S>& r, const FieldDesc& F, uint64_t i) {
  constexpr int U = S / 32;
  const uint64_t w0 = i * U;
  const uint32_t* src = F.words + w0;
  if (w0 + U <= F.nwords) {
    if constexpr (U == 2) {
      const uint2 v = ldg_v2(src);
      r.u[0] = v.x;
      r.u[1] = v.y;
    } else {
#pragma unroll
      for (int h = 0; h < U / 4; ++h) {
        const uint4 v = ldg_v4(src + 4 * h);
        r.u[4 * h + 0] = v.x;
        r.u[4 * h + 1] = v.y;
        r.u[4 * h + 2] = v.z;
        r.u[4 * h + 3] = v.w;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < U; ++k) r.u[k] = (w0 + k < F.nwords) ? __ldg(src + k) : 0u;
  }
  r.u[U] = (w0 + U < F.nwords) ? __ldg(src + U) : 0u;
}

// Writes fetched units into a shared-memory column with stride `stride`.
template <int S>
__device__ __forceinline__ void put_units(uint32_t* col, const UnitRegs<S>& r, int stride) {
#pragma unroll
  for (int k = 0; k <= S / 32; ++k) col[k * stride] = r.u[k];
}

}  // namespace dev
}  // namespace hd
