// decode_warp.cu -- single-pass gap-array decoding with warp-sized tiles.
//
// The gap array (Sec. III-C) gives every subsequence the position of its first
// codeword, so each thread decodes its own subsequence; the output index of
// its first symbol is the prefix sum of the codeword counts before it
// (Sec. III-B2 step 3), and Algorithm 1 (Sec. IV-B) stages the symbols in
// shared memory so that they leave in coalesced stores.  This kernel does the
// whole path in one pass over the stream with the warp as the unit of work:
//
//   tile     32 consecutive subsequences of S bits, one per lane; tiles go
//            round-robin over the warps of a cooperative (all-resident)
//            launch, and the units and gap entries of a warp's next tile are
//            loaded into registers while it decodes the current one;
//   decode   each lane walks its subsequence once, word by word straight from
//            registers, one shared-memory table lookup per codeword, and
//            stores each symbol in its own column of a per-warp scratch
//            (symbol j of lane l at 16-bit slot j*32 + l: lanes at the same j
//            share nothing but pairs of halves of one word, lanes a row apart
//            fall in the other half of the banks);
//   offsets  a warp scan of the counts gives each lane's offset inside the
//            tile; a decoupled look-back over per-tile states in global
//            memory (the aggregate published as soon as the tile is counted,
//            the inclusive prefix once its own prefix is known) gives the
//            tile's first output index;
//   write    the lanes copy their columns into the warp's window in output
//            order, two symbols per 32-bit store, and the warp writes the
//            window to global memory with 16-byte stores.
//
// After the table load no block-wide barrier is taken: a warp waiting for a
// predecessor's count leaves the SM's issue slots to the other warps.
//
// A lane holds at most cmax symbols in its column.  When every code has at
// least `minlen` bits and S / minlen <= cmax no lane can exceed that and the
// decode loop stores without checking; otherwise stores are checked, and a
// tile in which some lane overflowed writes its output in window-sized rounds
// whose overflowing lanes decode their subsequence again from the registers.
#include <cuda_runtime.h>

#include "common.cuh"
#include "decode_common.cuh"
#include "kernels.h"

namespace hd {
namespace {

using namespace dev;

constexpr uint32_t kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
  uint16_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint4 lds_v4(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a));
  return v;
}
__device__ __forceinline__ void sts_u16(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"(static_cast<uint16_t>(v)) : "memory");
}
__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Per-warp shared memory: two column scratches (one per round in flight;
// cmax + 2 rows of 32 lanes x 2 bytes each, one spare row that the copy may
// read past a lane's last symbol), then the window (32*cmax symbols + 16 for
// the alignment pad).
__host__ __device__ constexpr uint32_t col_bytes(uint32_t cmax) { return (cmax + 2) * 64u; }
__host__ __device__ constexpr uint32_t win_syms(uint32_t cmax) { return 32u * cmax + 16u; }
__host__ __device__ constexpr uint32_t warp_bytes(uint32_t cmax) {
  return (2u * col_bytes(cmax) + 2u * win_syms(cmax) + 15u) & ~15u;
}

// What the escape path needs of the decode tables (shared-memory limits,
// long-code symbols), passed by value to keep the decode loop's registers.
struct LongTab {
  const uint64_t* end;
  const uint32_t* base;
  const uint16_t* sorted;
  const uint16_t* long_syms;
  uint32_t long0, long_cap, maxlen;
  uint32_t sub_a;  // shared address of the second-level tables
  uint32_t sub_bits, nsub, sub_p0, K;
};

// Code of a table entry that is no direct hit (longer than K bits, a prefix
// with codes of several lengths, or no code at all): walk the canonical
// limits.  Returns length | symbol << 8 | (invalid << 31).  An invalid bit
// pattern counts as `lmin` bits, which keeps a lane's codeword count within
// S / lmin even for a corrupt stream.  Rare (codes longer than K bits), so it
// is a call rather than part of the decode loop.
template <class E>
__device__ __noinline__ uint32_t escape(LongTab T, uint32_t w, uint32_t e, uint32_t lmin) {
  uint32_t L = e & 0xFFu;
  const bool mixed = sizeof(E) == 2 ? (e & kLut16Mixed) != 0 : L != ((e >> 8) & 0xFFu);
  if (mixed) {
    while (L <= T.maxlen && static_cast<uint64_t>(w) >= T.end[L]) ++L;
    if (L > T.maxlen) return lmin | 0x80000000u;
  }
  const uint32_t rank = (w >> (32 - L)) + T.base[L];
  const uint32_t li = rank - T.long0;
  const uint32_t sym = li < T.long_cap ? T.long_syms[li] : __ldg(T.sorted + rank);
  return L | (sym << 8);
}

// A code longer than the first-level table (entry e at window w): the
// second-level table of its prefix when it has one and the code fits it, else
// the walk.  v receives the symbol (a second-level entry: raw, with length
// bits the copy masks off).
template <class E>
__device__ __forceinline__ uint32_t long_step(const LongTab* T, uint32_t w, uint32_t e,
                                              uint32_t lmin, uint32_t& v, bool& bad) {
  const uint32_t s = (w >> (32u - T->K)) - T->sub_p0;
  if (s < T->nsub) {
    const uint32_t q = (w << T->K) >> (32u - T->sub_bits);
    const uint32_t e2 = lds_u16(T->sub_a + 2u * ((s << T->sub_bits) | q));
    if (e2 >> 12) {
      v = e2;
      return T->K + (e2 >> 12);
    }
  }
  const uint32_t x = escape<E>(*T, w, e, lmin);
  v = (x >> 8) & 0xFFFFu;
  bad |= (x >> 31) != 0;
  return x & 0xFFu;
}

// Length of the codeword at window w; v receives its symbol (16-bit tables:
// the raw entry, whose length bits the copy masks off).
template <class E>
__device__ __forceinline__ uint32_t dec_step(uint32_t lut_a, uint32_t shift, const LongTab* T,
                                             uint32_t w, uint32_t lmin, uint32_t& v, bool& bad) {
  uint32_t e;
  if constexpr (sizeof(E) == 2) {
    e = lds_u16(lut_a + ((w >> shift) << 1));
    if (e >> 12) {
      v = e;
      return e >> 12;
    }
  } else {
    e = lds_u32(lut_a + ((w >> shift) << 2));
    if (!(e & kLongFlag)) {
      v = e & 0xFFFFu;
      return e >> 16;
    }
  }
  return long_step<E>(T, w, e, lmin, v, bad);
}

// Decodes the codewords that start in bits [pos, end) of a subsequence held
// in registers (r[k] = unit k, r[S/32] = the first unit after it), calling
// sink(v) for each in order.  BOUNDED = false: end = S (every codeword that
// starts in the subsequence).  Returns where the last codeword ended,
// relative to the subsequence start.
template <int S, class E, bool BOUNDED, class Sink>
__device__ __forceinline__ uint32_t walk(const uint32_t (&r)[S / 32 + 1], uint32_t pos,
                                         uint32_t end, uint32_t lut_a, uint32_t shift,
                                         const LongTab* T, uint32_t lmin, bool& bad, Sink&& sink) {
  constexpr int U = S / 32;
  uint32_t stop = 0xffffffffu;
#pragma unroll
  for (int k = 0; k < U; ++k) {
    const uint32_t hi = r[k], lo = r[k + 1];
    while (pos < 32) {
      if (BOUNDED && k * 32u + pos >= end) {
        stop = k * 32u + pos;
        pos = 0x40000000u;
        break;
      }
      uint32_t v;
      pos += dec_step<E>(lut_a, shift, T, __funnelshift_l(lo, hi, pos), lmin, v, bad);
      sink(v);
    }
    pos -= 32;
  }
  return stop != 0xffffffffu ? stop : S + pos;
}

// The decode loop for codebooks whose shortest code has lmin >= 32 / MAXW
// bits: at most MAXW codewords start in a 32-bit unit, so every unit takes
// exactly MAXW steps without a loop branch; a step past the unit's end
// (pos >= 32) changes nothing but stores into the slot after the lane's last
// symbol, which the next step or nobody reads.  A code longer than the
// first-level table reads its prefix's second-level table in a branch of its
// own; one longer than that too (rare: beyond K + sub_bits bits) sets `esc`
// and counts as lmin bits, and the caller decodes the whole subsequence again
// with walk (the loop itself holds no call).  16-bit tables only.  Needs a
// column of S / lmin + 1 slots (the unchecked case).  Returns as
// walk<.., false>.
template <int S, int MAXW>
__device__ __forceinline__ uint32_t walk_fixed(const uint32_t (&r)[S / 32 + 1], uint32_t pos,
                                               uint32_t lut_a, uint32_t shift, const LongTab* T,
                                               uint32_t lmin, bool& esc, uint32_t& a) {
  constexpr int U = S / 32;
#pragma unroll
  for (int k = 0; k < U; ++k) {
    const uint32_t hi = r[k], lo = r[k + 1];
#pragma unroll
    for (int st = 0; st < MAXW; ++st) {
      const bool in = pos < 32;
      const uint32_t w = __funnelshift_l(lo, hi, pos);
      const uint32_t p = w >> shift;
      uint32_t e = lds_u16(lut_a + (p << 1));
      uint32_t L = e >> 12;
      if (in && L == 0) {
        const uint32_t s = p - T->sub_p0;
        if (s < T->nsub) {
          const uint32_t sb = T->sub_bits;
          const uint32_t e2 = lds_u16(T->sub_a + 2u * ((s << sb) | ((w << T->K) >> (32u - sb))));
          if (e2 >> 12) {
            L = T->K + (e2 >> 12);
            e = e2;
          }
        }
        if (L == 0) {
          esc = true;
          L = lmin;
        }
      }
      sts_u16(a, e);
      a += in ? 64u : 0u;
      pos += in ? L : 0u;
    }
    pos -= 32;
  }
  return S + pos;
}

// Writes window indices [lo, hi) (16-byte aligned window; index r is virtual
// output index a0 + r, a0 a multiple of 8) to out_al, clipped to virtual
// indices below Xn.  The 16-byte aligned middle goes out as one bulk copy by
// the TMA engine, issued by lane 0 (the lanes ran fence_async_smem() after
// writing the window; lane 0 waits for the copy's read before the window is
// written again); the at most 7 symbols before and after it, plain.
__device__ __forceinline__ void flush_window(uint32_t win_a, const uint16_t* win, uint32_t lo,
                                             uint32_t hi, uint64_t a0, uint16_t* out_al,
                                             uint64_t Xn, int lane) {
  const uint32_t end =
      a0 + hi <= Xn ? hi : (Xn > a0 + lo ? static_cast<uint32_t>(Xn - a0) : lo);
  const uint32_t ra = (lo + 7) & ~7u, rb = end & ~7u;
  if (rb > ra) {
    if (lane < 8) {
      const uint32_t r = lo + lane;
      if (r < ra) out_al[a0 + r] = win[r];
    } else if (lane < 16) {
      const uint32_t r = rb + (lane - 8);
      if (r < end) out_al[a0 + r] = win[r];
    } else if (lane == 16) {
      if (!bulk_store(out_al + a0 + ra, win_a + 2 * ra, 2 * (rb - ra)))
        for (uint32_t r = ra; r < rb; ++r) out_al[a0 + r] = win[r];
    }
  } else {
    for (uint32_t r = lo + lane; r < end; r += 32) out_al[a0 + r] = win[r];
  }
}

template <int S>
struct WarpTileIn {
  UnitRegs<S> bits;
  uint32_t gap0, gap1;
};

template <int S>
__device__ __forceinline__ void fetch_warp_tile(WarpTileIn<S>& in, const FieldDesc& F, uint64_t g,
                                                int lane) {
  const uint64_t i = g * 32 + lane;
  if (i < F.nsub) {
    fetch_units<S>(in.bits, F, i);
    in.gap0 = __ldg(F.gap + i * F.gap_stride);
    in.gap1 = (i + 1 < F.nsub) ? __ldg(F.gap + (i + 1) * F.gap_stride) : 0u;
  } else {
    in.gap0 = in.gap1 = 0;
  }
}

// What a lane keeps of a decoded tile until the tile is written.
struct TileRes {
  uint32_t c;      // codewords of the lane's subsequence
  uint32_t o;      // offset of its first symbol within the tile
  uint32_t C;      // codewords of the tile (warp-uniform)
  uint32_t start;  // bit where the lane's first codeword starts
  uint32_t err;
  bool overflow;   // some lane's column overflowed (warp-uniform)
};

// Everything a warp needs to decode and write tiles of one field.
struct WarpCtx {
  const FieldDesc* F;
  const LongTab* T;  // in shared memory
  uint32_t lut_a, shift, lmin, cmax;
  bool unchecked, table_ok;
  uint32_t win_a;
  uint16_t* win;
  uint16_t* out_al;  // 16-byte aligned; virtual index X = output index + off0
  uint32_t off0;
  uint64_t Xn;       // n + off0
};

// Decodes tile g (bits in `in`) once: each lane's symbols into its column at
// col_a (lane offset included), then the warp scan of the counts.
template <int S, class E>
__device__ __forceinline__ TileRes decode_tile(const WarpCtx& W, const WarpTileIn<S>& in,
                                               uint64_t g, uint32_t col_a, int lane) {
  const FieldDesc& F = *W.F;
  const uint64_t i = g * 32 + lane;
  TileRes R{};
  uint32_t c = 0, err = 0;
  bool bad = false;
  uint32_t a = col_a;  // next column slot (64 bytes per row)
  auto store = [&](uint32_t v) {
    sts_u16(a, v);
    a += 64;
  };
  auto store_checked = [&](uint32_t v) {
    if (c < W.cmax) {
      sts_u16(a, v);
      a += 64;
    }
    ++c;
  };
  if (W.table_ok && (g + 1) * 32 < F.nsub) {
    // every lane's subsequence is followed by another: codewords start
    // anywhere in [gap0, S) and the last one must end at S + gap1
    R.start = in.gap0;
    if (R.start >= S) {
      err |= kErrGap;
    } else if (sizeof(E) == 2 && W.unchecked && W.lmin >= 8) {
      // four steps per unit (codes of 8 bits and more)
      bool esc = false;
      uint32_t fin = walk_fixed<S, 4>(in.bits.u, R.start, W.lut_a, W.shift, W.T, W.lmin, esc, a);
      if (esc) {  // a code beyond the second-level tables: decode again
        a = col_a;
        fin = walk<S, E, false>(in.bits.u, R.start, S, W.lut_a, W.shift, W.T, W.lmin, bad, store);
      }
      c = (a - col_a) >> 6;
      if (fin != S + in.gap1) err |= kErrGap;
    } else if (W.unchecked) {
      const uint32_t fin = walk<S, E, false>(in.bits.u, R.start, S, W.lut_a, W.shift, W.T, W.lmin,
                                              bad, store);
      c = (a - col_a) >> 6;
      if (fin != S + in.gap1) err |= kErrGap;
    } else {
      const uint32_t fin = walk<S, E, false>(in.bits.u, R.start, S, W.lut_a, W.shift, W.T, W.lmin,
                                              bad, store_checked);
      if (fin != S + in.gap1) err |= kErrGap;
    }
  } else if (W.table_ok && i < F.nsub) {
    // the field's last tile: the last subsequence ends at nbits
    const uint64_t rem = F.nbits - i * S;
    const uint32_t end = rem < S ? static_cast<uint32_t>(rem) : S;
    const uint32_t expect = (i + 1 < F.nsub) ? S + in.gap1 : static_cast<uint32_t>(rem);
    R.start = in.gap0;
    if (R.start > end || R.start >= S) {
      err |= kErrGap;
      R.start = end;
    }
    const uint32_t fin = walk<S, E, true>(in.bits.u, R.start, end, W.lut_a, W.shift, W.T, W.lmin,
                                           bad, store_checked);
    if (fin != expect) err |= kErrGap;
  }
  if (bad) err |= kErrCode;
  const uint32_t incl = warp_incl_scan(c, lane);
  R.c = c;
  R.o = incl - c;
  R.C = __shfl_sync(kFull, incl, 31);
  R.overflow = __any_sync(kFull, c > W.cmax);
  R.err = err;
  return R;
}

// Writes tile g (decoded into the column at col_a) to output index `base`
// on: the lanes copy their columns into the warp's window in output order,
// the warp stores the window (Algorithm 1).  A tile whose column overflowed
// goes in window-sized rounds, its overflowing lanes decoding again from the
// stream.
template <int S, class E>
__device__ __forceinline__ void write_tile(const WarpCtx& W, const TileRes& R, uint64_t g,
                                           uint64_t base, uint32_t col_a, int lane) {
  constexpr uint32_t kMask16 = sizeof(E) == 2 ? 0x0FFFu : 0xFFFFu;
  constexpr uint32_t kMask32 = kMask16 | (kMask16 << 16);
  const uint32_t c = R.c, o = R.o, C = R.C;
  // the previous tile's bulk copy must have read the window
  if (lane == 16) bulk_wait_read();
  __syncwarp();
  if (!R.overflow) {
    const uint64_t X0 = base + W.off0;
    const uint32_t pad = static_cast<uint32_t>(X0 & 7u);
    if (c) {
      const uint32_t x0 = pad + o;  // window index of the lane's first symbol
      const uint32_t par = x0 & 1u;
      // symbols j, j+1 of the column (rows 64 bytes apart) make one window
      // word when x0 + j is even
      uint32_t src = col_a;
      if (par) {
        sts_u16(W.win_a + 2 * x0, lds_u16(src) & kMask16);
        src += 64;
      }
      const uint32_t nfw = (c - par) >> 1;
      uint32_t dst = W.win_a + 2 * (x0 + par);
      for (uint32_t m = 0; m < nfw; ++m) {
        const uint32_t lo = lds_u16(src), hi = lds_u16(src + 64);
        sts_u32(dst, (lo | (hi << 16)) & kMask32);
        src += 128;
        dst += 4;
      }
      if ((c - par) & 1u) sts_u16(W.win_a + 2 * (x0 + c - 1), lds_u16(src) & kMask16);
    }
    fence_async_smem();
    __syncwarp();
    flush_window(W.win_a, W.win, pad, pad + C, X0 - pad, W.out_al, W.Xn, lane);
    __syncwarp();
    return;
  }
  const FieldDesc& F = *W.F;
  const uint32_t wcap = 32u * W.cmax;
  WarpTileIn<S> in;
  fetch_warp_tile<S>(in, F, g, lane);
  const uint64_t i = g * 32 + lane;
  for (uint32_t ws = 0; ws < C; ws += wcap) {
    const uint32_t we = C < ws + wcap ? C : ws + wcap;
    const uint64_t X0 = base + ws + W.off0;
    const uint32_t pad = static_cast<uint32_t>(X0 & 7u);
    const uint32_t lo = o > ws ? o : ws, hi = o + c < we ? o + c : we;
    if (lo < hi) {
      const uint32_t j0 = lo - o, j1 = hi - o;
      const uint32_t wb = W.win_a + 2 * (pad + o - ws);  // window address of symbol 0
      if (c <= W.cmax) {
        for (uint32_t j = j0; j < j1; ++j) {
          const uint32_t v = lds_u16(col_a + j * 64u);
          sts_u16(wb + 2 * j, v & kMask16);
        }
      } else {
        uint32_t j = 0;
        bool bad2 = false;
        auto put = [&](uint32_t v) {
          if (j >= j0 && j < j1) sts_u16(wb + 2 * j, v & kMask16);
          ++j;
        };
        const uint64_t rem = F.nbits - i * S;
        const uint32_t end = rem < S ? static_cast<uint32_t>(rem) : S;
        walk<S, E, true>(in.bits.u, R.start, end, W.lut_a, W.shift, W.T, W.lmin, bad2, put);
      }
    }
    fence_async_smem();
    __syncwarp();
    flush_window(W.win_a, W.win, pad, pad + (we - ws), X0 - pad, W.out_al, W.Xn, lane);
    if (lane == 16) bulk_wait_read();
    __syncwarp();
  }
}

// Tiles and rounds.  The decoding warps take the tiles round-robin in
// rounds: in round r, decoding warp w of block b decodes tile (r*G + b)*NW + w
// (G blocks of NW decoding warps), so a block-round covers NW consecutive
// tiles, a super-tile.  Each block has one more warp, its index warp: it
// waits until the decoding warps have counted a round (their counts are
// combined in shared memory), runs the look-back over super-tile states
// (about G super-tiles in flight instead of G*NW tiles, so a look-back ends
// within a round trip or two) and publishes each tile's first output index.
// Meanwhile the decoding warps decode their next round into a second column,
// so they only wait for a round's index once they are a whole decode ahead,
// and no decoding warp ever waits for another block.  The launch is
// cooperative, so every warp is resident: a super-tile waits only for
// smaller ones, whose blocks never wait for a larger one.
template <int S, int NW, class E>
__global__ void __launch_bounds__((NW + 1) * 32, 1)
    k_decode_warp(const __grid_constant__ DecodeParams P) {
  constexpr Lut kKind = sizeof(E) == 2 ? Lut::k16 : Lut::k32;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint64_t s_end[34];
  __shared__ uint32_t s_base[34];
  __shared__ uint32_t s_meta[3];
  __shared__ uint32_t s_lmin;
  __shared__ uint32_t s_cnt[2][NW];    // tile counts of a block-round
  __shared__ uint64_t s_first[2][NW];  // each tile's first output index
  __shared__ uint32_t s_done[2];       // decoding warps of the round that have counted
  __shared__ uint32_t s_ready[2];      // round whose indices are in s_first

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const FieldDesc& F = P.f0;
  const uint32_t cmax = P.cmax;
  // shared memory: first-level table | second-level tables | per-warp
  // columns and windows | long-code symbols
  const uint32_t lut_b = lut_bytes(kKind, P.K) + 2 * sub_cap(P.K);
  unsigned char* s_lut = smem;
  uint16_t* s_sub = reinterpret_cast<uint16_t*>(smem + lut_bytes(kKind, P.K));
  uint16_t* s_long = reinterpret_cast<uint16_t*>(smem + lut_b + NW * warp_bytes(cmax));
  load_table(F.table, P.K, F.alphabet, kKind, s_lut, s_end, s_base, s_meta, (NW + 1) * 32, s_long,
             P.long_cap);
  const uint32_t sub_n = F.table->nsub << F.table->sub_bits;  // entries in use (<= sub_cap(K))
  {
    const uint4* src = reinterpret_cast<const uint4*>(reinterpret_cast<const char*>(F.table) +
                                                      table_sub_off(P.K, F.alphabet));
    uint4* dst = reinterpret_cast<uint4*>(s_sub);
    for (uint32_t k = t; k < (sub_n + 7) / 8; k += (NW + 1) * 32) dst[k] = __ldg(src + k);
  }
  __shared__ LongTab s_lt;
  if (t == 0) {
    s_lmin = F.table->minlen;
    s_lt = LongTab{s_end,
                   s_base,
                   reinterpret_cast<const uint16_t*>(reinterpret_cast<const char*>(F.table) +
                                                     table_sorted_off(P.K)),
                   s_long,
                   F.table->long0,
                   P.long_cap,
                   F.table->maxlen,
                   smem_addr(s_sub),
                   F.table->sub_bits,
                   F.table->nsub,
                   F.table->sub_p0,
                   P.K};
    s_done[0] = s_done[1] = 0;
    s_ready[0] = s_ready[1] = 0xffffffffu;
  }
  __syncthreads();

  const uint64_t units = F.nunits;
  const uint64_t G = gridDim.x;
  const uint64_t supers = (units + NW - 1) / NW;
  // rounds of this block: super-tiles r*G + blockIdx.x below `supers`
  const uint64_t R = supers > blockIdx.x ? (supers - blockIdx.x + G - 1) / G : 0;

  if (warp == NW) {
    // ---- the index warp ----------------------------------------------------
    for (uint64_t r = 0; r < R; ++r) {
      const int b = static_cast<int>(r & 1);
      bool ok = true;
      if (lane == 0) {
        const uint64_t t0 = static_cast<uint64_t>(clock64());
        uint32_t nap = 32;
        while (*static_cast<volatile uint32_t*>(&s_done[b]) != NW) {
          if (static_cast<uint64_t>(clock64()) - t0 > 2 * P.timeout_cycles) {
            atomicExch(P.abort_flag, 1u);
            atomicOr(F.err, kErrTimeout);
            ok = false;
            break;
          }
          __nanosleep(nap);
          nap = nap < 256 ? 2 * nap : nap;
        }
      }
      __threadfence_block();
      if (!__shfl_sync(kFull, ok, 0)) return;  // the decoding warps give up on their own
      const uint32_t cw = lane < NW ? *static_cast<volatile uint32_t*>(&s_cnt[b][lane]) : 0u;
      const uint32_t incl = warp_incl_scan(cw, lane);
      const uint32_t total = __shfl_sync(kFull, incl, 31);
      const uint64_t excl = lookback_counts(P, r * G + blockIdx.x, 0, total, F.err);
      if (lane < NW) s_first[b][lane] = excl + (incl - cw);
      if (lane == 0) s_done[b] = 0;
      __threadfence_block();
      __syncwarp();
      if (lane == 0) *static_cast<volatile uint32_t*>(&s_ready[b]) = static_cast<uint32_t>(r);
    }
    return;
  }

  // ---- the decoding warps ---------------------------------------------------
  unsigned char* wreg = smem + lut_b + warp * warp_bytes(cmax);
  WarpCtx W;
  W.F = &F;
  W.T = &s_lt;
  W.table_ok = s_meta[1] == 0;
  W.lmin = s_lmin ? s_lmin : 1u;
  W.cmax = cmax;
  W.unchecked = (S + W.lmin - 1) / W.lmin <= cmax;
  W.lut_a = smem_addr(s_lut);
  W.shift = 32u - P.K;
  W.win = reinterpret_cast<uint16_t*>(wreg + 2 * col_bytes(cmax));
  W.win_a = smem_addr(W.win);
  W.off0 = static_cast<uint32_t>((reinterpret_cast<uintptr_t>(F.out) >> 1) & 7u);
  W.out_al = F.out - W.off0;
  W.Xn = F.n + W.off0;
  const uint32_t col0 = smem_addr(wreg) + 2u * lane;  // column of even rounds
  const uint32_t col1 = col0 + col_bytes(cmax);        // column of odd rounds
  auto tile_of = [&](uint64_t r) { return (r * G + blockIdx.x) * NW + warp; };

  // the count of this warp's tile of round r, for the index warp
  auto publish = [&](uint64_t r, uint32_t C) {
    const int b = static_cast<int>(r & 1);
    if (lane == 0) {
      s_cnt[b][warp] = C;
      __threadfence_block();
      atomicAdd(&s_done[b], 1u);
    }
    __syncwarp();
  };
  // first output index of this warp's tile of round r (bounded wait)
  auto first_index = [&](uint64_t r) -> uint64_t {
    const int b = static_cast<int>(r & 1);
    bool ok = true;
    if (lane == 0) {
      const uint64_t t0 = static_cast<uint64_t>(clock64());
      uint32_t nap = 32;
      while (*static_cast<volatile uint32_t*>(&s_ready[b]) != static_cast<uint32_t>(r)) {
        if (static_cast<uint64_t>(clock64()) - t0 > 3 * P.timeout_cycles) {
          atomicExch(P.abort_flag, 1u);
          atomicOr(F.err, kErrTimeout);
          ok = false;
          break;
        }
        __nanosleep(nap);
        nap = nap < 256 ? 2 * nap : nap;
      }
    }
    __threadfence_block();
    ok = __shfl_sync(kFull, ok, 0);
    return ok ? *static_cast<volatile uint64_t*>(&s_first[b][warp]) : 0ull;
  };

  if (R == 0) return;
  WarpTileIn<S> nxt;
  uint64_t g = tile_of(0);
  if (g < units) fetch_warp_tile<S>(nxt, F, g, lane);
  TileRes rw{};
  if (g < units) rw = decode_tile<S, E>(W, nxt, g, col0, lane);
  publish(0, g < units ? rw.C : 0u);
  if (R > 1 && tile_of(1) < units) fetch_warp_tile<S>(nxt, F, tile_of(1), lane);
  for (uint64_t r = 0; r < R; ++r) {
    const uint64_t gw = tile_of(r);
    // decode the next round before waiting for this one's output index
    TileRes rn{};
    if (r + 1 < R) {
      const uint64_t gn = tile_of(r + 1);
      if (gn < units) {
        const WarpTileIn<S> cur = nxt;
        if (r + 2 < R && tile_of(r + 2) < units) fetch_warp_tile<S>(nxt, F, tile_of(r + 2), lane);
        rn = decode_tile<S, E>(W, cur, gn, ((r + 1) & 1) ? col1 : col0, lane);
      }
      publish(r + 1, gn < units ? rn.C : 0u);
    }
    const uint64_t base = first_index(r);
    if (gw < units) {
      uint32_t err = rw.err;
      if (lane == 0 && gw + 1 == units && base + rw.C != F.n) err |= kErrCount;
      if (lane == 0 && !W.table_ok && gw == 0) err |= kErrTable;
      write_tile<S, E>(W, rw, gw, base, (r & 1) ? col1 : col0, lane);
      err = __reduce_or_sync(kFull, err);
      if (lane == 0 && err) atomicOr(F.err, err);
    }
    rw = rn;
  }
  if (lane == 16) bulk_wait_all();  // the last window copies are done
}

template <int S, int NW>
cudaError_t launch_snw(const DecodeParams& p, const LaunchShape& s, int num_sms,
                       cudaStream_t stream) {
  const size_t smem = warp_decode_smem_bytes(s);
  auto kern = s.lut16 ? k_decode_warp<S, NW, uint16_t> : k_decode_warp<S, NW, uint32_t>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (NW + 1) * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  uint64_t grid = static_cast<uint64_t>(per_sm) * num_sms;
  if (s.grid && s.grid < grid) grid = s.grid;
  const uint64_t blocks_needed = (p.f0.nunits + NW - 1) / NW;  // super-tiles
  if (grid > blocks_needed) grid = blocks_needed;
  if (grid == 0) return cudaSuccess;
  // cooperative: all blocks resident at once (the round-robin tiles rely on it)
  void* args[] = {const_cast<DecodeParams*>(&p)};
  e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern),
                                  dim3(static_cast<unsigned>(grid)), dim3((NW + 1) * 32), args, smem,
                                  stream);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_s(const DecodeParams& p, const LaunchShape& s, int num_sms,
                     cudaStream_t stream) {
  // threads / 32 warps per block: the index warp and threads / 32 - 1
  // decoding warps
  switch (s.threads) {
    case 128: return launch_snw<S, 3>(p, s, num_sms, stream);
    case 256: return launch_snw<S, 7>(p, s, num_sms, stream);
    case 512: return launch_snw<S, 15>(p, s, num_sms, stream);
    case 768: return launch_snw<S, 23>(p, s, num_sms, stream);
    case 1024: return launch_snw<S, 31>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t warp_decode_smem_bytes(const LaunchShape& s) {
  const size_t lut = dev::lut_bytes(s.lut16 ? dev::Lut::k16 : dev::Lut::k32, s.K);
  size_t b = lut + 2 * sub_cap(s.K);
  b += static_cast<size_t>(s.threads / 32 - 1) * warp_bytes(s.cmax);
  b += static_cast<size_t>(s.long_cap) * 2;
  return (b + 15) & ~static_cast<size_t>(15);
}

cudaError_t launch_decode_warp(const DecodeParams& p, const LaunchShape& s, int num_sms,
                               cudaStream_t stream) {
  if (p.cmax != s.cmax || s.cmax < 2 || s.cmax > 512 || (s.cmax & 1u) ||
      p.long_cap != s.long_cap || p.hdr || p.nfields != 1 || !p.unit_state || !p.abort_flag)
    return cudaErrorInvalidValue;
  switch (s.S) {
    case 64: return launch_s<64>(p, s, num_sms, stream);
    case 128: return launch_s<128>(p, s, num_sms, stream);
    case 256: return launch_s<256>(p, s, num_sms, stream);
    case 512: return launch_s<512>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hd
