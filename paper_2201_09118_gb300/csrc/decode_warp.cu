// decode_warp.cu -- single-pass gap-array decoding with warp-sized tiles.
//
// The gap array (Sec. III-C) gives every subsequence the position of its first
// codeword, so each thread decodes its own subsequence; the output index of
// its first symbol is the prefix sum of the codeword counts before it
// (Sec. III-B2 step 3), and Algorithm 1 (Sec. IV-B) stages the symbols in
// shared memory so that they leave in coalesced stores.  This kernel does the
// whole path in one pass over the stream with the warp as the unit of work:
//
//   tile     32 consecutive subsequences of S bits, one per lane, taken in
//            order from a global ticket; the units and gap entries of the
//            warp's next tile are loaded into registers while it decodes the
//            current one;
//   decode   each lane walks its subsequence once, word by word straight from
//            registers, one shared-memory table lookup per codeword, and
//            stores each symbol in its own column of a per-warp scratch
//            (symbol j of lane l in 32-bit slot (j/2)*32 + l, half j%2, so the
//            32 lanes always write 32 distinct banks);
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

// Per-warp shared memory: the column scratch ((cmax/2 + 2) rows of 32 lanes x
// 4 bytes, one spare row that the copy may read past a lane's last pair),
// then the window (32*cmax symbols + 16 for the alignment pad).
__host__ __device__ constexpr uint32_t col_bytes(uint32_t cmax) { return (cmax / 2 + 2) * 128u; }
__host__ __device__ constexpr uint32_t win_syms(uint32_t cmax) { return 32u * cmax + 16u; }
__host__ __device__ constexpr uint32_t warp_bytes(uint32_t cmax) {
  return (col_bytes(cmax) + 2u * win_syms(cmax) + 15u) & ~15u;
}

// Code of a table entry that is no direct hit (longer than K bits, a prefix
// with codes of several lengths, or no code at all): walk the canonical
// limits.  An invalid bit pattern sets `bad` and counts as `lmin` bits, which
// keeps a lane's codeword count within S / lmin even for a corrupt stream.
template <class E>
__device__ __forceinline__ uint32_t escape(const Tables& T, uint32_t w, uint32_t e, uint32_t lmin,
                                        uint32_t& v, bool& bad) {
  uint32_t L = e & 0xFFu;
  const bool mixed = sizeof(E) == 2 ? (e & kLut16Mixed) != 0 : L != ((e >> 8) & 0xFFu);
  if (mixed) {
    L = walk_len(T, w, L, bad);
    if (!L) {
      v = 0;
      return lmin;
    }
  }
  v = long_sym(T, w, L);
  return L;
}

// Length of the codeword at window w; v receives its symbol (16-bit tables:
// the raw entry, whose length bits the copy masks off).
template <class E>
__device__ __forceinline__ uint32_t dec_step(uint32_t lut_a, uint32_t shift, const Tables& T,
                                             uint32_t w, uint32_t lmin, uint32_t& v, bool& bad) {
  if constexpr (sizeof(E) == 2) {
    const uint32_t e = lds_u16(lut_a + ((w >> shift) << 1));
    const uint32_t L = e >> 12;
    if (L) {
      v = e;
      return L;
    }
    return escape<E>(T, w, e, lmin, v, bad);
  } else {
    const uint32_t e = lds_u32(lut_a + ((w >> shift) << 2));
    if (!(e & kLongFlag)) {
      v = e & 0xFFFFu;
      return e >> 16;
    }
    return escape<E>(T, w, e, lmin, v, bad);
  }
}

// Decodes the codewords that start in bits [pos, end) of a subsequence held
// in registers (r[k] = unit k, r[S/32] = the first unit after it), calling
// sink(v) for each in order.  BOUNDED = false: end = S (every codeword that
// starts in the subsequence).  Returns where the last codeword ended,
// relative to the subsequence start.
template <int S, class E, bool BOUNDED, class Sink>
__device__ __forceinline__ uint32_t walk(const uint32_t (&r)[S / 32 + 1], uint32_t pos,
                                         uint32_t end, uint32_t lut_a, uint32_t shift,
                                         const Tables& T, uint32_t lmin, bool& bad, Sink&& sink) {
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

// Writes window indices [lo, hi) (16-byte aligned window; index r is virtual
// output index a0 + r, a0 a multiple of 8) to out_al, clipped to virtual
// indices below Xn.
__device__ __forceinline__ void flush_window(uint32_t win_a, const uint16_t* win, uint32_t lo,
                                             uint32_t hi, uint64_t a0, uint16_t* out_al,
                                             uint64_t Xn, int lane) {
  const uint32_t nq = (hi + 7) >> 3;
  for (uint32_t q = (lo >> 3) + lane; q < nq; q += 32) {
    const uint32_t r0 = q << 3;
    const uint64_t Xq = a0 + r0;
    if (r0 >= lo && r0 + 8 <= hi && Xq + 8 <= Xn) {
      *reinterpret_cast<uint4*>(out_al + Xq) = lds_v4(win_a + 2 * r0);
    } else {
      const uint32_t b = r0 > lo ? r0 : lo;
      const uint32_t e = r0 + 8 < hi ? r0 + 8 : hi;
      for (uint32_t x = b; x < e; ++x)
        if (a0 + x < Xn) out_al[a0 + x] = win[x];
    }
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

template <int S, int NW, class E>
__global__ void __launch_bounds__(NW * 32, 1) k_decode_warp(const __grid_constant__ DecodeParams P) {
  constexpr Lut kKind = sizeof(E) == 2 ? Lut::k16 : Lut::k32;
  constexpr uint32_t kMask16 = sizeof(E) == 2 ? 0x0FFFu : 0xFFFFu;
  constexpr uint32_t kMask32 = kMask16 | (kMask16 << 16);
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint64_t s_end[34];
  __shared__ uint32_t s_base[34];
  __shared__ uint32_t s_meta[3];
  __shared__ uint32_t s_lmin;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const FieldDesc& F = P.f0;
  const uint32_t cmax = P.cmax;
  const uint32_t lut_b = lut_bytes(kKind, P.K);
  unsigned char* s_lut = smem;
  unsigned char* wreg = smem + lut_b + warp * warp_bytes(cmax);
  uint16_t* s_long = reinterpret_cast<uint16_t*>(smem + lut_b + NW * warp_bytes(cmax));
  load_table(F.table, P.K, F.alphabet, kKind, s_lut, s_end, s_base, s_meta, NW * 32, s_long,
             P.long_cap);
  if (t == 0) s_lmin = F.table->minlen;
  __syncthreads();

  const Tables T = make_tables(F, P.K, s_lut, s_end, s_base, s_meta, s_long, P.long_cap);
  const bool table_ok = s_meta[1] == 0;
  const uint32_t lmin = s_lmin ? s_lmin : 1u;
  const bool unchecked = (S + lmin - 1) / lmin <= cmax;
  const uint32_t lut_a = smem_addr(s_lut), shift = 32u - P.K;
  const uint32_t col_a = smem_addr(wreg) + 4u * lane;
  uint16_t* win = reinterpret_cast<uint16_t*>(wreg + col_bytes(cmax));
  const uint32_t win_a = smem_addr(win);
  const uint32_t wcap = 32u * cmax;  // window symbols per round
  const uint64_t units = F.nunits;
  const uint32_t off0 = static_cast<uint32_t>((reinterpret_cast<uintptr_t>(F.out) >> 1) & 7u);
  uint16_t* out_al = F.out - off0;  // 16-byte aligned; virtual index X = output index + off0
  const uint64_t Xn = F.n + off0;

  auto take = [&]() -> uint64_t {
    uint32_t g = 0;
    if (lane == 0) g = atomicAdd(P.ticket, 1u);
    return __shfl_sync(kFull, g, 0);
  };
  uint64_t g = take();
  WarpTileIn<S> nxt;
  if (g < units) fetch_warp_tile<S>(nxt, F, g, lane);
  while (g < units) {
    const WarpTileIn<S> cur = nxt;
    const uint64_t gn = take();
    if (gn < units) fetch_warp_tile<S>(nxt, F, gn, lane);

    // ---- decode: every codeword once, symbols into the lane's column -------
    const uint64_t i = g * 32 + lane;
    uint32_t c = 0, err = 0;
    bool bad = false;
    uint32_t start = 0;
    uint32_t a = col_a, d = 2;  // next column slot; slots alternate +2 / +126 bytes
    auto store = [&](uint32_t v) {
      sts_u16(a, v);
      a += d;
      d = 128u - d;
    };
    auto store_checked = [&](uint32_t v) {
      if (c < cmax) {
        sts_u16(a, v);
        a += d;
        d = 128u - d;
      }
      ++c;
    };
    if (table_ok && (g + 1) * 32 < F.nsub) {
      // every lane's subsequence is followed by another: codewords start
      // anywhere in [gap0, S) and the last one must end at S + gap1
      start = cur.gap0;
      if (start >= S) {
        err |= kErrGap;
      } else if (unchecked) {
        const uint32_t fin = walk<S, E, false>(cur.bits.u, start, S, lut_a, shift, T, lmin, bad,
                                                store);
        const uint32_t used = a - col_a;
        c = ((used >> 7) << 1) | ((used >> 1) & 1u);
        if (fin != S + cur.gap1) err |= kErrGap;
      } else {
        const uint32_t fin = walk<S, E, false>(cur.bits.u, start, S, lut_a, shift, T, lmin, bad,
                                                store_checked);
        if (fin != S + cur.gap1) err |= kErrGap;
      }
    } else if (table_ok && i < F.nsub) {
      // the field's last tile: the last subsequence ends at nbits
      const uint64_t rem = F.nbits - i * S;
      const uint32_t end = rem < S ? static_cast<uint32_t>(rem) : S;
      const uint32_t expect = (i + 1 < F.nsub) ? S + cur.gap1 : static_cast<uint32_t>(rem);
      start = cur.gap0;
      if (start > end || start >= S) {
        err |= kErrGap;
        start = end;
      }
      const uint32_t fin = walk<S, E, true>(cur.bits.u, start, end, lut_a, shift, T, lmin, bad,
                                             store_checked);
      if (fin != expect) err |= kErrGap;
    }
    if (bad) err |= kErrCode;

    // ---- offsets: warp scan, then look-back over tiles ----------------------
    const uint32_t incl = warp_incl_scan(c, lane);
    const uint32_t C = __shfl_sync(kFull, incl, 31);
    const uint32_t o = incl - c;
    const bool overflow = __any_sync(kFull, c > cmax);
    const uint64_t base = lookback_counts(P, g, 0, C, F.err);
    if (lane == 0 && g + 1 == units && base + C != F.n) err |= kErrCount;
    if (lane == 0 && !table_ok && g == 0) err |= kErrTable;

    // ---- write: columns -> window in output order -> global -----------------
    __syncwarp();
    if (!overflow) {
      const uint64_t X0 = base + off0;
      const uint32_t pad = static_cast<uint32_t>(X0 & 7u);
      if (c) {
        const uint32_t x0 = pad + o;       // window index of the lane's first symbol
        const uint32_t par = x0 & 1u;
        const uint32_t sel = par ? 0x5432u : 0x3210u;
        uint32_t src = col_a;
        uint32_t pa = lds_u32(src);
        if (par) sts_u16(win_a + 2 * x0, pa & kMask16);
        const uint32_t nfw = (c - par) >> 1;
        uint32_t dst = win_a + 2 * (x0 + par);
        for (uint32_t m = 0; m < nfw; ++m) {
          src += 128;
          const uint32_t pb = lds_u32(src);
          sts_u32(dst, __byte_perm(pa, pb, sel) & kMask32);
          dst += 4;
          pa = pb;
        }
        if ((c - par) & 1u) sts_u16(win_a + 2 * (x0 + c - 1), (par ? pa >> 16 : pa) & kMask16);
      }
      __syncwarp();
      flush_window(win_a, win, pad, pad + C, X0 - pad, out_al, Xn, lane);
    } else {
      // rounds of wcap symbols; lanes whose column overflowed decode again
      for (uint32_t ws = 0; ws < C; ws += wcap) {
        const uint32_t we = C < ws + wcap ? C : ws + wcap;
        const uint64_t X0 = base + ws + off0;
        const uint32_t pad = static_cast<uint32_t>(X0 & 7u);
        const uint32_t lo = o > ws ? o : ws, hi = o + c < we ? o + c : we;
        if (lo < hi) {
          const uint32_t j0 = lo - o, j1 = hi - o;
          const uint32_t wb = win_a + 2 * (pad + o - ws);  // window address of symbol 0
          if (c <= cmax) {
            for (uint32_t j = j0; j < j1; ++j) {
              const uint32_t v = lds_u16(col_a + (j >> 1) * 128u + (j & 1u) * 2u);
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
            walk<S, E, true>(cur.bits.u, start, end, lut_a, shift, T, lmin, bad2, put);
          }
        }
        __syncwarp();
        flush_window(win_a, win, pad, pad + (we - ws), X0 - pad, out_al, Xn, lane);
        __syncwarp();
      }
    }
    err = __reduce_or_sync(kFull, err);
    if (lane == 0 && err) atomicOr(F.err, err);
    __syncwarp();
    g = gn;
  }
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
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NW * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  uint64_t grid = static_cast<uint64_t>(per_sm) * num_sms;
  if (s.grid && s.grid < grid) grid = s.grid;
  const uint64_t blocks_needed = (p.f0.nunits + NW - 1) / NW;
  if (grid > blocks_needed) grid = blocks_needed;
  if (grid == 0) return cudaSuccess;
  kern<<<static_cast<unsigned>(grid), NW * 32, smem, stream>>>(p);
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_s(const DecodeParams& p, const LaunchShape& s, int num_sms,
                     cudaStream_t stream) {
  switch (s.threads) {
    case 128: return launch_snw<S, 4>(p, s, num_sms, stream);
    case 256: return launch_snw<S, 8>(p, s, num_sms, stream);
    case 512: return launch_snw<S, 16>(p, s, num_sms, stream);
    case 1024: return launch_snw<S, 32>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t warp_decode_smem_bytes(const LaunchShape& s) {
  const size_t lut = dev::lut_bytes(s.lut16 ? dev::Lut::k16 : dev::Lut::k32, s.K);
  size_t b = lut + static_cast<size_t>(s.threads / 32) * warp_bytes(s.cmax);
  b += static_cast<size_t>(s.long_cap) * 2;
  return (b + 15) & ~static_cast<size_t>(15);
}

cudaError_t launch_decode_warp(const DecodeParams& p, const LaunchShape& s, int num_sms,
                               cudaStream_t stream) {
  if (p.cmax != s.cmax || s.cmax < 2 || s.cmax > 512 || (s.cmax & 1u) ||
      p.long_cap != s.long_cap || p.hdr || p.nfields != 1 || !p.unit_state || !p.ticket ||
      !p.abort_flag)
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
