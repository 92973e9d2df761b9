// decode2.cu -- two-phase gap-array decoding: count, then decode and write.
//
// This is the structure of the gap-array decoder in Sec. III-C and Sec. IV-C:
// a "redundant decoding" pass finds how many codewords start in every
// subsequence, a prefix sum turns the counts into output indices (Sec. III-B2
// step 3), and a decode-and-write pass stages each block's symbols in a
// shared-memory window and writes them with coalesced stores (Algorithm 1,
// Sec. IV-B).  On GB300 the passes are persistent, look-back-free kernels:
//
//   k_count   every thread counts the codewords of one subsequence (start from
//             the gap array, bits staged in shared memory, decode-table lookups
//             for the lengths), checks that it ends where the next subsequence
//             starts and stores the count; each tile stores its total.
//   k_scan    one block turns the tile totals of the launch into exclusive
//             tile bases (a device-wide scan over tiles).
//   k_write   the block scans its per-thread counts and every thread decodes
//             its subsequence straight into the window at its output offset
//             (tile base from k_scan); the window is then written out.
//
// Tiles are B subsequences of S bits.  Blocks load the next tile's bits, gap
// entries and counts into registers while they decode the current tile.
#include <cuda_runtime.h>

#include <type_traits>

#include <algorithm>

#include "common.cuh"
#include "decode_common.cuh"
#include "kernels.h"

namespace hd {
namespace {

using namespace dev;

template <int S>
struct CountType {
  using T = uint8_t;  // S <= 128: at most 128 codewords start in a subsequence
};
template <>
struct CountType<256> {
  using T = uint16_t;
};
template <>
struct CountType<512> {
  using T = uint16_t;
};

// Block-wide sum (all B threads); ends with a barrier.
template <int B>
__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* s_warp) {
  constexpr int NW = B / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) s_warp[warp] = v;
  __syncthreads();
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) tot += s_warp[w];
  __syncthreads();
  return tot;
}

// dst[0 .. z) = v (dst 2-byte aligned): 32-bit stores where aligned.
__device__ __forceinline__ void fill_u16(uint16_t* dst, uint32_t z, uint32_t v) {
  uint32_t k = 0;
  if ((reinterpret_cast<uintptr_t>(dst) & 2u) && z) {
    dst[0] = static_cast<uint16_t>(v);
    k = 1;
  }
  const uint32_t v2 = (v & 0xFFFFu) * 0x10001u;
  for (; k + 2 <= z; k += 2) *reinterpret_cast<uint32_t*>(dst + k) = v2;
  if (k < z) dst[k] = static_cast<uint16_t>(v);
}

// What a thread needs of its subsequence of one tile, loaded ahead.
template <int S>
struct TileIn {
  UnitRegs<S> bits;
  uint32_t gap0, gap1;  // gap entries of this and the next subsequence
  uint32_t count;       // k_write: the subsequence's codeword count
  uint64_t base;        // k_write: the tile's first output index (thread 0)
  uint64_t qbase, olo, ohi;  // k_write values: q before the tile, its outliers (thread 0)
};

template <int S, int B, bool WRITE>
__device__ __forceinline__ void fetch_tile(TileIn<S>& in, const DecodeParams& P,
                                           const FieldDesc& F, uint64_t g) {
  using CT = typename CountType<S>::T;
  const uint64_t i = (g - F.unit_begin) * B + threadIdx.x;
  if (i < F.nsub) {
    fetch_units<S>(in.bits, F, i);
    in.gap0 = __ldg(F.gap + i * F.gap_stride);
    in.gap1 = (i + 1 < F.nsub) ? __ldg(F.gap + (i + 1) * F.gap_stride) : 0u;
    if (WRITE) in.count = reinterpret_cast<const CT*>(P.counts)[F.count_begin + i];
  }
  if (WRITE && threadIdx.x == 0) {
    in.base = P.tile_base[g] - P.tile_base[F.unit_begin];
    if (P.vout) {
      in.qbase = P.tile_qbase[g];
      in.olo = P.tile_obase[g];
      in.ohi = P.tile_obase[g + 1];
    }
  }
}

// Register caps that keep 4 blocks of 256 threads per SM.
template <int B>
__host__ __device__ constexpr int count_min_blocks() {
  return 1024 / B;
}
template <int B>
__host__ __device__ constexpr int write_min_blocks() {
  return 1024 / B;
}

// E = uint8_t: lengths only (8-bit table; with RUNS also the run table, for
// fields of short codes).  E = uint16_t / uint32_t: the symbols too (the
// decode-and-write kernel's table), and each tile's residue sum for decode +
// reconstruction.
template <int S, int B, class E, bool RUNS = false>
__global__ void __launch_bounds__(B, count_min_blocks<B>())
    k_count(const __grid_constant__ DecodeParams P) {
  using CT = typename CountType<S>::T;
  constexpr bool kSums = sizeof(E) > 1;
  constexpr Lut kKind =
      sizeof(E) == 1 ? (RUNS ? Lut::k8r : Lut::k8) : (sizeof(E) == 2 ? Lut::k16 : Lut::k32);
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* s_lut = smem;  // first-level table
  uint32_t* s_bits = reinterpret_cast<uint32_t*>(smem + lut_bytes(kKind, P.K));
  __shared__ uint64_t s_end[34];
  __shared__ uint32_t s_base[34];
  __shared__ uint32_t s_meta[3];
  __shared__ uint32_t s_warp[B / 32];
  __shared__ uint32_t s_lmin;

  const int t = threadIdx.x;
  uint32_t* col = s_bits + t;
  uint32_t cur_field = 0xffffffffu;
  const LaunchSize LS = launch_size(P);
  uint64_t g = LS.lo + blockIdx.x;
  TileIn<S> nxt;
  uint32_t nfi = 0;
  if (g < LS.units) {
    nfi = find_field(P, LS, g);
    fetch_tile<S, B, false>(nxt, P, field_of(P, LS, nfi), g);
  }
  for (; g < LS.units; g += gridDim.x) {
    const uint32_t fi = nfi;
    const FieldDesc& F = field_of(P, LS, fi);
    // this tile's bits go to shared memory (each thread touches only its own
    // column), then the registers take the next tile's loads
    const uint64_t i = (g - F.unit_begin) * B + t;
    if (i < F.nsub) put_units<S>(col, nxt.bits, B);
    const uint32_t gap0 = nxt.gap0, gap1 = nxt.gap1;
    const uint64_t gn = g + gridDim.x;
    if (gn < LS.units) {
      nfi = find_field(P, LS, gn);
      fetch_tile<S, B, false>(nxt, P, field_of(P, LS, nfi), gn);
    }
    if (fi != cur_field) {
      __syncthreads();
      load_table(F.table, P.K, F.alphabet, kKind, s_lut, s_end, s_base, s_meta, B);
      if (t == 0) s_lmin = F.table->minlen;
      cur_field = fi;
      __syncthreads();
    }
    const Tables T = make_tables(F, P.K, s_lut, s_end, s_base, s_meta, nullptr, 0);
    const bool table_ok = s_meta[1] == 0;
    const uint64_t tl = g - F.unit_begin;
    uint32_t c = 0, err = 0, ssum = 0;
    if (table_ok && i < F.nsub) {
      const uint64_t rem = F.nbits - i * S;
      const uint32_t end = rem < S ? static_cast<uint32_t>(rem) : S;
      uint32_t p = gap0;
      const uint32_t expect = (i + 1 < F.nsub) ? S + gap1 : static_cast<uint32_t>(rem);
      if (p > end || p >= S) {
        err |= kErrGap;
        p = end;
      }
      bool bad = false;
      const uint8_t* run8 = s_lut + (1u << P.K);
      const bool zr = RUNS && P.zero_runs && s_lmin == 1;
      while (p < end) {
        if constexpr (kSums) {
          uint32_t sym;
          p += code_sym_t<E>(T, peek<B>(col, p), sym, bad);
          ssum += sym;
          ++c;
        } else if constexpr (RUNS) {
          // several short codes per lookup when they all start before `end`
          const uint32_t w = peek<B>(col, p);
          const uint32_t r = run8[w >> T.shift];
          if (zr && !(w >> 31)) {
            // a run of the 1-bit code 0: as many codes as zero bits, up to
            // the end of the subsequence
            uint32_t z = w ? __clz(w) : 32u;
            z = min(z, end - p);
            p += z;
            c += z;
          } else if (r && p + (r & 15u) <= end) {
            p += r & 15u;
            c += r >> 4;
          } else {
            p += code_len8(T, w, bad);
            ++c;
          }
        } else {
          p += code_len8(T, peek<B>(col, p), bad);
          ++c;
        }
      }
      if (bad) err |= kErrCode;
      else if (p != expect) err |= kErrGap;
      reinterpret_cast<CT*>(P.counts)[F.count_begin + i] = static_cast<CT>(c);
    }
    if (err) atomicOr(F.err, err);
    if (t == 0 && !table_ok && tl == 0) atomicOr(F.err, kErrTable);
    const uint32_t C = block_sum<B>(c, s_warp);
    if (t == 0) P.tile_total[g] = C;
    if constexpr (kSums) {
      const uint32_t Ssum = block_sum<B>(ssum, s_warp);
      if (t == 0) P.tile_rsum[g] = Ssum - C * static_cast<uint32_t>(P.radius);
    }
  }
}

// One block: tile_base[g] = sum of tile_total[j] for j < g over the tiles of
// the launch (g in [unit_lo, units]; a range that starts later continues from
// tile_base[unit_lo]).
__global__ void __launch_bounds__(kScanThreads) k_scan(const __grid_constant__ DecodeParams P) {
  const LaunchSize LS = launch_size(P);
  scan_totals(P.tile_total, P.tile_base, LS.lo, LS.units, P.scan_end);
  if (P.tile_rsum) {
    __syncthreads();
    scan_totals(P.tile_rsum, P.tile_qbase, LS.lo, LS.units, nullptr);
  }
}

// Decode + reconstruction: each tile's first outlier, and the outliers'
// corrections (stored residue + radius for each code 0 counted as -radius)
// added to the q before the tile (g up to the launch's end).
__global__ void k_tile_outliers(const __grid_constant__ DecodeParams P) {
  const LaunchSize LS = launch_size(P);
  for (uint64_t g = LS.lo + blockIdx.x * 256ull + threadIdx.x; g <= LS.units;
       g += static_cast<uint64_t>(gridDim.x) * 256) {
    const uint64_t at = P.tile_base[g];
    uint64_t lo = 0, hi = P.n_out;
    while (lo < hi) {
      const uint64_t mid = (lo + hi) >> 1;
      if (P.out_idx[mid] < at)
        lo = mid + 1;
      else
        hi = mid;
    }
    P.tile_obase[g] = lo;
    P.tile_qbase[g] += static_cast<uint32_t>(P.out_corr[lo]);
  }
}

template <int S, int B, class E, bool VALUES>
__global__ void __launch_bounds__(B, write_min_blocks<B>())
    k_write(const __grid_constant__ DecodeParams P) {
  constexpr int W = S / 32 + 1;
  constexpr bool kPairs = std::is_same_v<E, PairEntry>;
  constexpr Lut kKind = kPairs ? Lut::kPair : sizeof(E) == 2 ? Lut::k16 : Lut::k32;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* s_lut = smem;
  uint32_t* s_bits = reinterpret_cast<uint32_t*>(smem + lut_bytes(kKind, P.K));
  uint16_t* s_out = reinterpret_cast<uint16_t*>(s_bits + W * B);  // window + 16
  uint16_t* s_long = s_out + P.window + 16;
  __shared__ uint64_t s_end[34];
  __shared__ uint32_t s_base[34];
  __shared__ uint32_t s_meta[3];
  __shared__ uint32_t s_warp[B / 32];
  __shared__ uint64_t s_tile_base;
  __shared__ uint32_t s_flush_end;
  __shared__ uint64_t s_vtile[3];  // values: q before the tile, its outlier range
  __shared__ int32_t s_vw[2 * 32];
  __shared__ uint32_t s_lmin, s_sym0;  // shortest code length, symbol of the first code

  const int t = threadIdx.x;
  uint32_t* col = s_bits + t;
  uint32_t cur_field = 0xffffffffu;
  const LaunchSize LS = launch_size(P);
  // the tiles come from a list when one is given (CR-class launches)
  auto tile_of = [&](uint64_t v) -> uint64_t { return P.tile_list ? P.tile_list[v] : v; };
  uint64_t u = LS.lo + blockIdx.x;
  uint64_t g_next = 0;
  TileIn<S> nxt;
  uint32_t nfi = 0;
  if (u < LS.units) {
    g_next = tile_of(u);
    nfi = find_field(P, LS, g_next);
    fetch_tile<S, B, true>(nxt, P, field_of(P, LS, nfi), g_next);
  }
  for (; u < LS.units; u += gridDim.x) {
    const uint64_t g = g_next;
    const uint32_t fi = nfi;
    const FieldDesc& F = field_of(P, LS, fi);
    const uint64_t i = (g - F.unit_begin) * B + t;
    if (i < F.nsub) put_units<S>(col, nxt.bits, B);
    const uint32_t gap0 = nxt.gap0, count0 = nxt.count;
    if (t == 0) {
      s_tile_base = nxt.base;
      if (VALUES) {
        s_vtile[0] = nxt.qbase;
        s_vtile[1] = nxt.olo;
        s_vtile[2] = nxt.ohi;
      }
    }
    const uint64_t un = u + gridDim.x;
    if (un < LS.units) {
      g_next = tile_of(un);
      nfi = find_field(P, LS, g_next);
      fetch_tile<S, B, true>(nxt, P, field_of(P, LS, nfi), g_next);
    }
    if (fi != cur_field) {
      __syncthreads();
      load_table(F.table, P.K, F.alphabet, kKind, s_lut, s_end, s_base, s_meta, B, s_long,
                 P.long_cap);
      if (t == 0) {
        s_lmin = F.table->minlen;
        s_sym0 = reinterpret_cast<const uint16_t*>(reinterpret_cast<const char*>(F.table) +
                                                   table_sorted_off(P.K))[0];
      }
      cur_field = fi;
      __syncthreads();
    }
    const Tables T = make_tables(F, P.K, s_lut, s_end, s_base, s_meta, s_long, P.long_cap);
    const bool table_ok = s_meta[1] == 0;
    const uint64_t tl = g - F.unit_begin;
    const bool valid = table_ok && i < F.nsub;
    uint32_t c = 0, gp = 0;
    if (valid) {
      c = count0;
      gp = min(gap0, static_cast<uint32_t>(S));
    }
    uint32_t C;
    const uint32_t o = block_excl_scan<B>(c, s_warp, &C);
    const uint64_t base = s_tile_base;
    if (t == 0 && tl + 1 == F.nunits && base + C != F.n) atomicOr(F.err, kErrCount);
    const bool zr = P.zero_runs && s_lmin == 1;
    const uint32_t sym0 = s_sym0;
    // codes out: the window is pre-filled with the 1-bit code's symbol, so
    // its runs need no stores (values: every position is written)
    const bool prefilled = zr && !VALUES;
    auto decode = [&](uint16_t* dst) {
                      uint32_t p = gp;
                      bool bad = false;
                      uint32_t j = 0;
                      if (zr) {
                        // runs of the 1-bit code 0 go out whole, the other
                        // codes one lookup each
                        while (j < c) {
                          const uint32_t w = peek<B>(col, p);
                          if (!(w >> 31)) {
                            uint32_t z = w ? __clz(w) : 32u;
                            z = min(z, c - j);
                            if (!prefilled) fill_u16(dst + j, z, sym0);
                            j += z;
                            p += z;
                          } else {
                            uint32_t s0;
                            p += code_sym_t<E>(T, w, s0, bad);
                            dst[j++] = static_cast<uint16_t>(s0);
                          }
                        }
                      }
                      if constexpr (kPairs) {
                        // two codes per lookup when both lie within the
                        // first-level bits (the entry's m = 2)
                        const uint32_t* pt = static_cast<const uint32_t*>(T.lut);
                        while (j + 1 < c) {
                          const uint32_t w = peek<B>(col, p);
                          const uint32_t e = pt[w >> T.shift];
                          if ((e >> 30) == 2u) {
                            dst[j] = static_cast<uint16_t>(e & 0x3FFu);
                            dst[j + 1] = static_cast<uint16_t>((e >> 10) & 0x3FFu);
                            p += ((e >> 26) & 15u) + ((e >> 22) & 15u);
                            j += 2;
                          } else {
                            uint32_t s0;
                            p += code_sym_pair(T, w, e, s0, bad);
                            dst[j++] = static_cast<uint16_t>(s0);
                          }
                        }
                      } else {
                        for (; j + 1 < c; j += 2) {
                          uint32_t s0, s1;
                          p += code_sym_t<E>(T, peek<B>(col, p), s0, bad);
                          p += code_sym_t<E>(T, peek<B>(col, p), s1, bad);
                          dst[j] = static_cast<uint16_t>(s0);
                          dst[j + 1] = static_cast<uint16_t>(s1);
                        }
                      }
                      if (j < c) {
                        uint32_t s0;
                        p += code_sym_t<E>(T, peek<B>(col, p), s0, bad);
                        dst[j] = static_cast<uint16_t>(s0);
                      }
                      if (bad) atomicOr(F.err, kErrCode);
                    };
    if (VALUES)
      window_write_values<B>(s_out, &s_flush_end, P.window, o, c, C, base, F.n, P,
                             static_cast<int32_t>(static_cast<uint32_t>(s_vtile[0])),
                             s_vtile[1], s_vtile[2], s_vw, decode);
    else
      window_write<B>(s_out, &s_flush_end, P.window, o, c, C, base, F.out, F.n, decode,
                      prefilled, (sym0 & 0xFFFFu) * 0x10001u);
  }
  if (!VALUES && t == 16) bulk_wait_all();  // the window copies are done
}

// Shared-memory window classes (the per-sequence compression-ratio classes of
// Algorithm 2, Sec. IV-C): tile g goes to class c when its codeword count is
// in (c*unit, (c+1)*unit], the last class taking every larger tile; each
// class keeps an unordered list of its tiles.
__global__ void k_classify(const __grid_constant__ DecodeParams P, uint32_t unit, uint32_t nclass,
                           uint32_t* counts, uint32_t* lists, uint64_t cap) {
  const LaunchSize LS = launch_size(P);
  for (uint64_t g = blockIdx.x * 256ull + threadIdx.x; g < LS.units;
       g += static_cast<uint64_t>(gridDim.x) * 256) {
    const uint32_t sym = P.tile_total[g];
    uint32_t c = sym ? (sym - 1) / unit : 0u;
    if (c >= nclass) c = nclass - 1;
    const uint32_t slot = atomicAdd(counts + c, 1u);
    lists[c * cap + slot] = static_cast<uint32_t>(g);
  }
}

template <class Kern>
cudaError_t launch_persistent(Kern kern, const DecodeParams& p, int B, size_t smem,
                              int num_sms, uint32_t grid_cap, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, B, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  uint64_t grid = static_cast<uint64_t>(per_sm) * num_sms;
  if (grid_cap && grid_cap < grid) grid = grid_cap;
  const uint64_t units = (p.unit_hi ? p.unit_hi : p.total_units) - p.unit_lo;
  if (grid > units) grid = units;
  if (grid == 0) return cudaSuccess;
  kern<<<static_cast<unsigned>(grid), B, smem, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_scan(const DecodeParams& p, cudaStream_t stream) {
  k_scan<<<1, kScanThreads, 0, stream>>>(p);
  return cudaGetLastError();
}

template <int S, int B, bool VALUES = false>
cudaError_t launch_write_sb(const DecodeParams& p, const LaunchShape& s, int num_sms,
                            cudaStream_t stream) {
  if constexpr (S <= 256) {
    if (s.lut16 && (s.runs & kShapePairs))
      return launch_persistent(k_write<S, B, PairEntry, VALUES>, p, B, two_phase_smem_bytes(s),
                               num_sms, s.grid, stream);
  }
  if (s.lut16)
    return launch_persistent(k_write<S, B, uint16_t, VALUES>, p, B, two_phase_smem_bytes(s),
                             num_sms, s.grid, stream);
  return launch_persistent(k_write<S, B, uint32_t, VALUES>, p, B, two_phase_smem_bytes(s),
                           num_sms, s.grid, stream);
}

size_t count_values_smem_bytes(const LaunchShape& s) {
  const size_t W = s.S / 32 + 1;
  const size_t b =
      dev::lut_bytes(s.lut16 ? dev::Lut::k16 : dev::Lut::k32, s.K) + W * s.threads * 4;
  return (b + 15) & ~static_cast<size_t>(15);
}

// Decode + reconstruction: counts and residue sums, the two scans, the
// outlier corrections, then values.
template <int S, int B>
cudaError_t launch_values_sb(const DecodeParams& p, const LaunchShape& s, int num_sms,
                             cudaStream_t stream) {
  cudaError_t e =
      s.lut16 ? launch_persistent(k_count<S, B, uint16_t>, p, B, count_values_smem_bytes(s),
                                  num_sms, s.grid, stream)
              : launch_persistent(k_count<S, B, uint32_t>, p, B, count_values_smem_bytes(s),
                                  num_sms, s.grid, stream);
  if (e != cudaSuccess) return e;
  e = launch_scan(p, stream);
  if (e != cudaSuccess) return e;
  const uint64_t units = p.unit_hi ? p.unit_hi : p.total_units;
  const uint64_t blocks = std::min<uint64_t>((units - p.unit_lo + 1 + 255) / 256, 4096);
  k_tile_outliers<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_write_sb<S, B, true>(p, s, num_sms, stream);
}

template <int S>
cudaError_t launch_values_s(const DecodeParams& p, const LaunchShape& s, int num_sms,
                            cudaStream_t stream) {
  switch (s.threads) {
    case 128: return launch_values_sb<S, 128>(p, s, num_sms, stream);
    case 256: return launch_values_sb<S, 256>(p, s, num_sms, stream);
    case 512: return launch_values_sb<S, 512>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <int S, int B>
cudaError_t launch_sb(const DecodeParams& p, const LaunchShape& s, int num_sms,
                      cudaStream_t stream) {
  cudaError_t e = s.runs ? launch_persistent(k_count<S, B, uint8_t, true>, p, B,
                                             count_smem_bytes(s), num_sms, s.grid, stream)
                         : launch_persistent(k_count<S, B, uint8_t, false>, p, B,
                                             count_smem_bytes(s), num_sms, s.grid, stream);
  if (e != cudaSuccess) return e;
  e = launch_scan(p, stream);
  if (e != cudaSuccess) return e;
  return launch_write_sb<S, B>(p, s, num_sms, stream);
}

template <int S>
cudaError_t launch_s(const DecodeParams& p, const LaunchShape& s, int num_sms,
                     cudaStream_t stream) {
  switch (s.threads) {
    case 128: return launch_sb<S, 128>(p, s, num_sms, stream);
    case 256: return launch_sb<S, 256>(p, s, num_sms, stream);
    case 512: return launch_sb<S, 512>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <int S>
cudaError_t launch_write_s(const DecodeParams& p, const LaunchShape& s, int num_sms,
                           cudaStream_t stream) {
  cudaError_t e = launch_scan(p, stream);
  if (e != cudaSuccess) return e;
  switch (s.threads) {
    case 128: return launch_write_sb<S, 128>(p, s, num_sms, stream);
    case 256: return launch_write_sb<S, 256>(p, s, num_sms, stream);
    case 512: return launch_write_sb<S, 512>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t two_phase_smem_bytes(const LaunchShape& s) {
  const size_t W = s.S / 32 + 1;
  const dev::Lut kind = s.lut16 && (s.runs & kShapePairs) && s.S <= 256 ? dev::Lut::kPair
                        : s.lut16                                       ? dev::Lut::k16
                                                                        : dev::Lut::k32;
  size_t b = dev::lut_bytes(kind, s.K) + W * s.threads * 4;
  b += (static_cast<size_t>(s.window) + 16) * 2;
  b += static_cast<size_t>(s.long_cap) * 2;
  return (b + 15) & ~static_cast<size_t>(15);
}

size_t count_smem_bytes(const LaunchShape& s) {
  const size_t W = s.S / 32 + 1;
  const size_t b = dev::lut_bytes(s.runs ? dev::Lut::k8r : dev::Lut::k8, s.K) + W * s.threads * 4;
  return (b + 15) & ~static_cast<size_t>(15);
}

size_t count_bytes_per_subsequence(uint32_t S) { return S > 128 ? 2 : 1; }

cudaError_t launch_decode_two_phase(const DecodeParams& p, const LaunchShape& s, int num_sms,
                                    cudaStream_t stream) {
  if (p.long_cap != s.long_cap || p.window != s.window || s.window < s.S) return cudaErrorInvalidValue;
  switch (s.S) {
    case 64: return launch_s<64>(p, s, num_sms, stream);
    case 128: return launch_s<128>(p, s, num_sms, stream);
    case 256: return launch_s<256>(p, s, num_sms, stream);
    case 512: return launch_s<512>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_decode_values(const DecodeParams& p, const LaunchShape& s, int num_sms,
                                 cudaStream_t stream) {
  if (p.long_cap != s.long_cap || p.window != s.window || s.window < s.S) return cudaErrorInvalidValue;
  if (!p.vout || !p.tile_rsum || !p.tile_qbase || !p.tile_obase || !p.out_corr)
    return cudaErrorInvalidValue;
  switch (s.S) {
    case 64: return launch_values_s<64>(p, s, num_sms, stream);
    case 128: return launch_values_s<128>(p, s, num_sms, stream);
    case 256: return launch_values_s<256>(p, s, num_sms, stream);
    case 512: return launch_values_s<512>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <int S>
cudaError_t launch_count_s(const DecodeParams& p, const LaunchShape& s, int num_sms,
                           cudaStream_t stream) {
  switch (s.threads) {
    case 128: return s.runs ? launch_persistent(k_count<S, 128, uint8_t, true>, p, 128, count_smem_bytes(s), num_sms, s.grid, stream)
                            : launch_persistent(k_count<S, 128, uint8_t, false>, p, 128, count_smem_bytes(s), num_sms, s.grid, stream);
    case 256: return s.runs ? launch_persistent(k_count<S, 256, uint8_t, true>, p, 256, count_smem_bytes(s), num_sms, s.grid, stream)
                            : launch_persistent(k_count<S, 256, uint8_t, false>, p, 256, count_smem_bytes(s), num_sms, s.grid, stream);
    case 512: return s.runs ? launch_persistent(k_count<S, 512, uint8_t, true>, p, 512, count_smem_bytes(s), num_sms, s.grid, stream)
                            : launch_persistent(k_count<S, 512, uint8_t, false>, p, 512, count_smem_bytes(s), num_sms, s.grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <int S>
cudaError_t launch_write_only_s(const DecodeParams& p, const LaunchShape& s, int num_sms,
                                cudaStream_t stream) {
  switch (s.threads) {
    case 128: return launch_write_sb<S, 128>(p, s, num_sms, stream);
    case 256: return launch_write_sb<S, 256>(p, s, num_sms, stream);
    case 512: return launch_write_sb<S, 512>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_phase(const DecodeParams& p, const LaunchShape& s, Phase phase, int num_sms,
                         cudaStream_t stream) {
  if (p.long_cap != s.long_cap || p.window != s.window || s.window < s.S) return cudaErrorInvalidValue;
  if (phase == Phase::kScan) return launch_scan(p, stream);
  const bool count = phase == Phase::kCount;
  switch (s.S) {
    case 64: return count ? launch_count_s<64>(p, s, num_sms, stream) : launch_write_only_s<64>(p, s, num_sms, stream);
    case 128: return count ? launch_count_s<128>(p, s, num_sms, stream) : launch_write_only_s<128>(p, s, num_sms, stream);
    case 256: return count ? launch_count_s<256>(p, s, num_sms, stream) : launch_write_only_s<256>(p, s, num_sms, stream);
    case 512: return count ? launch_count_s<512>(p, s, num_sms, stream) : launch_write_only_s<512>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_classify(const DecodeParams& p, uint32_t unit, uint32_t nclass,
                            uint32_t* counts, uint32_t* lists, uint64_t cap, cudaStream_t stream) {
  const uint64_t units = p.unit_hi ? p.unit_hi : p.total_units;
  if (units == 0) return cudaSuccess;
  const uint64_t blocks = (units + 255) / 256;
  k_classify<<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0, stream>>>(
      p, unit, nclass, counts, lists, cap);
  return cudaGetLastError();
}

cudaError_t launch_write(const DecodeParams& p, const LaunchShape& s, int num_sms,
                         cudaStream_t stream) {
  if (p.long_cap != s.long_cap || p.window != s.window || s.window < s.S) return cudaErrorInvalidValue;
  switch (s.S) {
    case 64: return launch_write_s<64>(p, s, num_sms, stream);
    case 128: return launch_write_s<128>(p, s, num_sms, stream);
    case 256: return launch_write_s<256>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hd
