// decode2.cu -- two-phase gap-array decoding: count, then decode and write.
//
// This is the structure of the gap-array decoder in Sec. III-C and Sec. IV-C:
// a "redundant decoding" pass finds how many codewords start in every
// subsequence, a prefix sum turns the counts into output indices (Sec. III-B2
// step 3), and a decode-and-write pass stages each block's symbols in a
// shared-memory window and writes them with coalesced stores (Algorithm 1,
// Sec. IV-B).  On GB300 both passes are persistent, look-back-free kernels:
//
//   k_count   every thread counts the codewords of one subsequence (start from
//             the gap array, bits staged in shared memory, decode-table lookups
//             for the lengths), checks that it ends where the next subsequence
//             starts, stores the count, and each tile adds its total to a
//             per-tile array and to the total of its 256-tile segment.
//   k_write   a warp sums the segment totals and tile totals before its tile
//             (one parallel round of loads), the block scans the per-thread
//             counts, and every thread decodes its subsequence straight into
//             the window at its output offset; the window is then written out.
//
// Tiles are B subsequences of S bits.
#include <cuda_runtime.h>

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

constexpr int kSegTiles = 256;

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

template <int S, int B>
__global__ void __launch_bounds__(B) k_count(const __grid_constant__ DecodeParams P) {
  using CT = typename CountType<S>::T;
  constexpr int W = S / 32 + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_lut = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_bits = s_lut + (1u << P.K);
  uint16_t* s_long = reinterpret_cast<uint16_t*>(s_bits + W * B);
  __shared__ uint64_t s_end[34];
  __shared__ uint32_t s_base[34];
  __shared__ uint32_t s_meta[3];
  __shared__ uint32_t s_warp[B / 32];

  const int t = threadIdx.x;
  uint32_t* col = s_bits + t;
  uint32_t cur_field = 0xffffffffu;
  const LaunchSize LS = launch_size(P);
  for (uint64_t g = blockIdx.x; g < LS.units; g += gridDim.x) {
    const uint32_t fi = find_field(P, LS, g);
    const FieldDesc& F = field_of(P, LS, fi);
    if (fi != cur_field) {
      __syncthreads();
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
    uint32_t c = 0, err = 0;
    if (table_ok && i < F.nsub) {
      stage_units<S>(col, F, i, B);
      const uint64_t rem = F.nbits - i * S;
      const uint32_t end = rem < S ? static_cast<uint32_t>(rem) : S;
      uint32_t p = F.gap[i * F.gap_stride];
      const uint32_t expect =
          (i + 1 < F.nsub) ? S + F.gap[(i + 1) * F.gap_stride] : static_cast<uint32_t>(rem);
      if (p > end || p >= S) {
        err |= kErrGap;
        p = end;
      }
      bool bad = false;
      while (p < end) {
        p += code_len(T, peek<B>(col, p), bad);
        ++c;
      }
      if (bad) err |= kErrCode;
      else if (p != expect) err |= kErrGap;
      reinterpret_cast<CT*>(P.counts)[F.count_begin + i] = static_cast<CT>(c);
    }
    if (err) atomicOr(F.err, err);
    if (t == 0 && !table_ok && tl == 0) atomicOr(F.err, kErrTable);
    const uint32_t C = block_sum<B>(c, s_warp);
    if (t == 0) {
      P.tile_total[g] = C;
      atomicAdd(reinterpret_cast<unsigned long long*>(P.seg_total + g / kSegTiles),
                static_cast<unsigned long long>(C));
    }
  }
}

// Warp: sum of the counts of tiles [a, b) (all of one field).  Whole 256-tile
// segments inside the range come from the segment totals, the ragged ends
// from the tile totals; every lane issues its loads at once.
__device__ __forceinline__ uint64_t tiles_prefix(const DecodeParams& P, uint64_t a, uint64_t b) {
  const int lane = threadIdx.x & 31;
  uint64_t sum = 0;
  if (b > a) {
    const uint64_t s0 = (a + kSegTiles - 1) / kSegTiles;  // first whole segment
    const uint64_t s1 = b / kSegTiles;                    // end of whole segments
    if (s0 < s1) {
      for (uint64_t j = a + lane; j < s0 * kSegTiles; j += 32) sum += P.tile_total[j];
      for (uint64_t s = s0 + lane; s < s1; s += 32) sum += P.seg_total[s];
      for (uint64_t j = s1 * kSegTiles + lane; j < b; j += 32) sum += P.tile_total[j];
    } else {
      for (uint64_t j = a + lane; j < b; j += 32) sum += P.tile_total[j];
    }
  }
  return warp_sum_u64(sum);
}

template <int S, int B>
__global__ void __launch_bounds__(B) k_write(const __grid_constant__ DecodeParams P) {
  using CT = typename CountType<S>::T;
  constexpr int W = S / 32 + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_lut = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_bits = s_lut + (1u << P.K);
  uint16_t* s_out = reinterpret_cast<uint16_t*>(s_bits + W * B);  // window + 16
  uint16_t* s_long = s_out + P.window + 16;
  __shared__ uint64_t s_end[34];
  __shared__ uint32_t s_base[34];
  __shared__ uint32_t s_meta[3];
  __shared__ uint32_t s_warp[B / 32];
  __shared__ uint64_t s_tile_base;
  __shared__ uint32_t s_flush_end;

  const int t = threadIdx.x;
  const int warp = t >> 5;
  uint32_t* col = s_bits + t;
  uint32_t cur_field = 0xffffffffu;
  const LaunchSize LS = launch_size(P);
  for (uint64_t g = blockIdx.x; g < LS.units; g += gridDim.x) {
    const uint32_t fi = find_field(P, LS, g);
    const FieldDesc& F = field_of(P, LS, fi);
    if (fi != cur_field) {
      __syncthreads();
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
    uint32_t c = 0, gp = 0;
    if (warp == 0) {
      const uint64_t base = tiles_prefix(P, F.unit_begin, g);
      if (t == 0) s_tile_base = base;
    }
    if (valid) {
      c = reinterpret_cast<const CT*>(P.counts)[F.count_begin + i];
      gp = min(static_cast<uint32_t>(F.gap[i * F.gap_stride]), static_cast<uint32_t>(S));
      stage_units<S>(col, F, i, B);
    }
    uint32_t C;
    const uint32_t o = block_excl_scan<B>(c, s_warp, &C);
    const uint64_t base = s_tile_base;
    if (t == 0 && tl + 1 == F.nunits && base + C != F.n) atomicOr(F.err, kErrCount);
    window_write<B>(s_out, &s_flush_end, P.window, o, c, C, base, F.out, F.n,
                    [&](uint16_t* dst) {
                      uint32_t p = gp;
                      bool bad = false;
                      for (uint32_t j = 0; j < c; ++j) {
                        uint32_t sym;
                        p += code_sym(T, peek<B>(col, p), sym, bad);
                        dst[j] = static_cast<uint16_t>(sym);
                      }
                      if (bad) atomicOr(F.err, kErrCode);
                    });
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
  if (grid > p.total_units) grid = p.total_units;
  if (grid == 0) return cudaSuccess;
  kern<<<static_cast<unsigned>(grid), B, smem, stream>>>(p);
  return cudaGetLastError();
}

template <int S, int B>
cudaError_t launch_sb(const DecodeParams& p, const LaunchShape& s, int num_sms,
                      cudaStream_t stream) {
  const size_t W = S / 32 + 1;
  const size_t lut = (static_cast<size_t>(1) << s.K) * 4;
  const size_t smem_count = ((lut + W * B * 4 + s.long_cap * 2) + 15) & ~static_cast<size_t>(15);
  cudaError_t e =
      launch_persistent(k_count<S, B>, p, B, smem_count, num_sms, s.grid, stream);
  if (e != cudaSuccess) return e;
  return launch_persistent(k_write<S, B>, p, B, two_phase_smem_bytes(s), num_sms, s.grid,
                           stream);
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
  const size_t smem = two_phase_smem_bytes(s);
  switch (s.threads) {
    case 128: return launch_persistent(k_write<S, 128>, p, 128, smem, num_sms, s.grid, stream);
    case 256: return launch_persistent(k_write<S, 256>, p, 256, smem, num_sms, s.grid, stream);
    case 512: return launch_persistent(k_write<S, 512>, p, 512, smem, num_sms, s.grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t two_phase_smem_bytes(const LaunchShape& s) {
  const size_t W = s.S / 32 + 1;
  size_t b = (static_cast<size_t>(1) << s.K) * 4 + W * s.threads * 4;
  b += (static_cast<size_t>(s.window) + 16) * 2;
  b += static_cast<size_t>(s.long_cap) * 2;
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
