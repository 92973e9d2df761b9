// decode.cu -- single-pass gap-array decode kernel: one persistent launch
// decodes a field without any per-subsequence buffer in global memory.  It
// serves hd_decode_static, whose scratch is a fixed device array too small
// for the count arrays of the two-phase decoder that the context entry points
// use; its only global scratch is one look-back state per tile.
//
// Geometry.  A subsequence is S bits (one thread); a tile is B subsequences
// (one block pass).  Tiles are handed out in order through an atomic ticket;
// a tile's output offset comes from a decoupled look-back over tiles whose
// warp reads 256 predecessor states per round trip.
//
// Per tile:
//   1. stage the tile's units in shared memory (one vector load per thread,
//      stored transposed so a warp's lanes always hit distinct banks);
//   2. start = i*S + gap[i] (Sec. III-C); decode the subsequence once into a
//      per-thread column of a shared-memory scratch (threads with more
//      codewords than the column holds decode again at step 5);
//   3. block scan of the codeword counts (Sec. III-B2 step 3);
//   4. look-back across tiles for the tile's first output index;
//   5. copy the symbols into the shared-memory window in output order and
//      write it out with coalesced 16-byte stores (Algorithm 1, Sec. IV-B).
#include <cuda_runtime.h>

#include "common.cuh"
#include "decode_common.cuh"
#include "kernels.h"

namespace hd {
namespace {

using namespace dev;

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

template <int S, int B>
__global__ void __launch_bounds__(B) k_decode(const __grid_constant__ DecodeParams P) {
  constexpr int W = S / 32 + 1;
  constexpr int NW = B / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_lut = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_bits = s_lut + (1u << P.K);
  uint16_t* s_out = reinterpret_cast<uint16_t*>(s_bits + W * B);  // window + 16
  uint16_t* s_scr = s_out + P.window + 16;                          // [cmax][B]
  uint16_t* s_long = s_scr + P.cmax * B;                            // [long_cap]

  __shared__ uint64_t s_end[34];
  __shared__ uint32_t s_base[34];
  __shared__ uint32_t s_meta[3];
  __shared__ uint32_t s_warp[NW];
  __shared__ uint64_t s_tile_base;
  __shared__ uint32_t s_ticket;
  __shared__ uint32_t s_field;

  const int t = threadIdx.x;
  const int warp = t >> 5;
  const uint32_t cmax = P.cmax;
  uint32_t cur_field = 0xffffffffu;
  uint32_t* col = s_bits + t;
  uint16_t* scr = s_scr + t;
  const LaunchSize LS = launch_size(P);

  for (;;) {
    if (t == 0) {
      const uint32_t g = atomicAdd(P.ticket, 1u);
      s_ticket = g;
      s_field = g < LS.units ? find_field(P, LS, g) : 0u;
    }
    __syncthreads();
    const uint64_t g = s_ticket;
    if (g >= LS.units) break;
    const uint32_t fi = s_field;
    const FieldDesc& F = field_of(P, LS, fi);
    if (fi != cur_field) {
      load_table(F.table, P.K, F.alphabet, Lut::k32, s_lut, s_end, s_base, s_meta, B, s_long,
                 P.long_cap);
      cur_field = fi;
      __syncthreads();
    }
    const Tables T = make_tables(F, P.K, s_lut, s_end, s_base, s_meta, s_long, P.long_cap);
    const bool table_ok = s_meta[1] == 0;

    const uint64_t tl = g - F.unit_begin;
    const uint64_t i = tl * B + t;
    const bool valid = table_ok && i < F.nsub;

    // ---- start, count, symbols into the scratch ---------------------------
    uint32_t s = 0, c = 0;
    bool scr_ok = false;
    if (valid) {
      stage_units<S>(col, F, i, B);
      const uint64_t rem = F.nbits - i * S;
      const uint32_t end = rem < S ? static_cast<uint32_t>(rem) : S;
      uint32_t err = 0;
      uint32_t gp = F.gap[i * F.gap_stride];
      const uint32_t expect =
          (i + 1 < F.nsub) ? S + F.gap[(i + 1) * F.gap_stride] : static_cast<uint32_t>(rem);
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
      if (err) atomicOr(F.err, err);
    }

    // ---- output offsets ----------------------------------------------------
    uint32_t C;
    const uint32_t o = block_excl_scan<B>(c, s_warp, &C);
    if (warp == 0) {
      const uint64_t excl = lookback_counts(P, g, F.unit_begin, C, F.err);
      if (t == 0) s_tile_base = excl;
    }
    __syncthreads();
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

template <int S, int B>
cudaError_t launch_t(const DecodeParams& p, const LaunchShape& s, int num_sms,
                     cudaStream_t stream) {
  const size_t smem = decode_smem_bytes(s);
  auto kern = k_decode<S, B>;
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

template <int S>
cudaError_t launch_s(const DecodeParams& p, const LaunchShape& s, int num_sms,
                     cudaStream_t stream) {
  switch (s.threads) {
    case 128: return launch_t<S, 128>(p, s, num_sms, stream);
    case 256: return launch_t<S, 256>(p, s, num_sms, stream);
    case 512: return launch_t<S, 512>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t decode_smem_bytes(const LaunchShape& s) {
  const size_t W = s.S / 32 + 1;
  size_t b = (static_cast<size_t>(1) << s.K) * 4 + W * s.threads * 4;
  b += (static_cast<size_t>(s.window) + 16) * 2;
  b += static_cast<size_t>(s.cmax) * s.threads * 2;
  b += static_cast<size_t>(s.long_cap) * 2;
  return (b + 15) & ~static_cast<size_t>(15);
}

cudaError_t launch_decode_single_pass(const DecodeParams& p, const LaunchShape& s, int num_sms,
                                      cudaStream_t stream) {
  if (p.cmax != s.cmax || s.cmax > s.S || p.long_cap != s.long_cap) return cudaErrorInvalidValue;
  switch (s.S) {
    case 64: return launch_s<64>(p, s, num_sms, stream);
    case 128: return launch_s<128>(p, s, num_sms, stream);
    case 256: return launch_s<256>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hd
