// sync.cu -- self-synchronisation (Sec. III-B, with the early exit of
// Sec. IV-A): finds the first codeword of every subsequence from the bitstream
// alone, and counts the codewords of each subsequence on the way.
//
//   k_guess one thread per tile guesses where the tile's first codeword
//           starts by decoding from kLeadBits before the tile's first bit (an
//           arbitrary position) up to that bit.
//   k_sync  one tile (B subsequences of S bits) per block pass, no waiting on
//           other tiles.  Every thread but the first (which takes the tile's
//           guess) first decodes, without writing, the whole preceding
//           subsequence from its nominal start up to its own first bit: Huffman
//           codes re-synchronise within a few codewords, so that lead-in
//           almost always lands on the true boundary, which becomes the
//           thread's start.  It then decodes
//           its own subsequence and stops past its end.  Then, in rounds, a
//           thread whose start differs from its
//           predecessor's stop walks the new and the old path side by side
//           until they meet at a common codeword boundary -- from there on
//           both coincide, so the old stop and count stay valid.  Rounds run
//           inside each warp first (shuffles, no block barrier) and then across
//           warp boundaries; they end when no start changes.  The kernel writes each
//           subsequence's start (as a gap entry) and codeword count, the
//           tile's count, and the tile's assumed start and final stop offsets.
//   k_fix   one block per field checks, in order, that every tile's assumed
//           start equals its predecessor's stop; a tile where it does not (the
//           guess was wrong) is synchronised again from the true start, which
//           may change its stop and so the next check.  With Huffman codes
//           this is rare, but streams that never re-synchronise (e.g. equal
//           length codes) are fixed tile by tile and still come out right.
//
// The gap entries and counts then feed the decode-and-write kernel.
#include <cuda_runtime.h>

#include "common.cuh"
#include "decode_common.cuh"
#include "kernels.h"

namespace hd {
namespace {

using namespace dev;

template <int S>
struct CountT {
  using T = uint8_t;
};
template <>
struct CountT<256> {
  using T = uint16_t;
};


// Decodes codewords (lengths only) from p while p < end; returns the stop.
// When the codebook has a 1-bit code (canonically the bit 0, every other code
// starting with 1), z zero bits at a codeword boundary are z such codes, taken
// with one leading-zero count: the same stop and count as one code at a time.
template <int STRIDE>
__device__ __forceinline__ uint32_t walk(const Tables& T, const uint32_t* col, uint32_t p,
                                         uint32_t end, uint32_t& c) {
  bool bad = false;
  if (T.end[1] != 0) {
    while (p < end) {
      const uint32_t w = peek<STRIDE>(col, p);
      if (!(w >> 31)) {
        uint32_t z = w ? __clz(w) : 32u;
        z = min(z, end - p);
        p += z;
        c += z;
      } else {
        p += code_len8(T, w, bad);
        ++c;
      }
    }
    return p;
  }
  while (p < end) {
    p += code_len8(T, peek<STRIDE>(col, p), bad);
    ++c;
  }
  return p;
}

// Replaces the path from s (stop e, count c) by the path from ns: the two are
// walked side by side until they share a codeword boundary.
template <int STRIDE>
__device__ __forceinline__ void repath(const Tables& T, const uint32_t* col, uint32_t end,
                                       uint32_t ns, uint32_t& s, uint32_t& e, uint32_t& c) {
  uint32_t a = ns, b = s, ca = 0, cb = 0;
  bool met = false, bad = false;
  for (;;) {
    if (a == b) {
      met = true;
      break;
    }
    if (a >= end && b >= end) break;
    if (a < b) {
      a += code_len8(T, peek<STRIDE>(col, a), bad);
      ++ca;
    } else {
      b += code_len8(T, peek<STRIDE>(col, b), bad);
      ++cb;
    }
  }
  if (met) {
    c = ca + (c - cb);
  } else {
    c = ca;
    e = a;
  }
  s = ns;
}

// Rounds inside one warp: lane l > 0 takes lane l-1's stop as its start
// until no start changes (lane 0 keeps its start).  Returns false if the
// round cap was hit.
template <int S, int B>
__device__ __forceinline__ bool warp_rounds(const Tables& T, const uint32_t* col, bool valid,
                                            uint32_t end, uint32_t& s, uint32_t& e,
                                            uint32_t& c) {
  const int lane = threadIdx.x & 31;
  for (int round = 0;; ++round) {
    const uint32_t e_prev = __shfl_up_sync(0xffffffffu, e, 1);
    const uint32_t ns = (valid && lane) ? e_prev - S : s;
    const bool changed = ns != s;
    if (!__any_sync(0xffffffffu, changed)) return true;
    if (round > 33) return false;
    if (changed) repath<B>(T, col, end, ns, s, e, c);
  }
}

// Synchronisation over one tile (every thread of the block calls it): rounds
// inside every warp, then rounds over warp boundaries -- lane 0 of warp w takes
// the stop of warp w-1's last lane (warp 0's lane 0 takes e_pred - S) and, if
// that changed its start, its warp runs its inner rounds again.  Returns false
// if a round cap was hit.
template <int S, int B>
__device__ __forceinline__ bool sync_rounds(const Tables& T, const uint32_t* col, bool valid,
                                            uint32_t end, uint32_t e_pred, uint32_t& s,
                                            uint32_t& e, uint32_t& c, uint32_t* s_e_last) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  bool ok = warp_rounds<S, B>(T, col, valid, end, s, e, c);
  for (uint32_t round = 0;; ++round) {
    if (lane == 31) s_e_last[warp] = e;
    __syncthreads();
    bool changed = false;
    if (lane == 0 && valid) {
      const uint32_t ns = (warp ? s_e_last[warp - 1] : e_pred) - S;
      changed = ns != s;
      if (changed) repath<B>(T, col, end, ns, s, e, c);
    }
    const bool any = __syncthreads_or(changed) != 0;
    if (!any) return ok;
    if (round > B / 32 + 1) return false;
    if (__any_sync(0xffffffffu, changed)) ok &= warp_rounds<S, B>(T, col, valid, end, s, e, c);
  }
}

// Bits the guess kernel decodes before each tile's first bit.
constexpr uint32_t kLeadBits = 1024;
constexpr int kGuessThreads = 128;

// One thread per tile: where does the tile's first codeword start?  The
// thread decodes (lengths only) from kLeadBits before the tile's first bit --
// an arbitrary position -- up to that bit; Huffman codes re-synchronise within
// a few codewords, so the walk almost always ends on the true boundary.  A
// wrong guess only costs time: the link-fix kernel re-synchronises such a
// tile from its true start.  The lead-in bits are staged in shared memory
// (one column per thread), the length table is read through the L1 cache
// (the tiles of one block may belong to different fields).
template <int B>
__global__ void __launch_bounds__(kGuessThreads) k_guess(const __grid_constant__ DecodeParams P,
                                                         uint32_t S) {
  constexpr int kWords = kLeadBits / 32 + 1;
  __shared__ uint32_t s_lead[kWords * kGuessThreads];
  const LaunchSize LS = launch_size(P);
  const int t = threadIdx.x;
  uint32_t* col = s_lead + t;
  for (uint64_t g0 = static_cast<uint64_t>(blockIdx.x) * kGuessThreads; g0 < LS.units;
       g0 += static_cast<uint64_t>(gridDim.x) * kGuessThreads) {
    const uint64_t g = g0 + t;
    uint64_t tl = 0;
    const FieldDesc* Fp = nullptr;
    uint32_t first = 0;  // first staged bit relative to the lead-in start
    if (g < LS.units) {
      Fp = &field_of(P, LS, find_field(P, LS, g));
      tl = g - Fp->unit_begin;
      if (tl > 0 && Fp->table->status == 0) {
        const uint64_t target = tl * B * S;  // a multiple of 32
        const uint64_t w0 = target >= kLeadBits ? target / 32 - kLeadBits / 32 : 0;
        first = static_cast<uint32_t>(target - 32 * w0);
        for (int k = 0; k < kWords; ++k)
          col[k * kGuessThreads] = w0 + k < Fp->nwords ? __ldg(Fp->words + w0 + k) : 0u;
      }
    }
    __syncwarp();
    if (g < LS.units) {
      uint32_t guess = 0;
      if (tl > 0 && Fp->table->status == 0) {
        const TableHeader* H = Fp->table;
        const uint8_t* len8 =
            reinterpret_cast<const uint8_t*>(H) + table_len8_off(P.K, Fp->alphabet);
        const uint32_t shift = 32u - P.K, maxlen = H->maxlen;
        const bool zr = H->end[1] != 0;  // a 1-bit code: runs of zero bits (see walk)
        uint32_t pos = 0;
        while (pos < first) {
          const uint32_t w = peek<kGuessThreads>(col, pos);
          if (zr && !(w >> 31)) {
            const uint32_t z = w ? __clz(w) : 32u;
            pos += min(z, first - pos);
            continue;
          }
          uint32_t L = __ldg(len8 + (w >> shift));
          if (L & kLen8Walk) {
            L &= 0x7Fu;
            while (L <= maxlen && static_cast<uint64_t>(w) >= H->end[L]) ++L;
            if (L > maxlen) L = 1;  // no codeword here: move on by one bit
          }
          pos += L;
        }
        guess = pos - first;
      }
      P.tile_guess[g] = static_cast<uint8_t>(guess);
    }
    __syncwarp();
  }
}

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

struct SyncShared {
  uint32_t* s_warp;
  uint32_t* s_e_last;
  uint32_t* s_x;  // [2]: broadcast slots
};

// Synchronises tile tl of field F given its first start a0 (guessed, or known
// to be true), writes the tile's gap entries, counts and totals, and returns
// the start it used.  tile_flag[g] records whether the field's last
// subsequence ran past nbits; hitting the round cap sets kErrNoSync.
template <int S, int B>
__device__ __forceinline__ uint32_t sync_tile(const DecodeParams& P, const FieldDesc& F,
                                              const Tables& T, bool table_ok, uint64_t g,
                                              uint32_t a0, uint32_t* s_bits,
                                              const SyncShared& sh) {
  using CT = typename CountT<S>::T;
  const int t = threadIdx.x;
  uint32_t* col = s_bits + t;
  const uint64_t tl = g - F.unit_begin;
  const uint64_t i = tl * B + t;
  const bool valid = table_ok && i < F.nsub;
  uint32_t end = 0;
  if (valid) {
    stage_units<S>(col, F, i, B);
    const uint64_t rem = F.nbits - i * S;
    end = rem < S ? static_cast<uint32_t>(rem) : S;
  }
  __syncthreads();  // the lead-in reads the previous thread's column
  uint32_t s = 0, e = 0, c = 0;
  if (valid) {
    // decode the preceding subsequence (whose column ends with this
    // subsequence's first unit) from its nominal start up to this
    // subsequence's first bit; its stop is this thread's start
    uint32_t c_lead = 0;
    s = t > 0 ? walk<B>(T, col - 1, 0, S, c_lead) - S : a0;
    e = walk<B>(T, col, s, end, c);
  }
  __syncthreads();
  uint32_t flags = 0;
  if (!sync_rounds<S, B>(T, col, valid, end, S + a0, s, e, c, sh.s_e_last)) flags |= 2u;
  if (valid && i + 1 == F.nsub && e != end) flags |= 1u;
  if (valid) {
    F.gap_out[i] = static_cast<uint8_t>(s);
    reinterpret_cast<CT*>(P.counts)[F.count_begin + i] = static_cast<CT>(c);
  }
  if (t == B - 1) sh.s_x[1] = e - S;
  if (t == 0 && (flags & 2u)) atomicOr(F.err, kErrNoSync);
  const bool overran = __syncthreads_or(flags & 1u) != 0;
  const uint32_t C = block_sum<B>(c, sh.s_warp);
  if (t == 0) {
    P.tile_total[g] = C;
    P.tile_a[g] = static_cast<uint8_t>(a0);
    P.tile_e[g + 1] = static_cast<uint8_t>(sh.s_x[1]);
    P.tile_flag[g] = overran ? 1u : 0u;
  }
  __syncthreads();
  return a0;
}

template <int S, int B>
__global__ void __launch_bounds__(B) k_sync(const __grid_constant__ DecodeParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint8_t* s_lut = smem;  // length table
  uint32_t* s_bits = reinterpret_cast<uint32_t*>(smem + lut_bytes(Lut::k8, P.K));
  __shared__ uint64_t s_end[34];
  __shared__ uint32_t s_base[34];
  __shared__ uint32_t s_meta[3];
  __shared__ uint32_t s_warp[B / 32];
  __shared__ uint32_t s_e_last[B / 32];
  __shared__ uint32_t s_x[2];
  const SyncShared sh{s_warp, s_e_last, s_x};

  uint32_t cur_field = 0xffffffffu;
  const LaunchSize LS = launch_size(P);
  for (uint64_t g = blockIdx.x; g < LS.units; g += gridDim.x) {
    const uint32_t fi = find_field(P, LS, g);
    const FieldDesc& F = field_of(P, LS, fi);
    if (fi != cur_field) {
      __syncthreads();
      load_table(F.table, P.K, F.alphabet, Lut::k8, s_lut, s_end, s_base, s_meta, B);
      cur_field = fi;
      __syncthreads();
    }
    const Tables T = make_tables(F, P.K, s_lut, s_end, s_base, s_meta, nullptr, 0);
    sync_tile<S, B>(P, F, T, s_meta[1] == 0, g, P.tile_guess[g], s_bits, sh);
  }
}

// Smallest tile g in [lo, g1) whose assumed start differs from where its
// predecessor stopped (tile_a[g] != tile_e[g]), or g1.  Reads both arrays as
// 16-byte vectors, B * 16 tiles per round, and stops at the first round that
// finds one.  All threads of the block call it.
template <int B>
__device__ __forceinline__ uint64_t first_broken(const DecodeParams& P, uint64_t lo, uint64_t g1,
                                                 unsigned long long* s_first) {
  const int t = threadIdx.x;
  if (t == 0) *s_first = g1;
  __syncthreads();
  const uint64_t q_end = (g1 + 15) / 16;
  for (uint64_t q0 = lo / 16; q0 < q_end; q0 += B) {
    const uint64_t q = q0 + t;
    uint64_t found = g1;
    if (q < q_end) {
      const uint4 a = *reinterpret_cast<const uint4*>(P.tile_a + 16 * q);
      const uint4 e = *reinterpret_cast<const uint4*>(P.tile_e + 16 * q);
      const uint32_t x[4] = {a.x ^ e.x, a.y ^ e.y, a.z ^ e.z, a.w ^ e.w};
#pragma unroll
      for (int k = 3; k >= 0; --k) {
#pragma unroll
        for (int j = 3; j >= 0; --j) {
          const uint64_t g = 16 * q + 4 * k + j;
          if (((x[k] >> (8 * j)) & 0xFFu) && g >= lo && g < g1) found = g;
        }
      }
      if (found < g1) atomicMin(s_first, static_cast<unsigned long long>(found));
    }
    if (__syncthreads_or(found < g1)) break;
  }
  const uint64_t f = *s_first;
  __syncthreads();
  return f;
}

// One block per field (blocks loop over fields): finds, in order, every tile whose assumed start is not
// where its predecessor stopped and synchronises it again from the true start
// (which can move its own stop, so the scan resumes right after it); then
// checks that the field's last subsequence ended at nbits.
template <int S, int B>
__global__ void __launch_bounds__(B) k_fix(const __grid_constant__ DecodeParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint8_t* s_lut = smem;  // length table
  uint32_t* s_bits = reinterpret_cast<uint32_t*>(smem + lut_bytes(Lut::k8, P.K));
  __shared__ uint64_t s_end[34];
  __shared__ uint32_t s_base[34];
  __shared__ uint32_t s_meta[3];
  __shared__ uint32_t s_warp[B / 32];
  __shared__ uint32_t s_e_last[B / 32];
  __shared__ uint32_t s_x[2];
  __shared__ unsigned long long s_first;
  const SyncShared sh{s_warp, s_e_last, s_x};

  const LaunchSize LS = launch_size(P);
  for (uint32_t fi = blockIdx.x; fi < LS.nfields; fi += gridDim.x) {
    const FieldDesc& F = field_of(P, LS, fi);
    if (F.nunits == 0) continue;
    __syncthreads();  // the previous field's table is no longer read
    load_table(F.table, P.K, F.alphabet, Lut::k8, s_lut, s_end, s_base, s_meta, B);
    __syncthreads();
    const Tables T = make_tables(F, P.K, s_lut, s_end, s_base, s_meta, nullptr, 0);
    const bool table_ok = s_meta[1] == 0;
    const uint64_t g0 = F.unit_begin, g1 = F.unit_begin + F.nunits;
    uint64_t cursor = g0 + 1;
    while (table_ok && cursor < g1) {
      const uint64_t gb = first_broken<B>(P, cursor, g1, &s_first);
      if (gb >= g1) break;
      sync_tile<S, B>(P, F, T, table_ok, gb, P.tile_e[gb], s_bits, sh);
      cursor = gb + 1;
    }
    if (threadIdx.x == 0) {
      if (!table_ok) atomicOr(F.err, kErrTable);
      else if (P.tile_flag[g1 - 1]) atomicOr(F.err, kErrCode);
    }
  }
}

template <int S, int B>
cudaError_t launch_sb(const DecodeParams& p, const LaunchShape& s, int num_sms,
                      cudaStream_t stream) {
  const size_t smem = sync_smem_bytes(s);
  auto ks = k_sync<S, B>;
  auto kf = k_fix<S, B>;
  cudaError_t e =
      cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks, B, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  uint64_t grid = static_cast<uint64_t>(per_sm) * num_sms;
  if (s.grid && s.grid < grid) grid = s.grid;
  if (grid > p.total_units) grid = p.total_units;
  if (grid == 0) return cudaSuccess;
  const uint64_t gblocks = (p.total_units + kGuessThreads - 1) / kGuessThreads;
  k_guess<B><<<static_cast<unsigned>(gblocks < 8192 ? gblocks : 8192), kGuessThreads, 0, stream>>>(
      p, S);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ks<<<static_cast<unsigned>(grid), B, smem, stream>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const uint32_t fix_grid = p.nfields < 1024u ? p.nfields : 1024u;
  if (fix_grid == 0) return cudaSuccess;
  kf<<<fix_grid, B, smem, stream>>>(p);
  return cudaGetLastError();
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

}  // namespace

size_t sync_smem_bytes(const LaunchShape& s) {
  const size_t W = s.S / 32 + 1;
  const size_t b = dev::lut_bytes(dev::Lut::k8, s.K) + W * s.threads * 4;
  return (b + 15) & ~static_cast<size_t>(15);
}

cudaError_t launch_sync(const DecodeParams& p, const LaunchShape& s, int num_sms,
                        cudaStream_t stream) {
  if (p.long_cap != s.long_cap) return cudaErrorInvalidValue;
  switch (s.S) {
    case 64: return launch_s<64>(p, s, num_sms, stream);
    case 128: return launch_s<128>(p, s, num_sms, stream);
    case 256: return launch_s<256>(p, s, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hd
