// encode_gpu.cu -- canonical-Huffman encoding on the GPU with gap-array
// emission (the step before the decoder; the gap array is the encoder-side
// output of Sec. III-C).
//
//   k_enc_count  one block per tile of kEncTile symbols: the tile's total code
//                bits (lengths read through the L1 cache); symbols without a
//                code set the error word.
//   (scan)       tile bit offsets = exclusive scan of the tile totals.
//   k_enc_write  one block per tile: a block scan of the threads' bit counts
//                places every thread's codewords; each thread assembles its
//                codewords in a 64-bit register and emits whole words into the
//                tile's words in shared memory (OR for the first and last word,
//                which it may share with its neighbours), which are then stored
//                (the two words a tile may share with its neighbour tiles with
//                atomicOr on the zeroed stream).  The thread that places a codeword starting at or
//                after a subsequence boundary j*S, with the previous codeword
//                starting before it, writes gap[j]; the end of the stream
//                closes the last open subsequence.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "decode_common.cuh"
#include "kernels.h"

namespace hd {
namespace {

using namespace dev;

constexpr int kEncThreads = 256;
constexpr int kEncPer = 16;  // symbols per thread
constexpr int kEncTile = kEncThreads * kEncPer;

// The thread's symbols (consecutive), 0 past n.
__device__ __forceinline__ void load_symbols(const uint16_t* codes, uint64_t n, uint64_t i0,
                                             uint32_t (&x)[kEncPer]) {
  if (i0 + kEncPer <= n && ((reinterpret_cast<uintptr_t>(codes + i0) & 15u) == 0)) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(codes + i0));
    const uint4 b = __ldg(reinterpret_cast<const uint4*>(codes + i0) + 1);
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      x[2 * k] = w[k] & 0xFFFFu;
      x[2 * k + 1] = w[k] >> 16;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kEncPer; ++k) x[k] = i0 + k < n ? __ldg(codes + i0 + k) : 0u;
  }
}

// Shared-memory copies of the code tables for alphabets up to kEncSmemAlphabet.
constexpr uint32_t kEncSmemAlphabet = 4096;

__global__ void __launch_bounds__(kEncThreads) k_enc_count(const __grid_constant__ EncodeParams E) {
  __shared__ uint32_t s_warp[kEncThreads / 32];
  __shared__ uint8_t s_len[kEncSmemAlphabet];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const bool smem_tab = E.alphabet <= kEncSmemAlphabet;
  if (smem_tab)
    for (uint32_t k = t; k < E.alphabet; k += kEncThreads) s_len[k] = E.lengths[k];
  __syncthreads();
  const uint8_t* lens = smem_tab ? s_len : E.lengths;
  const uint32_t amax = E.alphabet - 1;
  for (uint64_t tile = blockIdx.x; tile < E.tiles; tile += gridDim.x) {
    const uint64_t i0 = tile * kEncTile + static_cast<uint64_t>(t) * kEncPer;
    uint32_t x[kEncPer];
    load_symbols(E.codes, E.n, i0, x);
    const uint32_t m = i0 < E.n ? static_cast<uint32_t>(E.n - i0 < kEncPer ? E.n - i0 : kEncPer) : 0u;
    uint32_t bits = 0, xmax = 0, lmin = 32;
#pragma unroll
    for (int k = 0; k < kEncPer; ++k) {
      if (k < static_cast<int>(m)) {
        const uint32_t L = lens[min(x[k], amax)];
        xmax = max(xmax, x[k]);
        lmin = min(lmin, L);
        bits += L;
      }
    }
    if (m && (xmax > amax || lmin == 0)) atomicOr(E.err, 1u);
#pragma unroll
    for (int o = 16; o; o >>= 1) bits += __shfl_xor_sync(0xffffffffu, bits, o);
    if (lane == 0) s_warp[warp] = bits;
    __syncthreads();
    if (t == 0) {
      uint32_t tot = 0;
      for (int w = 0; w < kEncThreads / 32; ++w) tot += s_warp[w];
      E.tile_bits[tile] = tot;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads) k_enc_scan(const __grid_constant__ EncodeParams E) {
  scan_totals(E.tile_bits, E.tile_off, 0, E.tiles, E.total_out);
}

__global__ void __launch_bounds__(kEncThreads) k_enc_write(const __grid_constant__ EncodeParams E) {
  // a tile of kEncTile codewords of at most 32 bits spans at most kEncTile + 1 words
  __shared__ uint32_t s_w[kEncTile + 2];
  __shared__ uint32_t s_warp[kEncThreads / 32];
  __shared__ uint32_t s_cw[kEncSmemAlphabet];
  __shared__ uint8_t s_len[kEncSmemAlphabet];
  const int t = threadIdx.x;
  const uint32_t lgS = 31u - __clz(E.subseq_bits);  // S is a power of two
  const bool smem_tab = E.alphabet <= kEncSmemAlphabet;
  if (smem_tab)
    for (uint32_t k = t; k < E.alphabet; k += kEncThreads) {
      s_len[k] = E.lengths[k];
      s_cw[k] = E.codewords[k];
    }
  __syncthreads();
  const uint8_t* lens = smem_tab ? s_len : E.lengths;
  const uint32_t* cws = smem_tab ? s_cw : E.codewords;
  for (uint64_t tile = blockIdx.x; tile < E.tiles; tile += gridDim.x) {
    const uint64_t base = E.tile_off[tile];
    const uint64_t tile_end = E.tile_off[tile + 1];
    const uint64_t word0 = base >> 5;
    const uint32_t nw = tile_end > base ? static_cast<uint32_t>(((tile_end - 1) >> 5) - word0 + 1) : 0u;
    for (uint32_t k = t; k < nw; k += kEncThreads) s_w[k] = 0;
    const uint64_t i0 = tile * kEncTile + static_cast<uint64_t>(t) * kEncPer;
    uint32_t x[kEncPer];
    load_symbols(E.codes, E.n, i0, x);
    uint32_t len[kEncPer];
    uint32_t bits = 0;
#pragma unroll
    for (int k = 0; k < kEncPer; ++k) {
      len[k] = (i0 + k < E.n && x[k] < E.alphabet) ? lens[x[k]] : 0u;
      bits += len[k];
    }
    uint32_t total;
    const uint32_t excl = block_excl_scan<kEncThreads>(bits, s_warp, &total);
    const uint64_t off0 = base + excl;  // stream position of the thread's first codeword
    if (bits) {
      // assemble the thread's codewords in a 64-bit register, most significant
      // bit first, and emit whole words; the first and the last word may be
      // shared with the neighbouring threads (OR), the others are its own
      uint32_t r = static_cast<uint32_t>(off0 - (word0 << 5));
      uint32_t q = r >> 5;
      uint32_t nacc = r & 31;
      uint64_t acc = 0;
      bool first = true;
#pragma unroll
      for (int k = 0; k < kEncPer; ++k) {
        const uint32_t L = len[k];
        if (L) {
          acc |= static_cast<uint64_t>(cws[x[k]]) << (64 - nacc - L);
          nacc += L;
          if (nacc >= 32) {
            const uint32_t w = static_cast<uint32_t>(acc >> 32);
            if (first) atomicOr(&s_w[q], w);
            else s_w[q] = w;
            first = false;
            ++q;
            acc <<= 32;
            nacc -= 32;
          }
        }
      }
      // a last partial word is shared with the next thread's first one; a
      // range that ends on a word boundary left no partial word
      if (nacc) atomicOr(&s_w[q], static_cast<uint32_t>(acc >> 32));
      if (E.gap) {
        // gap[j] for every subsequence boundary j*S in (previous start, start]
        // of one of this thread's codewords; the end of the stream closes the
        // last subsequence.  Positions are taken relative to the start of the
        // subsequence holding the thread's first codeword (32-bit arithmetic:
        // the thread's codewords span at most 16 * 32 bits).
        const uint64_t j0 = off0 >> lgS;
        const uint64_t sub0 = j0 << lgS;
        const uint64_t nrel = E.nsub > j0 ? E.nsub - j0 : 0;  // subsequences from j0 on
        const uint32_t jmax = nrel < 0xFFFFFFFFull ? static_cast<uint32_t>(nrel) : 0xFFFFFFFFu;
        uint32_t r = static_cast<uint32_t>(off0 - sub0);
        int32_t rprev = INT32_MIN;  // the stream's first codeword opens subsequence 0
        if (i0 > 0) {
          const uint32_t xp = __ldg(E.codes + i0 - 1);
          rprev = static_cast<int32_t>(r) - static_cast<int32_t>(xp < E.alphabet ? lens[xp] : 0u);
        }
        // index of the stream's last codeword among the thread's, if it holds it
        const uint32_t klast =
            E.n > i0 && E.n - i0 <= kEncPer ? static_cast<uint32_t>(E.n - i0 - 1) : 0xFFFFFFFFu;
#pragma unroll
        for (int k = 0; k < kEncPer; ++k) {
          const uint32_t L = len[k];
          if (L) {
            const uint32_t jr = r >> lgS;
            const int32_t b = static_cast<int32_t>(jr << lgS);
            if (b > rprev && jr < jmax)
              E.gap[j0 + jr] = static_cast<uint8_t>(r - static_cast<uint32_t>(b));
            rprev = static_cast<int32_t>(r);
            r += L;
            if (static_cast<uint32_t>(k) == klast) {
              const uint32_t je = (static_cast<uint32_t>(rprev) >> lgS) + 1;
              if (je < jmax && (je << lgS) <= r)
                E.gap[j0 + je] = static_cast<uint8_t>(r - (je << lgS));
            }
          }
        }
      }
    }
    __syncthreads();
    for (uint32_t k = t; k < nw; k += kEncThreads) {
      uint32_t* dst = E.words + word0 + k;
      if (k == 0 || k + 1 == nw) atomicOr(dst, s_w[k]);  // possibly shared with a neighbour
      else *dst = s_w[k];
    }
    __syncthreads();
  }
}

// Symbol histogram: per-block counts in shared memory (alphabets up to
// kHistSmem) or straight global atomics, summed into hist[alphabet].
constexpr uint32_t kHistSmem = 8192;

__global__ void __launch_bounds__(kEncThreads) k_histogram(const uint16_t* codes, uint64_t n,
                                                           uint32_t alphabet,
                                                           unsigned long long* hist,
                                                           uint32_t* err) {
  __shared__ uint32_t s_h[kHistSmem];
  const bool local = alphabet <= kHistSmem;
  if (local)
    for (uint32_t k = threadIdx.x; k < alphabet; k += kEncThreads) s_h[k] = 0;
  __syncthreads();
  bool bad = false;
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(kEncThreads) + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * kEncThreads) {
    const uint32_t x = __ldg(codes + i);
    if (x >= alphabet) {
      bad = true;
    } else if (local) {
      atomicAdd(&s_h[x], 1u);
    } else {
      atomicAdd(hist + x, 1ull);
    }
  }
  if (bad) atomicOr(err, 1u);
  __syncthreads();
  if (local)
    for (uint32_t k = threadIdx.x; k < alphabet; k += kEncThreads)
      if (s_h[k]) atomicAdd(hist + k, static_cast<unsigned long long>(s_h[k]));
}

}  // namespace

cudaError_t launch_histogram(const uint16_t* codes, uint64_t n, uint32_t alphabet,
                             unsigned long long* hist, uint32_t* err, int num_sms,
                             cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  uint64_t grid = (n + kEncThreads * 16ull - 1) / (kEncThreads * 16ull);
  if (grid > 4ull * num_sms) grid = 4ull * num_sms;
  k_histogram<<<static_cast<unsigned>(grid), kEncThreads, 0, stream>>>(codes, n, alphabet, hist,
                                                                      err);
  return cudaGetLastError();
}

uint64_t encode_tiles(uint64_t n) { return (n + kEncTile - 1) / kEncTile; }

cudaError_t launch_encode_count(const EncodeParams& e, int num_sms, cudaStream_t stream) {
  if (e.tiles == 0) return cudaSuccess;
  const uint64_t grid = e.tiles < 8ull * num_sms ? e.tiles : 8ull * num_sms;
  k_enc_count<<<static_cast<unsigned>(grid), kEncThreads, 0, stream>>>(e);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  k_enc_scan<<<1, kScanThreads, 0, stream>>>(e);
  return cudaGetLastError();
}

cudaError_t launch_encode_write(const EncodeParams& e, int num_sms, cudaStream_t stream) {
  if (e.tiles == 0) return cudaSuccess;
  const uint64_t grid = e.tiles < 8ull * num_sms ? e.tiles : 8ull * num_sms;
  k_enc_write<<<static_cast<unsigned>(grid), kEncThreads, 0, stream>>>(e);
  return cudaGetLastError();
}

}  // namespace hd
