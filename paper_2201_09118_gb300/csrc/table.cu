// table.cu -- builds the shared-memory decode table of each field's canonical
// codebook on the GPU and clears the per-launch look-back state.
//
// The paper keeps the codebook in global memory and relies on the cache
// (Sec. IV-B); here every decode block copies a direct-lookup table into shared
// memory instead, so a codeword is resolved with one shared-memory load.  The
// table is derived from the code lengths alone because the codes are canonical
// (RFC 1951 Sec. 3.2.2 assignment).
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace hd {

namespace {

constexpr int kPrepThreads = 1024;

__device__ __forceinline__ const FieldDesc& field_at(const PrepParams& p, bool single, uint32_t i) {
  return single ? p.f0 : p.fields[i];
}

// Block `sl` of `nsl` builds the table of one field: every block computes the
// header and the sorted symbols (the same values), and fills entries
// sl*kPrepThreads + t + k*nsl*kPrepThreads of the first- and second-level
// tables.
__device__ void build_table(const FieldDesc& F, uint32_t K, uint32_t sl, uint32_t nsl) {
  __shared__ uint32_t cnt[34];
  __shared__ uint32_t s_maxlen, s_bad, s_nused;
  __shared__ uint64_t s_end[34];
  __shared__ uint32_t s_start[34];
  __shared__ uint32_t s_base[34];
  __shared__ uint32_t wcnt[kPrepThreads / 32][34];
  __shared__ uint32_t run[34];

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint32_t A = F.alphabet;
  TableHeader* H = const_cast<TableHeader*>(F.table);
  char* tb = reinterpret_cast<char*>(H);
  uint32_t* lut = reinterpret_cast<uint32_t*>(tb + kTableHeaderBytes);
  uint16_t* sorted = reinterpret_cast<uint16_t*>(tb + table_sorted_off(K));
  uint16_t* lut16 = reinterpret_cast<uint16_t*>(tb + table_lut16_off(K, A));
  uint8_t* len8 = reinterpret_cast<uint8_t*>(tb + table_len8_off(K, A));
  uint8_t* run8 = reinterpret_cast<uint8_t*>(tb + table_run8_off(K, A));
  uint32_t* pair = reinterpret_cast<uint32_t*>(tb + table_pair_off(K, A));
  const bool with16 = lut16_usable(K, A);

  if (t < 34) {
    cnt[t] = 0;
    run[t] = 0;
  }
  if (t == 0) {
    s_maxlen = 0;
    s_bad = 0;
    s_nused = 0;
  }
  __syncthreads();
  for (uint32_t s = t; s < A; s += kPrepThreads) {
    const uint32_t L = F.lengths[s];
    if (L > kMaxCodeLen) {
      atomicOr(&s_bad, 1u);
    } else if (L) {
      atomicAdd(&cnt[L], 1u);
      atomicMax(&s_maxlen, L);
      atomicAdd(&s_nused, 1u);
    }
  }
  __syncthreads();
  if (t == 0) {
    // Kraft sum in units of 2^-32 must not exceed 1
    uint64_t kraft = 0;
    for (int L = 1; L <= 32; ++L) kraft += static_cast<uint64_t>(cnt[L]) << (32 - L);
    if (kraft > (1ull << 32)) s_bad = 1;
    uint64_t code = 0;
    uint32_t start = 0;
    s_end[0] = 0;
    s_start[0] = 0;
    s_base[0] = 0;
    for (int L = 1; L <= 33; ++L) {
      const uint64_t c_prev = (L >= 2) ? cnt[L - 1] : 0;
      if (L <= 32) {
        code = (code + c_prev) << 1;  // first canonical code of length L
        s_start[L] = start;
        s_base[L] = start - static_cast<uint32_t>(code);
        s_end[L] = (code + cnt[L]) << (32 - L);
        start += cnt[L];
      } else {
        s_start[L] = start;
        s_base[L] = 0;
        s_end[L] = s_end[32];
      }
    }
    H->status = s_bad;
    H->maxlen = s_maxlen;
    H->nused = s_nused;
    H->K = K;
    H->long0 = s_start[K + 1 <= 33 ? K + 1 : 33];
    uint32_t lmin = 0;
    for (int L = 32; L >= 1; --L)
      if (cnt[L]) lmin = L;
    H->minlen = lmin;
    H->sub_bits = 0;
    H->nsub = 0;
    H->sub_p0 = 0;
    for (int L = 0; L < 34; ++L) {
      H->end[L] = s_end[L];
      H->base[L] = s_base[L];
    }
  }
  __syncthreads();
  if (s_bad) return;

  // Rank of each symbol among the symbols of its length, in symbol order:
  // within a warp via match/popc, across warps via per-length counters.
  for (uint32_t c0 = 0; c0 < A; c0 += kPrepThreads) {
    for (int k = t; k < (kPrepThreads / 32) * 34; k += kPrepThreads) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    const uint32_t s = c0 + t;
    const uint32_t L = s < A ? F.lengths[s] : 0u;
    const uint32_t same = __match_any_sync(0xffffffffu, L);
    const uint32_t rank_w = __popc(same & ((1u << lane) - 1u));
    if (L && rank_w == 0) wcnt[warp][L] = __popc(same);
    __syncthreads();
    if (t >= 1 && t <= 32) {
      uint32_t acc = run[t];
      for (int w = 0; w < kPrepThreads / 32; ++w) {
        const uint32_t v = wcnt[w][t];
        wcnt[w][t] = acc;
        acc += v;
      }
      run[t] = acc;
    }
    __syncthreads();
    if (L) sorted[s_start[L] + wcnt[warp][L] + rank_w] = static_cast<uint16_t>(s);
    __syncthreads();
  }

  // First-level table: entry p covers all windows whose top K bits equal p.
  const uint32_t maxlen = s_maxlen;
  for (uint32_t p = sl * kPrepThreads + t; p < (1u << K); p += nsl * kPrepThreads) {
    const uint32_t w = p << (32 - K);
    uint32_t L = 1;
    while (L <= 32 && static_cast<uint64_t>(w) >= s_end[L]) ++L;
    uint32_t e, e16, e8, r8 = 0, pe;
    if (L <= K && L <= maxlen) {
      const uint32_t rank = (w >> (32 - L)) + s_base[L];
      e = (L << 16) | sorted[rank];
      e16 = (L << 12) | (sorted[rank] & 0xFFFu);
      e8 = L;
      // the two-code entry: a second code wholly within the K bits joins
      // the first when both symbols fit 10 bits
      pe = (1u << 30) | (L << 26) | (sorted[rank] & 0xFFFu);
      if (A <= 1024 && L < K) {
        const uint32_t rem = K - L, w2 = w << L;
        uint32_t L2 = 1;
        while (L2 <= rem && static_cast<uint64_t>(w2) >= s_end[L2]) ++L2;
        if (L2 <= rem && L2 <= maxlen) {
          const uint32_t sym1 = sorted[(w2 >> (32 - L2)) + s_base[L2]];
          pe = (2u << 30) | (L << 26) | (L2 << 22) | ((sym1 & 0x3FFu) << 10) |
               (sorted[rank] & 0x3FFu);
        }
      }
      // further codes wholly within the K known bits: a code of length
      // L2 <= the bits left is fixed by them (the limits are left-aligned)
      uint32_t used = L, m = 1;
      while (m < 7 && used < K) {
        const uint32_t rem = K - used;
        const uint32_t w2 = w << used;
        uint32_t L2 = 1;
        while (L2 <= rem && static_cast<uint64_t>(w2) >= s_end[L2]) ++L2;
        if (L2 > rem || L2 > maxlen) break;
        used += L2;
        ++m;
      }
      r8 = (m << 4) | used;
    } else {
      // length of the code at the last window with this prefix
      const uint32_t w_last = w | ((1u << (32 - K)) - 1u);
      uint32_t Lx = L;
      while (Lx <= 32 && static_cast<uint64_t>(w_last) >= s_end[Lx]) ++Lx;
      const uint32_t lmin = L <= maxlen ? L : 33u;
      const uint32_t lmax = Lx <= maxlen ? Lx : 0xFFu;
      e = kLongFlag | (lmax << 8) | lmin;
      e16 = lmin | (lmin == lmax ? 0u : kLut16Mixed);
      e8 = lmin == lmax ? lmin : (kLen8Walk | lmin);
      pe = e16;  // m = 0
    }
    lut[p] = e;
    if (with16) {
      lut16[p] = static_cast<uint16_t>(e16);
      pair[p] = pe;
    }
    len8[p] = static_cast<uint8_t>(e8);
    run8[p] = static_cast<uint8_t>(r8);
  }

  // Second-level tables of the 16-bit table.  Canonical codes longer than K
  // bits are the windows from end[K] on, so their prefixes are consecutive:
  // [end[K] >> (32-K), ceil(end[maxlen] / 2^(32-K))).  Each gets sub_bits more
  // bits (as many as the longest code needs, at most 8, and as the sub_cap(K)
  // entries allow); the most probable long codes come first.
  __shared__ uint32_t s_sub[3];  // sub_bits, nsub, sub_p0
  if (t == 0) {
    uint32_t kb = 0, ns = 0, p0 = 0;
    if (with16 && maxlen > K) {
      const uint32_t sh = 32 - K;
      p0 = static_cast<uint32_t>(s_end[K] >> sh);
      const uint64_t p1 = (s_end[maxlen] + (1ull << sh) - 1) >> sh;
      kb = maxlen - K < 8 ? maxlen - K : 8;
      const uint64_t nlong = p1 > p0 ? p1 - p0 : 0;
      const uint32_t cap = sub_cap(K) >> kb;
      ns = static_cast<uint32_t>(nlong < cap ? nlong : cap);
    }
    s_sub[0] = kb;
    s_sub[1] = ns;
    s_sub[2] = p0;
    H->sub_bits = kb;
    H->nsub = ns;
    H->sub_p0 = p0;
  }
  __syncthreads();
  const uint32_t kb = s_sub[0], ns = s_sub[1], p0 = s_sub[2];
  uint16_t* sub = reinterpret_cast<uint16_t*>(tb + table_sub_off(K, A));
  for (uint32_t idx = sl * kPrepThreads + t; idx < (ns << kb); idx += nsl * kPrepThreads) {
    const uint32_t w = ((p0 + (idx >> kb)) << (32 - K)) | ((idx & ((1u << kb) - 1u)) << (32 - K - kb));
    uint32_t L = K + 1;
    while (L <= maxlen && static_cast<uint64_t>(w) >= s_end[L]) ++L;
    uint16_t x = 0;
    if (L <= K + kb && L <= maxlen) {
      const uint32_t rank = (w >> (32 - L)) + s_base[L];
      x = static_cast<uint16_t>(((L - K) << 12) | (sorted[rank] & 0xFFFu));
    }
    sub[idx] = x;
  }
}

__global__ void __launch_bounds__(kPrepThreads) k_prepare(const __grid_constant__ PrepParams P) {
  const uint32_t b = blockIdx.x;
  if (b < P.table_blocks) {
    const uint32_t nf = P.hdr ? P.hdr->nfields : P.nfields;
    const bool single = !P.hdr && P.nfields == 1;
    const uint32_t nsl = P.slices ? P.slices : 1u;
    for (uint32_t x = b; x < nf * nsl; x += P.table_blocks) {
      __syncthreads();  // the previous field's shared state is no longer read
      build_table(field_at(P, single, x / nsl), P.K, x % nsl, nsl);
    }
    return;
  }
  // clear the per-launch control region (error words, segment totals)
  const uint64_t zb = b - P.table_blocks;
  const uint4 z = make_uint4(0, 0, 0, 0);
  for (uint64_t i = zb * kPrepThreads + threadIdx.x; i < P.zero_vec;
       i += static_cast<uint64_t>(P.zero_blocks) * kPrepThreads)
    P.zero_ptr[i] = z;
}

}  // namespace

cudaError_t launch_prepare(const PrepParams& p, cudaStream_t stream) {
  const uint32_t zb = p.zero_blocks;
  const uint32_t grid = p.table_blocks + zb;
  if (grid == 0) return cudaSuccess;
  k_prepare<<<grid, kPrepThreads, 0, stream>>>(p);
  return cudaGetLastError();
}

size_t table_bytes(uint32_t K, uint32_t alphabet) {
  const size_t b = table_pair_off(K, alphabet) + (static_cast<size_t>(4) << K);
  return (b + 255) & ~static_cast<size_t>(255);
}

}  // namespace hd
