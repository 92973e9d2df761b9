// decode.cu -- the persistent Huffman decode kernel (gap-array and
// self-synchronising variants).
//
// Geometry.  A subsequence is S bits (one thread), a tile is B subsequences
// (one block pass), a work unit is M consecutive tiles.  Work units are handed
// out in order through an atomic ticket; the output offset of a unit comes
// from a decoupled look-back over units, so one launch decodes a whole field
// (or many fields) in a single pass over the bitstream.  Grouping M tiles per
// look-back step keeps the look-back chain short at full bandwidth.
//
// Per work unit:
//   A. for each tile: stage the tile's units in shared memory, find every
//      subsequence's first codeword and count the codewords that start in it;
//        - gap array (Sec. III-C): start = i*S + gap[i], counted by the
//          "redundant decoding" pass of Sec. IV-C;
//        - self-synchronisation (Sec. III-B, IV-A): every thread decodes its
//          subsequence from i*S without writing; a thread whose start differs
//          from its predecessor's stop position walks its new and old paths
//          side by side until they meet at a common codeword boundary, after
//          which the old stop position and count hold.  Rounds stop when no
//          start changes (block vote).  The first tile of a unit takes its
//          start from a warp that re-synchronises the 32 subsequences before
//          the unit; later tiles continue from the previous tile.
//   B. look-back across units for the unit's first output index (for the
//      self-synchronising variant it also checks that the unit's start equals
//      the verified stop of the previous unit, and re-runs A if not);
//   C. for each tile: decode again into the shared-memory window and write it
//      out with coalesced 16-byte stores (Algorithm 1, Sec. IV-B).
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

// Walks a new path from `ns` and the old path from `s` (stop `e`, count `c`)
// until they share a codeword boundary or both pass `end`; afterwards s, e, c
// describe the path from ns.
template <int STRIDE, bool COUNT>
__device__ __forceinline__ void merge_paths(const Tables& T, const uint32_t* col, uint32_t end,
                                            uint32_t ns, uint32_t& s, uint32_t& e,
                                            uint32_t& c) {
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
  if (COUNT) c = met ? ca + (c - cb) : ca;
  if (!met) e = a;
  s = ns;
}

// Intra-sequence synchronisation over one tile (all threads).  Thread 0's
// predecessor stopped at e_pred (so thread 0 starts at e_pred - S).  Returns
// false if the round cap was hit.
template <int S, int B>
__device__ __forceinline__ bool sync_rounds(const Tables& T, const uint32_t* col, bool valid,
                                            uint32_t end, uint32_t e_pred, uint32_t& s,
                                            uint32_t& e, uint32_t& c, uint32_t* s_e_last) {
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
    if (changed) merge_paths<B, true>(T, col, end, ns, s, e, c);
  }
}

// Warp 0: guesses where the work unit starting at subsequence i_u begins, by
// self-synchronising the 32 subsequences before it (lane 0 starts at its
// nominal position).  Returns the offset of the first codeword boundary at or
// after i_u*S as seen from there.
template <int S>
__device__ __forceinline__ uint32_t presync_guess(const Tables& T, uint32_t* s_pre,
                                                  const FieldDesc& F, uint64_t i_u) {
  const int lane = threadIdx.x & 31;
  uint32_t* col = s_pre + lane;
  stage_units<S>(col, F, i_u - 32 + lane, 32);
  __syncwarp();
  bool bad = false;
  uint32_t p = 0;
  while (p < S) p += code_len(T, peek<32>(col, p), bad);
  uint32_t s = 0, e = p, c = 0;
  for (int round = 0; round < 40; ++round) {
    const uint32_t e_prev = __shfl_up_sync(0xffffffffu, e, 1);
    const uint32_t ns = lane ? e_prev - S : s;
    const bool changed = ns != s;
    if (!__any_sync(0xffffffffu, changed)) break;
    if (changed) merge_paths<32, false>(T, col, S, ns, s, e, c);
  }
  return __shfl_sync(0xffffffffu, e, 31) - S;
}

// Look-back of the self-synchronising variant (warp 0).  Returns 0 when the
// unit's assumed start is verified (and publishes the inclusive state), or 1
// when the previous unit's verified stop differs: then *true_start is that
// stop offset and *excl_out the previous unit's inclusive count.
__device__ __forceinline__ uint32_t lookback_sync(const DecodeParams& P, uint64_t g,
                                                  uint64_t first_unit, uint32_t a_self,
                                                  uint32_t e_self, uint64_t C, uint32_t* err,
                                                  uint64_t* excl_out, uint32_t* true_start) {
  const int lane = threadIdx.x & 31;
  uint64_t* st = P.unit_state;
  if (g == first_unit) {
    if (lane == 0) st_relaxed(st + g, pack_state(kStateInc, a_self, e_self, C));
    *excl_out = 0;
    return 0;
  }
  if (lane == 0) st_relaxed(st + g, pack_state(kStateAgg, a_self, e_self, C));
  uint64_t excl = 0;
  int64_t j = static_cast<int64_t>(g) - 1;
  const int64_t lo = static_cast<int64_t>(first_unit);
  uint32_t carry_a = a_self;
  const uint64_t t0 = now_ns();
  for (;;) {
    const int64_t idx = j - lane;
    const bool before = idx < lo;
    const uint64_t s = before ? kStateInc : ld_relaxed(st + idx);
    const uint32_t flag = static_cast<uint32_t>(s >> 62);
    const uint32_t a_l = static_cast<uint32_t>(s >> 56) & 63u;
    const uint32_t e_l = static_cast<uint32_t>(s >> 50) & 63u;
    uint32_t succ_a = __shfl_up_sync(0xffffffffu, a_l, 1);
    if (lane == 0) succ_a = carry_a;
    const bool link_ok = before || (flag != 0u && e_l == succ_a);
    const uint32_t inc = __ballot_sync(0xffffffffu, flag == 2u);
    const uint32_t notready = __ballot_sync(0xffffffffu, flag == 0u);
    const uint32_t broken = __ballot_sync(0xffffffffu, !link_ok && flag != 0u);
    const uint32_t need = inc ? (((inc & (0u - inc)) << 1) - 1u) : 0xffffffffu;
    bool wait = (notready & need) != 0;
    bool restart = false;
    if (!wait && (broken & need)) {
      const uint32_t first_broken = __ffs(broken & need) - 1;
      if (first_broken == 0 && (inc & 1u) && j == static_cast<int64_t>(g) - 1) {
        *true_start = __shfl_sync(0xffffffffu, e_l, 0);
        *excl_out = __shfl_sync(0xffffffffu, s & kValMask50, 0);
        return 1;
      }
      // an earlier unit's start is wrong; it will publish a fix, and the
      // units after it may change too, so the walk starts over
      wait = true;
      restart = true;
    }
    if (wait) {
      bool go = true;
      if (lane == 0) go = backoff_wait(P, t0);
      go = __shfl_sync(0xffffffffu, go, 0);
      if (!go) {
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
    excl += warp_sum_u64((need >> lane) & 1u ? (s & kValMask50) : 0ull);
    if (inc) break;
    carry_a = __shfl_sync(0xffffffffu, a_l, 31);
    j -= 32;
  }
  if (lane == 0) st_relaxed(st + g, pack_state(kStateInc, a_self, e_self, excl + C));
  *excl_out = excl;
  return 0;
}

template <int S, int B, bool SS>
__global__ void __launch_bounds__(B) k_decode(const __grid_constant__ DecodeParams P) {
  constexpr int W = S / 32 + 1;
  constexpr int NW = B / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_lut = reinterpret_cast<uint32_t*>(smem);
  uint32_t* s_bits = s_lut + (1u << P.K);
  uint32_t* s_pre = s_bits + W * B;  // self-sync only: 32 staged subsequences
  uint16_t* s_out = reinterpret_cast<uint16_t*>(s_pre + (SS ? W * 32 : 0));
  uint16_t* s_cnt = s_out + P.window + 16;                // [M][B] codeword counts
  uint8_t* s_start = reinterpret_cast<uint8_t*>(s_cnt + P.M * B);  // [M][B] starts (self-sync)

  __shared__ uint64_t s_end[34];
  __shared__ uint32_t s_base[34];
  __shared__ uint32_t s_meta[2];
  __shared__ uint32_t s_warp[NW];
  __shared__ uint32_t s_e_last[NW];
  __shared__ uint32_t s_tileC[kMaxTilesPerUnit];
  __shared__ uint64_t s_unit_base;
  __shared__ uint32_t s_ticket;
  __shared__ uint32_t s_field;
  __shared__ uint32_t s_flush_end;
  __shared__ uint32_t s_a, s_tile_e, s_resync, s_true_start;

  const int t = threadIdx.x;
  const int lane = t & 31;
  const int warp = t >> 5;
  uint32_t cur_field = 0xffffffffu;
  uint32_t* col = s_bits + t;

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
      load_table(F.table, P.K, s_lut, s_end, s_base, s_meta, B);
      cur_field = fi;
      __syncthreads();
    }
    const Tables T{s_lut, s_end, s_base,
                   reinterpret_cast<const uint16_t*>(reinterpret_cast<const char*>(F.table) +
                                                     kTableHeaderBytes + (4u << P.K)),
                   s_meta[0], 32u - P.K};
    const bool table_ok = s_meta[1] == 0;

    const uint64_t ul = g - F.unit_begin;
    const uint64_t i_u = ul * P.M * B;
    const uint32_t m_cnt =
        static_cast<uint32_t>(min(static_cast<uint64_t>(P.M), (F.nsub - i_u + B - 1) / B));

    // ---- A: starts and counts of every tile of the unit ------------------
    uint32_t err_data = 0;   // errors in the data itself (gap variant)
    uint32_t err_sync = 0;   // errors along the synchronised path (self-sync)
    uint32_t unit_e = 0;     // self-sync: stop offset past the unit's last subsequence
    auto phase_a = [&](uint32_t a0) -> uint64_t {
      uint64_t total = 0;
      uint32_t e_pred = S + a0;
      err_sync = 0;
      for (uint32_t m = 0; m < m_cnt; ++m) {
        const uint64_t i = i_u + static_cast<uint64_t>(m) * B + t;
        const bool valid = table_ok && i < F.nsub;
        uint32_t end = 0;
        if (valid) {
          stage_units<S>(col, F, i, B);
          const uint64_t rem = F.nbits - i * S;
          end = rem < S ? static_cast<uint32_t>(rem) : S;
        }
        uint32_t c = 0;
        if constexpr (!SS) {
          if (valid) {
            uint32_t gp = F.gap[i * F.gap_stride];
            const uint32_t expect = (i + 1 < F.nsub) ? S + F.gap[(i + 1) * F.gap_stride]
                                                     : static_cast<uint32_t>(F.nbits - i * S);
            if (gp > end || gp >= S) {
              err_data |= kErrGap;
              gp = end;
            }
            uint32_t p = gp;
            bool bad = false;
            while (p < end) {
              p += code_len(T, peek<B>(col, p), bad);
              ++c;
              if (bad) break;
            }
            if (bad) err_data |= kErrCode;
            else if (p != expect) err_data |= kErrGap;
          }
        } else {
          uint32_t s = 0, e = 0;
          if (valid) {
            bool bad = false;
            uint32_t p = 0;
            while (p < end) {
              p += code_len(T, peek<B>(col, p), bad);
              ++c;
            }
            e = p;
          }
          if (!sync_rounds<S, B>(T, col, valid, end, e_pred, s, e, c, s_e_last))
            err_sync |= kErrNoSync;
          if (valid && i + 1 == F.nsub && e != end) err_sync |= kErrCode;
          s_start[m * B + t] = static_cast<uint8_t>(s);
          if (t == B - 1) s_tile_e = e;
        }
        s_cnt[m * B + t] = static_cast<uint16_t>(c);
        uint32_t C;
        block_excl_scan<B>(c, s_warp, &C);
        if (t == 0) s_tileC[m] = C;
        total += C;
        if constexpr (SS) {
          e_pred = s_tile_e;  // written before the scan's barriers
          __syncthreads();    // everyone read s_tile_e before the next tile rewrites it
        }
      }
      unit_e = e_pred - S;
      return total;
    };

    uint32_t a0 = 0;
    if constexpr (SS) {
      if (warp == 0) {
        const uint32_t guess = (ul > 0 && table_ok) ? presync_guess<S>(T, s_pre, F, i_u) : 0u;
        if (lane == 0) s_a = guess;
      }
      __syncthreads();
      a0 = s_a;
    }
    uint64_t C = phase_a(a0);

    // ---- B: unit offset by look-back --------------------------------------
    if constexpr (!SS) {
      if (err_data) atomicOr(F.err, err_data);
      if (warp == 0) {
        const uint64_t excl = lookback_counts(P, g, F.unit_begin, C, F.err);
        if (t == 0) s_unit_base = excl;
      }
      __syncthreads();
    } else {
      if (warp == 0) {
        uint64_t excl = 0;
        uint32_t ts = 0;
        const uint32_t r = lookback_sync(P, g, F.unit_begin, a0, unit_e, C, F.err, &excl, &ts);
        if (t == 0) {
          s_resync = r;
          s_true_start = ts;
          s_unit_base = excl;
        }
      }
      __syncthreads();
      if (s_resync) {
        a0 = s_true_start;
        C = phase_a(a0);
        if (t == 0)
          st_relaxed(P.unit_state + g, pack_state(kStateInc, a0, unit_e, s_unit_base + C));
      }
      if (err_sync) atomicOr(F.err, err_sync);
      if (P.sync_only) {
        for (uint32_t m = 0; m < m_cnt; ++m) {
          const uint64_t i = i_u + static_cast<uint64_t>(m) * B + t;
          if (table_ok && i < F.nsub) F.gap_out[i] = s_start[m * B + t];
        }
        if (t == 0 && !table_ok && ul == 0) atomicOr(F.err, kErrTable);
        __syncthreads();
        continue;
      }
    }
    const uint64_t unit_base = s_unit_base;
    if (t == 0) {
      if (ul + 1 == F.nunits && unit_base + C != F.n) atomicOr(F.err, kErrCount);
      if (!table_ok && ul == 0) atomicOr(F.err, kErrTable);
    }

    // ---- C: decode into the shared-memory window, coalesced stores --------
    uint64_t tile_base = unit_base;
    bool bad_any = false;
    for (uint32_t m = 0; m < m_cnt; ++m) {
      const uint64_t i = i_u + static_cast<uint64_t>(m) * B + t;
      const bool valid = table_ok && i < F.nsub;
      uint32_t gp = 0;
      const uint32_t c = s_cnt[m * B + t];
      if (valid) {
        stage_units<S>(col, F, i, B);
        if constexpr (SS) gp = s_start[m * B + t];
        else gp = min(static_cast<uint32_t>(F.gap[i * F.gap_stride]), static_cast<uint32_t>(S));
      }
      uint32_t Cm;
      const uint32_t o = block_excl_scan<B>(c, s_warp, &Cm);
      window_write<B>(s_out, &s_flush_end, P.window, o, c, Cm, tile_base, F.out, F.n,
                      [&](uint16_t* dst) {
                        uint32_t p = gp;
                        bool bad = false;
                        for (uint32_t j = 0; j < c; ++j) {
                          uint32_t sym;
                          p += code_sym(T, peek<B>(col, p), sym, bad);
                          dst[j] = static_cast<uint16_t>(sym);
                        }
                        bad_any |= bad;
                      });
      tile_base += Cm;
    }
    if (SS && bad_any) atomicOr(F.err, kErrCode);
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
  size_t b = (static_cast<size_t>(1) << s.K) * 4 + W * s.threads * 4;
  if (self_sync) b += W * 32 * 4;
  b += (static_cast<size_t>(s.window) + 16) * 2;
  b += static_cast<size_t>(s.M) * s.threads * 2;
  if (self_sync) b += static_cast<size_t>(s.M) * s.threads;
  return (b + 15) & ~static_cast<size_t>(15);
}

cudaError_t launch_decode(const DecodeParams& p, const LaunchShape& s, bool self_sync,
                          int num_sms, cudaStream_t stream) {
  if (s.M < 1 || s.M > kMaxTilesPerUnit || p.M != s.M) return cudaErrorInvalidValue;
  return self_sync ? launch_v<true>(p, s, num_sms, stream)
                   : launch_v<false>(p, s, num_sms, stream);
}

}  // namespace hd
