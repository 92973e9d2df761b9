// lorenzo.cu -- the reconstruction after the decoder: cuSZ's first-order
// Lorenzo predictor inverted on prequantized integers (the second half of the
// end-to-end decompression the paper measures in Sec. V-B2).
//
// A code c stands for the residue d = c - R; code 0 marks an outlier whose
// residue is looked up in the ascending outlier list.  The prequantized value
// q is the inclusive prefix sum of d along every axis, and the output is
// float32(q) * float32(2 eb).
//
// 1D: reduce, scan, reconstruct: residue sums of tiles of 8192 codes, an
// exclusive scan of the tile sums, and a pass that scans each tile again
// from its prefix and writes the floats (8 bytes per code moved).  (Decode +
// reconstruction of 1D fields runs instead inside the decoder's kernels.)
// 3D with many slices and rows of at most 1024 codes, the slice path:
//   k_lorenzo_slice     one block per slice: per-warp column sums of residues,
//                       one barrier, then each warp streams its rows (x prefix
//                       by lane and warp scans, y sums in registers) from the
//                       carry of the rows above, writing int32;
//   k_lorenzo_zscan     the sum along z, float32 values in place of the int32s.
// Otherwise (2D, few slices, long rows) the band path, per group of slices:
//   k_lorenzo_warpband  one warp per band of rows in registers (rows up to
//   / k_lorenzo_band    1024 codes), or one block per band in shared memory:
//                       x and in-band y prefixes as int32, band column totals;
//   k_lorenzo_bandscan  exclusive scan of the band totals over the bands of
//                       each slice (the y carry of every band);
//   k_lorenzo_zscan     adds the band carry, runs the sum along z (carried
//                       between groups in `plane`) and writes the float32
//                       values in place of the int32s.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace hd {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint64_t kWarpBandMaxRow = 1024;  // rows handled by one warp in registers

// Residue of an outlier: binary search of position i in the outlier list.
__device__ __noinline__ int32_t outlier_residue(const uint64_t* idx, const int32_t* val,
                                                uint64_t n_out, uint32_t* err, uint64_t i) {
  uint64_t lo = 0, hi = n_out;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (idx[mid] < i)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo < n_out && idx[lo] == i) return val[lo];
  atomicOr(err, kErrOutlier);
  return 0;
}

__device__ __forceinline__ int32_t residue(const LorenzoParams& P, uint32_t c, uint64_t i) {
  return c ? static_cast<int32_t>(c) - P.radius
           : outlier_residue(P.out_idx, P.out_val, P.n_out, P.err, i);
}

__device__ __forceinline__ float value(const LorenzoParams& P, int32_t q) {
  return __fmul_rn(__int2float_rn(q), P.ebx2);
}

__device__ __forceinline__ int32_t warp_incl(int32_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(~0u, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// Eight codes of a 16-byte vector -> residues.  Branch-free unless a code is
// 0 (an outlier): one test per vector finds a zero half-word (it may also
// fire for a zero low half-word's borrow, which only costs the slow path).
__device__ __forceinline__ bool has_zero_half(uint32_t w) {
  return ((w - 0x00010001u) & ~w & 0x80008000u) != 0;
}

__device__ __forceinline__ void residues8(const LorenzoParams& P, uint4 u, uint64_t i,
                                          int32_t* d) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
  if (has_zero_half(u.x) | has_zero_half(u.y) | has_zero_half(u.z) | has_zero_half(u.w)) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      d[2 * k] = residue(P, w[k] & 0xffffu, i + 2 * k);
      d[2 * k + 1] = residue(P, w[k] >> 16, i + 2 * k + 1);
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    d[2 * k] = static_cast<int32_t>(w[k] & 0xffffu) - P.radius;
    d[2 * k + 1] = static_cast<int32_t>(w[k] >> 16) - P.radius;
  }
}

// ---- 1D ---------------------------------------------------------------------

constexpr int k1Vec = 8;   // codes per 16-byte load
constexpr int k1Rows = 4;  // loads per thread per tile
constexpr uint64_t k1Tile = static_cast<uint64_t>(kThreads) * k1Vec * k1Rows;

// Tile sums of the residues (threads loop over the tiles).
__global__ void __launch_bounds__(kThreads) k_lorenzo_1d_sums(LorenzoParams P, uint64_t tiles) {
  __shared__ int32_t s_part[kWarps];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const uint64_t base = tile * k1Tile;
    int32_t sum = 0;
    uint4 u[k1Rows];
#pragma unroll
    for (int r = 0; r < k1Rows; ++r) {
      const uint64_t i0 = base + (static_cast<uint64_t>(r) * kThreads + t) * k1Vec;
      if (i0 + k1Vec <= P.n) u[r] = __ldcs(reinterpret_cast<const uint4*>(P.codes + i0));
    }
#pragma unroll
    for (int r = 0; r < k1Rows; ++r) {
      const uint64_t i0 = base + (static_cast<uint64_t>(r) * kThreads + t) * k1Vec;
      int32_t d[k1Vec];
      if (i0 + k1Vec <= P.n) {
        residues8(P, u[r], i0, d);
      } else {
#pragma unroll
        for (int j = 0; j < k1Vec; ++j) d[j] = i0 + j < P.n ? residue(P, P.codes[i0 + j], i0 + j) : 0;
      }
#pragma unroll
      for (int j = 0; j < k1Vec; ++j) sum += d[j];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(~0u, sum, o);
    if (lane == 0) s_part[w] = sum;
    __syncthreads();
    if (t == 0) {
      int32_t total = 0;
#pragma unroll
      for (int k = 0; k < kWarps; ++k) total += s_part[k];
      P.tile_prefix[tile] = total;
    }
    __syncthreads();
  }
}

// Exclusive scan of the tile sums in place (one block).
constexpr int k1ScanThreads = 1024;

__global__ void __launch_bounds__(k1ScanThreads) k_lorenzo_1d_scan(int32_t* a, uint64_t tiles) {
  __shared__ int32_t s_w[k1ScanThreads / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const uint64_t per = (tiles + k1ScanThreads - 1) / k1ScanThreads;
  const uint64_t lo = min(tiles, per * t), hi = min(tiles, lo + per);
  int32_t sum = 0;
  for (uint64_t k = lo; k < hi; ++k) sum += a[k];
  const int32_t incl = warp_incl(sum, lane);
  if (lane == 31) s_w[w] = incl;
  __syncthreads();
  int32_t run = incl - sum;
  for (int k = 0; k < w; ++k) run += s_w[k];
  for (uint64_t k = lo; k < hi; ++k) {
    const int32_t v = a[k];
    a[k] = run;
    run += v;
  }
}

// Exclusive prefix of (residue + radius) over the outlier list (one block):
// the correction of q for the outliers before a position, whose codes 0 a
// residue sum over codes counts as -radius.
__global__ void __launch_bounds__(k1ScanThreads) k_outlier_prefix(const int32_t* val, uint64_t n,
                                                                  int32_t radius, int32_t* corr) {
  __shared__ int32_t s_w[k1ScanThreads / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const uint64_t per = (n + k1ScanThreads - 1) / k1ScanThreads;
  const uint64_t lo = min(n, per * t), hi = min(n, lo + per);
  int32_t sum = 0;
  for (uint64_t k = lo; k < hi; ++k) sum += val[k] + radius;
  const int32_t incl = warp_incl(sum, lane);
  if (lane == 31) s_w[w] = incl;
  __syncthreads();
  int32_t run = incl - sum;
  for (int k = 0; k < w; ++k) run += s_w[k];
  for (uint64_t k = lo; k < hi; ++k) {
    corr[k] = run;
    run += val[k] + radius;
  }
  if (t == k1ScanThreads - 1) corr[n] = run;
}

// Reconstruction of one tile from its prefix.
__global__ void __launch_bounds__(kThreads) k_lorenzo_1d(LorenzoParams P) {
  __shared__ int32_t s_warp[k1Rows][kWarps];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const uint64_t tile = blockIdx.x;
  const uint64_t base = tile * k1Tile;
  // element (r, t, j) of the tile is base + (r * kThreads + t) * 8 + j
  int32_t v[k1Rows][k1Vec];
  int32_t ex[k1Rows];
#pragma unroll
  for (int r = 0; r < k1Rows; ++r) {
    const uint64_t i0 = base + (static_cast<uint64_t>(r) * kThreads + t) * k1Vec;
    if (i0 + k1Vec <= P.n) {
      residues8(P, __ldcs(reinterpret_cast<const uint4*>(P.codes + i0)), i0, v[r]);
    } else {
#pragma unroll
      for (int j = 0; j < k1Vec; ++j)
        v[r][j] = i0 + j < P.n ? residue(P, P.codes[i0 + j], i0 + j) : 0;
    }
#pragma unroll
    for (int j = 1; j < k1Vec; ++j) v[r][j] += v[r][j - 1];
    const int32_t incl = warp_incl(v[r][k1Vec - 1], lane);
    ex[r] = incl - v[r][k1Vec - 1];
    if (lane == 31) s_warp[r][w] = incl;
  }
  __syncthreads();
  int32_t agg = P.tile_prefix[tile], pre[k1Rows];
#pragma unroll
  for (int r = 0; r < k1Rows; ++r) {
#pragma unroll
    for (int k = 0; k < kWarps; ++k) {
      if (k == w) pre[r] = agg;
      agg += s_warp[r][k];
    }
  }
#pragma unroll
  for (int r = 0; r < k1Rows; ++r) {
    const uint64_t i0 = base + (static_cast<uint64_t>(r) * kThreads + t) * k1Vec;
    const int32_t off = pre[r] + ex[r];
    float o[k1Vec];
#pragma unroll
    for (int j = 0; j < k1Vec; ++j) o[j] = value(P, off + v[r][j]);
    if (i0 + k1Vec <= P.n) {
      float4* dst = reinterpret_cast<float4*>(P.out + i0);
      __stcs(dst, make_float4(o[0], o[1], o[2], o[3]));
      __stcs(dst + 1, make_float4(o[4], o[5], o[6], o[7]));
    } else {
#pragma unroll
      for (int j = 0; j < k1Vec; ++j)
        if (i0 + j < P.n) P.out[i0 + j] = o[j];
    }
  }
}

// ---- 2D / 3D ------------------------------------------------------------------

// VEC: nx % 8 == 0 (16-byte loads of codes, int4 rows in shared memory).
template <bool VEC>
__global__ void __launch_bounds__(kThreads) k_lorenzo_band(LorenzoParams P) {
  extern __shared__ int4 s_raw[];
  int32_t* s = reinterpret_cast<int32_t*>(s_raw);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const uint64_t zz = blockIdx.x / P.nb;  // slice within the launch
  const uint64_t b = blockIdx.x - zz * P.nb;
  const uint64_t y0 = b * P.yb;
  const uint32_t h = static_cast<uint32_t>(min(static_cast<uint64_t>(P.yb), P.ny - y0));
  const uint32_t nx = static_cast<uint32_t>(P.nx);
  const uint64_t start = ((P.z_lo + zz) * P.ny + y0) * P.nx;
  const uint32_t count = h * nx;
  if (VEC) {
#pragma unroll 4
    for (uint32_t k = t * 8; k < count; k += kThreads * 8) {
      int32_t d[8];
      residues8(P, *reinterpret_cast<const uint4*>(P.codes + start + k), start + k, d);
      reinterpret_cast<int4*>(s + k)[0] = make_int4(d[0], d[1], d[2], d[3]);
      reinterpret_cast<int4*>(s + k)[1] = make_int4(d[4], d[5], d[6], d[7]);
    }
  } else {
    for (uint32_t k = t; k < count; k += kThreads) s[k] = residue(P, P.codes[start + k], start + k);
  }
  __syncthreads();
  // prefix along x: one warp per row
  for (uint32_t r = w; r < h; r += kWarps) {
    int32_t* row = s + r * nx;
    int32_t carry = 0;
    if (VEC) {
      for (uint32_t x0 = 0; x0 < nx; x0 += 128) {
        const uint32_t x = x0 + lane * 4;
        int4 a = x < nx ? *reinterpret_cast<const int4*>(row + x) : make_int4(0, 0, 0, 0);
        a.y += a.x;
        a.z += a.y;
        a.w += a.z;
        const int32_t incl = warp_incl(a.w, lane);
        const int32_t e = incl - a.w + carry;
        if (x < nx)
          *reinterpret_cast<int4*>(row + x) = make_int4(a.x + e, a.y + e, a.z + e, a.w + e);
        carry += __shfl_sync(~0u, incl, 31);
      }
    } else {
      for (uint32_t x0 = 0; x0 < nx; x0 += 32) {
        const uint32_t x = x0 + lane;
        const int32_t a = x < nx ? row[x] : 0;
        const int32_t incl = warp_incl(a, lane);
        if (x < nx) row[x] = incl + carry;
        carry += __shfl_sync(~0u, incl, 31);
      }
    }
  }
  __syncthreads();
  // prefix along y inside the band; the band's column totals
  int32_t* band = P.band + (zz * P.nb + b) * P.nx;
  for (uint32_t x = t; x < nx; x += kThreads) {
    int32_t run = 0;
    for (uint32_t r = 0; r < h; ++r) {
      run += s[r * nx + x];
      s[r * nx + x] = run;
    }
    band[x] = run;
  }
  __syncthreads();
  int32_t* g = reinterpret_cast<int32_t*>(P.out) + start;
  if (VEC) {
    for (uint32_t k = t * 4; k < count; k += kThreads * 4)
      *reinterpret_cast<int4*>(g + k) = *reinterpret_cast<const int4*>(s + k);
  } else {
    for (uint32_t k = t; k < count; k += kThreads) g[k] = s[k];
  }
}

// Rows up to 1024 codes, one warp per band of rows, everything in
// registers: lane l holds the 8-code chunks l, l + 32, .. of a row; a row's
// prefix is a lane scan per chunk plus one warp scan per chunk column, and the
// column sums run in registers while the rows stream through (no shared
// memory, no barriers).  R rows of raw codes are loaded before any is
// processed.  `col` enters with the band's y carry (x prefix included) and
// leaves with the prefix of the band's last row.
template <int K, bool VEC>
__device__ __forceinline__ void load_row(const LorenzoParams& P, int lane, uint64_t row0,
                                         uint32_t r, uint32_t h, uint4 (&raw)[K]) {
  const uint32_t nx = static_cast<uint32_t>(P.nx);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t x = 8u * (lane + 32u * k);
    raw[k] = VEC && r < h && x < nx
                 ? __ldcg(reinterpret_cast<const uint4*>(P.codes + row0 +
                                                         static_cast<uint64_t>(r) * nx + x))
                 : make_uint4(0, 0, 0, 0);
  }
}

template <int K, bool VEC>
__device__ __forceinline__ void row_residues(const LorenzoParams& P, int lane, uint64_t rs,
                                             const uint4 (&raw)[K], int k, int32_t (&v)[8]) {
  const uint32_t nx = static_cast<uint32_t>(P.nx);
  const uint32_t x = 8u * (lane + 32u * k);
  if (VEC) {
    if (x < nx) {
      residues8(P, raw[k], rs + x, v);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = 0;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      v[j] = x + j < nx ? residue(P, P.codes[rs + x + j], rs + x + j) : 0;
  }
}

// Rows stream through a ring of R rows of raw codes: the load of row r + R
// is issued as soon as row r has been taken out of the ring.
template <int K, bool VEC, int R>
__device__ __forceinline__ void warp_rows(const LorenzoParams& P, int lane, uint64_t row0,
                                          uint32_t h, int32_t (&col)[K][8]) {
  const uint32_t nx = static_cast<uint32_t>(P.nx);
  int32_t* inter = reinterpret_cast<int32_t*>(P.out);
  uint4 raw[R][K];
#pragma unroll
  for (int p = 0; p < R; ++p) load_row<K, VEC>(P, lane, row0, p, h, raw[p]);
  for (uint32_t r0 = 0; r0 < h; r0 += R) {
#pragma unroll
    for (int p = 0; p < R; ++p) {
      const uint32_t r = r0 + p;
      if (r >= h) break;
      const uint64_t rs = row0 + static_cast<uint64_t>(r) * nx;
      uint4 cur[K];
#pragma unroll
      for (int k = 0; k < K; ++k) cur[k] = raw[p][k];
      load_row<K, VEC>(P, lane, row0, r + R, h, raw[p]);
      int32_t carry = 0;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const uint32_t x = 8u * (lane + 32u * k);
        int32_t v[8];
        row_residues<K, VEC>(P, lane, rs, cur, k, v);
#pragma unroll
        for (int j = 1; j < 8; ++j) v[j] += v[j - 1];
        const int32_t incl = warp_incl(v[7], lane);
        const int32_t e = incl - v[7] + carry;
        carry += __shfl_sync(~0u, incl, 31);
#pragma unroll
        for (int j = 0; j < 8; ++j) col[k][j] += v[j] + e;
        if (VEC) {
          if (x < nx) {
            int4* dst = reinterpret_cast<int4*>(inter + rs + x);
            dst[0] = make_int4(col[k][0], col[k][1], col[k][2], col[k][3]);
            dst[1] = make_int4(col[k][4], col[k][5], col[k][6], col[k][7]);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (x + j < nx) inter[rs + x + j] = col[k][j];
        }
      }
    }
  }
}

// Residue sums per column over h rows (no scans), through the same ring.
template <int K, bool VEC, int R>
__device__ __forceinline__ void warp_colsums(const LorenzoParams& P, int lane, uint64_t row0,
                                             uint32_t h, int32_t (&acc)[K][8]) {
  const uint32_t nx = static_cast<uint32_t>(P.nx);
  uint4 raw[R][K];
#pragma unroll
  for (int p = 0; p < R; ++p) load_row<K, VEC>(P, lane, row0, p, h, raw[p]);
  for (uint32_t r0 = 0; r0 < h; r0 += R) {
#pragma unroll
    for (int p = 0; p < R; ++p) {
      const uint32_t r = r0 + p;
      if (r >= h) break;
      const uint64_t rs = row0 + static_cast<uint64_t>(r) * nx;
      uint4 cur[K];
#pragma unroll
      for (int k = 0; k < K; ++k) cur[k] = raw[p][k];
      load_row<K, VEC>(P, lane, row0, r + R, h, raw[p]);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        int32_t v[8];
        row_residues<K, VEC>(P, lane, rs, cur, k, v);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[k][j] += v[j];
      }
    }
  }
}

// x prefix of a row held as in warp_rows (in place).
template <int K>
__device__ __forceinline__ void warp_row_prefix(int lane, int32_t (&a)[K][8]) {
  int32_t carry = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int j = 1; j < 8; ++j) a[k][j] += a[k][j - 1];
    const int32_t incl = warp_incl(a[k][7], lane);
    const int32_t e = incl - a[k][7] + carry;
    carry += __shfl_sync(~0u, incl, 31);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[k][j] += e;
  }
}

// Band path: warps loop over the bands of the launch (the grid is one
// resident wave); each writes its band's local prefix and column totals.
constexpr int kWarpBandThreads = 128;

template <int K, bool VEC, int R>
__global__ void __launch_bounds__(kWarpBandThreads, K <= 2 ? 4 : 3)
    k_lorenzo_warpband(LorenzoParams P) {
  constexpr int W = kWarpBandThreads / 32;
  const int lane = threadIdx.x & 31;
  const uint64_t total = (P.z_hi - P.z_lo) * P.nb;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * W;
  const uint32_t nx = static_cast<uint32_t>(P.nx);
  for (uint64_t gw = static_cast<uint64_t>(blockIdx.x) * W + (threadIdx.x >> 5); gw < total;
       gw += stride) {
    const uint64_t zz = gw / P.nb;
    const uint64_t b = gw - zz * P.nb;
    const uint64_t y0 = b * P.yb;
    const uint32_t h = static_cast<uint32_t>(min(static_cast<uint64_t>(P.yb), P.ny - y0));
    const uint64_t row0 = ((P.z_lo + zz) * P.ny + y0) * P.nx;
    int32_t col[K][8];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < 8; ++j) col[k][j] = 0;
    warp_rows<K, VEC, R>(P, lane, row0, h, col);
    int32_t* band = P.band + gw * P.nx;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint32_t x = 8u * (lane + 32u * k);
      if (VEC) {
        if (x < nx) {
          int4* dst = reinterpret_cast<int4*>(band + x);
          dst[0] = make_int4(col[k][0], col[k][1], col[k][2], col[k][3]);
          dst[1] = make_int4(col[k][4], col[k][5], col[k][6], col[k][7]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (x + j < nx) band[x + j] = col[k][j];
      }
    }
  }
}

// Slice path (3D grids with many slices, rows up to 1024 codes): one block of
// kSliceWarps warps per slice, warp w taking an equal share of its rows.
// Each warp first sums the residues of its rows per column (no scans) into
// shared memory; after the one barrier, a warp's y carry is the x prefix of
// the column sums of the warps above it, and it streams its rows as a band
// warp (their codes read again, now from L2), writing the slice's x-y prefix
// as int32.  The z kernel follows.
constexpr int kSliceWarps = 4;
constexpr int kSliceThreads = 32 * kSliceWarps;

template <int K, bool VEC, int R>
__global__ void __launch_bounds__(kSliceThreads, 4) k_lorenzo_slice(LorenzoParams P) {
  extern __shared__ int4 s_raw[];
  int32_t* s_tot = reinterpret_cast<int32_t*>(s_raw);  // [kSliceWarps][nx]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t nx = static_cast<uint32_t>(P.nx);
  const uint32_t ny = static_cast<uint32_t>(P.ny);
  const uint32_t rpw = (ny + kSliceWarps - 1) / kSliceWarps;
  const uint32_t r_lo = min(ny, w * rpw);
  const uint32_t h = min(ny, r_lo + rpw) - r_lo;
  for (uint64_t z = P.z_lo + blockIdx.x; z < P.z_hi; z += gridDim.x) {
    const uint64_t row0 = (z * P.ny + r_lo) * P.nx;
    int32_t a[K][8];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < 8; ++j) a[k][j] = 0;
    warp_colsums<K, VEC, R>(P, lane, row0, h, a);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint32_t x = 8u * (lane + 32u * k);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (x + j < nx) s_tot[w * nx + x + j] = a[k][j];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < 8; ++j) a[k][j] = 0;
    for (int v = 0; v < w; ++v) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const uint32_t x = 8u * (lane + 32u * k);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (x + j < nx) a[k][j] += s_tot[v * nx + x + j];
      }
    }
    __syncthreads();  // s_tot is rewritten for the next slice
    warp_row_prefix<K>(lane, a);
    warp_rows<K, VEC, R>(P, lane, row0, h, a);
  }
}

constexpr int kScanBatch = 8;
constexpr int kZBatch = 16;
constexpr int kColThreads = 128;

__global__ void __launch_bounds__(kColThreads) k_lorenzo_bandscan(LorenzoParams P) {
  const uint64_t units = (P.z_hi - P.z_lo) * P.nx;
  for (uint64_t g = static_cast<uint64_t>(blockIdx.x) * kColThreads + threadIdx.x; g < units;
       g += static_cast<uint64_t>(gridDim.x) * kColThreads) {
    const uint64_t zz = g / P.nx;
    const uint64_t x = g - zz * P.nx;
    int32_t* col = P.band + zz * P.nb * P.nx + x;
    int32_t run = 0;
    for (uint64_t b0 = 0; b0 < P.nb; b0 += kScanBatch) {
      int32_t v[kScanBatch];
#pragma unroll
      for (int k = 0; k < kScanBatch; ++k) v[k] = b0 + k < P.nb ? col[(b0 + k) * P.nx] : 0;
#pragma unroll
      for (int k = 0; k < kScanBatch; ++k) {
        if (b0 + k < P.nb) col[(b0 + k) * P.nx] = run;
        run += v[k];
      }
    }
  }
}

template <int V>
struct IntV;
template <>
struct IntV<1> {
  static __device__ __forceinline__ void load(const int32_t* p, int32_t* v) { v[0] = *p; }
};
template <>
struct IntV<2> {
  static __device__ __forceinline__ void load(const int32_t* p, int32_t* v) {
    const int2 a = *reinterpret_cast<const int2*>(p);
    v[0] = a.x;
    v[1] = a.y;
  }
};
template <>
struct IntV<4> {
  static __device__ __forceinline__ void load(const int32_t* p, int32_t* v) {
    const int4 a = *reinterpret_cast<const int4*>(p);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
  }
};

template <int V>
__device__ __forceinline__ void store_values(float* p, const float* f) {
  if (V == 4)
    __stcs(reinterpret_cast<float4*>(p), make_float4(f[0], f[1], f[2], f[3]));
  else if (V == 2)
    __stcs(reinterpret_cast<float2*>(p), make_float2(f[0], f[V - 1]));
  else
    __stcs(p, f[0]);
}

// The sum along z and the float32 conversion, in place.  V adjacent columns
// of one row per thread (16- or 8-byte accesses when nx allows), kZBatch
// slices loaded before they are summed; BAND adds the y carry of each band
// (band path).  Threads loop over the plane (the grid is one resident wave).
template <int V, bool BAND>
__global__ void __launch_bounds__(kColThreads) k_lorenzo_zscan(LorenzoParams P) {
  const uint64_t plane = P.ny * P.nx;
  const uint64_t units = plane / V;
  const uint64_t band_stride = P.nb * P.nx;
  const int32_t* inter = reinterpret_cast<const int32_t*>(P.out);
  for (uint64_t u = static_cast<uint64_t>(blockIdx.x) * kColThreads + threadIdx.x; u < units;
       u += static_cast<uint64_t>(gridDim.x) * kColThreads) {
    const uint64_t g = u * V;
    const uint64_t y = g / P.nx;
    const uint64_t x = g - y * P.nx;
    const int32_t* band = BAND ? P.band + (y / P.yb) * P.nx + x : nullptr;
    int32_t run[V];
#pragma unroll
    for (int c = 0; c < V; ++c) run[c] = P.z_lo ? P.plane[g + c] : 0;
    for (uint64_t z0 = P.z_lo; z0 < P.z_hi; z0 += kZBatch) {
      int32_t v[kZBatch][V];
#pragma unroll
      for (int k = 0; k < kZBatch; ++k) {
        const uint64_t z = z0 + k;
        if (z < P.z_hi) {
          IntV<V>::load(inter + z * plane + g, v[k]);
          if (BAND) {
            int32_t c[V];
            IntV<V>::load(band + (z - P.z_lo) * band_stride, c);
#pragma unroll
            for (int j = 0; j < V; ++j) v[k][j] += c[j];
          }
        } else {
#pragma unroll
          for (int j = 0; j < V; ++j) v[k][j] = 0;
        }
      }
#pragma unroll
      for (int k = 0; k < kZBatch; ++k) {
        const uint64_t z = z0 + k;
        float f[V];
#pragma unroll
        for (int j = 0; j < V; ++j) {
          run[j] += v[k][j];
          f[j] = value(P, run[j]);
        }
        if (z < P.z_hi) store_values<V>(P.out + z * plane + g, f);
      }
    }
    if (P.z_hi < P.nz) {
#pragma unroll
      for (int c = 0; c < V; ++c) P.plane[g + c] = run[c];
    }
  }
}

// Blocks of one resident wave (at most `want`) for a kernel.
template <class Kernel>
unsigned wave_blocks(Kernel kernel, int threads, size_t smem, int num_sms, uint64_t want) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const uint64_t wave = static_cast<uint64_t>(per_sm) * static_cast<uint64_t>(num_sms);
  return static_cast<unsigned>(std::max<uint64_t>(1, std::min(want, wave)));
}

}  // namespace

uint64_t lorenzo_tiles_1d(uint64_t n) { return (n + k1Tile - 1) / k1Tile; }

uint32_t lorenzo_rows_per_band(uint64_t nx) {
  if (nx <= kWarpBandMaxRow) return 8;
  return static_cast<uint32_t>(std::min<uint64_t>(32, std::max<uint64_t>(1, 16384 / nx)));
}

size_t lorenzo_band_smem(uint32_t yb, uint64_t nx) {
  return nx <= kWarpBandMaxRow ? 0 : 4ull * yb * nx;
}

cudaError_t launch_outlier_prefix(const int32_t* val, uint64_t n_out, int32_t radius,
                                  int32_t* corr, cudaStream_t st) {
  k_outlier_prefix<<<1, k1ScanThreads, 0, st>>>(val, n_out, radius, corr);
  return cudaGetLastError();
}

cudaError_t launch_lorenzo_1d(const LorenzoParams& P, int num_sms, cudaStream_t st) {
  const uint64_t tiles = lorenzo_tiles_1d(P.n);
  if (!tiles) return cudaSuccess;
  k_lorenzo_1d_sums<<<wave_blocks(k_lorenzo_1d_sums, kThreads, 0, num_sms, tiles), kThreads, 0,
                      st>>>(P, tiles);
  k_lorenzo_1d_scan<<<1, k1ScanThreads, 0, st>>>(P.tile_prefix, tiles);
  k_lorenzo_1d<<<static_cast<unsigned>(tiles), kThreads, 0, st>>>(P);
  return cudaGetLastError();
}

template <bool BAND>
void launch_zscan(const LorenzoParams& P, int num_sms, cudaStream_t st) {
  const uint64_t plane = P.ny * P.nx;
  auto go = [&](auto kernel, uint64_t units) {
    kernel<<<wave_blocks(kernel, kColThreads, 0, num_sms, (units + kColThreads - 1) / kColThreads),
             kColThreads, 0, st>>>(P);
  };
  if (P.nx % 4 == 0)
    go(k_lorenzo_zscan<4, BAND>, plane / 4);
  else if (P.nx % 2 == 0)
    go(k_lorenzo_zscan<2, BAND>, plane / 2);
  else
    go(k_lorenzo_zscan<1, BAND>, plane);
}

template <int K, int R>
void launch_warpband(const LorenzoParams& P, int num_sms, cudaStream_t st) {
  const uint64_t warps = (P.z_hi - P.z_lo) * P.nb;
  const uint64_t want = (warps + kWarpBandThreads / 32 - 1) / (kWarpBandThreads / 32);
  if (P.nx % 8 == 0) {
    auto k = k_lorenzo_warpband<K, true, R>;
    k<<<wave_blocks(k, kWarpBandThreads, 0, num_sms, want), kWarpBandThreads, 0, st>>>(P);
  } else {
    auto k = k_lorenzo_warpband<K, false, 1>;
    k<<<wave_blocks(k, kWarpBandThreads, 0, num_sms, want), kWarpBandThreads, 0, st>>>(P);
  }
}

bool lorenzo_slice_path(uint64_t nx, uint64_t nz, int num_sms) {
  return nx <= kWarpBandMaxRow && nz >= 2ull * static_cast<uint64_t>(num_sms);
}

template <int K, int R>
void launch_slice(const LorenzoParams& P, int num_sms, cudaStream_t st) {
  const size_t smem = 4ull * kSliceWarps * P.nx;
  const uint64_t nzc = P.z_hi - P.z_lo;
  if (P.nx % 8 == 0) {
    auto k = k_lorenzo_slice<K, true, R>;
    k<<<wave_blocks(k, kSliceThreads, smem, num_sms, nzc), kSliceThreads, smem, st>>>(P);
  } else {
    auto k = k_lorenzo_slice<K, false, 1>;
    k<<<wave_blocks(k, kSliceThreads, smem, num_sms, nzc), kSliceThreads, smem, st>>>(P);
  }
}

cudaError_t launch_lorenzo_whole_slices(const LorenzoParams& P, int num_sms, cudaStream_t st) {
  const uint64_t nzc = P.z_hi - P.z_lo;
  if (!nzc || !P.ny || !P.nx) return cudaSuccess;
  const uint64_t chunks = (P.nx + 255) / 256;
  if (chunks == 1)
    launch_slice<1, 4>(P, num_sms, st);
  else if (chunks == 2)
    launch_slice<2, 4>(P, num_sms, st);
  else if (chunks == 3)
    launch_slice<3, 2>(P, num_sms, st);
  else
    launch_slice<4, 1>(P, num_sms, st);
  launch_zscan<false>(P, num_sms, st);
  return cudaGetLastError();
}

cudaError_t launch_lorenzo_slices(const LorenzoParams& P, int num_sms, cudaStream_t st) {
  const uint64_t nzc = P.z_hi - P.z_lo;
  if (!nzc || !P.ny || !P.nx) return cudaSuccess;
  if (P.nx <= kWarpBandMaxRow) {
    const uint64_t chunks = (P.nx + 255) / 256;
    if (chunks == 1)
      launch_warpband<1, 4>(P, num_sms, st);
    else if (chunks == 2)
      launch_warpband<2, 4>(P, num_sms, st);
    else if (chunks == 3)
      launch_warpband<3, 2>(P, num_sms, st);
    else
      launch_warpband<4, 2>(P, num_sms, st);
  } else {
    const size_t smem = lorenzo_band_smem(P.yb, P.nx);
    const bool vec = P.nx % 8 == 0;
    if (smem > 48 * 1024) {
      cudaError_t e = vec ? cudaFuncSetAttribute(k_lorenzo_band<true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(smem))
                          : cudaFuncSetAttribute(k_lorenzo_band<false>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(smem));
      if (e != cudaSuccess) return e;
    }
    const unsigned band_blocks = static_cast<unsigned>(nzc * P.nb);
    if (vec)
      k_lorenzo_band<true><<<band_blocks, kThreads, smem, st>>>(P);
    else
      k_lorenzo_band<false><<<band_blocks, kThreads, smem, st>>>(P);
  }
  const uint64_t scan_units = nzc * P.nx;
  k_lorenzo_bandscan<<<wave_blocks(k_lorenzo_bandscan, kColThreads, 0, num_sms,
                                   (scan_units + kColThreads - 1) / kColThreads),
                       kColThreads, 0, st>>>(P);
  launch_zscan<true>(P, num_sms, st);
  return cudaGetLastError();
}

}  // namespace hd
