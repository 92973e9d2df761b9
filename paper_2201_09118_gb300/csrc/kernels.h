// kernels.h -- host-side launchers of the decode kernels (C++ linkage, used
// by the C-ABI layer).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "common.cuh"

namespace hd {

// Builds every field's decode table and clears the per-launch control region.
cudaError_t launch_prepare(const PrepParams& p, cudaStream_t stream);

// Bytes of a decode table with K index bits for an alphabet (256-byte multiple).
size_t table_bytes(uint32_t K, uint32_t alphabet);

struct LaunchShape {
  uint32_t S;        // decoder subsequence bits
  uint32_t threads;  // threads per block = subsequences per tile
  uint32_t window;   // output window (symbols)
  uint32_t K;        // table bits
  uint32_t cmax;     // scratch symbols per subsequence
  uint32_t long_cap; // symbols of long codes kept in shared memory
  uint32_t grid;     // persistent blocks (0: full occupancy)
  uint32_t lut16;    // 1: the decode-and-write kernel uses 16-bit first-level entries
  uint32_t runs;     // bit 0: the count kernel takes several short codes per lookup (run
                     // table); bit 1: runs of a 1-bit code are counted and written whole;
                     // bit 2 (kShapePairs): the decode-and-write kernel of 16-bit tables
                     // takes two codes per lookup (two-code table, S up to 256)
  uint32_t decoder;  // 0 automatic, 1 two phases, 2 one pass (hd_config.decoder)
};

constexpr uint32_t kShapePairs = 4u;

// Dynamic shared memory of the single-pass gap-array kernel.
size_t decode_smem_bytes(const LaunchShape& s);

// Two-phase gap-array decode (count kernel, then decode-and-write kernel).
cudaError_t launch_decode_two_phase(const DecodeParams& p, const LaunchShape& s, int num_sms,
                                    cudaStream_t stream);

// Dynamic shared memory of the decode-and-write kernel (s.window = window).
size_t two_phase_smem_bytes(const LaunchShape& s);

// Dynamic shared memory of the count kernel.
size_t count_smem_bytes(const LaunchShape& s);

// Bytes per stored codeword count for subsequences of S bits.
size_t count_bytes_per_subsequence(uint32_t S);

// One kernel of the two-phase gap-array decode, for launches over a tile
// range (p.unit_lo, p.unit_hi) such as the chunks of a pipelined host decode.
enum class Phase { kCount, kScan, kWrite };
cudaError_t launch_phase(const DecodeParams& p, const LaunchShape& s, Phase phase, int num_sms,
                         cudaStream_t stream);

// Sorts the tiles of a launch into nclass window classes by codeword count
// (class c: counts in (c*unit, (c+1)*unit], the last class unbounded);
// counts[c] (zeroed by the caller) receives the class sizes and
// lists[c*cap ..] the tiles.  For CR-class decodes (Sec. IV-C, Algorithm 2).
cudaError_t launch_classify(const DecodeParams& p, uint32_t unit, uint32_t nclass,
                            uint32_t* counts, uint32_t* lists, uint64_t cap, cudaStream_t stream);

// Decode + 1D Lorenzo reconstruction of one gap-array field (float32 values
// to p.vout instead of codes): the count kernel also sums each tile's
// residues (symbol tables), the tile scan scans both, a kernel adds each
// tile's outlier corrections (p.out_corr: exclusive prefix of residue +
// radius over the outliers) and the decode-and-write kernel writes values.
cudaError_t launch_decode_values(const DecodeParams& p, const LaunchShape& s, int num_sms,
                                 cudaStream_t stream);

// Tile scan and decode-and-write kernel, for fields whose counts and gap
// entries are already in place (self-synchronisation writes them).
cudaError_t launch_write(const DecodeParams& p, const LaunchShape& s, int num_sms,
                         cudaStream_t stream);

// Self-synchronisation (Sec. III-B, IV-A) without waiting between tiles: the
// synchronising kernel guesses each tile's first start and writes per-
// subsequence starts (F.gap_out) and codeword counts, tile totals and tile
// links; a one-block-per-field kernel then re-synchronises, in order, the
// tiles whose guess was wrong.
cudaError_t launch_sync(const DecodeParams& p, const LaunchShape& s, int num_sms,
                        cudaStream_t stream);

// Dynamic shared memory of the synchronising kernels.
size_t sync_smem_bytes(const LaunchShape& s);

// Single-pass gap-array decode (Sec. III-C): one persistent kernel whose
// tiles take their output offsets from a look-back over per-tile states
// (p.unit_state, p.ticket, p.abort_flag zeroed before the launch); needs no
// per-subsequence scratch in global memory.
cudaError_t launch_decode_single_pass(const DecodeParams& p, const LaunchShape& s, int num_sms,
                                      cudaStream_t stream);

// One-pass gap-array decode of a single field with warp-sized tiles
// (decode_warp.cu): s.threads / 32 warps per block in a cooperative launch,
// each warp decoding tiles of 32 subsequences (round-robin over the grid's
// warps) once into a column scratch of s.cmax symbols per lane, offsets from a
// look-back over p.unit_state (one state per tile, zeroed with p.abort_flag
// before the launch), Algorithm 1's window per warp.
cudaError_t launch_decode_warp(const DecodeParams& p, const LaunchShape& s, int num_sms,
                               cudaStream_t stream);

// Dynamic shared memory of the one-pass decoder.
size_t warp_decode_smem_bytes(const LaunchShape& s);

// GPU encoder: symbol tiles of a stream of n symbols; per-tile code bits and
// their scan (tile_off[tiles] = stream bits); then the stream and gap array.
uint64_t encode_tiles(uint64_t n);
cudaError_t launch_histogram(const uint16_t* codes, uint64_t n, uint32_t alphabet,
                             unsigned long long* hist, uint32_t* err, int num_sms,
                             cudaStream_t stream);
cudaError_t launch_encode_count(const EncodeParams& e, int num_sms, cudaStream_t stream);
cudaError_t launch_encode_write(const EncodeParams& e, int num_sms, cudaStream_t stream);

// Lorenzo reconstruction (lorenzo.cu).  1D: tile sums, their scan and the
// reconstruction pass (P.tile_prefix holds lorenzo_tiles_1d(n) entries).  2D/3D:
// band, band-scan and z kernels over the slices [P.z_lo, P.z_hi); P.yb =
// lorenzo_rows_per_band(nx); shared memory of the band kernel:
// lorenzo_band_smem(P.yb, P.nx) (0 for rows up to 1024 codes).
uint64_t lorenzo_tiles_1d(uint64_t n);
uint32_t lorenzo_rows_per_band(uint64_t nx);
size_t lorenzo_band_smem(uint32_t yb, uint64_t nx);
cudaError_t launch_lorenzo_1d(const LorenzoParams& p, int num_sms, cudaStream_t stream);
cudaError_t launch_lorenzo_slices(const LorenzoParams& p, int num_sms, cudaStream_t stream);
// Slice path for 3D grids: one block per slice (x and y prefixes), then the
// z kernel; used when lorenzo_slice_path(nx, nz, num_sms).  Needs no band or
// plane buffers (one launch covers all slices).
bool lorenzo_slice_path(uint64_t nx, uint64_t nz, int num_sms);
// corr[k] = sum over outliers j < k of (val[j] + radius), k = 0 .. n_out.
cudaError_t launch_outlier_prefix(const int32_t* val, uint64_t n_out, int32_t radius,
                                  int32_t* corr, cudaStream_t stream);
cudaError_t launch_lorenzo_whole_slices(const LorenzoParams& p, int num_sms, cudaStream_t stream);

}  // namespace hd
