// common.cuh -- device data structures shared by the decode-table kernel and
// the decode kernels of the GB300 Huffman decoder.
#pragma once

#include <cstdint>

namespace hd {

constexpr uint32_t kMaxCodeLen = 32;
constexpr uint32_t kTableHeaderBytes = 512;

// Decode-table header, written by the table kernel.  A decode table is, in
// order: the header (kTableHeaderBytes), the 32-bit first-level table
// (uint32[2^K]), the symbols sorted by (code length, symbol) (uint16[A]), the
// 16-bit first-level table (uint16[2^K], only when A <= 4096 and K <= 15),
// the first-level length table (uint8[2^K]) and the run table (uint8[2^K]);
// offsets below.
//
// Canonical codes occupy, for each length L, the left-aligned 32-bit interval
//   [first[L] << (32-L), (first[L] + count[L]) << (32-L)),
// and these intervals are consecutive in L, so the length of the codeword at a
// left-aligned 32-bit window w is the smallest L with w < end[L], and its rank
// among codes sorted by (length, symbol) is (w >> (32-L)) - first[L] + start[L].
struct TableHeader {
  uint32_t status;   // 0 = valid length table; else bad (Kraft sum > 1, length > 32)
  uint32_t maxlen;   // longest code length in use (0 if no symbol is used)
  uint32_t nused;    // symbols with a code
  uint32_t K;        // first-level index bits
  uint64_t end[34];  // end[L]: exclusive left-aligned limit of codes of length <= L
  uint32_t base[34]; // start[L] - first[L] (mod 2^32): rank = (w >> (32-L)) + base[L]
  uint32_t long0;    // rank of the first code longer than K (codes sorted by length)
  uint32_t minlen;   // shortest code length in use (0 if no symbol is used)
  // second-level tables of the 16-bit table (table_sub_off): first-level
  // prefixes sub_p0 .. sub_p0 + nsub - 1 hold codes longer than K bits, and
  // sub-table s resolves, by the sub_bits bits after the prefix, every code
  // of prefix sub_p0 + s that is at most K + sub_bits long
  uint32_t sub_bits;
  uint32_t nsub;
  uint32_t sub_p0;
};
static_assert(sizeof(TableHeader) <= kTableHeaderBytes, "table header too large");

// First-level entry: bit 31 clear -> (len << 16) | symbol with len <= K;
// bit 31 set -> the code is longer than K bits (or the prefix is no code):
// bits 0..7 hold the smallest length a code with this prefix can have (33 if
// none can), bits 8..15 the largest when every window with this prefix is a
// valid code (else 0xFF).  Canonical lengths grow with the window value, so
// when the two are equal every code under the prefix has that length;
// otherwise the length is found by walking end[] from the smallest.
constexpr uint32_t kLongFlag = 0x80000000u;

// 16-bit first-level entry (alphabets up to 4096, K <= 15): bits 12..15 hold
// the length (1..15) and bits 0..11 the symbol of a code of at most K bits;
// length 0 marks a longer code (or no code): bits 0..7 then hold the smallest
// length under the prefix and bit 11 is set when the prefix holds codes of
// several lengths (the length is then found by walking end[]).
constexpr uint32_t kLut16Mixed = 0x800u;

// 8-bit first-level length entry: the code length when every code under the
// prefix has the same length (this includes all codes of at most K bits);
// else 0x80 | the smallest length under the prefix (33: no code).
constexpr uint32_t kLen8Walk = 0x80u;

__host__ __device__ constexpr uint64_t table_sorted_off(uint32_t K) {
  return kTableHeaderBytes + (static_cast<uint64_t>(4) << K);
}
__host__ __device__ constexpr uint64_t table_lut16_off(uint32_t K, uint32_t A) {
  return (table_sorted_off(K) + 2ull * A + 15) & ~static_cast<uint64_t>(15);
}
__host__ __device__ constexpr uint64_t table_len8_off(uint32_t K, uint32_t A) {
  return table_lut16_off(K, A) + (static_cast<uint64_t>(2) << K);
}
// First-level run entry (uint8[2^K] after the length table): the codes that
// lie wholly within the K bits of the window, decoded one after another from
// the first: (m << 4) | bits with m in 1..7 codes; 0 when the first code is
// longer than K bits (or is no code).
__host__ __device__ constexpr uint64_t table_run8_off(uint32_t K, uint32_t A) {
  return table_len8_off(K, A) + (static_cast<uint64_t>(1) << K);
}
// Second-level tables (uint16[kSubCap] after the run table, 16-byte aligned):
// entry (s << sub_bits) | q is ((L - K) << 12) | symbol for the code of length
// L <= K + sub_bits whose first K + sub_bits bits are prefix sub_p0 + s then q,
// else 0 (a longer code, or no code: the limits are walked).
constexpr uint32_t kSubCap = 4096;
// Second-level entries in use for K first-level bits: all kSubCap below 14
// bits; half of them from 14 bits on, where fewer codes are longer than the
// first level and the one-pass decoder's shared memory holds a first-level
// table twice as large (the prefixes past the capacity keep the walk of the
// canonical limits).
__host__ __device__ constexpr uint32_t sub_cap(uint32_t K) {
  return K >= 14 ? kSubCap / 2 : kSubCap;
}
__host__ __device__ constexpr uint64_t table_sub_off(uint32_t K, uint32_t A) {
  return (table_run8_off(K, A) + (static_cast<uint64_t>(1) << K) + 15) &
         ~static_cast<uint64_t>(15);
}
// Two-code first-level entry (uint32[2^K] after the second-level tables,
// 16-byte aligned), read by the decode-and-write kernel of fields under four
// bits per code: bits 30..31 hold m, the codes of at most K bits that lie
// wholly within the prefix's K bits, counted from the first up to two.
//   m = 2: first length (bits 26..29), second length (22..25), second symbol
//          (10..19), first symbol (0..9) -- alphabets up to 1024 only;
//   m = 1: first length (26..29) and symbol (0..11);
//   m = 0: the first code is longer than K bits (or is no code): the low bits
//          as in the 16-bit entry (smallest length, kLut16Mixed).
__host__ __device__ constexpr uint64_t table_pair_off(uint32_t K, uint32_t A) {
  return table_sub_off(K, A) + 2ull * kSubCap;
}

__host__ __device__ constexpr bool lut16_usable(uint32_t K, uint32_t A) {
  return A <= 4096 && K <= 15;
}

// Per-field work description (device memory for batches, a kernel parameter
// for single fields).
struct FieldDesc {
  const uint32_t* words;   // bitstream
  uint64_t nwords;         // units readable in `words`
  uint64_t nbits;          // valid bits
  uint64_t nsub;           // decoder subsequences = ceil(nbits / S)
  const uint8_t* gap;      // gap array of the stream (NULL: self-synchronisation)
  uint32_t gap_stride;     // decoder S / stream S
  uint32_t alphabet;
  const uint8_t* lengths;  // code lengths [alphabet]
  const TableHeader* table;// decode table built from `lengths`
  uint16_t* out;           // decoded symbols [n]
  uint64_t n;              // expected symbol count
  uint64_t unit_begin;     // index of this field's first tile in the launch
  uint64_t nunits;         // tiles of this field
  uint32_t* err;           // error bits of this field
  uint8_t* gap_out;        // self-synchronisation: subsequence starts written here
  uint64_t count_begin;    // first entry of this field's per-subsequence counts
};

// Error bits (per field).
enum : uint32_t {
  kErrCode = 1u,     // a bit pattern that is no codeword
  kErrGap = 2u,      // gap entry out of range or not at a codeword boundary
  kErrCount = 4u,    // decoded symbol count differs from n
  kErrTimeout = 8u,  // a look-back wait gave up
  kErrNoSync = 16u,  // self-synchronisation hit its round cap
  kErrTable = 32u,   // invalid code-length table
  kErrOutlier = 64u, // reconstruction: code 0 at a position the outlier list lacks
};

// Sizes of a launch kept in device memory.  Graph launches read their field
// and tile counts from here (the host rewrites it before every replay), so one
// captured graph serves every batch within the capacity it was captured for.
struct LaunchHeader {
  uint64_t total_units;  // tiles
  uint32_t nfields;
  uint32_t pad;
};

struct DecodeParams {
  FieldDesc f0;             // the field when nfields == 1 and hdr == NULL
  const FieldDesc* fields;  // device array (always used when hdr != NULL)
  const LaunchHeader* hdr;  // non-NULL: nfields and total_units are read from here;
                            // the two fields below then hold the capacity
  uint32_t nfields;
  uint32_t K;               // first-level table bits for this launch
  uint32_t window;          // shared-memory output window, symbols (Alg. 1 buffer)
  uint32_t cmax;            // scratch symbols per subsequence (<= S)
  uint32_t long_cap;        // sorted symbols of long codes kept in shared memory
  uint64_t total_units;     // tiles in the launch
  uint64_t unit_lo;         // two-phase kernels: process tiles [unit_lo, unit_hi) only
  uint64_t unit_hi;         // (0: up to total_units); k_scan continues from tile_base[unit_lo]
  uint64_t* scan_end;       // k_scan also stores tile_base[unit_hi] here (host-mapped; may be NULL)
  const uint32_t* tile_list;  // k_write: tiles to process are tile_list[unit_lo .. unit_hi) (NULL: the range itself)
  uint64_t* unit_state;     // look-back state per tile (zeroed before launch)
  uint32_t* ticket;         // dynamic tile counter (zeroed before launch)
  uint32_t* abort_flag;     // set when any wait times out (zeroed before launch)
  uint64_t timeout_cycles;  // per-wait limit in SM clock cycles
  void* counts;             // two-phase decode: codewords per subsequence (u8, or u16 for S=256)
  uint32_t* tile_total;     // two-phase decode: codewords per tile
  uint64_t* tile_base;      // exclusive scan of tile_total over the launch ([units + 1])
  uint8_t* tile_a;          // self-synchronisation: start offset each tile assumed
  uint8_t* tile_e;          // self-synchronisation: tile_e[g + 1] = where tile g stopped, minus S
  uint8_t* tile_flag;       // self-synchronisation: 1 = last subsequence overran nbits
  uint8_t* tile_guess;      // self-synchronisation: guessed start offset of each tile
  // decode + 1D Lorenzo reconstruction of one field (values instead of codes):
  // k_count also sums each tile's residues, k_scan scans those sums, a tile
  // kernel adds the outlier corrections, k_write writes float32 values
  uint32_t* tile_rsum;      // residue sum (code - radius) of each tile, two's complement
  uint64_t* tile_qbase;     // q before each tile ([units + 1]; the low 32 bits count)
  uint64_t* tile_obase;     // first outlier at or after each tile's first output ([units + 1])
  float* vout;              // values [n] (16-byte aligned)
  int32_t radius;
  float ebx2;               // float32(2 eb)
  const uint64_t* out_idx;  // outlier positions, ascending [n_out]
  const int32_t* out_val;   // outlier residues [n_out]
  uint64_t n_out;
  const int32_t* out_corr;  // exclusive prefix of (residue + radius) over the outliers [n_out + 1]
  uint32_t* verr;           // kErrOutlier
  // fields of short codes: where the shortest code has 1 bit (canonically
  // the bit 0), a run of zero bits at a codeword boundary is a run of that
  // code's symbol, counted and written as a whole
  uint32_t zero_runs;
};

struct PrepParams {
  FieldDesc f0;
  const FieldDesc* fields;
  const LaunchHeader* hdr;  // as in DecodeParams
  uint32_t nfields;         // field count, or the capacity when hdr != NULL
  uint32_t table_blocks;    // blocks that build tables (each loops over fields)
  uint32_t slices;          // blocks per field table (0 = 1): each fills 1/slices of the entries
  uint32_t K;
  uint4* zero_ptr;          // region cleared before the decode kernel
  uint64_t zero_vec;        // its size in 16-byte vectors
  uint32_t zero_blocks;
};

// GPU encoder (encode_gpu.cu).
struct EncodeParams {
  const uint16_t* codes;      // symbols [n]
  uint64_t n;
  const uint8_t* lengths;     // code lengths [alphabet]
  const uint32_t* codewords;  // canonical codewords [alphabet], right-aligned
  uint32_t alphabet;
  uint32_t subseq_bits;       // S of the gap array
  uint64_t tiles;             // symbol tiles
  uint32_t* tile_bits;        // code bits per tile
  uint64_t* tile_off;         // stream offset of each tile [tiles + 1]
  uint64_t* total_out;        // stream length (may be NULL)
  uint32_t* words;            // stream, zeroed before the write kernel
  uint8_t* gap;               // gap array [nsub] or NULL
  uint64_t nsub;
  uint32_t* err;              // bit 0: a symbol without a code
};

// Lorenzo reconstruction (lorenzo.cu): codes -> residues -> prefix sums
// along every axis -> float32 values 2 eb q.
struct LorenzoParams {
  const uint16_t* codes;     // quantization codes [n], x fastest (16-byte aligned)
  float* out;                // values [n] (16-byte aligned); 2D/3D: also the int32 intermediate
  uint64_t n;
  uint64_t nx, ny, nz;       // extents (1D: nx = n, ny = nz = 1)
  int32_t radius;            // residue = code - radius; code 0 = outlier
  float ebx2;                // float32(2 eb)
  const uint64_t* out_idx;   // outlier positions, ascending [n_out]
  const int32_t* out_val;    // outlier residues [n_out]
  uint64_t n_out;
  uint32_t* err;             // error bits
  // 2D/3D: bands of yb rows within a slice; launches cover slices [z_lo, z_hi)
  uint32_t yb;
  uint64_t nb;               // bands per slice
  int32_t* band;             // per (slice of the launch, band, x): band column totals
  int32_t* plane;            // running z-sum of every (y, x) between launches [ny * nx]
  uint64_t z_lo, z_hi;
  // 1D: exclusive prefix of the residue sums of each tile
  int32_t* tile_prefix;
};

// Look-back state word: flag in bits 62..63, value in bits 0..61.
constexpr uint64_t kStateAgg = 1ull << 62;
constexpr uint64_t kStateInc = 2ull << 62;
constexpr uint64_t kStateValMask = (1ull << 62) - 1;

}  // namespace hd
