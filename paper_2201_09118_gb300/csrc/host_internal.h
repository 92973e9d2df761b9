// host_internal.h -- host-side helpers shared by the C-ABI translation units.
#pragma once

#include <cstdint>

namespace hd {

// Optimal code lengths (<= max_len) for a histogram; lengths_out[alphabet].
int build_code_lengths(const uint64_t* freq, uint32_t alphabet, uint32_t max_len,
                       uint8_t* lengths_out);

// Canonical codewords for a length table (RFC 1951 Sec. 3.2.2 assignment).
// Returns HD_ERR_ARG for lengths > 32 or a Kraft sum above 1.
int canonical_codewords(const uint8_t* lengths, uint32_t alphabet, uint32_t* codes);

// Units a stream of nbits occupies with subsequences of S bits (incl. guard).
inline uint64_t stream_words(uint64_t nbits, uint32_t S) {
  const uint64_t nsub = (nbits + S - 1) / S;
  return nsub * (S / 32) + 1;
}

}  // namespace hd
