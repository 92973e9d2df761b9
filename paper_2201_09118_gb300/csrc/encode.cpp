// encode.cpp -- host-side canonical-Huffman encoder with gap-array output
// (hd_encode).  It produces the decoder's test inputs; the paper does not
// optimise encoding (Sec. VI) and neither does this file beyond packing a
// 64-bit accumulator.
#include <cstring>
#include <vector>

#include "hd.h"
#include "host_internal.h"

namespace hd {

int canonical_codewords(const uint8_t* lengths, uint32_t alphabet, uint32_t* codes) {
  uint64_t per_len[33] = {0};
  for (uint32_t s = 0; s < alphabet; ++s) {
    if (lengths[s] > 32) return HD_ERR_ARG;
    ++per_len[lengths[s]];
  }
  per_len[0] = 0;
  uint64_t kraft = 0;  // in units of 2^-32
  for (int L = 1; L <= 32; ++L) kraft += per_len[L] << (32 - L);
  if (kraft > (1ull << 32)) return HD_ERR_ARG;
  // first code of each length: shorter codes come first, each length's block
  // starts right after the previous block, shifted to the new length
  uint64_t first[33];
  uint64_t next_code = 0;
  first[0] = 0;
  for (int L = 1; L <= 32; ++L) {
    next_code = (next_code + per_len[L - 1]) << 1;
    first[L] = next_code;
  }
  for (uint32_t s = 0; s < alphabet; ++s)
    codes[s] = lengths[s] ? static_cast<uint32_t>(first[lengths[s]]++) : 0u;
  return HD_OK;
}

}  // namespace hd

extern "C" int hd_encode(const uint16_t* codes, uint64_t n, const uint8_t* lengths,
                         uint32_t alphabet, uint32_t subseq_bits, uint32_t* words_out,
                         uint64_t words_cap, uint8_t* gap_out, uint64_t gap_cap,
                         hd_stream_info* info) {
  if (!info || !lengths || (n && !codes)) return HD_ERR_ARG;
  if (alphabet < 1 || alphabet > 65536) return HD_ERR_ARG;
  if (subseq_bits != 64 && subseq_bits != 128 && subseq_bits != 256) return HD_ERR_ARG;
  std::vector<uint32_t> cw(alphabet);
  int rc = hd::canonical_codewords(lengths, alphabet, cw.data());
  if (rc) return rc;
  uint64_t nbits = 0;
  for (uint64_t i = 0; i < n; ++i) {
    const uint16_t x = codes[i];
    if (x >= alphabet || lengths[x] == 0) return HD_ERR_SYMBOL;
    nbits += lengths[x];
  }
  const uint32_t S = subseq_bits;
  info->nbits = nbits;
  info->nsub = (nbits + S - 1) / S;
  info->nwords = hd::stream_words(nbits, S);
  if (!words_out || words_cap < info->nwords) return HD_ERR_CAPACITY;
  if (gap_out && gap_cap < info->nsub) return HD_ERR_CAPACITY;
  std::memset(words_out, 0, info->nwords * sizeof(uint32_t));

  uint64_t acc = 0;   // pending bits, most significant first
  uint32_t nacc = 0;  // number of pending bits (< 32 between symbols)
  uint64_t wi = 0;
  uint64_t pos = 0;   // stream position of the current codeword
  uint64_t sub = 0;   // next subsequence whose gap entry is still open
  for (uint64_t i = 0; i < n; ++i) {
    const uint16_t x = codes[i];
    const uint32_t L = lengths[x];
    if (gap_out) {
      while (sub * S <= pos && sub < info->nsub) {
        gap_out[sub] = static_cast<uint8_t>(pos - sub * S);
        ++sub;
      }
    }
    acc |= static_cast<uint64_t>(cw[x]) << (64 - nacc - L);
    nacc += L;
    if (nacc >= 32) {
      words_out[wi++] = static_cast<uint32_t>(acc >> 32);
      acc <<= 32;
      nacc -= 32;
    }
    pos += L;
  }
  if (nacc) words_out[wi++] = static_cast<uint32_t>(acc >> 32);
  if (gap_out) {
    while (sub < info->nsub) {
      gap_out[sub] = static_cast<uint8_t>(nbits - sub * S);
      ++sub;
    }
  }
  return HD_OK;
}
