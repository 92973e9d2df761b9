// codebook.cpp -- host-side code-length construction for hd_build_codebook.
//
// Huffman code lengths (Sec. II-B) are computed with Moffat and Katajainen's
// in-place method on the weights sorted ascending; when the longest code
// exceeds the limit, optimal length-limited lengths come from package-merge,
// tracked here only through the number of leaves each level selects.
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <vector>

#include "hd.h"
#include "host_internal.h"

namespace hd {

// Code lengths for ascending weights w[0..m) (m >= 2).  On return len[k] is
// the length of the symbol with the k-th smallest weight.
static void huffman_sorted(const std::vector<uint64_t>& w, std::vector<uint32_t>& len) {
  const size_t m = w.size();
  std::vector<uint64_t> a(w.begin(), w.end());
  // phase 1: internal nodes, each slot holding a weight or a parent index
  size_t leaf = 2, root = 0;
  a[0] += a[1];
  for (size_t next = 1; next + 1 < m; ++next) {
    if (leaf >= m || a[root] < a[leaf]) {
      a[next] = a[root];
      a[root++] = next;
    } else {
      a[next] = a[leaf++];
    }
    if (leaf >= m || (root < next && a[root] < a[leaf])) {
      a[next] += a[root];
      a[root++] = next;
    } else {
      a[next] += a[leaf++];
    }
  }
  // phase 2: depths of the internal nodes
  a[m - 2] = 0;
  for (size_t next = m - 2; next-- > 0;) a[next] = a[a[next]] + 1;
  // phase 3: leaf depths, deepest first
  len.assign(m, 0);
  int64_t avail = 1, used = 0, depth = 0;
  int64_t r = static_cast<int64_t>(m) - 2, nx = static_cast<int64_t>(m) - 1;
  while (avail > 0) {
    while (r >= 0 && static_cast<int64_t>(a[r]) == depth) {
      ++used;
      --r;
    }
    while (avail > used) {
      len[nx--] = static_cast<uint32_t>(depth);
      --avail;
    }
    avail = 2 * used;
    ++depth;
    used = 0;
  }
}

// Package-merge for ascending weights w[0..m), limit L (m <= 2^L).  Level
// lists are built bottom-up; the selection then only needs, per level, how
// many of the first k items are leaves (a prefix of the sorted leaves) and how
// many are packages (which select the first 2*p items one level deeper).
static void package_merge_sorted(const std::vector<uint64_t>& w, uint32_t L,
                                 std::vector<uint32_t>& len) {
  const size_t m = w.size();
  std::vector<std::vector<uint64_t>> wt(L + 1);
  std::vector<std::vector<uint8_t>> is_leaf(L + 1);
  wt[L] = w;
  is_leaf[L].assign(m, 1);
  for (uint32_t l = L; l >= 2; --l) {
    const std::vector<uint64_t>& prev = wt[l];
    const size_t np = prev.size() / 2;
    std::vector<uint64_t>& cur = wt[l - 1];
    std::vector<uint8_t>& lf = is_leaf[l - 1];
    cur.reserve(m + np);
    lf.reserve(m + np);
    size_t i = 0, j = 0;
    while (i < m || j < np) {
      const bool take_leaf = (j >= np) || (i < m && w[i] <= prev[2 * j] + prev[2 * j + 1]);
      if (take_leaf) {
        cur.push_back(w[i++]);
        lf.push_back(1);
      } else {
        cur.push_back(prev[2 * j] + prev[2 * j + 1]);
        lf.push_back(0);
        ++j;
      }
    }
  }
  len.assign(m, 0);
  size_t k = 2 * m - 2;  // items chosen at the top level
  for (uint32_t l = 1; l <= L && k > 0; ++l) {
    size_t leaves = 0;
    for (size_t q = 0; q < k; ++q) leaves += is_leaf[l][q];
    for (size_t q = 0; q < leaves; ++q) len[q] += 1;
    k = 2 * (k - leaves);
  }
}

int build_code_lengths(const uint64_t* freq, uint32_t alphabet, uint32_t max_len,
                       uint8_t* lengths_out) {
  std::vector<uint32_t> sym;
  for (uint32_t s = 0; s < alphabet; ++s)
    if (freq[s]) sym.push_back(s);
  std::fill(lengths_out, lengths_out + alphabet, 0);
  const size_t m = sym.size();
  if (m == 0) return HD_OK;
  if (m == 1) {
    lengths_out[sym[0]] = 1;
    return HD_OK;
  }
  if (max_len < 32 && m > (static_cast<size_t>(1) << max_len)) return HD_ERR_ARG;
  std::stable_sort(sym.begin(), sym.end(),
                   [&](uint32_t a, uint32_t b) { return freq[a] < freq[b]; });
  std::vector<uint64_t> w(m);
  for (size_t k = 0; k < m; ++k) w[k] = freq[sym[k]];
  std::vector<uint32_t> len;
  huffman_sorted(w, len);
  if (len[0] > max_len) package_merge_sorted(w, max_len, len);
  for (size_t k = 0; k < m; ++k) lengths_out[sym[k]] = static_cast<uint8_t>(len[k]);
  return HD_OK;
}

}  // namespace hd

extern "C" int hd_build_codebook_freq(const uint64_t* freq, uint32_t alphabet, uint32_t max_len,
                                      uint8_t* lengths_out) {
  if (alphabet < 2 || alphabet > 65536 || max_len < 1 || max_len > 32) return HD_ERR_ARG;
  if (!freq || !lengths_out) return HD_ERR_ARG;
  return hd::build_code_lengths(freq, alphabet, max_len, lengths_out);
}

extern "C" int hd_build_codebook(const uint16_t* codes, uint64_t n, uint32_t alphabet,
                                 uint32_t max_len, uint8_t* lengths_out) {
  if (alphabet < 2 || alphabet > 65536 || max_len < 1 || max_len > 32) return HD_ERR_ARG;
  if ((n && !codes) || !lengths_out) return HD_ERR_ARG;
  std::vector<uint64_t> freq(alphabet, 0);
  for (uint64_t i = 0; i < n; ++i) {
    if (codes[i] >= alphabet) return HD_ERR_SYMBOL;
    ++freq[codes[i]];
  }
  return hd::build_code_lengths(freq.data(), alphabet, max_len, lengths_out);
}
