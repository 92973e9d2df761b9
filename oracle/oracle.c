/*
 * oracle.c -- CPU oracle for canonical-Huffman coding of uint16 quantization
 * codes and for the decoding the GPU path performs.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously correct
 * reference the CUDA decoder is checked against.  Only the test suite, the
 * package's smoke check and the benchmark's CPU-baseline leg load it; the
 * product library never does, and the two share no code, header or table.
 *
 * Each routine writes out the definition of what it computes:
 *   or_histogram          symbol counts
 *   or_huffman_depths     Huffman's construction (Sec. II-B): repeatedly merge
 *                         the two lightest nodes; ties broken by (weight, id),
 *                         leaves have id = symbol, merged nodes A, A+1, ...
 *   or_package_merge      optimal length-limited code lengths (Larmore and
 *                         Hirschberg's package-merge), used when the Huffman
 *                         depth exceeds the limit (32 bits here)
 *   or_code_lengths       Huffman, falling back to package-merge
 *   or_canonical_codes    canonical codewords from lengths (RFC 1951 3.2.2)
 *   or_encode             MSB-first packing of codewords into 32-bit units
 *                         (Sec. III-B2 "units"), zero padding to whole
 *                         subsequences plus one zero guard unit
 *   or_gap_build          gap array, non-negative convention: offset from the
 *                         subsequence boundary i*S to the first codeword
 *                         boundary at or after it (Sec. III-C)
 *   or_gap_paper          gap array, the paper's signed convention: offset back
 *                         to the start of the codeword that contains bit i*S
 *                         (Sec. III-C, the example [0, 0, -2, -1] of Fig. 1)
 *   or_subseq_counts      codewords starting inside each subsequence (the
 *                         per-subsequence counts that are prefix-summed into
 *                         output indices, Sec. III-B2 step 3)
 *   or_decode             decoding by walking the code tree one bit at a time
 *   or_sync_points        the self-synchronisation fixed point (Sec. III-B2,
 *                         Fig. 1): threads start at evenly spaced positions,
 *                         decode without writing past their subsequence, and a
 *                         thread's start is replaced by its predecessor's stop
 *                         position until no start changes
 *
 * Status codes: 0 ok, -1 bad argument, -2 capacity, -3 symbol without a
 * codeword, -4 corrupt stream, -5 no synchronisation within the round limit,
 * -8 out of host memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_CAPACITY (-2)
#define OR_ERR_SYMBOL (-3)
#define OR_ERR_CORRUPT (-4)
#define OR_ERR_NOSYNC (-5)
#define OR_ERR_NOMEM (-8)

/* ------------------------------------------------------------------------ */
/* histogram                                                                */
/* ------------------------------------------------------------------------ */

int or_histogram(const uint16_t *x, uint64_t n, uint32_t alphabet, uint64_t *freq) {
  if (alphabet < 1 || alphabet > 65536) return OR_ERR_ARG;
  memset(freq, 0, (size_t)alphabet * sizeof(uint64_t));
  for (uint64_t i = 0; i < n; ++i) {
    if (x[i] >= alphabet) return OR_ERR_SYMBOL;
    freq[x[i]] += 1;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Huffman code lengths                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t w;
  uint32_t id;
} hnode;

static int hless(hnode a, hnode b) { return a.w < b.w || (a.w == b.w && a.id < b.id); }

static void heap_push(hnode *h, uint32_t *size, hnode v) {
  uint32_t i = (*size)++;
  h[i] = v;
  while (i > 0) {
    uint32_t p = (i - 1) / 2;
    if (!hless(h[i], h[p])) break;
    hnode t = h[i];
    h[i] = h[p];
    h[p] = t;
    i = p;
  }
}

static hnode heap_pop(hnode *h, uint32_t *size) {
  hnode top = h[0];
  h[0] = h[--(*size)];
  uint32_t i = 0;
  for (;;) {
    uint32_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < *size && hless(h[l], h[m])) m = l;
    if (r < *size && hless(h[r], h[m])) m = r;
    if (m == i) break;
    hnode t = h[i];
    h[i] = h[m];
    h[m] = t;
    i = m;
  }
  return top;
}

/* depth[s] = depth of leaf s in the Huffman tree (0 for unused symbols).
 * A lone used symbol gets depth 1 (a one-bit code "0"). */
int or_huffman_depths(const uint64_t *freq, uint32_t alphabet, uint32_t *depth) {
  if (alphabet < 1 || alphabet > 65536) return OR_ERR_ARG;
  memset(depth, 0, (size_t)alphabet * sizeof(uint32_t));
  uint32_t used = 0;
  for (uint32_t s = 0; s < alphabet; ++s) used += freq[s] > 0;
  if (used == 0) return OR_OK;
  if (used == 1) {
    for (uint32_t s = 0; s < alphabet; ++s)
      if (freq[s]) depth[s] = 1;
    return OR_OK;
  }
  uint32_t total = 2 * alphabet;
  hnode *heap = (hnode *)malloc(sizeof(hnode) * alphabet);
  uint32_t *parent = (uint32_t *)malloc(sizeof(uint32_t) * total);
  uint32_t *d = (uint32_t *)calloc(total, sizeof(uint32_t));
  if (!heap || !parent || !d) {
    free(heap);
    free(parent);
    free(d);
    return OR_ERR_NOMEM;
  }
  uint32_t hs = 0;
  for (uint32_t s = 0; s < alphabet; ++s)
    if (freq[s]) heap_push(heap, &hs, (hnode){freq[s], s});
  uint32_t next = alphabet;
  while (hs > 1) {
    hnode a = heap_pop(heap, &hs);
    hnode b = heap_pop(heap, &hs);
    parent[a.id] = next;
    parent[b.id] = next;
    heap_push(heap, &hs, (hnode){a.w + b.w, next});
    ++next;
  }
  uint32_t root = next - 1;
  /* a parent is always created after its children: walk ids downwards */
  d[root] = 0;
  for (uint32_t id = root; id-- > alphabet;) d[id] = d[parent[id]] + 1;
  for (uint32_t s = 0; s < alphabet; ++s)
    if (freq[s]) depth[s] = d[parent[s]] + 1;
  free(heap);
  free(parent);
  free(d);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* package-merge (coin collector): optimal code lengths bounded by L          */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t w;
  int32_t leaf;  /* symbol for a leaf coin, -1 for a package */
  uint32_t a, b; /* for a package: the two items of the next deeper list */
} pm_item;

typedef struct {
  uint64_t w;
  uint32_t s;
} pm_leaf;

static int pm_leaf_cmp(const void *x, const void *y) {
  const pm_leaf *p = (const pm_leaf *)x, *q = (const pm_leaf *)y;
  if (p->w != q->w) return p->w < q->w ? -1 : 1;
  return p->s < q->s ? -1 : (p->s > q->s);
}

int or_package_merge(const uint64_t *freq, uint32_t alphabet, uint32_t L, uint8_t *len) {
  if (alphabet < 1 || alphabet > 65536 || L < 1 || L > 32) return OR_ERR_ARG;
  memset(len, 0, alphabet);
  uint32_t m = 0;
  for (uint32_t s = 0; s < alphabet; ++s) m += freq[s] > 0;
  if (m == 0) return OR_OK;
  if (m == 1) {
    for (uint32_t s = 0; s < alphabet; ++s)
      if (freq[s]) len[s] = 1;
    return OR_OK;
  }
  if (L < 32 && (uint64_t)m > (1ull << L)) return OR_ERR_ARG;
  pm_leaf *leaves = (pm_leaf *)malloc(sizeof(pm_leaf) * m);
  pm_item **lists = (pm_item **)calloc(L + 1, sizeof(pm_item *));
  uint32_t *cnt = (uint32_t *)calloc(L + 1, sizeof(uint32_t));
  uint8_t **sel = (uint8_t **)calloc(L + 1, sizeof(uint8_t *));
  if (!leaves || !lists || !cnt || !sel) goto nomem;
  {
    uint32_t k = 0;
    for (uint32_t s = 0; s < alphabet; ++s)
      if (freq[s]) leaves[k++] = (pm_leaf){freq[s], s};
    qsort(leaves, m, sizeof(pm_leaf), pm_leaf_cmp);
  }
  /* the deepest list (denomination 2^-L) holds the leaf coins only */
  lists[L] = (pm_item *)malloc(sizeof(pm_item) * m);
  if (!lists[L]) goto nomem;
  for (uint32_t i = 0; i < m; ++i) lists[L][i] = (pm_item){leaves[i].w, (int32_t)leaves[i].s, 0, 0};
  cnt[L] = m;
  /* list l-1 = merge(leaf coins, packages of adjacent pairs of list l) */
  for (uint32_t l = L; l >= 2; --l) {
    uint32_t np = cnt[l] / 2;
    lists[l - 1] = (pm_item *)malloc(sizeof(pm_item) * (m + np));
    if (!lists[l - 1]) goto nomem;
    uint32_t i = 0, j = 0, k = 0;
    while (i < m || j < np) {
      int take_leaf;
      if (i >= m) take_leaf = 0;
      else if (j >= np) take_leaf = 1;
      else take_leaf = leaves[i].w <= lists[l][2 * j].w + lists[l][2 * j + 1].w;
      if (take_leaf) {
        lists[l - 1][k++] = (pm_item){leaves[i].w, (int32_t)leaves[i].s, 0, 0};
        ++i;
      } else {
        lists[l - 1][k++] =
            (pm_item){lists[l][2 * j].w + lists[l][2 * j + 1].w, -1, 2 * j, 2 * j + 1};
        ++j;
      }
    }
    cnt[l - 1] = k;
  }
  /* choose the 2m-2 cheapest items of the top list; every leaf coin reached
   * from a chosen item adds one bit to that symbol's length */
  for (uint32_t l = 1; l <= L; ++l) {
    sel[l] = (uint8_t *)calloc(cnt[l] ? cnt[l] : 1, 1);
    if (!sel[l]) goto nomem;
  }
  for (uint32_t i = 0; i < 2 * m - 2; ++i) sel[1][i] = 1;
  for (uint32_t l = 1; l <= L; ++l) {
    for (uint32_t i = 0; i < cnt[l]; ++i) {
      if (!sel[l][i]) continue;
      const pm_item *it = &lists[l][i];
      if (it->leaf >= 0) {
        len[it->leaf] += 1;
      } else {
        sel[l + 1][it->a] = 1;
        sel[l + 1][it->b] = 1;
      }
    }
  }
  for (uint32_t l = 0; l <= L; ++l) {
    free(lists[l]);
    free(sel[l]);
  }
  free(lists);
  free(sel);
  free(cnt);
  free(leaves);
  return OR_OK;
nomem:
  if (lists)
    for (uint32_t l = 0; l <= L; ++l) free(lists[l]);
  if (sel)
    for (uint32_t l = 0; l <= L; ++l) free(sel[l]);
  free(lists);
  free(sel);
  free(cnt);
  free(leaves);
  return OR_ERR_NOMEM;
}

/* Huffman lengths; package-merge at `max_len` when the Huffman tree is deeper. */
int or_code_lengths(const uint64_t *freq, uint32_t alphabet, uint32_t max_len, uint8_t *len) {
  if (alphabet < 1 || alphabet > 65536 || max_len < 1 || max_len > 32) return OR_ERR_ARG;
  uint32_t *depth = (uint32_t *)malloc(sizeof(uint32_t) * alphabet);
  if (!depth) return OR_ERR_NOMEM;
  int rc = or_huffman_depths(freq, alphabet, depth);
  if (rc) {
    free(depth);
    return rc;
  }
  uint32_t dmax = 0;
  for (uint32_t s = 0; s < alphabet; ++s)
    if (depth[s] > dmax) dmax = depth[s];
  if (dmax <= max_len) {
    for (uint32_t s = 0; s < alphabet; ++s) len[s] = (uint8_t)depth[s];
    free(depth);
    return OR_OK;
  }
  free(depth);
  return or_package_merge(freq, alphabet, max_len, len);
}

/* ------------------------------------------------------------------------ */
/* canonical codewords (RFC 1951 3.2.2)                                      */
/* ------------------------------------------------------------------------ */

int or_canonical_codes(const uint8_t *len, uint32_t alphabet, uint32_t *code) {
  if (alphabet < 1 || alphabet > 65536) return OR_ERR_ARG;
  uint64_t bl_count[34] = {0};
  for (uint32_t s = 0; s < alphabet; ++s) {
    if (len[s] > 32) return OR_ERR_ARG;
    if (len[s]) bl_count[len[s]] += 1;
  }
  /* Kraft: sum 2^-len <= 1, in units of 2^-32 */
  uint64_t kraft = 0;
  for (uint32_t l = 1; l <= 32; ++l) kraft += bl_count[l] << (32 - l);
  if (kraft > (1ull << 32)) return OR_ERR_ARG;
  uint64_t next[34] = {0};
  uint64_t c = 0;
  for (uint32_t bits = 1; bits <= 32; ++bits) {
    c = (c + bl_count[bits - 1]) << 1;
    next[bits] = c;
  }
  for (uint32_t s = 0; s < alphabet; ++s) {
    code[s] = 0;
    if (len[s]) code[s] = (uint32_t)(next[len[s]]++);
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* stream format helpers                                                    */
/* ------------------------------------------------------------------------ */

/* number of subsequences and of 32-bit units the packed stream occupies */
void or_stream_size(uint64_t nbits, uint32_t S, uint64_t *nsub, uint64_t *nwords) {
  uint64_t ns = (nbits + S - 1) / S;
  *nsub = ns;
  *nwords = (ns * S + 31) / 32 + 1;
}

static int get_bit(const uint32_t *words, uint64_t b) {
  return (int)((words[b >> 5] >> (31 - (b & 31))) & 1u);
}

/* ------------------------------------------------------------------------ */
/* encoder                                                                  */
/* ------------------------------------------------------------------------ */

/* Appends the codeword of each symbol, most significant bit first; bit b of the
 * stream is bit 31 - (b mod 32) of unit floor(b / 32).  `code`/`len` may be any
 * prefix code (the paper's Listing 1 codebook is not canonical). */
int or_encode(const uint16_t *x, uint64_t n, const uint8_t *len, const uint32_t *code,
              uint32_t alphabet, uint32_t S, uint32_t *words, uint64_t words_cap,
              uint64_t *nbits_out, uint64_t *nwords_out) {
  if (S < 1) return OR_ERR_ARG;
  uint64_t nbits = 0;
  for (uint64_t i = 0; i < n; ++i) {
    if (x[i] >= alphabet) return OR_ERR_SYMBOL;
    if (len[x[i]] == 0) return OR_ERR_SYMBOL;
    nbits += len[x[i]];
  }
  uint64_t nsub, nwords;
  or_stream_size(nbits, S, &nsub, &nwords);
  *nbits_out = nbits;
  *nwords_out = nwords;
  if (words_cap < nwords) return OR_ERR_CAPACITY;
  memset(words, 0, nwords * sizeof(uint32_t));
  uint64_t pos = 0;
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t l = len[x[i]], c = code[x[i]];
    for (uint32_t b = l; b-- > 0;) {
      if ((c >> b) & 1u) words[pos >> 5] |= 0x80000000u >> (pos & 31);
      ++pos;
    }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* gap arrays and per-subsequence counts (from the codeword boundaries)      */
/* ------------------------------------------------------------------------ */

/* gap[i] = (first codeword boundary >= i*S) - i*S, where the boundaries are the
 * codeword starts and the stream end nbits. */
int or_gap_build(const uint16_t *x, uint64_t n, const uint8_t *len, uint32_t S, uint64_t nbits,
                 uint8_t *gap, uint64_t gap_cap) {
  uint64_t nsub = (nbits + S - 1) / S;
  if (gap_cap < nsub) return OR_ERR_CAPACITY;
  uint64_t pos = 0, k = 0; /* pos = start of codeword k */
  for (uint64_t i = 0; i < nsub; ++i) {
    uint64_t b = i * S;
    while (k < n && pos < b) {
      pos += len[x[k]];
      ++k;
    }
    /* pos is now the first boundary >= b (a codeword start, or nbits) */
    if (pos - b > 255) return OR_ERR_ARG;
    gap[i] = (uint8_t)(pos - b);
  }
  return OR_OK;
}

/* gap[i] = (start of the codeword containing bit i*S) - i*S  (<= 0). */
int or_gap_paper(const uint16_t *x, uint64_t n, const uint8_t *len, uint32_t S, uint64_t nbits,
                 int32_t *gap, uint64_t gap_cap) {
  uint64_t nsub = (nbits + S - 1) / S;
  if (gap_cap < nsub) return OR_ERR_CAPACITY;
  uint64_t start = 0, k = 0; /* codeword k occupies [start, start + len) */
  for (uint64_t i = 0; i < nsub; ++i) {
    uint64_t b = i * S;
    while (k < n && start + len[x[k]] <= b) {
      start += len[x[k]];
      ++k;
    }
    gap[i] = (int32_t)((int64_t)start - (int64_t)b);
  }
  return OR_OK;
}

/* counts[i] = number of codewords whose first bit lies in [i*S, (i+1)*S) */
int or_subseq_counts(const uint16_t *x, uint64_t n, const uint8_t *len, uint32_t S,
                     uint64_t nbits, uint32_t *counts, uint64_t cap) {
  uint64_t nsub = (nbits + S - 1) / S;
  if (cap < nsub) return OR_ERR_CAPACITY;
  memset(counts, 0, nsub * sizeof(uint32_t));
  uint64_t pos = 0;
  for (uint64_t k = 0; k < n; ++k) {
    counts[pos / S] += 1;
    pos += len[x[k]];
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* decoder: walk the code tree one bit at a time                            */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t child[2];
  int32_t sym; /* >= 0 at a leaf */
} tnode;

typedef struct {
  tnode *node;
  uint32_t count;
} tree;

static int tree_build(const uint32_t *code, const uint8_t *len, uint32_t alphabet, tree *t) {
  uint64_t cap = 1;
  for (uint32_t s = 0; s < alphabet; ++s) cap += len[s];
  t->node = (tnode *)malloc(sizeof(tnode) * cap);
  if (!t->node) return OR_ERR_NOMEM;
  t->count = 1;
  t->node[0] = (tnode){{-1, -1}, -1};
  for (uint32_t s = 0; s < alphabet; ++s) {
    uint32_t l = len[s];
    if (!l) continue;
    if (l > 32) return OR_ERR_ARG;
    int32_t cur = 0;
    for (uint32_t b = l; b-- > 0;) {
      if (t->node[cur].sym >= 0) return OR_ERR_ARG; /* a shorter codeword is a prefix */
      int bit = (int)((code[s] >> b) & 1u);
      if (t->node[cur].child[bit] < 0) {
        t->node[t->count] = (tnode){{-1, -1}, -1};
        t->node[cur].child[bit] = (int32_t)t->count++;
      }
      cur = t->node[cur].child[bit];
    }
    if (t->node[cur].sym >= 0 || t->node[cur].child[0] >= 0 || t->node[cur].child[1] >= 0)
      return OR_ERR_ARG; /* duplicate codeword, or a prefix of a longer one */
    t->node[cur].sym = (int32_t)s;
  }
  return OR_OK;
}

/* Decodes bits [start_bit, nbits) of the stream.  Errors: a bit pattern that is
 * no codeword, or a codeword cut off by nbits -> corrupt; more than out_cap
 * symbols -> capacity. */
int or_decode(const uint32_t *words, uint64_t nwords, uint64_t start_bit, uint64_t nbits,
              const uint32_t *code, const uint8_t *len, uint32_t alphabet, uint16_t *out,
              uint64_t out_cap, uint64_t *n_out) {
  if (nbits > nwords * 32 || start_bit > nbits) return OR_ERR_ARG;
  tree t = {0, 0};
  int rc = tree_build(code, len, alphabet, &t);
  if (rc) {
    free(t.node);
    return rc;
  }
  uint64_t k = 0;
  int32_t cur = 0;
  rc = OR_OK;
  for (uint64_t b = start_bit; b < nbits; ++b) {
    cur = t.node[cur].child[get_bit(words, b)];
    if (cur < 0) {
      rc = OR_ERR_CORRUPT;
      break;
    }
    if (t.node[cur].sym >= 0) {
      if (k >= out_cap) {
        rc = OR_ERR_CAPACITY;
        break;
      }
      out[k++] = (uint16_t)t.node[cur].sym;
      cur = 0;
    }
  }
  if (rc == OR_OK && cur != 0) rc = OR_ERR_CORRUPT;
  *n_out = k;
  free(t.node);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* self-synchronisation fixed point                                         */
/* ------------------------------------------------------------------------ */

/* From `pos`, decode whole codewords without writing while pos < limit.
 * A codeword that runs past nbits ends the walk at nbits.  A bit pattern that
 * is no codeword (possible from a wrong start with an incomplete code) is
 * skipped one bit at a time; from a true boundary of a valid stream neither
 * case occurs, so the fixed point below does not depend on this choice. */
static uint64_t advance(const tree *t, const uint32_t *words, uint64_t nbits, uint64_t pos,
                        uint64_t limit) {
  while (pos < limit && pos < nbits) {
    int32_t cur = 0;
    uint64_t p = pos;
    for (;;) {
      if (p >= nbits) {
        return nbits;
      }
      cur = t->node[cur].child[get_bit(words, p)];
      ++p;
      if (cur < 0) {
        p = pos + 1;
        break;
      }
      if (t->node[cur].sym >= 0) break;
    }
    pos = p;
  }
  return pos < nbits ? pos : nbits;
}

/* sync[i]: start of subsequence i's first codeword.  Round r: every thread i
 * decodes from sync[i] until it reaches (i+1)*S and stops at e[i]; then each
 * sync[i+1] that differs from e[i] is replaced by e[i].  Thread 0 starts at a
 * true boundary, so after round r at least threads 0..r hold true starts;
 * rounds stop when nothing changes (at most nsub rounds). */
int or_sync_points(const uint32_t *words, uint64_t nwords, uint64_t nbits, const uint32_t *code,
                   const uint8_t *len, uint32_t alphabet, uint32_t S, uint64_t *sync,
                   uint64_t cap, uint32_t max_rounds, uint32_t *rounds_out) {
  if (nbits > nwords * 32 || S < 1) return OR_ERR_ARG;
  uint64_t nsub = (nbits + S - 1) / S;
  if (cap < nsub) return OR_ERR_CAPACITY;
  tree t = {0, 0};
  int rc = tree_build(code, len, alphabet, &t);
  if (rc) {
    free(t.node);
    return rc;
  }
  uint64_t *e = (uint64_t *)malloc(sizeof(uint64_t) * (nsub ? nsub : 1));
  if (!e) {
    free(t.node);
    return OR_ERR_NOMEM;
  }
  for (uint64_t i = 0; i < nsub; ++i) sync[i] = i * S;
  uint32_t r = 0;
  int converged = nsub <= 1;
  while (!converged && r < max_rounds) {
    ++r;
    for (uint64_t i = 0; i < nsub; ++i) e[i] = advance(&t, words, nbits, sync[i], (i + 1) * S);
    int changed = 0;
    for (uint64_t i = 1; i < nsub; ++i) {
      if (sync[i] != e[i - 1]) {
        sync[i] = e[i - 1];
        changed = 1;
      }
    }
    converged = !changed;
  }
  *rounds_out = r;
  free(e);
  free(t.node);
  return converged ? OR_OK : OR_ERR_NOSYNC;
}
