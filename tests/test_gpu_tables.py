"""The per-prefix decode tables the kernels build (first-level entries, length
table and run table, read back through hd_inspect_tables) against a walk of
the canonical codes written here from their definition (Sec. II-B; the codes
themselves from the oracle's RFC 1951 assignment, pinned in test_oracle.py).

For every K-bit prefix p the expected entries follow from the codes alone:
  * a code of at most K bits that p starts with: its length and symbol; the
    run entry counts the codes that lie wholly within p's K bits, decoded one
    after another (at most 7), and the bits they take; the two-code entry
    holds the first two of them when there are two and the alphabet's
    symbols fit 10 bits;
  * otherwise the codes longer than K bits that start with p: the shortest
    length, and whether the prefix is "mixed" (codes of several lengths under
    it, or windows under it that are no code); no code at all reads as 33.
Integer tables, so the comparison is exact.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MIXED16 = 0x800
WALK8 = 0x80


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_09118_gb300 import hd
    c = hd.Context(0)
    yield c
    c.close()


def expected_tables(lengths, K):
    lengths = np.asarray(lengths, np.int64)
    codes = oracle.canonical_codes(lengths.astype(np.uint8)).astype(np.int64)
    short = {}  # (length, code) -> symbol, codes of at most K bits
    long_by_prefix = {}  # prefix -> list of lengths of longer codes under it
    for s in np.nonzero(lengths)[0]:
        L, cw = int(lengths[s]), int(codes[s])
        if L <= K:
            short[(L, cw)] = int(s)
        else:
            long_by_prefix.setdefault(cw >> (L - K), []).append(L)
    n = 1 << K
    lut16 = np.zeros(n, np.uint16)
    len8 = np.zeros(n, np.uint8)
    run8 = np.zeros(n, np.uint8)
    pair = np.zeros(n, np.uint32)
    A = lengths.size

    def code_at(p, used):
        # the code of at most K - used bits at bit offset `used` of prefix p
        rem = K - used
        for L in range(1, rem + 1):
            cw = (p >> (rem - L)) & ((1 << L) - 1)
            if (L, cw) in short:
                return L, short[(L, cw)]
        return None

    for p in range(n):
        first = code_at(p, 0)
        if first is not None:
            L, s = first
            lut16[p] = (L << 12) | (s & 0xFFF)
            len8[p] = L
            used, m = L, 1
            second = None
            while m < 7 and used < K:
                nxt = code_at(p, used)
                if nxt is None:
                    break
                if m == 1:
                    second = nxt
                used += nxt[0]
                m += 1
            run8[p] = (m << 4) | used
            if second is not None and A <= 1024:
                pair[p] = ((2 << 30) | (L << 26) | (second[0] << 22) | ((second[1] & 0x3FF) << 10)
                           | (s & 0x3FF))
            else:
                pair[p] = (1 << 30) | (L << 26) | (s & 0xFFF)
        else:
            ls = long_by_prefix.get(p, [])
            if not ls:
                lmin, mixed = 33, True
            else:
                lmin = min(ls)
                covered = sum(2 ** (32 - L) for L in ls)
                mixed = min(ls) != max(ls) or covered != 2 ** (32 - K)
            lut16[p] = lmin | (MIXED16 if mixed else 0)
            len8[p] = (WALK8 | lmin) if mixed else lmin
            run8[p] = 0
            pair[p] = lut16[p]
    return {"lut16": lut16, "len8": len8, "run8": run8, "pair": pair}


def fibonacci_lengths():
    fib = [1, 1]
    while len(fib) < 34:
        fib.append(fib[-1] + fib[-2])
    return oracle.code_lengths(np.array(fib, np.uint64), 32)


def skew_freq():
    k = np.arange(1024)
    f = np.where(np.abs(k - 512) <= 120, np.floor(3e4 * np.exp(-np.abs(k - 512) / 6.0)), 0)
    f = np.maximum(f, (np.abs(k - 512) <= 120).astype(np.float64))
    f[512] = 4e6
    return f.astype(np.uint64)


CODEBOOKS = {
    # lengths {1, 2, 3, 3}: runs of short codes end exactly at K bits
    "1-2-3-3": lambda: np.array([1, 2, 3, 3], np.uint8),
    # depths up to 32: codes far beyond the first level, long prefixes of one
    # length and mixed ones
    "fibonacci32": fibonacci_lengths,
    # a 1-bit code for the centre symbol (fields under 1.25 bits per code)
    # with a tail of codes up to 20+ bits
    "skew": lambda: oracle.code_lengths(skew_freq()),
    # a dense 1024-symbol codebook (about 9 bits per code) with codes of 14+
    "dense": lambda: oracle.code_lengths(
        oracle.histogram(synth.laplace_codes(400000, scale=60.0, seed=4), 1024)
        .astype(np.uint64)),
    # an incomplete code (one used symbol: Kraft sum 1/2): prefixes with no code
    "one_symbol": lambda: np.array([0, 0, 1, 0, 0, 0, 0, 0], np.uint8),
    # 4096 symbols: symbols past 10 bits, so no two-code entries
    "wide4096": lambda: oracle.code_lengths(
        oracle.histogram(synth.laplace_codes(300000, scale=3.0, center=2048, alphabet=4096,
                                             seed=5), 4096).astype(np.uint64)),
}


@pytest.mark.parametrize("K", [8, 11, 13, 15])
@pytest.mark.parametrize("book", sorted(CODEBOOKS))
def test_tables_match_the_canonical_codes(ctx, book, K):
    lengths = np.asarray(CODEBOOKS[book](), np.uint8)
    A = max(2, lengths.size)
    dev = torch.from_numpy(np.ascontiguousarray(lengths)).cuda()
    got = ctx.inspect_tables(dev, A, K)
    want = expected_tables(lengths, K)
    for name in ("lut16", "len8", "run8", "pair"):
        bad = np.nonzero(got[name] != want[name])[0]
        assert bad.size == 0, (name, [(int(p), int(got[name][p]), int(want[name][p]))
                                      for p in bad[:6]])


def test_tables_reject_a_length_table_that_is_no_prefix_code(ctx):
    from paper_2201_09118_gb300 import hd
    dev = torch.from_numpy(np.array([1, 1, 1], np.uint8)).cuda()  # Kraft sum 3/2
    with pytest.raises(hd.HDError) as e:
        ctx.inspect_tables(dev, 3, 10)
    assert e.value.code == hd.HD_ERR_CORRUPT
