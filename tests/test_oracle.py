"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints for its worked examples (tests/golden/), a textbook worked example
(RFC 1951), closed forms (Fibonacci weights), brute-force enumeration over tiny
alphabets, and invariants that any correct prefix coder must satisfy.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------


def _codebook(spec):
    """'A=00 B=10 ...' -> (symbol letters, lengths uint8, codes uint32)."""
    letters, lens, codes = [], [], []
    for item in spec:
        s, bits = item.split("=")
        letters.append(s)
        lens.append(len(bits))
        codes.append(int(bits, 2))
    return letters, np.array(lens, np.uint8), np.array(codes, np.uint32)


def _bits_to_words(bits: str):
    n = len(bits)
    nwords = (n + 31) // 32 + 1
    w = np.zeros(nwords, np.uint32)
    for i, ch in enumerate(bits):
        if ch == "1":
            w[i >> 5] |= np.uint32(0x80000000 >> (i & 31))
    return w, n


def _words_to_bits(words, nbits):
    return "".join(str((int(words[b >> 5]) >> (31 - (b & 31))) & 1) for b in range(nbits))


def _kraft(lengths):
    return sum(Fraction(1, 2 ** int(l)) for l in lengths if l)


def _cost(freq, lengths):
    return int(sum(int(f) * int(l) for f, l in zip(freq, lengths)))


# ----------------------------------------------------------------------------
# worked examples printed in the paper
# ----------------------------------------------------------------------------


def test_listing1_decodes_example(golden):
    g = golden("listing1_selfsync.txt")
    letters, lens, codes = _codebook(g["codebook"])
    words, nbits = _bits_to_words(g["bits"][0])
    out = oracle.decode(words, nbits, codes, lens)
    assert "".join(letters[s] for s in out) == g["decode"][0]


def test_listing1_self_synchronises_after_skipped_bit(golden):
    g = golden("listing1_selfsync.txt")
    letters, lens, codes = _codebook(g["codebook"])
    words, nbits = _bits_to_words(g["bits"][0])
    out = oracle.decode(words, nbits, codes, lens, start_bit=1)
    got = "".join(letters[s] for s in out)
    assert got == g["decode_skip1"][0]
    # after the 4 wrong symbols (8 bits) the tail equals the correct decode
    assert got[4:] == g["decode"][0][4:]


def test_fig1_encoding_matches_figure_rows(golden):
    g = golden("fig1_gap_array.txt")
    letters, lens, codes = _codebook(g["codebook"])
    x = np.array([letters.index(c) for c in g["string"][0]], np.uint16)
    S = int(g["subsequence_bits"][0])
    words, nbits = oracle.encode(x, lens, codes, S)
    assert _words_to_bits(words, nbits) == g["row0"][0] + g["row1"][0]
    assert oracle.decode(words, nbits, codes, lens).tolist() == x.tolist()


def test_fig1_gap_array_paper_convention(golden):
    g = golden("fig1_gap_array.txt")
    letters, lens, codes = _codebook(g["codebook"])
    x = np.array([letters.index(c) for c in g["string"][0]], np.uint16)
    S = int(g["subsequence_bits"][0])
    words, nbits = oracle.encode(x, lens, codes, S)
    assert oracle.gap_paper(x, lens, S, nbits).tolist() == [int(v) for v in g["gap"]]
    starts_paper = [i * S + int(v) for i, v in enumerate(g["gap"])]
    assert starts_paper == [int(v) for v in g["sync_points"]]


def test_fig1_build_convention_and_self_sync(golden):
    """The non-negative convention points at the first codeword boundary at or
    after each subsequence start; the self-synchronisation fixed point finds the
    same positions from the bitstream alone."""
    g = golden("fig1_gap_array.txt")
    letters, lens, codes = _codebook(g["codebook"])
    x = np.array([letters.index(c) for c in g["string"][0]], np.uint16)
    S = int(g["subsequence_bits"][0])
    words, nbits = oracle.encode(x, lens, codes, S)
    gb = oracle.gap_build(x, lens, S, nbits)
    assert gb.tolist() == [0, 0, 1, 2]
    # relation between the conventions: the straddling codeword's length
    gp = oracle.gap_paper(x, lens, S, nbits)
    starts = np.cumsum([0] + [int(lens[s]) for s in x])
    for i in range(len(gp)):
        if gp[i] < 0:
            k = int(np.searchsorted(starts, i * S + gp[i]))
            assert gb[i] == gp[i] + int(lens[x[k]])
        else:
            assert gb[i] == 0
    sync, rounds = oracle.sync_points(words, nbits, codes, lens, S)
    assert sync.tolist() == [i * S + int(v) for i, v in enumerate(gb)]
    assert rounds >= 1


def test_table_compression_ratio_one_gap_byte_per_128_bits(golden):
    g = golden("table_compression_ratio.txt")
    ss = [float(v) for v in g["opt_self_sync"]]
    ga = [float(v) for v in g["opt_gap_array"]]
    for a, b in zip(ss, ga):
        # both printed to 2 decimals: |a - b*17/16| <= 0.005 + 0.005*17/16
        assert abs(a - b * 17.0 / 16.0) <= 0.0105
    # the oracle's format carries exactly one byte per 128-bit subsequence
    x = synth.laplace_codes(4096, seed=5)
    c = oracle.compress(x, 1024, S=128)
    nsub, nwords = oracle.stream_size(c["nbits"], 128)
    assert c["gap"].size == nsub == -(-c["nbits"] // 128)
    assert nwords == nsub * 4 + 1
    ratio = (nsub * 16 + nsub) / (nsub * 16)
    assert ratio == 17 / 16


# ----------------------------------------------------------------------------
# canonical codes
# ----------------------------------------------------------------------------


def test_rfc1951_canonical_example(golden):
    g = golden("rfc1951_canonical.txt")
    lens = np.array([int(v) for v in g["lengths"]], np.uint8)
    codes = oracle.canonical_codes(lens)
    got = [format(int(c), f"0{int(l)}b") for c, l in zip(codes, lens)]
    assert got == g["codes"]


def test_canonical_codes_prefix_free_and_ordered():
    rng = np.random.default_rng(3)
    for trial in range(20):
        A = int(rng.integers(2, 300))
        freq = rng.integers(0, 1000, A).astype(np.uint64)
        freq[rng.integers(0, A)] += 1
        freq[rng.integers(0, A)] += 1
        lens = oracle.code_lengths(freq, 32)
        codes = oracle.canonical_codes(lens)
        words = sorted((format(int(codes[s]), f"0{int(lens[s])}b"), s)
                       for s in range(A) if lens[s])
        # lexicographic order of codewords == order by (length, symbol)
        assert [s for _, s in words] == sorted(
            (s for s in range(A) if lens[s]), key=lambda s: (int(lens[s]), s))
        cw = [w for w, _ in words]
        for a, b in zip(cw, cw[1:]):
            assert not b.startswith(a)


def test_canonical_rejects_oversubscribed_lengths():
    with pytest.raises(oracle.OracleError) as e:
        oracle.canonical_codes(np.array([1, 1, 1], np.uint8))
    assert e.value.code == oracle.ERR_ARG


# ----------------------------------------------------------------------------
# Huffman lengths
# ----------------------------------------------------------------------------


def _brute_force_optimal_cost(freq, max_len):
    """min sum f*len over all length vectors with Kraft <= 1 (Kraft-McMillan)."""
    used = [f for f in freq if f > 0]
    best = None
    for ls in itertools.product(range(1, max_len + 1), repeat=len(used)):
        if sum(Fraction(1, 2 ** l) for l in ls) <= 1:
            c = sum(f * l for f, l in zip(used, ls))
            best = c if best is None else min(best, c)
    return best


@pytest.mark.parametrize("seed", range(12))
def test_huffman_cost_equals_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    A = int(rng.integers(2, 7))
    freq = rng.integers(1, 50, A).astype(np.uint64)
    lens = oracle.code_lengths(freq, 32)
    assert _cost(freq, lens) == _brute_force_optimal_cost(list(map(int, freq)), A - 1)
    assert _kraft(lens) == 1


@pytest.mark.parametrize("seed", range(8))
def test_package_merge_cost_equals_brute_force(seed):
    rng = np.random.default_rng(200 + seed)
    A = int(rng.integers(6, 10))
    L = 4
    # geometric-ish weights make the unconstrained Huffman tree deeper than L
    freq = (2.0 ** rng.uniform(0, 9, A)).astype(np.uint64) + 1
    lens = oracle.package_merge(freq, L)
    assert int(lens.max()) <= L
    assert _kraft(lens) <= 1
    assert _cost(freq, lens) == _brute_force_optimal_cost(list(map(int, freq)), L)


def test_fibonacci_weights_closed_form_and_length_limit():
    # Fibonacci weights F1..F40 give the caterpillar tree: depths 39,39,38,...,1
    fib = [1, 1]
    while len(fib) < 40:
        fib.append(fib[-1] + fib[-2])
    freq = np.array(fib, np.uint64)
    d = oracle.huffman_depths(freq)
    assert d.tolist() == [39, 39] + list(range(38, 0, -1))
    lens = oracle.code_lengths(freq, 32)
    assert int(lens.max()) == 32
    assert _kraft(lens) == 1
    # the limited code must stay a valid, decodable prefix code
    codes = oracle.canonical_codes(lens)
    x = np.repeat(np.arange(40, dtype=np.uint16), 3)
    words, nbits = oracle.encode(x, lens, codes, 64)
    assert oracle.decode(words, nbits, codes, lens).tolist() == x.tolist()


def test_kraft_equality_random_histograms():
    rng = np.random.default_rng(7)
    for _ in range(30):
        A = int(rng.choice([2, 3, 17, 256, 1024, 4096]))
        freq = rng.integers(0, 10 ** int(rng.integers(1, 6)), A).astype(np.uint64)
        freq[0] += 1
        freq[-1] += 1
        lens = oracle.code_lengths(freq, 32)
        assert _kraft(lens) == 1
        assert all((lens > 0) == (freq > 0))


# ----------------------------------------------------------------------------
# histogram (the symbol frequencies Huffman's construction starts from, Sec. II-B)
# ----------------------------------------------------------------------------


def test_histogram_fig1_string_counted_by_hand(golden):
    # BACACCBDBAAEBBA: A at 2, 4, 10, 11, 15; B at 1, 7, 9, 13, 14; C at 3, 5, 6;
    # D at 8; E at 12 (1-based positions, counted by hand)
    string = golden("fig1_gap_array.txt")["string"][0]
    assert string == "BACACCBDBAAEBBA"
    x = np.array(["ABCDE".index(ch) for ch in string], np.uint16)
    assert oracle.histogram(x, 5).tolist() == [5, 5, 3, 1, 1]
    # unused symbols of a larger alphabet count zero
    assert oracle.histogram(x, 9).tolist() == [5, 5, 3, 1, 1, 0, 0, 0, 0]


def test_histogram_against_independent_count():
    from collections import Counter
    x = synth.laplace_codes(200003, scale=40.0, seed=21)
    x[::997] = 1023  # the alphabet's last symbol
    x[5] = 0
    ref = Counter(int(v) for v in x.tolist())
    got = oracle.histogram(x, 1024)
    assert got.dtype == np.uint64 and got.size == 1024
    for sym in range(1024):
        assert int(got[sym]) == ref.get(sym, 0), sym
    assert int(got.sum()) == x.size


def test_histogram_edges_and_errors():
    assert oracle.histogram(np.zeros(0, np.uint16), 4).tolist() == [0, 0, 0, 0]
    x = np.array([65535, 0, 65535], np.uint16)
    h = oracle.histogram(x, 65536)
    assert int(h[65535]) == 2 and int(h[0]) == 1 and int(h.sum()) == 3
    with pytest.raises(oracle.OracleError) as e:
        oracle.histogram(np.array([0, 4, 1], np.uint16), 4)  # 4 is outside [0, 4)
    assert e.value.code == oracle.ERR_SYMBOL


def test_single_and_no_symbol():
    freq = np.zeros(8, np.uint64)
    assert oracle.code_lengths(freq).tolist() == [0] * 8
    freq[5] = 10
    lens = oracle.code_lengths(freq)
    assert lens.tolist() == [0, 0, 0, 0, 0, 1, 0, 0]
    codes = oracle.canonical_codes(lens)
    x = np.full(100, 5, np.uint16)
    words, nbits = oracle.encode(x, lens, codes, 64)
    assert nbits == 100
    assert oracle.decode(words, nbits, codes, lens).tolist() == x.tolist()


# ----------------------------------------------------------------------------
# encoder / decoder
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("S", [8, 64, 128, 256])
def test_round_trip_laplace(S):
    x = synth.laplace_codes(20000, seed=11)
    c = oracle.compress(x, 1024, S=S)
    assert oracle.decode(c["words"], c["nbits"], c["codes"], c["lengths"]).tolist() == x.tolist()
    # padding: whole subsequences plus a zero guard unit, and padding is zero
    nsub, nwords = oracle.stream_size(c["nbits"], S)
    assert c["words"].size == nwords
    assert _words_to_bits(c["words"], nwords * 32)[c["nbits"]:] == "0" * (nwords * 32 - c["nbits"])


def test_decode_errors():
    # incomplete code {0, 10}: '11' is no codeword
    lens = np.array([1, 2, 0], np.uint8)
    codes = np.array([0b0, 0b10, 0], np.uint32)
    words, nbits = _bits_to_words("0101100")
    with pytest.raises(oracle.OracleError) as e:
        oracle.decode(words, nbits, codes, lens)
    assert e.value.code == oracle.ERR_CORRUPT
    # truncated codeword at the end of the stream
    words, nbits = _bits_to_words("0101")
    with pytest.raises(oracle.OracleError) as e:
        oracle.decode(words, nbits, codes, lens)
    assert e.value.code == oracle.ERR_CORRUPT
    # a codebook that is not prefix-free is rejected
    with pytest.raises(oracle.OracleError):
        oracle.decode(words, 2, np.array([0b0, 0b01], np.uint32), np.array([1, 2], np.uint8))


def test_empty_stream():
    c = oracle.compress(np.zeros(0, np.uint16), 16, S=128)
    assert c["nbits"] == 0 and c["gap"].size == 0
    assert oracle.decode(c["words"], 0, c["codes"], c["lengths"]).size == 0


# ----------------------------------------------------------------------------
# gap arrays, counts, synchronisation points
# ----------------------------------------------------------------------------


def _boundaries(x, lens):
    return np.concatenate([[0], np.cumsum(lens[x].astype(np.int64))])


@pytest.mark.parametrize("S", [64, 128, 256])
def test_gap_and_counts_against_boundaries(S):
    x = synth.laplace_codes(30000, scale=6.0, seed=21)
    c = oracle.compress(x, 1024, S=S)
    b = _boundaries(x, c["lengths"])
    nsub = c["gap"].size
    starts = b[:-1]
    for i in range(nsub):
        nxt = b[np.searchsorted(b, i * S)]
        assert c["gap"][i] == nxt - i * S
        assert 0 <= c["gap"][i] <= 31
    counts = oracle.subseq_counts(x, c["lengths"], S, c["nbits"])
    assert counts.tolist() == np.bincount(starts // S, minlength=nsub).tolist()
    assert int(counts.sum()) == x.size
    gp = oracle.gap_paper(x, c["lengths"], S, c["nbits"])
    for i in range(nsub):
        k = np.searchsorted(b, i * S, side="right") - 1
        assert gp[i] == b[k] - i * S


@pytest.mark.parametrize("S", [64, 128])
def test_sync_points_equal_gap_starts(S):
    x = synth.laplace_codes(50000, scale=30.0, seed=33)
    c = oracle.compress(x, 1024, S=S)
    sync, rounds = oracle.sync_points(c["words"], c["nbits"], c["codes"], c["lengths"], S)
    assert sync.tolist() == [i * S + int(g) for i, g in enumerate(c["gap"])]
    # Huffman codes re-synchronise quickly: a handful of rounds, not nsub
    assert rounds <= 8


def test_sync_points_non_synchronising_code():
    """Equal-length codes never re-synchronise from a misaligned start, so the
    true starts can only propagate from thread 0, one subsequence per round."""
    A = 8
    lens = np.full(A, 3, np.uint8)
    codes = oracle.canonical_codes(lens)
    x = (np.arange(300) % A).astype(np.uint16)
    S = 64
    words, nbits = oracle.encode(x, lens, codes, S)
    gap = oracle.gap_build(x, lens, S, nbits)
    sync, rounds = oracle.sync_points(words, nbits, codes, lens, S)
    assert sync.tolist() == [i * S + int(g) for i, g in enumerate(gap)]
    nsub = gap.size
    # every start not on a multiple of 3 has to be fixed by propagation
    assert rounds >= nsub - 1
    with pytest.raises(oracle.OracleError) as e:
        oracle.sync_points(words, nbits, codes, lens, S, max_rounds=2)
    assert e.value.code == oracle.ERR_NOSYNC
