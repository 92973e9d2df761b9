"""GPU parity: the CUDA decoder (through the C ABI) against the CPU oracle.

Every stream decoded here is produced by the oracle's encoder and every
expected value is the oracle's decode (which the pins in test_oracle.py tie to
the paper).  Decoding is integer work, so parity is bit-exact.
"""
import zlib

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CANARY = 0xABCD


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_09118_gb300 import hd
    c = hd.Context(0)
    yield c
    c.close()


def dev_field(c, with_gap=True):
    from paper_2201_09118_gb300 import hd
    enc = {"words": c["words"], "gap": c["gap"], "nbits": c["nbits"], "subseq_bits": c["S"]}
    return hd.DeviceField.upload(enc, c["lengths"], c["n"], with_gap=with_gap)


def run_decode(ctx, c, with_gap=True, stream=None):
    f = dev_field(c, with_gap)
    out = torch.full((c["n"] + 64,), CANARY, dtype=torch.int32).to(torch.int16).cuda()
    ctx.decode(f, out, stream)
    st = ctx.status(stream)
    res = out.cpu().numpy().view(np.uint16)
    return st, res


def expect(c):
    return oracle.decode(c["words"], c["nbits"], c["codes"], c["lengths"], n_cap=max(1, c["n"]))


def check(ctx, c, with_gap=True):
    from paper_2201_09118_gb300 import hd
    st, res = run_decode(ctx, c, with_gap)
    assert st == hd.HD_OK
    ref = expect(c)
    assert ref.size == c["n"]
    got = res[:c["n"]]
    if not np.array_equal(got, ref):
        bad = np.nonzero(got != ref)[0]
        raise AssertionError(f"{bad.size} mismatches, first at {bad[:8].tolist()}")
    assert np.all(res[c["n"]:] == np.uint16(CANARY)), "write past the output"


# ---------------------------------------------------------------------------


@pytest.mark.parametrize("with_gap", [True, False], ids=["gap", "selfsync"])
def test_laplace_2pow20(ctx, with_gap):
    x = synth.laplace_codes(1 << 20, scale=2.0, seed=1000)
    c = oracle.compress(x, 1024, S=128)
    check(ctx, c, with_gap)


def test_sync_points_equal_gap_array(ctx):
    x = synth.laplace_codes(300001, scale=20.0, seed=77)
    for S in (64, 128, 256):
        c = oracle.compress(x, 1024, S=S)
        f = dev_field(c, with_gap=False)
        nsub = c["gap"].size
        gout = torch.full((nsub + 16,), 255, dtype=torch.uint8, device="cuda")
        ctx.sync_points(f, gout)
        assert ctx.status() == 0
        got = gout.cpu().numpy()
        sync, _ = oracle.sync_points(c["words"], c["nbits"], c["codes"], c["lengths"], S)
        ref = (sync - np.arange(nsub, dtype=np.uint64) * S).astype(np.uint8)
        assert np.array_equal(got[:nsub], ref)
        assert np.array_equal(got[:nsub], c["gap"])
        assert np.all(got[nsub:] == 255)


# strategy, decoder: gap arrays through the two-phase kernels (1) and the
# one-pass kernel (2); self-synchronisation always runs two phases
STRATEGIES = [(True, 1), (True, 2), (False, 0)]
STRATEGY_IDS = ["gap-2phase", "gap-1pass", "selfsync"]


@pytest.mark.parametrize("S", [64, 128, 256])
@pytest.mark.parametrize("threads", [128, 256, 512])
@pytest.mark.parametrize("with_gap,decoder", STRATEGIES, ids=STRATEGY_IDS)
def test_launch_shapes(ctx, S, threads, with_gap, decoder):
    x = synth.laplace_codes(200003, scale=30.0, seed=S + threads)
    c = oracle.compress(x, 1024, S=S)
    try:
        for window, K in ((S, 8), (1024, 11), (0, 12), (8192, 13), (0, 14), (2048, 15)):
            ctx.set_config(subseq_bits=S, threads=threads, window=max(window, S) if window else 0,
                           lut_bits=K, decoder=decoder)
            check(ctx, c, with_gap)
            if with_gap:
                assert ctx.get_config()["decoder"] == decoder
    finally:
        ctx.reset_config()


def mixed_cr_codes(n_seg=8, seg=1 << 18, seed=77):
    """A field whose compressibility changes along it: segments quantized at
    error bounds from 1e-2 (about 1 bit per code) to 1e-6 (about 8 bits)."""
    parts = []
    for k in range(n_seg):
        eb = [1e-2, 1e-6, 1e-3, 1e-5, 1e-2, 1e-4, 1e-6, 1e-2][k % 8]
        parts.append(synth.smooth_codes_1d(seg, eb, alphabet=1024, seed=seed + k))
    return np.concatenate(parts)


@pytest.mark.parametrize("classes", [2, 8, 32])
@pytest.mark.parametrize("threads", [128, 512])
def test_cr_class_launches(ctx, classes, threads):
    # Algorithm 2 shaping: tiles sorted into window classes, one launch per class
    x = mixed_cr_codes()
    c = oracle.compress(x, 1024, S=128)
    try:
        ctx.set_config(threads=threads, cr_classes=classes)
        check(ctx, c, True)
        assert ctx.get_config()["cr_classes"] == classes
        # corrupt count still detected, nothing written past n
        cc = dict(c)
        cc["n"] = c["n"] - 1
        st, res = run_decode(ctx, cc, True)
        assert st == hd_codes().HD_ERR_CORRUPT
        assert np.all(res[cc["n"]:] == np.uint16(CANARY))
    finally:
        ctx.reset_config()


def hd_codes():
    from paper_2201_09118_gb300 import hd
    return hd


@pytest.mark.parametrize("dec_S", [128, 256, 512])
def test_decoder_subsequence_multiple_of_stream(ctx, dec_S):
    x = synth.laplace_codes(100000, scale=3.0, seed=5)
    c = oracle.compress(x, 1024, S=64)
    try:
        ctx.set_config(subseq_bits=dec_S)
        check(ctx, c, True)
    finally:
        ctx.reset_config()


@pytest.mark.parametrize("with_gap,decoder", STRATEGIES, ids=STRATEGY_IDS)
@pytest.mark.parametrize("case", ["n1", "n2", "n3", "one_symbol", "two_symbols_skew",
                                  "fibonacci32", "alphabet256", "alphabet4096", "skew1e-2",
                                  "uniform_equal_lengths", "ragged"])
def test_edge_cases(ctx, case, with_gap, decoder):
    rng = np.random.default_rng(zlib.crc32(case.encode()))
    A = 1024
    if case == "n1":
        x = np.array([517], np.uint16)
    elif case == "n2":
        x = np.array([3, 900], np.uint16)
    elif case == "n3":
        x = np.array([3, 900, 3], np.uint16)
    elif case == "one_symbol":
        x = np.full(300000, 512, np.uint16)
    elif case == "two_symbols_skew":
        x = np.where(rng.random(200000) < 0.999, 512, 7).astype(np.uint16)
    elif case == "fibonacci32":
        # Fibonacci histogram F1..F34: Huffman depth 33, limited to 32 bits
        fib = [1, 1]
        while len(fib) < 34:
            fib.append(fib[-1] + fib[-2])
        x = rng.permutation(np.repeat(np.arange(34, dtype=np.uint16), fib))
        A = 64
    elif case == "alphabet256":
        x = synth.smooth_codes_1d(150000, 1e-5, alphabet=256, seed=8)
        A = 256
    elif case == "alphabet4096":
        x = synth.smooth_codes_1d(150000, 1e-6, alphabet=4096, seed=9)
        A = 4096
    elif case == "skew1e-2":
        x = synth.smooth_codes_1d(400000, 1e-2, seed=10)
    elif case == "uniform_equal_lengths":
        x = (np.arange(70000) % 8).astype(np.uint16)
        A = 8
    else:  # ragged
        x = synth.laplace_codes(777777, scale=7.0, seed=11)
    c = oracle.compress(x, A, S=128)
    if case == "fibonacci32":
        assert int(c["lengths"].max()) == 32
    try:
        ctx.set_config(decoder=decoder)
        check(ctx, c, with_gap)
    finally:
        ctx.reset_config()


def test_decode_host(ctx):
    from paper_2201_09118_gb300 import hd
    x = synth.laplace_codes(500000, scale=4.0, seed=12)
    c = oracle.compress(x, 1024, S=128)
    enc = {"words": c["words"], "gap": c["gap"], "nbits": c["nbits"], "subseq_bits": 128}
    got = ctx.decode_host(enc, c["lengths"], c["n"])
    assert np.array_equal(got, expect(c))
    got2 = ctx.decode_host(enc, c["lengths"], c["n"], with_gap=False)
    assert np.array_equal(got2, expect(c))
    assert hd.HD_OK == 0


@pytest.mark.parametrize("shape", [None, {"subseq_bits": 256, "threads": 512, "lut_bits": 14},
                                   {"subseq_bits": 128, "threads": 128, "lut_bits": 12}])
def test_decode_host_pipelined(ctx, shape):
    # large enough to be copied, decoded and copied back in overlapped chunks
    from paper_2201_09118_gb300 import hd
    x = synth.laplace_codes(1 << 24, scale=30.0, seed=15)
    c = oracle.compress(x, 1024, S=128)
    enc = {"words": c["words"], "gap": c["gap"], "nbits": c["nbits"], "subseq_bits": 128}
    try:
        if shape:
            ctx.set_config(**shape)
        out = np.full(c["n"] + 32, CANARY, dtype=np.uint16)
        l0 = ctx.launch_count()
        got = ctx.decode_host(enc, c["lengths"], c["n"], out=out)
        assert ctx.launch_count() - l0 > 4  # several chunks
        assert np.array_equal(got, expect(c))
        assert np.all(out[c["n"]:] == CANARY)
        # a count that does not match the stream is reported, nothing written past n
        out2 = np.full(c["n"] + 32, CANARY, dtype=np.uint16)
        with pytest.raises(hd.HDError) as e:
            ctx.decode_host(enc, c["lengths"], c["n"] - 1, out=out2)
        assert e.value.code == hd.HD_ERR_CORRUPT
        assert np.all(out2[c["n"] - 1:] == CANARY)
    finally:
        ctx.reset_config()


def test_batch_mixed_fields(ctx):
    from paper_2201_09118_gb300 import hd
    specs = synth.batch_spec(12, lo=1 << 10, hi=1 << 18, seed=55)
    comps, fields, outs = [], [], []
    for sp in specs:
        x = synth.smooth_codes_1d(sp.n, sp.rel_eb, alphabet=sp.alphabet, seed=sp.seed)
        c = oracle.compress(x, sp.alphabet, S=128)
        comps.append(c)
        fields.append(dev_field(c, True))
        outs.append(torch.full((c["n"] + 16,), CANARY, dtype=torch.int32).to(torch.int16).cuda())
    ctx.decode_batch(fields, outs)
    rc, st = ctx.batch_status(len(fields))
    assert rc == hd.HD_OK and np.all(st == 0)
    for c, o in zip(comps, outs):
        r = o.cpu().numpy().view(np.uint16)
        assert np.array_equal(r[:c["n"]], expect(c))
        assert np.all(r[c["n"]:] == np.uint16(CANARY))


# ---------------------------------------------------------------------------
# corrupt and invalid inputs: error codes, no hang, nothing written past n
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("with_gap,decoder", STRATEGIES, ids=STRATEGY_IDS)
def test_corrupt_streams(ctx, with_gap, decoder):
    ctx.set_config(decoder=decoder)
    try:
        corrupt_streams(ctx, with_gap)
    finally:
        ctx.reset_config()


def corrupt_streams(ctx, with_gap):
    from paper_2201_09118_gb300 import hd
    x = synth.laplace_codes(200000, scale=6.0, seed=13)
    c = oracle.compress(x, 1024, S=128)
    # claimed symbol count differs from the stream
    for dn in (-1, 1):
        cc = dict(c)
        cc["n"] = c["n"] + dn
        st, res = run_decode(ctx, cc, with_gap)
        assert st == hd.HD_ERR_CORRUPT
        assert np.all(res[cc["n"]:] == np.uint16(CANARY))
    # truncated stream
    cc = dict(c)
    cc["nbits"] = c["nbits"] - 5
    st, res = run_decode(ctx, cc, with_gap)
    assert st == hd.HD_ERR_CORRUPT
    assert np.all(res[cc["n"]:] == np.uint16(CANARY))
    # flipped bits: either still a valid stream of n symbols or detected
    rng = np.random.default_rng(3)
    for _ in range(5):
        cc = dict(c)
        w = c["words"].copy()
        b = int(rng.integers(0, c["nbits"]))
        w[b >> 5] ^= np.uint32(1 << (31 - (b & 31)))
        cc["words"] = w
        st, res = run_decode(ctx, cc, with_gap)
        assert st in (hd.HD_OK, hd.HD_ERR_CORRUPT)
        assert np.all(res[cc["n"]:] == np.uint16(CANARY))
    if with_gap:
        # entries at multiples of 4 are read by every decoder subsequence size
        # (128 to 512 bits over a 128-bit stream): a wrong one must be caught
        for k, bad in ((4 * (len(c["gap"]) // 8), lambda v: 200),
                       (4 * (len(c["gap"]) // 12), lambda v: v ^ 1)):
            cc = dict(c)
            g = c["gap"].copy()
            g[k] = bad(int(g[k]))
            cc["gap"] = g
            st, res = run_decode(ctx, cc, True)
            assert st == hd.HD_ERR_CORRUPT
            assert np.all(res[cc["n"]:] == np.uint16(CANARY))
        # an entry a wider decoder subsequence skips: caught, or not needed
        cc = dict(c)
        g = c["gap"].copy()
        g[4 * (len(g) // 8) + 1] ^= 1
        cc["gap"] = g
        st, res = run_decode(ctx, cc, True)
        if st == hd.HD_OK:
            assert np.array_equal(res[:c["n"]], expect(c))
        else:
            assert st == hd.HD_ERR_CORRUPT


def test_invalid_codebook_and_arguments(ctx):
    from paper_2201_09118_gb300 import hd
    x = synth.laplace_codes(10000, seed=14)
    c = oracle.compress(x, 1024, S=128)
    cc = dict(c)
    L = c["lengths"].copy()
    L[0] = 1  # Kraft sum > 1
    L[1] = 1
    cc["lengths"] = L
    st, _ = run_decode(ctx, cc, True)
    assert st == hd.HD_ERR_ARG
    f = dev_field(c)
    out = torch.empty(c["n"] + 8, dtype=torch.int16, device="cuda")
    bad = hd.DeviceField(f.words, f.nbits, f.gap, 96, f.lengths, f.alphabet, f.n)
    with pytest.raises(hd.HDError) as e:
        ctx.decode(bad, out)
    assert e.value.code == hd.HD_ERR_ARG
    mis = hd.DeviceField(f.words[1:], f.nbits, f.gap, 128, f.lengths, f.alphabet, f.n)
    with pytest.raises(hd.HDError) as e:
        ctx.decode(mis, out)
    assert e.value.code == hd.HD_ERR_ARG


@pytest.mark.parametrize("decoder", [1, 2], ids=["2phase", "1pass"])
@pytest.mark.parametrize("shift", [1, 3, 7])
def test_unaligned_output(ctx, shift, decoder):
    x = synth.laplace_codes(99991, scale=3.0, seed=15)
    c = oracle.compress(x, 1024, S=128)
    f = dev_field(c)
    buf = torch.full((c["n"] + 32,), CANARY, dtype=torch.int32).to(torch.int16).cuda()
    ctx.set_config(decoder=decoder)
    try:
        ctx.decode(f, buf[shift:])
        assert ctx.status() == 0
    finally:
        ctx.reset_config()
    r = buf.cpu().numpy().view(np.uint16)
    assert np.all(r[:shift] == np.uint16(CANARY))
    assert np.array_equal(r[shift:shift + c["n"]], x)
    assert np.all(r[shift + c["n"]:] == np.uint16(CANARY))


@pytest.mark.parametrize("case", ["skew1e-2", "one_symbol", "mixed"])
@pytest.mark.parametrize("with_gap", [True, False], ids=["gap", "selfsync"])
@pytest.mark.parametrize("S,threads,window", [(128, 128, 0), (128, 512, 256), (256, 256, 1024),
                                              (128, 256, 4096)])
def test_pre_filled_windows_of_1bit_runs(ctx, case, with_gap, S, threads, window):
    # fields under 1.25 bits per code: the two-phase write kernel fills each
    # window pass with the 1-bit code's symbol and stores only the other
    # codes; small windows make tiles take several passes, and the output
    # starts at an odd symbol so the window's pad is nonzero
    rng = np.random.default_rng(S + threads + window)
    if case == "skew1e-2":
        x = synth.smooth_codes_1d(500001, 1e-2, seed=31)
    elif case == "one_symbol":
        x = np.full(262147, 512, np.uint16)
    else:  # long runs of the 1-bit code broken by bursts of other codes
        x = np.full(400003, 512, np.uint16)
        for k in rng.integers(0, x.size - 300, 60):
            x[k:k + rng.integers(1, 300)] = rng.integers(0, 1024, 1)[0]
    c = oracle.compress(x, 1024, S=128)
    assert c["nbits"] / c["n"] < 1.25
    f = dev_field(c, with_gap)
    buf = torch.full((c["n"] + 40,), CANARY, dtype=torch.int32).to(torch.int16).cuda()
    ctx.set_config(decoder=1 if with_gap else 0, subseq_bits=S, threads=threads, window=window)
    try:
        ctx.decode(f, buf[3:])
        assert ctx.status() == 0
    finally:
        ctx.reset_config()
    r = buf.cpu().numpy().view(np.uint16)
    assert np.all(r[:3] == np.uint16(CANARY))
    assert np.array_equal(r[3:3 + c["n"]], expect(c))
    assert np.all(r[3 + c["n"]:] == np.uint16(CANARY))


@pytest.mark.parametrize("A,scale", [(1024, 1.0), (256, 2.5), (4096, 1.5)])
@pytest.mark.parametrize("with_gap", [True, False], ids=["gap", "selfsync"])
@pytest.mark.parametrize("S,threads,window", [(64, 128, 0), (128, 512, 512), (256, 256, 0),
                                              (128, 128, 2048)])
def test_two_code_lookups(ctx, A, scale, with_gap, S, threads, window):
    # fields of 1.25 to 4 bits per code: the two-phase write kernel takes the
    # first two codes of a first-level prefix with one lookup when both lie
    # within it (alphabets up to 1024; a 4096-symbol field keeps one code per
    # lookup), the window in several passes, the output at an odd offset
    x = synth.laplace_codes(600001, scale=scale, center=A // 2, alphabet=A, seed=A + S + threads)
    c = oracle.compress(x, A, S=S if S < 256 else 128)
    bits = c["nbits"] / c["n"]
    assert 1.25 <= bits < 4.0, bits
    f = dev_field(c, with_gap)
    buf = torch.full((c["n"] + 40,), CANARY, dtype=torch.int32).to(torch.int16).cuda()
    ctx.set_config(decoder=1 if with_gap else 0, subseq_bits=S, threads=threads, window=window)
    try:
        ctx.decode(f, buf[5:])
        assert ctx.status() == 0
    finally:
        ctx.reset_config()
    r = buf.cpu().numpy().view(np.uint16)
    assert np.all(r[:5] == np.uint16(CANARY))
    assert np.array_equal(r[5:5 + c["n"]], x)
    assert np.all(r[5 + c["n"]:] == np.uint16(CANARY))


# ---------------------------------------------------------------------------
# full-size workload: the 512^3 field of Lorenzo codes
# ---------------------------------------------------------------------------


@pytest.fixture(scope="module")
def cube():
    x = synth.field3d_codes(512, rel_eb=1e-4, noise=0.01, seed=1001)
    return x, oracle.compress(x, 1024, S=128)


@pytest.mark.parametrize("with_gap", [True, False], ids=["gap", "selfsync"])
def test_full_512cube(ctx, cube, with_gap):
    x, c = cube
    assert c["n"] == 512 ** 3
    st, res = run_decode(ctx, c, with_gap)
    assert st == 0
    assert np.array_equal(res[:c["n"]], x)
    assert np.all(res[c["n"]:] == np.uint16(CANARY))


@pytest.mark.parametrize("with_gap", [True, False], ids=["gap", "selfsync"])
def test_full_512cube_in_the_benchmark_launch_shape(cube, with_gap):
    # the benchmark times the shape the autotuner picks for this field
    from paper_2201_09118_gb300 import hd
    x, c = cube
    tctx = hd.Context(0)
    f = dev_field(c, with_gap)
    out = torch.full((c["n"] + 64,), CANARY, dtype=torch.int32).to(torch.int16).cuda()
    best = tctx.autotune([f], [out])
    assert best["threads"] in (128, 256, 512, 1024)
    out.fill_(CANARY - 65536)
    tctx.decode(f, out)
    assert tctx.status() == 0
    assert tctx.get_config()["threads"] == best["threads"]
    res = out.cpu().numpy().view(np.uint16)
    assert np.array_equal(res[:c["n"]], x)
    assert np.all(res[c["n"]:] == np.uint16(CANARY))
    tctx.close()


def test_full_512cube_matches_oracle_decode(ctx, cube):
    x, c = cube
    assert np.array_equal(expect(c), x)
