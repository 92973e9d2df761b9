"""GPU parity of the one-pass gap-array decoder (hd_config.decoder = 2).

Each warp decodes a tile of 32 subsequences once, takes its output index from
a look-back over the tiles before it and writes through its own window
(Sec. III-C start points, Sec. III-B2 output indices, Algorithm 1).  Every
expected value is the CPU oracle's decode of the oracle's own encoding; the
path is integer work, so parity is bit-exact.
"""
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


def dev_field(c):
    from paper_2201_09118_gb300 import hd
    enc = {"words": c["words"], "gap": c["gap"], "nbits": c["nbits"], "subseq_bits": c["S"]}
    return hd.DeviceField.upload(enc, c["lengths"], c["n"], with_gap=True)


def decode(ctx, c, n=None, **cfg):
    n = c["n"] if n is None else n
    f = dev_field(dict(c, n=n))
    out = torch.full((n + 64,), CANARY, dtype=torch.int32).to(torch.int16).cuda()
    ctx.set_config(decoder=2, **cfg)
    try:
        ctx.decode(f, out)
        st = ctx.status()
        assert ctx.get_config()["decoder"] == 2
    finally:
        ctx.reset_config()
    return st, out.cpu().numpy().view(np.uint16)


def check(ctx, c, **cfg):
    st, res = decode(ctx, c, **cfg)
    assert st == 0, f"status {st}"
    ref = oracle.decode(c["words"], c["nbits"], c["codes"], c["lengths"], n_cap=c["n"])
    got = res[:c["n"]]
    if not np.array_equal(got, ref):
        bad = np.nonzero(got != ref)[0]
        raise AssertionError(f"{bad.size} mismatches, first at {bad[:8].tolist()}")
    assert np.all(res[c["n"]:] == np.uint16(CANARY)), "write past the output"


@pytest.mark.parametrize("S", [128, 256, 512])
@pytest.mark.parametrize("threads", [128, 256, 512, 768, 1024])
def test_warps_per_block_and_subsequence_bits(ctx, S, threads):
    # 331,337 codes at ~4.3 bits: tiles of 32 subsequences with a ragged last
    # tile (nsub not a multiple of 32, nbits not a multiple of S)
    x = synth.laplace_codes(331337, scale=5.0, seed=S * 7 + threads)
    c = oracle.compress(x, 1024, S=128)
    check(ctx, c, subseq_bits=S, threads=threads)


@pytest.mark.parametrize("K", [8, 10, 12, 13, 14, 15])
def test_table_bits(ctx, K):
    # K = 8: most codes are longer than the table and take the escape path
    x = synth.laplace_codes(250000, scale=40.0, seed=K)
    c = oracle.compress(x, 1024, S=128)
    check(ctx, c, lut_bits=K)


@pytest.mark.parametrize("S", [128, 256])
def test_column_overflow_rounds(ctx, S):
    # compressibility changes along the field (about 1 bit per code at 1e-2,
    # 8 at 1e-6): the column is sized from the mean code length, so lanes in
    # the 1-bit segments overflow it and their tiles write in several window
    # rounds, decoding those lanes again
    parts = [synth.smooth_codes_1d(1 << 17, eb, alphabet=1024, seed=40 + k)
             for k, eb in enumerate([1e-6, 1e-2, 1e-5, 1e-2, 1e-6, 1e-3])]
    x = np.concatenate(parts)
    c = oracle.compress(x, 1024, S=128)
    check(ctx, c, subseq_bits=S)


@pytest.mark.parametrize("A", [8192, 65536])
def test_wide_alphabets_use_32bit_tables(ctx, A):
    # alphabets beyond 4096 symbols take the 32-bit first-level table
    rng = np.random.default_rng(A)
    x = np.clip(np.rint(rng.normal(A // 2, A / 16, 200000)), 0, A - 1).astype(np.uint16)
    c = oracle.compress(x, A, S=128)
    check(ctx, c)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 1000, 4097])
def test_small_fields(ctx, n):
    x = synth.laplace_codes(n, scale=2.0, seed=n)
    c = oracle.compress(x, 1024, S=128)
    check(ctx, c)


def test_repeated_decodes_reset_the_tile_states(ctx):
    # the ticket and look-back states are cleared for every decode
    x = synth.laplace_codes(700001, scale=9.0, seed=21)
    c = oracle.compress(x, 1024, S=128)
    for _ in range(4):
        check(ctx, c)


def test_count_mismatch_reported_nothing_past_n(ctx):
    from paper_2201_09118_gb300 import hd
    x = synth.laplace_codes(400000, scale=6.0, seed=22)
    c = oracle.compress(x, 1024, S=128)
    for dn in (-1000, -1, 1, 1000):
        st, res = decode(ctx, c, n=c["n"] + dn)
        assert st == hd.HD_ERR_CORRUPT
        assert np.all(res[c["n"] + dn:] == np.uint16(CANARY))
        if dn > 0:
            assert np.array_equal(res[:c["n"]], x)


def test_full_512cube_one_pass(ctx):
    x = synth.field3d_codes(512, rel_eb=1e-4, noise=0.01, seed=1001)
    c = oracle.compress(x, 1024, S=128)
    for cfg in ({}, {"subseq_bits": 512, "threads": 512, "lut_bits": 12}):
        st, res = decode(ctx, c, **cfg)
        assert st == 0
        assert np.array_equal(res[:c["n"]], x)
        assert np.all(res[c["n"]:] == np.uint16(CANARY))


def test_lookback_wait_limit_reports_timeout_and_context_stays_usable(ctx):
    # failure detection without hanging the GPU: a one-cycle limit makes every
    # look-back wait that finds a predecessor not yet counted give up; the
    # decode reports HD_ERR_TIMEOUT, writes nothing past its output, and the
    # next decode with the default limit is exact
    from paper_2201_09118_gb300 import hd
    x = synth.laplace_codes(1 << 23, scale=20.0, seed=71)
    c = oracle.compress(x, 1024, S=128)
    statuses = []
    try:
        ctx.set_wait_limit(1)
        for _ in range(6):
            st, res = decode(ctx, c)
            statuses.append(st)
            assert st in (hd.HD_OK, hd.HD_ERR_TIMEOUT)
            assert np.all(res[c["n"]:] == np.uint16(CANARY))
            if st == hd.HD_OK:
                assert np.array_equal(res[:c["n"]], x)
    finally:
        ctx.set_wait_limit(0)
    assert hd.HD_ERR_TIMEOUT in statuses
    st, res = decode(ctx, c)
    assert st == hd.HD_OK and np.array_equal(res[:c["n"]], x)


@pytest.fixture(scope="module")
def cube128():
    # the 3D workload's generator at 128^3: codes of 8 to 19 bits, so the
    # fixed-step decode loop and the second-level tables (codes longer than
    # the first-level table) run
    x = synth.field3d_codes(128, rel_eb=1e-4, noise=0.01, seed=1001)
    c = oracle.compress(x, 1024, S=128)
    assert int(c["lengths"][c["lengths"] > 0].min()) >= 8
    return x, c


@pytest.mark.parametrize("S", [128, 256, 512])
@pytest.mark.parametrize("threads", [256, 512, 768, 1024])
@pytest.mark.parametrize("K", [11, 13, 14])
def test_long_codes_fixed_steps_and_second_level_tables(ctx, cube128, S, threads, K):
    x, c = cube128
    st, res = decode(ctx, c, subseq_bits=S, threads=threads, lut_bits=K)
    assert st == 0
    assert np.array_equal(res[:c["n"]], x)
    assert np.all(res[c["n"]:] == np.uint16(CANARY))


def test_wrong_gap_entries_of_long_code_streams(ctx, cube128):
    # a wrong entry at a decoder subsequence's start is caught by the end
    # check of the subsequence before it; an entry a wider decoder subsequence
    # skips changes nothing; nothing is written past the output
    from paper_2201_09118_gb300 import hd
    x, c = cube128
    for S, k, bad in ((128, 1001, lambda v: v ^ 1), (256, 2 * 2002, lambda v: 31 - v),
                      (512, 4 * 3003, lambda v: (v + 3) % 32)):
        g = c["gap"].copy()
        g[k] = bad(int(g[k]))
        st, res = decode(ctx, dict(c, gap=g), subseq_bits=S)
        assert st == hd.HD_ERR_CORRUPT
        assert np.all(res[c["n"]:] == np.uint16(CANARY))
    g = c["gap"].copy()
    g[4 * 1234 + 2] ^= 1
    st, res = decode(ctx, dict(c, gap=g), subseq_bits=512)
    assert st == hd.HD_OK and np.array_equal(res[:c["n"]], x)
