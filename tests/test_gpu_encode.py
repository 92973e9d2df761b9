"""GPU encoder (hd_encode_device) and histogram (hd_histogram_device) against
the oracle: every stream word, every gap entry and the bit count identical to
the oracle's encoding of the same symbols with the same code lengths."""
import zlib

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_09118_gb300 import hd
    c = hd.Context(0)
    yield c
    c.close()


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint16).view(np.int16)).cuda()


def check_same_as_oracle(ctx, x, alphabet, S):
    c = oracle.compress(x, alphabet, S=S)
    lengths = c["lengths"]
    e = ctx.encode(to_dev(x), lengths, S)
    assert e["nbits"] == c["nbits"]
    got_w = e["words"].cpu().numpy().view(np.uint32)
    assert got_w.size == c["words"].size
    if not np.array_equal(got_w, c["words"]):
        bad = np.nonzero(got_w != c["words"])[0]
        raise AssertionError(f"{bad.size} words differ, first at {bad[:8].tolist()}")
    got_g = e["gap"].cpu().numpy()
    assert np.array_equal(got_g[:e["nsub"]], c["gap"])
    return e, c


@pytest.mark.parametrize("S", [64, 128, 256])
def test_encode_laplace_matches_oracle(ctx, S):
    x = synth.laplace_codes(1 << 20, scale=2.0, seed=1000)
    check_same_as_oracle(ctx, x, 1024, S)


@pytest.mark.parametrize("case", ["n1", "n2", "one_symbol", "tile_edge", "ragged",
                                  "alphabet4096", "skew1e-2", "fibonacci32", "odd_offset"])
def test_encode_edge_cases(ctx, case):
    rng = np.random.default_rng(zlib.crc32(case.encode()))
    A = 1024
    if case == "n1":
        x = np.array([7], np.uint16)
    elif case == "n2":
        x = np.array([7, 900], np.uint16)
    elif case == "one_symbol":
        x = np.full(10000, 512, np.uint16)
    elif case == "tile_edge":
        x = synth.laplace_codes(4096 * 3, scale=3.0, seed=2)  # whole symbol tiles
    elif case == "ragged":
        x = synth.laplace_codes(4096 * 5 + 17, scale=9.0, seed=3)
    elif case == "alphabet4096":
        A = 4096
        x = rng.integers(0, 4096, 300001).astype(np.uint16)
    elif case == "skew1e-2":
        x = synth.smooth_codes_1d(200000, 1e-2, alphabet=1024, seed=4)
    elif case == "fibonacci32":
        # exact Fibonacci counts force 32-bit codes (length limit)
        fib = [1, 1]
        while len(fib) < 34:
            fib.append(fib[-1] + fib[-2])
        x = np.repeat(np.arange(34, dtype=np.uint16), fib)
        rng.shuffle(x)
        A = 64
    elif case == "odd_offset":
        x = synth.laplace_codes(70001, scale=5.0, seed=5)
    for S in (64, 128, 256):
        if case == "odd_offset":
            # symbols starting at an odd element: unaligned vector loads
            buf = to_dev(np.concatenate([np.zeros(1, np.uint16), x]))
            c = oracle.compress(x, A, S=S)
            e = ctx.encode(buf[1:], c["lengths"], S)
            assert e["nbits"] == c["nbits"]
            assert np.array_equal(e["words"].cpu().numpy().view(np.uint32), c["words"])
            assert np.array_equal(e["gap"].cpu().numpy()[:e["nsub"]], c["gap"])
        else:
            check_same_as_oracle(ctx, x, A, S)


def test_encode_then_decode_round_trip(ctx):
    from paper_2201_09118_gb300 import hd
    x = synth.field3d_codes(128, rel_eb=1e-4, noise=0.01, seed=7)
    xd = to_dev(x)
    freq = ctx.histogram(xd, 1024)
    assert np.array_equal(freq, np.bincount(x, minlength=1024))
    lengths = hd.hd_build_codebook_freq(freq, 32)
    e = ctx.encode(xd, lengths, 128)
    f = hd.DeviceField(e["words"], e["nbits"], e["gap"], 128,
                       torch.from_numpy(lengths).cuda(), 1024, x.size)
    out = torch.empty(x.size, dtype=torch.int16, device="cuda")
    ctx.decode(f, out)
    assert ctx.status() == 0
    assert np.array_equal(out.cpu().numpy().view(np.uint16), x)


def test_encode_errors(ctx):
    from paper_2201_09118_gb300 import hd
    x = np.array([1, 2, 3, 5], np.uint16)
    L = np.zeros(8, np.uint8)
    L[[1, 2, 3]] = 2  # symbol 5 has no code
    with pytest.raises(hd.HDError) as e:
        ctx.encode(to_dev(x), L, 128)
    assert e.value.code == hd.HD_ERR_SYMBOL
    with pytest.raises(hd.HDError) as e:
        ctx.histogram(to_dev(np.array([1, 9], np.uint16)), 8)
    assert e.value.code == hd.HD_ERR_SYMBOL
    bad = np.array([1, 1, 1, 1], np.uint8)  # Kraft sum 2
    with pytest.raises(hd.HDError) as e:
        ctx.encode(to_dev(np.array([0, 1], np.uint16)), bad, 128)
    assert e.value.code == hd.HD_ERR_ARG


def test_encode_empty(ctx):
    e = ctx.encode(torch.empty(0, dtype=torch.int16, device="cuda"),
                   np.array([1, 1], np.uint8), 128)
    assert e["nbits"] == 0 and e["nsub"] == 0 and e["nwords"] == 1
    assert int(e["words"].cpu()[0]) == 0


def test_encode_full_512cube_matches_oracle(ctx):
    x = synth.field3d_codes(512, rel_eb=1e-4, noise=0.01, seed=1001)
    check_same_as_oracle(ctx, x, 1024, 128)
