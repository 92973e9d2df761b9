"""GPU parity of the Lorenzo reconstruction after the decoder
(hd_reconstruct_device) and of decode + reconstruction (hd_decompress_device)
against the CPU oracle, bit for bit on the float32 output.

Grids cover 1D tiles with ragged tails, 2D rows with and without the 16-byte
path (nx % 8), one-row bands with large shared memory, 3D slice groups of
every size (automatic, 1, odd, all slices), outliers, q beyond 2^24 (float
rounding), and the full 512^3 workload.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from oracle import lorenzo as olz

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


def quantized(dims, rel_eb=1e-3, radius=512, seed=5, noise=1e-2):
    shape = tuple(reversed(dims))
    f = synth.fourier_field(shape, noise=noise, kmax=4, seed=seed)
    g = synth.lorenzo_quantize(f, rel_eb, radius=radius)
    g["field"] = f
    return g


def to_dev(g):
    codes = torch.from_numpy(g["codes"].view(np.int16)).cuda()
    idx = torch.from_numpy(g["out_idx"].view(np.int64)).cuda()
    val = torch.from_numpy(g["out_val"]).cuda()
    return codes, idx, val


def run(ctx, g, dims, radius, chunk=0):
    from paper_2201_09118_gb300 import hd
    codes, idx, val = to_dev(g)
    n = int(np.prod(dims))
    out = torch.full((n + 8,), float("nan"), dtype=torch.float32, device="cuda")
    L = hd.lorenzo_params(dims, radius, g["eb"], idx, val, chunk)
    ctx.reconstruct(codes, L, out)
    st = ctx.status()
    r = out.cpu().numpy()
    assert np.all(np.isnan(r[n:])), "write past the grid"
    return st, r[:n]


def expect(g, dims, radius):
    return olz.reconstruct(g["codes"], dims, radius, g["eb"], g["out_idx"], g["out_val"])


def same_bits(a, b):
    return np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("n", [1, 7, 8191, 8192, 8193, 3 * 8192 + 5, (1 << 20) + 13])
def test_1d_tiles_and_tails(ctx, n):
    g = quantized((n,), rel_eb=1e-4, radius=64, seed=n % 97)
    st, got = run(ctx, g, (n,), 64)
    assert st == 0
    assert same_bits(got, expect(g, (n,), 64))


@pytest.mark.parametrize("dims", [(3600, 1800), (500, 37), (64, 1000), (16384, 3), (20000, 5),
                                  (49152, 2), (1, 300), (8, 1)])
def test_2d_grids(ctx, dims):
    g = quantized(dims, rel_eb=1e-3, radius=16, seed=sum(dims) % 89)
    assert g["out_idx"].size > 0
    st, got = run(ctx, g, dims, 16)
    assert st == 0
    assert same_bits(got, expect(g, dims, 16))


@pytest.mark.parametrize("dims,chunk,radius", [
    ((512, 512, 64), 0, 512), ((512, 512, 64), 1, 512), ((512, 512, 64), 7, 512),
    ((512, 512, 64), 64, 512), ((67, 53, 37), 0, 512), ((67, 53, 37), 5, 32),
    ((500, 500, 100), 0, 512), ((8, 8, 8), 3, 32), ((1, 1, 40), 0, 512)])
def test_3d_grids_and_slice_groups(ctx, dims, chunk, radius):
    g = quantized(dims, rel_eb=1e-4, radius=radius, seed=sum(dims) % 83)
    assert g["out_idx"].size > 0
    st, got = run(ctx, g, dims, radius, chunk)
    assert st == 0
    assert same_bits(got, expect(g, dims, radius))


@pytest.mark.parametrize("dims,radius", [((64, 48, 320), 512), ((64, 48, 320), 32),
                                         ((999, 2, 305), 32), ((7, 5, 400), 512),
                                         ((1024, 4, 304), 512), ((1, 3, 330), 32)])
def test_3d_slice_path(ctx, dims, radius):
    # at least two slices per SM and rows up to 1024 codes: one block per slice
    g = quantized(dims, rel_eb=1e-4, radius=radius, seed=sum(dims) % 79)
    assert g["out_idx"].size > 0
    st, got = run(ctx, g, dims, radius)
    assert st == 0
    assert same_bits(got, expect(g, dims, radius))


def test_error_bound_on_the_field(ctx):
    dims = (96, 80, 72)
    g = quantized(dims, rel_eb=1e-4, radius=512, seed=3)
    st, got = run(ctx, g, dims, 512)
    assert st == 0
    f = g["field"].reshape(-1).astype(np.float64)
    assert np.all(np.abs(got - f) <= g["eb"] * (1 + 1e-6) + 2.0 ** -23 * np.abs(f))


def test_float_rounding_beyond_2_24(ctx):
    n = 20000
    codes = np.full(n, 512, np.uint16)
    codes[[0, 9000]] = 0
    g = {"codes": codes, "eb": 0.05, "out_idx": np.array([0, 9000], np.uint64),
         "out_val": np.array([(1 << 24) + 1, 3], np.int32)}
    st, got = run(ctx, g, (n,), 512)
    assert st == 0
    want = expect(g, (n,), 512)
    assert same_bits(got, want)
    assert got[0] == np.float32(1 << 24) * np.float32(0.1)


@pytest.mark.parametrize("dims", [(5000,), (40, 30), (16, 8, 9)])
def test_missing_outlier_reported(ctx, dims):
    from paper_2201_09118_gb300 import hd
    n = int(np.prod(dims))
    codes = np.full(n, 512, np.uint16)
    codes[n // 2] = 0
    g = {"codes": codes, "eb": 1.0, "out_idx": np.zeros(0, np.uint64),
         "out_val": np.zeros(0, np.int32)}
    st, _ = run(ctx, g, dims, 512)
    assert st == hd.HD_ERR_CORRUPT
    # the next good call reports success again
    g2 = quantized(dims, radius=512)
    st, got = run(ctx, g2, dims, 512)
    assert st == 0 and same_bits(got, expect(g2, dims, 512))


def test_arguments_checked(ctx):
    from paper_2201_09118_gb300 import hd
    codes = torch.zeros(1024, dtype=torch.int16, device="cuda")
    out = torch.zeros(1024 + 4, dtype=torch.float32, device="cuda")
    lib = hd.load()
    cases = [hd.lorenzo_params((1024,), 0, 1.0), hd.lorenzo_params((1024,), 40000, 1.0),
             hd.lorenzo_params((1024,), 512, float("inf")),
             hd.lorenzo_params((49153, 1), 512, 1.0)]
    bad_dim = hd.lorenzo_params((1024,), 512, 1.0)
    bad_dim.ndim = 4
    cases.append(bad_dim)
    for L in cases:
        rc = lib.hd_reconstruct_device(ctx.handle, ctypes.c_void_p(codes.data_ptr()),
                                       ctypes.byref(L), ctypes.c_void_p(out.data_ptr()), None)
        assert rc == hd.HD_ERR_ARG
    L = hd.lorenzo_params((1020,), 512, 1.0)
    rc = lib.hd_reconstruct_device(ctx.handle, ctypes.c_void_p(codes.data_ptr()), ctypes.byref(L),
                                   ctypes.c_void_p(out.data_ptr() + 4), None)
    assert rc == hd.HD_ERR_ARG  # output not 16-byte aligned
    L = hd.lorenzo_params((0, 5), 512, 1.0)
    assert lib.hd_reconstruct_device(ctx.handle, None, ctypes.byref(L), None, None) == hd.HD_OK


def _device_field(c):
    from paper_2201_09118_gb300 import hd
    enc = {"words": c["words"], "gap": c["gap"], "nbits": c["nbits"], "subseq_bits": c["S"]}
    return hd.DeviceField.upload(enc, c["lengths"], c["n"], with_gap=True)


@pytest.mark.parametrize("dims", [(70001,), (360, 180), (64, 48, 40)])
def test_decompress_small(ctx, dims):
    from paper_2201_09118_gb300 import hd
    g = quantized(dims, rel_eb=1e-4, radius=512, seed=17)
    c = oracle.compress(g["codes"], 1024, S=128)
    dec = oracle.decode(c["words"], c["nbits"], c["codes"], c["lengths"], n_cap=c["n"])
    want = olz.reconstruct(dec, dims, 512, g["eb"], g["out_idx"], g["out_val"])
    _, idx, val = to_dev(g)
    out = torch.empty(int(np.prod(dims)), dtype=torch.float32, device="cuda")
    ctx.decompress(_device_field(c), hd.lorenzo_params(dims, 512, g["eb"], idx, val), out)
    assert ctx.status() == 0
    assert same_bits(out.cpu().numpy(), want)


def test_decompress_512_cube(ctx):
    """The 512^3 workload (134,217,728 codes): decode + reconstruction on the
    GPU against the oracle's reconstruction of the same codes (the oracle's
    decode returns its encoder's input, pinned in the oracle tests)."""
    from paper_2201_09118_gb300 import hd
    g = synth.field3d_quantized(512, 1e-4, 0.01, 1001, keep_field=True)
    dims = (512, 512, 512)
    c = oracle.compress(g["codes"], 1024, S=128)
    want = olz.reconstruct(g["codes"], dims, 512, g["eb"], g["out_idx"], g["out_val"])
    _, idx, val = to_dev(g)
    out = torch.empty(512 ** 3, dtype=torch.float32, device="cuda")
    f = _device_field(c)
    ctx.decompress(f, hd.lorenzo_params(dims, 512, g["eb"], idx, val), out)
    assert ctx.status() == 0
    got = out.cpu().numpy()
    assert same_bits(got, want)
    fl = g["field"].reshape(-1).astype(np.float64)
    assert np.all(np.abs(got - fl) <= g["eb"] * (1 + 1e-6) + 2.0 ** -23 * np.abs(fl))


def _compressed_1d(n, rel_eb, radius, seed):
    g = quantized((n,), rel_eb=rel_eb, radius=radius, seed=seed, noise=1e-4)
    c = oracle.compress(g["codes"], 2 * radius, S=128)
    return g, c


@pytest.mark.parametrize("n,rel_eb,radius", [(1, 1e-3, 64), (7, 1e-3, 64), (5000, 1e-4, 16),
                                             ((1 << 20) + 3, 1e-4, 512),
                                             ((1 << 22) + 1, 1e-6, 2048)])
def test_fused_1d_equals_oracle_and_separate(ctx, n, rel_eb, radius):
    """1D gap-array fields decode straight into values (no codes in HBM);
    bit for bit the oracle's reconstruction of the oracle's decode, and the
    same as decode-then-reconstruct."""
    from paper_2201_09118_gb300 import hd
    g, c = _compressed_1d(n, rel_eb, radius, seed=n % 101)
    dec = oracle.decode(c["words"], c["nbits"], c["codes"], c["lengths"], n_cap=c["n"])
    want = olz.reconstruct(dec, (n,), radius, g["eb"], g["out_idx"], g["out_val"])
    _, idx, val = to_dev(g)
    f = _device_field(c)
    outs = []
    for separate in (False, True):
        out = torch.full((n + 8,), float("nan"), dtype=torch.float32, device="cuda")
        ctx.decompress(f, hd.lorenzo_params((n,), radius, g["eb"], idx, val, separate=separate),
                       out)
        assert ctx.status() == 0
        r = out.cpu().numpy()
        assert np.all(np.isnan(r[n:]))
        outs.append(r[:n])
    assert same_bits(outs[0], want)
    assert same_bits(outs[1], want)


def test_fused_1d_several_window_passes(ctx):
    # a small output window forces several passes per tile (q carried across)
    from paper_2201_09118_gb300 import hd
    n = 300_001
    g, c = _compressed_1d(n, 1e-2, 64, seed=3)  # ~1-2 bits per code: crowded tiles
    want = olz.reconstruct(g["codes"], (n,), 64, g["eb"], g["out_idx"], g["out_val"])
    _, idx, val = to_dev(g)
    f = _device_field(c)
    try:
        ctx.set_config(subseq_bits=256, threads=256, window=1024)
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        ctx.decompress(f, hd.lorenzo_params((n,), 64, g["eb"], idx, val), out)
        assert ctx.status() == 0
        assert same_bits(out.cpu().numpy(), want)
    finally:
        ctx.reset_config()


def test_fused_1d_heavy_outliers_and_large_q(ctx):
    from paper_2201_09118_gb300 import hd
    n = 200_000
    rng = np.random.default_rng(9)
    codes = rng.integers(1, 16, n).astype(np.uint16)
    out_idx = np.sort(rng.choice(n, size=n // 5, replace=False)).astype(np.uint64)
    codes[out_idx.astype(np.int64)] = 0
    out_val = rng.integers(-3000, 3000, out_idx.size).astype(np.int32)
    out_val[0] = (1 << 24) + 1
    g = {"codes": codes, "eb": 0.05, "out_idx": out_idx, "out_val": out_val}
    c = oracle.compress(codes, 16, S=128)
    want = olz.reconstruct(codes, (n,), 8, 0.05, out_idx, out_val)
    _, idx, val = to_dev(g)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx.decompress(_device_field(c), hd.lorenzo_params((n,), 8, 0.05, idx, val), out)
    assert ctx.status() == 0
    assert same_bits(out.cpu().numpy(), want)


def test_fused_1d_missing_outlier_and_corrupt_stream(ctx):
    from paper_2201_09118_gb300 import hd
    n = 50_000
    codes = np.full(n, 512, np.uint16)
    codes[[10, 40_000]] = 0
    c = oracle.compress(codes, 1024, S=128)
    f = _device_field(c)
    out = torch.full((n + 8,), float("nan"), dtype=torch.float32, device="cuda")
    idx = torch.tensor([10], dtype=torch.int64, device="cuda")
    val = torch.tensor([5], dtype=torch.int32, device="cuda")
    ctx.decompress(f, hd.lorenzo_params((n,), 512, 1.0, idx, val), out)
    assert ctx.status() == hd.HD_ERR_CORRUPT  # position 40,000 has no stored residue
    # a stream claiming one symbol more than it holds: corrupt, nothing past n
    bad = hd.DeviceField(f.words, f.nbits, f.gap, f.subseq_bits, f.lengths, f.alphabet, n + 1)
    out2 = torch.full((n + 9,), float("nan"), dtype=torch.float32, device="cuda")
    idx2 = torch.tensor([10, 40_000], dtype=torch.int64, device="cuda")
    val2 = torch.tensor([5, 6], dtype=torch.int32, device="cuda")
    ctx.decompress(bad, hd.lorenzo_params((n + 1,), 512, 1.0, idx2, val2), out2)
    assert ctx.status() == hd.HD_ERR_CORRUPT
    assert np.all(np.isnan(out2.cpu().numpy()[n + 1:]))


def test_fused_1d_hacc_size(ctx):
    """280,953,867 codes (the HACC particle count), rel. error bound 1e-4:
    fused decode + reconstruction against the oracle's reconstruction."""
    from paper_2201_09118_gb300 import hd
    n = 280_953_867
    g, c = _compressed_1d(n, 1e-4, 512, seed=1002)
    want = olz.reconstruct(g["codes"], (n,), 512, g["eb"], g["out_idx"], g["out_val"])
    _, idx, val = to_dev(g)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx.decompress(_device_field(c), hd.lorenzo_params((n,), 512, g["eb"], idx, val), out)
    assert ctx.status() == 0
    assert same_bits(out.cpu().numpy(), want)


@pytest.mark.parametrize("mode", ["selfsync", "cr_classes", "tuned"])
def test_1d_decompress_other_paths(ctx, mode):
    """1D decompression when the fused path does not apply (self-synchronised
    field, CR-class launches) or runs in an autotuned shape."""
    from paper_2201_09118_gb300 import hd
    n = 400_003
    g, c = _compressed_1d(n, 1e-4, 512, seed=77)
    want = olz.reconstruct(g["codes"], (n,), 512, g["eb"], g["out_idx"], g["out_val"])
    enc = {"words": c["words"], "gap": c["gap"], "nbits": c["nbits"], "subseq_bits": c["S"]}
    f = hd.DeviceField.upload(enc, c["lengths"], c["n"], with_gap=mode != "selfsync")
    _, idx, val = to_dev(g)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    try:
        if mode == "cr_classes":
            ctx.set_config(cr_classes=4)
        if mode == "tuned":
            ctx.autotune([f], [torch.empty(n, dtype=torch.int16, device="cuda")])
        ctx.decompress(f, hd.lorenzo_params((n,), 512, g["eb"], idx, val), out)
        assert ctx.status() == 0
        assert same_bits(out.cpu().numpy(), want)
    finally:
        ctx.reset_config()
