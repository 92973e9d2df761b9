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
