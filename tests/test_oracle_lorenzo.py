"""Pins of the Lorenzo reconstruction oracle (CPU only).

The oracle computes q as prefix sums along every axis.  These tests check it
against what fixes the result independently of that formulation: the
predictor's own recurrence evaluated point by point (brute force), closed
forms (a single residue fills an orthant; a constant residue gives products
of coordinates), the generator's prequantized integers, and the error bound
the quantizer guarantees on the original field.
"""
import itertools

import numpy as np
import pytest

import synth
from oracle import lorenzo

R = 512


def _recurrence_q(d, shape):
    """q by the first-order Lorenzo predictor, point by point: q = d + the
    inclusion-exclusion sum of the already reconstructed neighbours one step
    back along any non-empty subset of the axes (zero outside the domain)."""
    d = d.reshape(shape)
    q = np.zeros(shape, np.int64)
    nd = len(shape)
    subsets = [s for k in range(1, nd + 1) for s in itertools.combinations(range(nd), k)]
    for p in itertools.product(*[range(v) for v in shape]):
        pred = 0
        for s in subsets:
            nb = list(p)
            inside = True
            for ax in s:
                nb[ax] -= 1
                inside &= nb[ax] >= 0
            if inside:
                pred += (-1) ** (len(s) + 1) * q[tuple(nb)]
        q[p] = d[p] + pred
    return q.reshape(-1)


@pytest.mark.parametrize("dims", [(13,), (7, 5), (6, 5, 4), (1, 1, 9), (4, 1, 3)])
def test_brute_force_predictor_recurrence(dims):
    rng = np.random.default_rng(sum(dims))
    n = int(np.prod(dims))
    codes = rng.integers(R - 40, R + 40, n).astype(np.uint16)
    out_idx = np.sort(rng.choice(n, size=max(1, n // 7), replace=False)).astype(np.uint64)
    codes[out_idx.astype(np.int64)] = 0
    out_val = rng.integers(-5000, 5000, out_idx.size).astype(np.int32)
    x, q = lorenzo.reconstruct(codes, dims, R, 0.25, out_idx, out_val, return_q=True)
    d = codes.astype(np.int64) - R
    d[out_idx.astype(np.int64)] = out_val
    assert np.array_equal(q, _recurrence_q(d, tuple(reversed(dims))))
    assert np.array_equal(x, q.astype(np.float32) * np.float32(0.5))


def test_single_residue_fills_its_orthant():
    dims = (6, 4, 3)  # nx, ny, nz: a transposed axis order would fail
    x0, y0, z0 = 2, 1, 1
    codes = np.full(int(np.prod(dims)), R, np.uint16)
    codes[(z0 * dims[1] + y0) * dims[0] + x0] = R + 1
    q = lorenzo.reconstruct(codes, dims, R, 1.0, return_q=True)[1].reshape(3, 4, 6)
    z, y, x = np.meshgrid(np.arange(3), np.arange(4), np.arange(6), indexing="ij")
    assert np.array_equal(q, ((x >= x0) & (y >= y0) & (z >= z0)).astype(np.int64))


@pytest.mark.parametrize("dims", [(9,), (5, 7), (4, 3, 5)])
def test_constant_residue_gives_coordinate_products(dims):
    # d = 1 everywhere: q counts the points below and at p, i.e. the product
    # of (coordinate + 1) over the axes
    codes = np.full(int(np.prod(dims)), R + 1, np.uint16)
    q = lorenzo.reconstruct(codes, dims, R, 1.0, return_q=True)[1]
    grids = np.meshgrid(*[np.arange(v) + 1 for v in reversed(dims)], indexing="ij")
    assert np.array_equal(q, np.prod(grids, axis=0).reshape(-1))


def test_centre_codes_give_zero():
    x = lorenzo.reconstruct(np.full(60, R, np.uint16), (3, 4, 5), R, 0.1)
    assert x.dtype == np.float32 and not np.any(x)


@pytest.mark.parametrize("shape,rel_eb,radius", [
    ((5000,), 1e-4, 512), ((48, 70), 1e-3, 16), ((12, 17, 23), 1e-3, 8), ((20, 20, 20), 1e-5, 512)])
def test_generator_round_trip_within_error_bound(shape, rel_eb, radius):
    f = synth.fourier_field(shape, noise=1e-2, kmax=4, seed=11)
    g = synth.lorenzo_quantize(f, rel_eb, radius=radius, keep_q=True)
    dims = tuple(reversed(shape))
    x, q = lorenzo.reconstruct(g["codes"], dims, radius, g["eb"], g["out_idx"], g["out_val"],
                               return_q=True)
    assert np.array_equal(q, g["q"].reshape(-1))
    if radius < 512:
        assert g["out_idx"].size > 0  # the outlier path is exercised
    # the quantizer's bound |2 eb q - x| <= eb, plus the float32 roundings of
    # 2 eb and of the product
    err = np.abs(x.astype(np.float64) - f.reshape(-1).astype(np.float64))
    bound = g["eb"] * (1 + 1e-6) + 2.0 ** -23 * np.abs(f.reshape(-1).astype(np.float64))
    assert np.all(err <= bound)


def test_outlier_list_must_match_code_zero():
    codes = np.array([R, 0, R, 0], np.uint16)
    with pytest.raises(lorenzo.ReconstructError):
        lorenzo.reconstruct(codes, (4,), R, 1.0, np.array([1], np.uint64), np.array([3], np.int32))
    with pytest.raises(lorenzo.ReconstructError):
        lorenzo.reconstruct(codes, (4,), R, 1.0, np.array([3, 1], np.uint64),
                            np.array([3, 4], np.int32))
    x = lorenzo.reconstruct(codes, (4,), R, 1.0, np.array([1, 3], np.uint64),
                            np.array([3, -4], np.int32))
    assert np.array_equal(x, np.float32([0, 6, 6, -2]))


def test_float_rounding_is_one_product_of_float32s():
    # q beyond 2^24 rounds to nearest even when converted; 2 eb rounds once
    codes = np.array([0], np.uint16)
    q0 = (1 << 24) + 1
    x = lorenzo.reconstruct(codes, (1,), R, 0.05, np.array([0], np.uint64),
                            np.array([q0], np.int32))
    assert x[0] == np.float32(1 << 24) * np.float32(0.1)
    assert float(np.float32(0.1)) != 0.1  # 2 eb is not exact in float32
