"""Checks of the seeded input generators (test and benchmark inputs only).

The generators hold none of the decoder's arithmetic; these tests pin them to
what they claim to produce: cuSZ-style Lorenzo quantization codes that
reconstruct every non-outlier value within the error bound, and a discrete
Laplace distribution with its closed-form centre probability.
"""
import math

import numpy as np
import pytest

import synth


def _inverse_lorenzo(d: np.ndarray) -> np.ndarray:
    """Undo the first-order Lorenzo residue: a cumulative sum along every axis."""
    q = d.astype(np.int64)
    for ax in range(q.ndim):
        q = np.cumsum(q, axis=ax)
    return q


@pytest.mark.parametrize("shape", [(4096,), (48, 64), (16, 20, 24)])
@pytest.mark.parametrize("rel_eb", [1e-2, 1e-3])
def test_lorenzo_codes_reconstruct_within_error_bound(shape, rel_eb):
    f = synth.fourier_field(shape, noise=1e-3, kmax=4, seed=7)
    codes, eb, out_frac = synth.lorenzo_codes(f, rel_eb, radius=512)
    assert codes.dtype == np.uint16 and codes.size == f.size
    assert out_frac == 0.0  # smooth field, wide radius: no outliers to keep aside
    d = codes.astype(np.int64).reshape(shape) - 512
    q = _inverse_lorenzo(d)
    err = np.abs(f.astype(np.float64) - 2.0 * eb * q)
    assert err.max() <= eb * (1 + 1e-9)
    assert math.isclose(eb, rel_eb * (float(f.max()) - float(f.min())), rel_tol=1e-12)


def test_lorenzo_outliers_get_code_zero():
    f = np.zeros(64, np.float32)
    f[10] = 1.0  # a jump far beyond the radius at this error bound
    codes, eb, out_frac = synth.lorenzo_codes(f, 1e-4, radius=8)
    assert codes[10] == 0 and codes[11] == 0  # +jump and -jump residues
    assert np.all(np.delete(codes, [10, 11]) == 8)
    assert math.isclose(out_frac, 2 / 64)


def test_laplace_centre_probability_closed_form():
    x = synth.laplace_codes(1 << 20, scale=2.0, seed=1)
    assert x.min() >= 0 and x.max() < 1024
    # P(k) proportional to exp(-|k - 512| / b): P(centre) = tanh(1 / (2b))
    p0 = math.tanh(1.0 / 4.0)
    got = np.count_nonzero(x == 512) / x.size
    assert abs(got - p0) < 4 * math.sqrt(p0 * (1 - p0) / x.size)
    # symmetric around the centre
    assert abs(float(np.mean(x.astype(np.float64))) - 512.0) < 0.02


def test_generators_are_seeded():
    a = synth.laplace_codes(1000, seed=3)
    b = synth.laplace_codes(1000, seed=3)
    c = synth.laplace_codes(1000, seed=4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_batch_spec_ranges():
    spec = synth.batch_spec(n_fields=256)
    assert len(spec) == 256
    ns = np.array([s.n for s in spec])
    assert ns.min() >= 1 << 16 and ns.max() <= 1 << 26
    assert {s.alphabet for s in spec} <= {256, 1024, 4096}
    assert all(1e-6 <= s.rel_eb <= 1e-2 for s in spec)
    # log-uniform: the median size is near the geometric mean of the range
    assert abs(math.log2(float(np.median(ns))) - 21) < 1.0


def test_lorenzo_radius_boundary_and_outlier_list():
    # a 1D field whose residues are exactly +-(R-1) and +-R (eb = 0.5 so that
    # q = round(x)): |d| < R is coded as d + R, |d| >= R goes to the outlier list
    R = 8
    q = np.cumsum([0, R - 1, -(R - 1), R, -R, 3]).astype(np.float64)
    x = np.concatenate([q, [0.0, float(q.max() - q.min())]])  # fix the range
    rel = 0.5 / (x.max() - x.min())
    g = synth.lorenzo_quantize(x, rel, radius=R, keep_q=True)
    assert np.array_equal(g["q"], np.round(x).astype(np.int64))
    d = np.diff(np.concatenate([[0], g["q"]]))
    inl = np.abs(d) < R
    assert np.array_equal(g["codes"][inl], (d[inl] + R).astype(np.uint16))
    assert np.all(g["codes"][~inl] == 0)
    assert np.array_equal(g["out_idx"], np.flatnonzero(~inl).astype(np.uint64))
    assert np.array_equal(g["out_val"], d[~inl].astype(np.int32))
    assert g["codes"][1] == 2 * R - 1 and g["codes"][2] == 1


def test_field3d_quantized_outliers_match_zero_codes():
    g = synth.field3d_quantized(24, rel_eb=1e-4, noise=0.01, seed=5, keep_field=True)
    assert g["codes"].size == 24 ** 3 and g["field"].shape == (24, 24, 24)
    zero = np.flatnonzero(g["codes"] == 0).astype(np.uint64)
    assert np.array_equal(zero, g["out_idx"])
    assert g["out_val"].dtype == np.int32 and g["out_val"].size == zero.size
    assert np.all(np.abs(g["out_val"].astype(np.int64)) >= 512)
