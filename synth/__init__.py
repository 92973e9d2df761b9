"""Seeded synthetic inputs: uint16 quantization-code arrays shaped like the
paper's workloads.

This module generates *inputs only*.  It holds none of the Huffman arithmetic
(no histogram, code lengths, codewords, packing or decoding) and is imported by
both the CPU oracle's tests and the GPU path's tests and benchmark, so the two
sides decode exactly the same code arrays.

The paper evaluates cuSZ quantization codes of eight SDRBench-style datasets
(Sec. V-A3, Table "datasets": HACC 280,953,867 points, CESM-ATM 26x1800x3600,
Nyx 512^3, ...).  Those datasets are not available, so these generators stand
in for them:

* ``laplace_codes``      i.i.d. discrete Laplace codes around the centre bin.
* ``fourier_field``      smooth float32 fields (1D/2D/3D) made of random
                         Fourier modes with 1/|k|^2 amplitudes plus Gaussian
                         noise.
* ``lorenzo_quantize``   cuSZ-style error-bounded quantization followed by the
                         integer first-order Lorenzo predictor, giving the
                         residue codes the decoder consumes and the outliers
                         (residues beyond the radius) kept aside for the
                         reconstruction after it.  The paper does not
                         describe this step (it only cites cuSZ); it is a
                         test-input generator here and is never timed.
* ``lorenzo_codes``      the codes alone.
* ``batch_spec``         the size / alphabet / error-bound mix of a batch of
                         independent fields.

All randomness comes from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "laplace_codes",
    "fourier_field",
    "lorenzo_quantize",
    "lorenzo_codes",
    "smooth_codes_1d",
    "field3d_codes",
    "field3d_quantized",
    "batch_spec",
    "FieldSpec",
    "code_stats",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def laplace_codes(n: int, scale: float = 2.0, center: int = 512,
                  alphabet: int = 1024, seed: int = 1000) -> np.ndarray:
    """``n`` i.i.d. codes with P(k) proportional to exp(-|k-center|/scale) on [0, alphabet)."""
    k = np.arange(alphabet, dtype=np.float64)
    pmf = np.exp(-np.abs(k - center) / scale)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    u = _rng(seed).random(n)
    idx = np.searchsorted(cdf, u, side="right")
    np.minimum(idx, alphabet - 1, out=idx)
    return idx.astype(np.uint16)


def _random_modes(rng: np.random.Generator, ndim: int, n_modes: int, kmax: int):
    """Integer wave vectors (last component >= 1), amplitude 1/|k|^2, random phase."""
    ks = []
    while len(ks) < n_modes:
        k = rng.integers(-kmax, kmax + 1, size=ndim)
        k[-1] = abs(int(k[-1]))
        if k[-1] == 0:
            continue
        ks.append(k)
    ks = np.array(ks, dtype=np.int64)
    amp = 1.0 / np.sum(ks.astype(np.float64) ** 2, axis=1)
    phase = rng.random(n_modes) * 2.0 * math.pi
    return ks, amp, phase


def fourier_field(shape, n_modes: int = 64, noise: float = 0.01, kmax: int = 8,
                  seed: int = 1001) -> np.ndarray:
    """float32 field = sum of ``n_modes`` Fourier modes + N(0, (noise*range)^2).

    For 2D/3D the smooth part is one inverse real FFT of a spectrum holding the
    chosen modes (last-axis wavenumber in [1, N/2)), so a mode with coefficient
    a*exp(i*phi) contributes a*cos(2*pi*k.x/N + phi).  In 1D the smooth part is
    evaluated on a coarse grid of at most 2^20 points and linearly interpolated,
    which keeps 10^8-point fields cheap to generate.
    """
    import scipy.fft as sfft

    shape = tuple(int(s) for s in shape)
    rng = _rng(seed)
    ndim = len(shape)
    ks, amp, phase = _random_modes(rng, ndim, n_modes, kmax)
    if ndim == 1:
        n = shape[0]
        m = min(n, 1 << 20)
        x = np.arange(m, dtype=np.float64) / m
        coarse = np.zeros(m, dtype=np.float64)
        for k, a, p in zip(ks[:, 0], amp, phase):
            coarse += a * np.cos(2.0 * math.pi * k * x + p)
        if m == n:
            smooth = coarse.astype(np.float32)
        else:
            smooth = np.interp(np.arange(n, dtype=np.float64) * (m / n),
                               np.arange(m, dtype=np.float64), coarse).astype(np.float32)
    else:
        half = shape[:-1] + (shape[-1] // 2 + 1,)
        spec = np.zeros(half, dtype=np.complex64)
        total = float(np.prod(shape))
        for k, a, p in zip(ks, amp, phase):
            kk = k.copy()
            kk[-1] = min(int(kk[-1]), shape[-1] // 2 - 1)
            idx = tuple(int(kk[d]) % shape[d] for d in range(ndim - 1)) + (int(kk[-1]),)
            spec[idx] += np.complex64(0.5 * total * a * complex(math.cos(p), math.sin(p)))
        smooth = sfft.irfftn(spec, s=shape, workers=-1).astype(np.float32, copy=False)
        del spec
    rng_noise = _rng(seed + 7919)
    sigma = noise * float(smooth.max() - smooth.min())
    if sigma > 0:
        # chunked to bound the float64 temporaries numpy would otherwise create
        flat = smooth.reshape(-1)
        step = 1 << 24
        for s in range(0, flat.size, step):
            e = min(flat.size, s + step)
            flat[s:e] += rng_noise.standard_normal(e - s, dtype=np.float32) * np.float32(sigma)
    return smooth


def lorenzo_quantize(field: np.ndarray, rel_eb: float, radius: int = 512,
                     keep_q: bool = False) -> dict:
    """cuSZ-style codes with their outliers: q = round(x / 2eb) (half away
    from zero), integer first-order Lorenzo residue d (zero outside the
    domain), code = d + radius when |d| < radius, else 0 with d kept aside.

    Returns a dict: ``codes`` (uint16, flat, x fastest), ``eb``,
    ``out_idx`` (uint64, ascending flat positions of code 0), ``out_val``
    (int32 residues there), ``out_frac`` and, with ``keep_q``, ``q`` (int64,
    the prequantized values, shaped like the field).
    """
    field = np.asarray(field)
    lo = float(field.min())
    hi = float(field.max())
    eb = rel_eb * (hi - lo) if hi > lo else rel_eb
    scaled = field.astype(np.float64) / (2.0 * eb)
    q = (np.sign(scaled) * np.floor(np.abs(scaled) + 0.5)).astype(np.int64)
    del scaled
    d = q.copy() if keep_q else q
    # (1 - S_x)(1 - S_y)(1 - S_z) q: the 1D/2D/3D Lorenzo residue
    for ax in range(d.ndim):
        sl_hi = [slice(None)] * d.ndim
        sl_lo = [slice(None)] * d.ndim
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(None, -1)
        d[tuple(sl_hi)] -= d[tuple(sl_lo)].copy()
    d = d.reshape(-1)
    inlier = np.abs(d) < radius
    codes = np.where(inlier, d + radius, 0).astype(np.uint16)
    out_idx = np.flatnonzero(~inlier).astype(np.uint64)
    out_val = d[out_idx.astype(np.int64)]
    if out_val.size and (out_val.min() < -(1 << 31) or out_val.max() >= (1 << 31)):
        raise ValueError("outlier residue outside int32")
    res = {
        "codes": codes,
        "eb": eb,
        "out_idx": out_idx,
        "out_val": out_val.astype(np.int32),
        "out_frac": float(out_idx.size) / max(1, d.size),
    }
    if keep_q:
        res["q"] = q
    return res


def lorenzo_codes(field: np.ndarray, rel_eb: float, radius: int = 512):
    """The codes of ``lorenzo_quantize``: ``(codes uint16, eb, outlier_fraction)``."""
    r = lorenzo_quantize(field, rel_eb, radius)
    return r["codes"], r["eb"], r["out_frac"]


def smooth_codes_1d(n: int, rel_eb: float, alphabet: int = 1024, noise: float = 1e-4,
                    seed: int = 1002) -> np.ndarray:
    """1D smooth field -> 1D Lorenzo codes with radius alphabet/2 (skew sweep, batches)."""
    f = fourier_field((n,), noise=noise, kmax=64, seed=seed)
    codes, _, _ = lorenzo_codes(f, rel_eb, radius=alphabet // 2)
    return codes


def field3d_codes(side: int = 512, rel_eb: float = 1e-4, noise: float = 0.01,
                  seed: int = 1001) -> np.ndarray:
    """The 3D workload: side^3 smooth field + noise, 3D Lorenzo, radius 512."""
    return field3d_quantized(side, rel_eb, noise, seed)["codes"]


def field3d_quantized(side: int = 512, rel_eb: float = 1e-4, noise: float = 0.01,
                      seed: int = 1001, keep_field: bool = False) -> dict:
    """``lorenzo_quantize`` of the 3D workload (codes, eb, outliers); with
    ``keep_field`` also the float32 field itself under ``field``."""
    f = fourier_field((side, side, side), noise=noise, kmax=8, seed=seed)
    r = lorenzo_quantize(f, rel_eb, radius=512)
    if keep_field:
        r["field"] = f
    return r


@dataclass
class FieldSpec:
    n: int
    alphabet: int
    rel_eb: float
    seed: int


def batch_spec(n_fields: int = 256, lo: int = 1 << 16, hi: int = 1 << 26,
               alphabets=(256, 1024, 4096), eb_lo: float = 1e-6, eb_hi: float = 1e-2,
               seed: int = 1003):
    """Sizes log-uniform in [lo, hi], alphabets uniform, error bounds log-uniform."""
    rng = _rng(seed)
    out = []
    for f in range(n_fields):
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        a = int(alphabets[int(rng.integers(0, len(alphabets)))])
        eb = float(math.exp(rng.uniform(math.log(eb_lo), math.log(eb_hi))))
        out.append(FieldSpec(n=n, alphabet=a, rel_eb=eb, seed=seed + 1 + f))
    return out


def code_stats(codes: np.ndarray, alphabet: int) -> dict:
    """Empirical entropy (bits/symbol) and the share of the centre bin."""
    cnt = np.bincount(codes, minlength=alphabet).astype(np.float64)
    p = cnt[cnt > 0] / cnt.sum()
    return {
        "entropy_bits": float(-(p * np.log2(p)).sum()),
        "p_center": float(cnt[alphabet // 2] / cnt.sum()),
        "p_outlier": float(cnt[0] / cnt.sum()),
    }
