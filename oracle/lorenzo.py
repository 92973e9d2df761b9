"""CPU oracle of the Lorenzo reconstruction that follows the decoder (test
infrastructure only; the same import rules as the rest of ``oracle``).

The paper's end-to-end measurement (Sec. V-B2, cuSZ decompression) is the
Huffman decode followed by cuSZ's Lorenzo reconstruction, which the paper
cites but never defines.  This module reads it as cuSZ's first-order Lorenzo
predictor on prequantized integers, zero outside the domain:

* a code c in [1, 2R) stands for the residue d = c - R; code 0 marks an
  outlier whose residue is stored aside (position, value);
* the prequantized value q is the inclusive prefix sum of d along every axis
  (the inverse of the predictor's inclusion-exclusion difference);
* the reconstructed value is 2 eb q, rounded to float32 in one defined way:
  float32(q) * float32(2 eb), both roundings to nearest even.

Plain numpy in int64; no blocking or reordering beyond the definition.
"""
from __future__ import annotations

import numpy as np


class ReconstructError(ValueError):
    pass


def ebx2_f32(eb: float) -> np.float32:
    """The float32 step 2 eb (the double product rounded once to float32)."""
    return np.float32(2.0 * float(eb))


def residues(codes, radius: int, out_idx=None, out_val=None) -> np.ndarray:
    """Flat int64 residues: code - radius, outliers' stored values at code 0.

    The outlier list must name exactly the positions whose code is 0, in
    ascending order; anything else is rejected."""
    c = np.asarray(codes, dtype=np.uint16).reshape(-1)
    d = c.astype(np.int64) - int(radius)
    idx = np.zeros(0, np.int64) if out_idx is None else np.asarray(out_idx).astype(np.int64)
    val = np.zeros(0, np.int64) if out_val is None else np.asarray(out_val).astype(np.int64)
    if idx.shape != val.shape:
        raise ReconstructError("outlier positions and values differ in length")
    if idx.size and (np.any(np.diff(idx) <= 0) or idx[0] < 0 or idx[-1] >= c.size):
        raise ReconstructError("outlier positions not ascending or out of range")
    zero = np.flatnonzero(c == 0)
    if zero.size != idx.size or not np.array_equal(zero, idx):
        raise ReconstructError("outlier list does not match the positions of code 0")
    d[idx] = val
    return d


def prequantized(d, dims) -> np.ndarray:
    """q: inclusive prefix sums of the residues along every axis.  ``dims`` is
    (nx,), (nx, ny) or (nx, ny, nz) with nx varying fastest."""
    shape = tuple(int(v) for v in reversed(dims))
    q = np.asarray(d, dtype=np.int64).reshape(shape)
    for ax in range(q.ndim):
        q = np.cumsum(q, axis=ax)
    return q


def reconstruct(codes, dims, radius: int, eb: float, out_idx=None, out_val=None,
                return_q: bool = False):
    """Flat float32 reconstruction (and, with ``return_q``, the int64 q)."""
    n = int(np.prod([int(v) for v in dims])) if len(dims) else 0
    if np.asarray(codes).size != n:
        raise ReconstructError("code count differs from the grid size")
    q = prequantized(residues(codes, radius, out_idx, out_val), dims).reshape(-1)
    if q.size and np.abs(q).max() >= (1 << 31):
        raise ReconstructError("prequantized value outside int32")
    x = q.astype(np.float32) * ebx2_f32(eb)
    return (x, q) if return_q else x
