"""Low-precision copies of A (oracle, test infrastructure).

The paper computes in one precision only; the streamed low-precision copies are an extension
of the x-subproblem's inexactness (an approximate Hessian, §2 after Eq. (6)).  Definitions:

* ``bf16_rne(x)``: the bfloat16 value nearest to the float32 value x, ties to the value
  whose last significand bit is 0 (round to nearest even).  bfloat16 = 1 sign, 8 exponent,
  7 fraction bits (the top 16 bits of a float32).
* ``split_hi_lo(A)``: hi = bf16_rne(A32), lo = bf16_rne(A32 - hi) (difference in float32).
* ``e4m3_rne(x)``: the FP8 E4M3 (OCP "FN" variant: bias 7, no infinities, max 448) value
  nearest to x, ties to even, saturating to +-448.
* ``quantize_fp8_rows(A)``: per-row scale s_i = amax_i / 448 (float32 division; s_i = 1 for
  an all-zero row) and codes e4m3_rne(a_ij / s_i) (float32 division).

Implemented from the format definitions by enumeration of the representable values, not by
bit tricks.  Pinned against torch's CPU bfloat16 / float8_e4m3fn casts and hand-checked values.
"""
from __future__ import annotations

import numpy as np


def _bf16_grid_neighbors(x32):
    """Round toward zero to bf16 and the next bf16 away from zero (both as float32)."""
    bits = x32.view(np.uint32)
    low = (bits & np.uint32(0xFFFF0000)).view(np.float32)
    up_bits = (bits & np.uint32(0xFFFF0000)) + np.uint32(0x10000)
    up = up_bits.view(np.float32)
    return low, up


def bf16_rne(x):
    """float32 array -> float32 array holding the nearest bf16 values (ties to even)."""
    x32 = np.ascontiguousarray(x, dtype=np.float32)
    low, up = _bf16_grid_neighbors(x32)
    # distances measured exactly in float64
    dl = np.abs(x32.astype(np.float64) - low.astype(np.float64))
    du = np.abs(up.astype(np.float64) - x32.astype(np.float64))
    low_even = ((low.view(np.uint32) >> np.uint32(16)) & np.uint32(1)) == 0
    pick_up = (du < dl) | ((du == dl) & ~low_even)
    out = np.where(pick_up, up, low).astype(np.float32)
    exact = low == x32
    out[exact] = x32[exact]
    return out


def bf16_bits(x):
    return (bf16_rne(x).view(np.uint32) >> np.uint32(16)).astype(np.uint16)


def split_hi_lo(A):
    A32 = np.ascontiguousarray(A, dtype=np.float32)
    hi = bf16_rne(A32)
    lo = bf16_rne((A32 - hi).astype(np.float32))
    return hi, lo


def e4m3_values():
    """All 256 E4M3FN code values (NaN for the two NaN codes)."""
    vals = np.empty(256, dtype=np.float64)
    for c in range(256):
        s = -1.0 if c & 0x80 else 1.0
        e = (c >> 3) & 0xF
        f = c & 0x7
        if e == 0xF and f == 0x7:
            vals[c] = np.nan
        elif e == 0:
            vals[c] = s * (f / 8.0) * 2.0 ** (-6)
        else:
            vals[c] = s * (1.0 + f / 8.0) * 2.0 ** (e - 7)
    return vals


_E4M3 = e4m3_values()
_POS_CODES = np.array([c for c in range(0x7F) if not np.isnan(_E4M3[c])], dtype=np.int64)
_POS_VALS = _E4M3[_POS_CODES]          # increasing, 0 .. 448


def e4m3_rne_codes(x):
    """float array -> uint8 E4M3 codes, nearest value with ties to even code, saturating."""
    x = np.asarray(x, dtype=np.float64)
    a = np.minimum(np.abs(x), 448.0)
    j = np.searchsorted(_POS_VALS, a, side="left")       # first value >= a
    j = np.clip(j, 0, _POS_VALS.size - 1)
    i = np.clip(j - 1, 0, _POS_VALS.size - 1)
    vi, vj = _POS_VALS[i], _POS_VALS[j]
    di, dj = a - vi, vj - a
    ci, cj = _POS_CODES[i], _POS_CODES[j]
    pick_j = (dj < di) | ((dj == di) & (cj % 2 == 0))
    code = np.where(pick_j, cj, ci)
    code = np.where(vj == a, cj, code)
    neg = (x < 0) & (code != 0)
    code = code | np.where(neg, 0x80, 0)
    return code.astype(np.uint8)


def e4m3_decode(codes):
    return _E4M3[np.asarray(codes, dtype=np.int64)]


def quantize_fp8_rows(A):
    """Returns (codes uint8 (m, n), scales float32 (m,)): a_ij ~= scales_i * e4m3(codes_ij)."""
    A32 = np.ascontiguousarray(A, dtype=np.float32)
    amax = np.max(np.abs(A32), axis=1) if A32.shape[1] else np.zeros(A32.shape[0], np.float32)
    scales = (amax / np.float32(448.0)).astype(np.float32)
    scales[scales == 0] = np.float32(1.0)
    q = (A32 / scales[:, None]).astype(np.float32)
    return e4m3_rne_codes(q), scales
