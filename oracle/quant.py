"""Reference roundings for the reduced-precision leaf tiers.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper computes in FP32 only (Section 6.1). The BF16 and FP8 tiers are
this project's additions; these functions state the roundings those tiers
use, written from the IEEE-754 formats themselves (bit fields and
round-half-to-even), not from any library conversion:

  * bf16_rn(x): FP32 -> BF16 (1 sign, 8 exponent, 7 fraction bits),
    round to nearest, ties to even; NaN stays NaN.
  * split_bf16(x): hi = bf16_rn(x), lo = bf16_rn(x - hi), the difference
    taken in FP32 (exact, since hi is within one BF16 half-ulp of x).
  * split3_bf16(x): hi = bf16_rn(x), mid = bf16_rn(x - hi),
    lo = bf16_rn(x - hi - mid), both differences in FP32 (exact: x - hi has
    at most 16 significant bits and x - hi - mid at most 8, so lo holds it
    and hi + mid + lo == x).
  * e4m3_rn_sat(x): FP32 -> OCP FP8 E4M3 (bias 7, largest finite 448,
    smallest subnormal 2^-9, no infinities), round to nearest even,
    saturating to +-448.
  * fp8_block_quant(X): per 128 x 128 block scale s = amax/448 (s = 1 when
    amax = 0), code q = e4m3_rn_sat(x / s), both divisions in FP32.
"""
from __future__ import annotations

import numpy as np


def bf16_rn(x) -> np.ndarray:
    """FP32 -> BF16 round-to-nearest-even, returned as FP32 values."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    out = r.astype(np.uint32).view(np.float32)
    nan = np.isnan(f)
    if nan.any():
        out = out.copy()
        out[nan] = np.float32("nan")
    return out.reshape(f.shape)


def split_bf16(x) -> tuple[np.ndarray, np.ndarray]:
    """Two-term BF16 split: x ~ hi + lo with hi = bf16(x), lo = bf16(x - hi)."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    hi = bf16_rn(f)
    lo = bf16_rn((f - hi).astype(np.float32))
    return hi, lo


def split3_bf16(x) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Three-term BF16 split: x = hi + mid + lo with hi = bf16(x),
    mid = bf16(x - hi), lo = bf16(x - hi - mid)."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    hi = bf16_rn(f)
    r = (f - hi).astype(np.float32)
    mid = bf16_rn(r)
    lo = bf16_rn((r - mid).astype(np.float32))
    return hi, mid, lo


def e4m3_rn_sat(x) -> np.ndarray:
    """FP32 -> E4M3 (finite-only variant), nearest-even, saturating. Returned
    as FP32 values of the codes. NaN stays NaN."""
    f = np.asarray(x, dtype=np.float32).astype(np.float64)
    a = np.abs(f)
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.clip(e, -6, 8)          # exponent of the binade; -6 is the subnormal binade too
    q = np.exp2(e - 3)             # spacing of representable values (3 fraction bits)
    # log2 of a float can land a hair off at exact powers of two: fix the binade
    over = a >= np.exp2(e + 1)
    e = np.where(over & (e < 8), e + 1, e)
    under = (a < np.exp2(e)) & (e > -6)
    e = np.where(under, e - 1, e)
    q = np.exp2(e - 3)
    r = np.rint(a / q) * q         # np.rint rounds half to even; a/q is exact
    r = np.minimum(r, 448.0)
    out = (np.sign(f) * r).astype(np.float32)
    out[np.isnan(f)] = np.float32("nan")
    return out


def fp8_block_quant(X, block: int = 128):
    """Quantise a 2-D FP32 array with one FP32 scale per block x block tile.

    Returns (codes as FP32 values, scales of shape (ceil(r/block), ceil(c/block)))
    such that X ~ codes * scale of the element's block."""
    X = np.asarray(X, dtype=np.float32)
    r, c = X.shape
    gr, gc = -(-r // block), -(-c // block)
    scales = np.ones((gr, gc), dtype=np.float32)
    codes = np.zeros_like(X)
    for bi in range(gr):
        for bj in range(gc):
            t = X[bi * block:(bi + 1) * block, bj * block:(bj + 1) * block]
            amax = np.float32(np.max(np.abs(t))) if t.size else np.float32(0)
            s = np.float32(amax / np.float32(448.0)) if amax > 0 else np.float32(1.0)
            scales[bi, bj] = s
            codes[bi * block:(bi + 1) * block, bj * block:(bj + 1) * block] = \
                e4m3_rn_sat((t / s).astype(np.float32))
    return codes, scales
