"""The split-BF16 tiers' products in exact arithmetic.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper computes the SgemmLeaf of Section 6.1 in FP32. The split tiers are
this project's way of reaching FP32 accuracy on BF16 tensor cores: every
FP32 operand element is written as a sum of BF16 parts (``quant.split_bf16``
gives two, ``quant.split3_bf16`` three) and the leaf sums a fixed set of
products of parts:

  * BF16x3: hi*hi + hi*lo + lo*hi (the product lo*lo is dropped);
  * BF16x6: hi*hi + hi*mid + mid*hi + mid*mid + hi*lo + lo*hi (mid*lo, lo*mid
    and lo*lo are dropped).

``split_block_f64`` evaluates alpha * (that sum) + beta * C for one block of
the result with every product and sum in FP64. Products of two BF16 values
are exact in FP64 and the sums over K lose only FP64 rounding, so this is
the value a tier would return if its accumulation were exact: its distance
from ``sgemm.sgemm_block_f64`` is the error the representation alone
causes, and a GPU result's distance from it is the accumulation error.
A matrix product from numpy serves as a step.
"""
from __future__ import annotations

import numpy as np

import workloads as W

from . import quant as Q

PRODUCTS = {
    "bf16x3": ((0, 0), (0, 1), (1, 0)),
    "bf16x6": ((0, 0), (0, 1), (1, 0), (1, 1), (0, 2), (2, 0)),
}


def _op_rows(flat, rows_stored, cols_stored, ld, trans, r0, r1):
    """Rows r0..r1 of op(X) (op(X) = X, or X^T when trans) as a dense
    (r1 - r0, K) FP32 array."""
    X = W.col_major(flat, rows_stored, cols_stored, ld)
    Y = X.t() if trans else X
    return np.ascontiguousarray(Y[r0:r1].numpy(), dtype=np.float32)


def parts(x, method: str):
    """The BF16 parts of x the method uses, as FP64 arrays."""
    if method == "bf16x3":
        ps = Q.split_bf16(x)
    elif method == "bf16x6":
        ps = Q.split3_bf16(x)
    else:
        raise ValueError(method)
    return [np.asarray(t, dtype=np.float64) for t in ps]


def split_block_f64(p, i0: int, j0: int, bm: int, bn: int, method: str) -> np.ndarray:
    """Rows [i0, i0+bm) x columns [j0, j0+bn) of alpha * sum over the method's
    products of op(A)_s * op(B)_t + beta * C, in FP64, clipped to the M x N
    result. ``p`` is a ``workloads.SgemmProblem``."""
    bm = max(0, min(bm, p.M - i0))
    bn = max(0, min(bn, p.N - j0))
    if bm == 0 or bn == 0:
        return np.zeros((bm, bn))
    ar, ac = W.stored_shape(p.M, p.K, p.transA)
    br, bc = W.stored_shape(p.K, p.N, p.transB)
    # op(A) rows i0.. (K columns); op(B)^T rows j0.. (K columns)
    a = _op_rows(p.A, ar, ac, p.lda, p.transA, i0, i0 + bm)
    bt = _op_rows(p.B, br, bc, p.ldb, not p.transB, j0, j0 + bn)
    pa, pb = parts(a, method), parts(bt, method)
    acc = np.zeros((bm, bn))
    for s, t in PRODUCTS[method]:
        acc += pa[s] @ pb[t].T
    out = p.alpha * acc
    if p.beta != 0.0:
        Cb = W.col_major(p.C, p.M, p.N, p.ldc)[i0:i0 + bm, j0:j0 + bn].numpy().astype(np.float64)
        out = out + p.beta * Cb
    return out
