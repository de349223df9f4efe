"""FP64 reference of the block-scaled FP8 sgemm leaf.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper computes in FP32 only (Section 6.1); the FP8 tier is this
project's addition. Its result is defined as the sgemm definition applied to
the dequantised operands:

    C <- alpha * deq(op(A)) * deq(op(B)) + beta * C,

where op(A) (M x K) and op(B)^T (N x K) are each quantised per 128 x 128
block with ``quant.fp8_block_quant`` (scale s = amax/448, code
q = e4m3_rn_sat(x/s)) and deq(x) = q * s of the element's block, all in FP64
after the quantisation. A matrix product from numpy serves as a step. The
error of the tier against the unquantised FP64 product is measured with
``sgemm.sgemm_block_f64`` on the original FP32 inputs.
"""
from __future__ import annotations

import numpy as np

from . import quant as Q

BLOCK = 128


def _op_rows(p, which: str, r0: int, r1: int) -> np.ndarray:
    """Rows [r0, r1) of op(A) (which='A', M x K) or of op(B)^T (which='B',
    N x K) as an FP32 array, read from the column-major buffers.

    op(A)(i, k) is A[i + k*lda], or A[k + i*lda] when A is transposed;
    op(B)^T(j, k) = op(B)(k, j) is B[j + k*ldb] when B is transposed, else
    B[k + j*ldb]."""
    if which == "A":
        buf, ld, rows_contiguous, nrows = p.A.numpy(), p.lda, not p.transA, p.M
    else:
        buf, ld, rows_contiguous, nrows = p.B.numpy(), p.ldb, p.transB, p.N
    if nrows == 0 or p.K == 0:
        return np.zeros((max(0, r1 - r0), p.K), dtype=np.float32)
    item = buf.itemsize
    strides = (item, item * ld) if rows_contiguous else (item * ld, item)
    view = np.lib.stride_tricks.as_strided(buf, shape=(nrows, p.K), strides=strides,
                                           writeable=False)
    return np.array(view[r0:r1], dtype=np.float32)


def quantize_panel(p, which: str, r0: int, r1: int):
    """Codes and scales of the 128-row blocks covering rows [r0, r1) of
    op(A) / op(B)^T (r0 a multiple of 128). Returns (codes, scales, rows)."""
    nrows = p.M if which == "A" else p.N
    r1 = min(r1, nrows)
    Y = _op_rows(p, which, r0, r1)
    codes, scales = Q.fp8_block_quant(Y, BLOCK)
    return codes, scales, r1 - r0


def _dequant(codes, scales) -> np.ndarray:
    s = np.repeat(np.repeat(scales.astype(np.float64), BLOCK, 0), BLOCK, 1)
    return codes.astype(np.float64) * s[: codes.shape[0], : codes.shape[1]]


def fp8_sgemm_block_f64(p, i0: int, j0: int, bm: int, bn: int) -> np.ndarray:
    """Rows [i0, i0+bm) x columns [j0, j0+bn) of alpha*deq(op(A))*deq(op(B)) +
    beta*C in FP64, as a (rows, cols) array (clipped to M x N)."""
    bm = max(0, min(bm, p.M - i0))
    bn = max(0, min(bn, p.N - j0))
    if bm == 0 or bn == 0:
        return np.zeros((bm, bn))
    # whole 128-row blocks: a block's scale depends on all of its rows
    a0, a1 = (i0 // BLOCK) * BLOCK, min(-(-(i0 + bm) // BLOCK) * BLOCK, p.M)
    b0, b1 = (j0 // BLOCK) * BLOCK, min(-(-(j0 + bn) // BLOCK) * BLOCK, p.N)
    qa, sa, _ = quantize_panel(p, "A", a0, a1)
    qb, sb, _ = quantize_panel(p, "B", b0, b1)
    da = _dequant(qa, sa)[i0 - a0: i0 - a0 + bm]
    db = _dequant(qb, sb)[j0 - b0: j0 - b0 + bn]
    out = p.alpha * (da @ db.T)
    if p.beta != 0.0:
        Cv = p.C.numpy()
        C = np.stack([Cv[i0 + j * p.ldc: i0 + bm + j * p.ldc] for j in range(j0, j0 + bn)], axis=1)
        out = out + p.beta * C.astype(np.float64)
    return out
