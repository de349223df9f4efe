"""FP64 definition of the sgemm leaf, and the error metric.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows Section 6.1 (the SgemmLeaf node of the sgemm example: arguments A,
lda, B, ldb, C, ldc, k, alpha, beta; A and B ``in``, C ``in out`` per
Section 2.3). Reading taken where the paper is silent: column-major storage,
op(A) = A or A^T and op(B) = B or B^T chosen by flags (the example's own form
is op(A) = A, op(B) = B^T), explicit M and N, and the BLAS convention that
beta == 0 means C is not read.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from .build import build

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, f64, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        fp = ctypes.c_void_p
        lib.oracle_sgemm_block_f64.argtypes = [
            i32, i32, i64, i64, i64, f64, fp, i64, fp, i64, f64, fp, i64,
            i64, i64, i64, i64, fp, i64]
        lib.oracle_sgemm_block_f64.restype = i32
        lib.oracle_num_threads.restype = i32
        lib.oracle_set_num_threads.argtypes = [i32]
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


def _ptr(t: torch.Tensor) -> int:
    assert t.dtype == torch.float32 and t.device.type == "cpu" and t.is_contiguous()
    return t.data_ptr()


def sgemm_block_f64(p, i0: int, j0: int, bm: int, bn: int) -> np.ndarray:
    """Rows [i0, i0+bm) x columns [j0, j0+bn) of alpha*op(A)*op(B) + beta*C in
    FP64, clipped to the M x N result. ``p`` is a ``workloads.SgemmProblem``
    (or any object with the same fields). Returns a (rows, cols) array."""
    bm = max(0, min(bm, p.M - i0))
    bn = max(0, min(bn, p.N - j0))
    out = np.zeros((bn, bm), dtype=np.float64)  # column-major bm x bn
    if bm and bn:
        lib = _load()
        empty = torch.zeros(1, dtype=torch.float32)
        A = p.A if p.A.numel() else empty
        B = p.B if p.B.numel() else empty
        C = p.C if p.C.numel() else empty
        rc = lib.oracle_sgemm_block_f64(
            int(p.transA), int(p.transB), p.M, p.N, p.K, float(p.alpha),
            _ptr(A), p.lda, _ptr(B), p.ldb, float(p.beta), _ptr(C), p.ldc,
            i0, j0, bm, bn, out.ctypes.data, bm)
        if rc != 0:
            raise MemoryError("oracle panel allocation failed")
    return out.T


def sgemm_f64(p) -> np.ndarray:
    """The whole M x N result in FP64, as an (M, N) array."""
    return sgemm_block_f64(p, 0, 0, p.M, p.N)


def normwise_rel_err(got, ref) -> float:
    """||got - ref||_F / ||ref||_F with FP64 accumulation (0/0 -> 0)."""
    g = np.asarray(got, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    num = float(np.sqrt(np.sum((g - r) ** 2)))
    den = float(np.sqrt(np.sum(r ** 2)))
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return num / den


def block_errors(blocks):
    """Normwise relative error over a list of (got, ref) blocks taken together:
    sqrt(sum ||got-ref||^2) / sqrt(sum ||ref||^2)."""
    num = 0.0
    den = 0.0
    for got, ref in blocks:
        g = np.asarray(got, dtype=np.float64)
        r = np.asarray(ref, dtype=np.float64)
        num += float(np.sum((g - r) ** 2))
        den += float(np.sum(r ** 2))
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return float(np.sqrt(num / den))
