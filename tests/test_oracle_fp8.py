"""Pins of the oracle's block-scaled FP8 product (CPU only).

* Integer operands whose every 128 x 128 block holds a +-448: the scale of
  every block is exactly 1 and every other entry (|x| <= 16) is an exact
  E4M3 code, so the FP8 product must equal Python's exact integer sums.
* Quantisation bounds: against the unquantised FP64 product, each operand
  element moves by at most 2^-4 of itself (normal codes) or half the
  smallest subnormal spacing times the scale.
* A block of zeros keeps scale 1 and contributes nothing.
"""
import random

import numpy as np
import pytest
import torch

import workloads as W
from oracle import fp8 as F
from oracle import quant as Q
from oracle import sgemm as O


def _int_problem(M, N, K, transA, transB, seed):
    """Integer entries in [-16, 16] with a 448 in every 128x128 block of
    op(A) and op(B)^T, so all block scales are 1."""
    rnd = random.Random(seed)
    opA = np.array([[rnd.randint(-16, 16) for _ in range(K)] for _ in range(M)], np.float32)
    opBt = np.array([[rnd.randint(-16, 16) for _ in range(K)] for _ in range(N)], np.float32)
    for X in (opA, opBt):
        for r in range(0, X.shape[0], 128):
            for c in range(0, X.shape[1], 128):
                X[r, c] = 448.0 if (r + c) % 256 == 0 else -448.0
    C = np.array([[rnd.randint(-4, 4) for _ in range(N)] for _ in range(M)], np.float32)
    As = opA.T if transA else opA
    Bs = opBt if transB else opBt.T

    def flat(X):
        r, c = X.shape
        f = torch.zeros(r * c, dtype=torch.float32)
        W.col_major(f, r, c, r).copy_(torch.from_numpy(np.ascontiguousarray(X)))
        return f, r

    A, lda = flat(As)
    B, ldb = flat(Bs)
    Cf, ldc = flat(C)
    p = W.SgemmProblem(M, N, K, transA, transB, 2.0, 0.5, A, lda, B, ldb, Cf, ldc)
    return p, opA, opBt, C


@pytest.mark.parametrize("transA,transB", [(False, True), (True, False)])
def test_exact_integer_case(transA, transB):
    M, N, K = 140, 130, 260
    p, opA, opBt, C = _int_problem(M, N, K, transA, transB, seed=3)
    got = F.fp8_sgemm_block_f64(p, 0, 0, M, N)
    a = opA.astype(np.int64)
    b = opBt.astype(np.int64)
    exact = 2 * (a @ b.T) + C.astype(np.float64) * 0.5
    assert np.array_equal(got, exact)
    # scales are all exactly one
    _, s, _ = F.quantize_panel(p, "A", 0, M)
    assert (s == 1.0).all()


def test_quantisation_error_bound_and_definition():
    p = W.sgemm_problem(200, 150, 300, seed=7, alpha=1.0, beta=0.0)
    got = F.fp8_sgemm_block_f64(p, 0, 0, p.M, p.N)
    ref = O.sgemm_f64(p)
    err = O.normwise_rel_err(got, ref)
    assert 1e-3 < err < 6e-2  # quantised, but within the FP8 tier's bound
    # an output sub-block computed alone equals the same block of the whole
    sub = F.fp8_sgemm_block_f64(p, 130, 20, 50, 60)
    assert np.allclose(sub, got[130:180, 20:80], rtol=1e-12, atol=1e-12)


def test_elementwise_quantisation_bound():
    g = torch.Generator().manual_seed(5)
    X = (torch.randn(256, 384, generator=g) * torch.exp(2 * torch.randn(256, 1, generator=g))).numpy()
    codes, s = Q.fp8_block_quant(X)
    deq = codes.astype(np.float64) * np.repeat(np.repeat(s, 128, 0), 128, 1)
    err = np.abs(deq - X)
    sub = np.repeat(np.repeat(s, 128, 0), 128, 1) * 2.0 ** -10  # half the subnormal spacing
    assert (err <= np.maximum(2.0 ** -4 * np.abs(X), sub) * (1 + 1e-6)).all()


def test_zero_block():
    p = W.sgemm_problem(128, 128, 256, seed=9, beta=0.0)
    Av = W.col_major(p.A, 128, 256, p.lda)
    Av[:, :128] = 0.0
    _, s, _ = F.quantize_panel(p, "A", 0, 128)
    assert s[0, 0] == 1.0
    got = F.fp8_sgemm_block_f64(p, 0, 0, 128, 128)
    assert np.isfinite(got).all()
