"""Pins of the oracle's sgemm definition (CPU only).

Each check ties the FP64 oracle to a fact it does not compute itself: closed
forms of special matrices, exact integer arithmetic, a matrix-vector route
through the product, and the NaN/beta conventions. A plausible slip in the
oracle (a dropped alpha or beta term, a swapped transpose, a wrong leading
dimension, a transposed operand) fails at least one of them; the planted
mistakes at the end show it.
"""
import math
import random

import numpy as np
import pytest
import torch

import workloads as W
from oracle import sgemm as O

TRANS = [(False, False), (False, True), (True, False), (True, True)]


def _problem_from(Aop, Bop, C, alpha, beta, transA, transB, pad=0):
    """Build a problem whose op(A), op(B) are the given (M,K), (K,N) arrays."""
    M, K = Aop.shape
    _, N = Bop.shape
    As = Aop.T if transA else Aop
    Bs = Bop.T if transB else Bop

    def flat(X, ld):
        r, c = X.shape
        f = torch.full((max(ld * c, 0),), float("nan"), dtype=torch.float32)
        if r * c:
            W.col_major(f, r, c, ld).copy_(torch.as_tensor(np.asarray(X, np.float32)))
        return f

    lda, ldb, ldc = As.shape[0] + pad, Bs.shape[0] + pad, M + pad
    return W.SgemmProblem(M, N, K, transA, transB, alpha, beta,
                          flat(As, lda), lda, flat(Bs, ldb), ldb, flat(C, ldc), ldc)


@pytest.mark.parametrize("transA,transB", TRANS)
def test_identity_gives_scaled_copy(transA, transB):
    # A = I (M = K): sum_p I(i,p) opB(p,j) = opB(i,j), so C = alpha*op(B) + beta*C
    rng = np.random.default_rng(1)
    M, N = 7, 5
    Bop = rng.standard_normal((M, N)).astype(np.float32)
    C = rng.standard_normal((M, N)).astype(np.float32)
    p = _problem_from(np.eye(M, dtype=np.float32), Bop, C, 1.5, -0.25, transA, transB, pad=3)
    got = O.sgemm_f64(p)
    want = 1.5 * Bop.astype(np.float64) - 0.25 * C.astype(np.float64)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("transA,transB", TRANS)
def test_rank_one_closed_form(transA, transB):
    # every column of op(A) is u, every row of op(B) is v: C = alpha*K*u v^T + beta*C
    M, N, K = 6, 4, 9
    u = np.arange(1, M + 1, dtype=np.float32) - 3
    v = np.arange(1, N + 1, dtype=np.float32) * 2 - 5
    Aop = np.repeat(u[:, None], K, axis=1)
    Bop = np.repeat(v[None, :], K, axis=0)
    C = np.full((M, N), 3.0, np.float32)
    p = _problem_from(Aop, Bop, C, 2.0, 0.5, transA, transB, pad=1)
    got = O.sgemm_f64(p)
    want = 2.0 * K * np.outer(u, v).astype(np.float64) + 0.5 * 3.0
    assert np.array_equal(got, want)


def test_rotations_compose():
    # R(a) R(b)^T = R(a - b); R(a) R(b) = R(a + b). The two differ unless sin(b) = 0,
    # so a swapped transpose of B is caught.
    a, b = 0.7, 0.3

    def R(t):
        return np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])

    Ra, Rb = R(a).astype(np.float32), R(b).astype(np.float32)
    zero = np.zeros((2, 2), np.float32)
    # NT form: op(B) = B^T with B stored as Rb
    p = W.SgemmProblem(2, 2, 2, False, True, 1.0, 0.0,
                       torch.tensor(Ra.T.reshape(-1)), 2, torch.tensor(Rb.T.reshape(-1)), 2,
                       torch.tensor(zero.reshape(-1)), 2)
    assert np.allclose(O.sgemm_f64(p), R(a - b), atol=2e-7)
    p.transB = False
    assert np.allclose(O.sgemm_f64(p), R(a + b), atol=2e-7)


@pytest.mark.parametrize("transA,transB", TRANS)
def test_selection_matrix_gathers_rows(transA, transB):
    # op(A)(i, s(i)) = 1 and 0 elsewhere: C(i, j) = alpha * opB(s(i), j)
    M, K, N = 5, 8, 3
    s = [7, 0, 3, 3, 5]
    Aop = np.zeros((M, K), np.float32)
    for i, k in enumerate(s):
        Aop[i, k] = 1.0
    rng = np.random.default_rng(3)
    Bop = rng.standard_normal((K, N)).astype(np.float32)
    p = _problem_from(Aop, Bop, np.zeros((M, N), np.float32), -2.0, 0.0, transA, transB, pad=2)
    got = O.sgemm_f64(p)
    assert np.array_equal(got, -2.0 * Bop[s].astype(np.float64))


@pytest.mark.parametrize("transA,transB", TRANS)
def test_integer_matrices_match_exact_arithmetic(transA, transB):
    # integers in [-8, 8]: compare with Python's exact integer sums
    M, N, K = 5, 4, 11
    rnd = random.Random(7)
    Aop = [[rnd.randint(-8, 8) for _ in range(K)] for _ in range(M)]
    Bop = [[rnd.randint(-8, 8) for _ in range(N)] for _ in range(K)]
    C = [[rnd.randint(-8, 8) for _ in range(N)] for _ in range(M)]
    p = _problem_from(np.array(Aop, np.float32), np.array(Bop, np.float32),
                      np.array(C, np.float32), 2.0, 3.0, transA, transB, pad=1)
    got = O.sgemm_f64(p)
    for i in range(M):
        for j in range(N):
            exact = 2 * sum(Aop[i][q] * Bop[q][j] for q in range(K)) + 3 * C[i][j]
            assert got[i, j] == exact


def test_beta_zero_does_not_read_c_and_padding_is_not_read():
    p = W.sgemm_problem(9, 7, 5, seed=4, pad=3, beta=0.0)
    p.C.fill_(float("nan"))
    got = O.sgemm_f64(p)
    assert np.isfinite(got).all()
    # the leading-dimension slack of A and B holds NaN (see workloads): unread
    p2 = W.sgemm_problem(9, 7, 5, seed=4, pad=3, beta=0.5)
    assert np.isfinite(O.sgemm_f64(p2)).all()


def test_empty_dimensions():
    p = W.sgemm_problem(4, 3, 0, seed=5, alpha=2.0, beta=0.5)
    C = W.col_major(p.C, 4, 3, p.ldc).double().numpy()
    assert np.array_equal(O.sgemm_f64(p), 0.5 * C)  # K = 0: only beta*C remains
    assert O.sgemm_f64(W.sgemm_problem(0, 3, 4, seed=5)).shape == (0, 3)
    assert O.sgemm_f64(W.sgemm_problem(3, 0, 4, seed=5)).shape == (3, 0)


@pytest.mark.parametrize("transA,transB", TRANS)
def test_freivalds_matrix_vector_route(transA, transB):
    # (alpha op(A) op(B) + beta C) x  =  alpha op(A) (op(B) x) + beta C x
    p = W.sgemm_problem(70, 50, 90, seed=6, transA=transA, transB=transB,
                        alpha=0.75, beta=-1.25, pad=2)
    got = O.sgemm_f64(p)
    ar, ac = p.a_shape
    br, bc = p.b_shape
    A = W.col_major(p.A, ar, ac, p.lda).double().numpy()
    B = W.col_major(p.B, br, bc, p.ldb).double().numpy()
    C = W.col_major(p.C, p.M, p.N, p.ldc).double().numpy()
    opA = A.T if transA else A
    opB = B.T if transB else B
    x = np.random.default_rng(8).standard_normal(p.N)
    lhs = got @ x
    rhs = 0.75 * (opA @ (opB @ x)) - 1.25 * (C @ x)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-10)


def test_blocks_agree_with_whole_and_clip():
    p = W.sgemm_problem(300, 200, 64, seed=9, beta=0.5)
    full = O.sgemm_f64(p)
    for (i0, j0) in W.sample_blocks(p.M, p.N, bs=128, count=4):
        blk = O.sgemm_block_f64(p, i0, j0, 128, 128)
        assert np.array_equal(blk, full[i0:i0 + 128, j0:j0 + 128])


def test_normwise_metric():
    ref = np.array([[3.0, 0.0], [0.0, 4.0]])
    assert O.normwise_rel_err(ref, ref) == 0.0
    assert O.normwise_rel_err(ref + np.array([[0, 0], [0, 0.5]]), ref) == pytest.approx(0.1)
    assert O.block_errors([(ref, ref), (ref * 0, ref)]) == pytest.approx(math.sqrt(0.5))


# ---------------------------------------------------------------------------
# Planted mistakes: wrong variants of the oracle (on the CPU) must fail a pin.
# ---------------------------------------------------------------------------

def _variant(p, mistake):
    ar, ac = p.a_shape
    br, bc = p.b_shape
    A = W.col_major(p.A, ar, ac, p.lda).double().numpy()
    B = W.col_major(p.B, br, bc, p.ldb).double().numpy()
    C = W.col_major(p.C, p.M, p.N, p.ldc).double().numpy()
    opA = A.T if p.transA else A
    opB = B.T if p.transB else B
    alpha, beta = p.alpha, p.beta
    if mistake == "swap_transB":
        opB = B if p.transB else B.T
    if mistake == "drop_beta":
        beta = 0.0
    if mistake == "drop_alpha":
        alpha = 1.0
    if mistake == "transpose_result":
        return (alpha * (opA @ opB) + beta * C).T.copy()
    return alpha * (opA @ opB) + beta * C


@pytest.mark.parametrize("mistake", ["swap_transB", "drop_beta", "drop_alpha",
                                     "transpose_result"])
def test_planted_mistakes_are_caught(mistake):
    caught = False
    # identity pin with a non-symmetric square B
    rng = np.random.default_rng(1)
    Bop = rng.standard_normal((4, 4)).astype(np.float32)
    C = rng.standard_normal((4, 4)).astype(np.float32)
    p = _problem_from(np.eye(4, dtype=np.float32), Bop, C, 1.5, -0.25, False, True)
    want = 1.5 * Bop.astype(np.float64) - 0.25 * C.astype(np.float64)
    got = _variant(p, mistake)
    caught |= not (got.shape == want.shape and np.array_equal(got, want))
    assert caught
