"""Pins of the split-BF16 products in exact arithmetic (``oracle.split``), CPU only.

The split tiers are defined by which products of BF16 parts they sum. These
tests tie ``split_block_f64`` to what that definition fixes independently of
the oracle's own code: exact integer products, inputs whose parts are known,
and the size of the representation error the definition implies (a dropped
or doubled cross term, a wrong sign or a missing part moves it by orders of
magnitude). They also record, for the record of what the method can reach,
that two BF16 parts are not enough on inputs with log-normal row scales:
there BF16x3 misses 5e-6 normwise in exact arithmetic, and BF16x6 does not.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import quant as Q
from oracle import sgemm as O
from oracle import split as S


@pytest.mark.parametrize("method", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("transA,transB", [(False, True), (True, False)])
def test_integer_inputs_exact(method, transA, transB):
    # integers in [-8, 8] are BF16 values: hi = x and the other parts vanish,
    # so every method gives the exact product
    p = W.sgemm_problem(70, 50, 90, seed=2, transA=transA, transB=transB, alpha=2.0, beta=0.5, dist="int8")
    got = S.split_block_f64(p, 0, 0, p.M, p.N, method)
    assert np.array_equal(got, O.sgemm_f64(p))


def test_bf16x3_drops_exactly_the_lo_lo_product():
    # operands with 16 significant bits: the two-term split is exact (hi +
    # lo == x), so BF16x3 differs from the exact product by alpha * lo_A lo_B
    # alone
    p = W.sgemm_problem(40, 30, 64, seed=5, alpha=1.0, beta=0.0)
    for t in (p.A, p.B):
        t.copy_((t.view(torch.int32) & 0xFFFFFF00).view(torch.float32))
    exact = O.sgemm_f64(p)
    got = S.split_block_f64(p, 0, 0, p.M, p.N, "bf16x3")
    a = W.col_major(p.A, p.M, p.K, p.lda).numpy()
    bt = W.col_major(p.B, p.N, p.K, p.ldb).numpy()
    lo_a = Q.split_bf16(a)[1].astype(np.float64)
    lo_b = Q.split_bf16(bt)[1].astype(np.float64)
    assert np.allclose(exact - got, lo_a @ lo_b.T, rtol=0, atol=1e-12 * np.abs(exact).max())
    # BF16x6 keeps mid*mid (the two-term split's lo*lo): exact up to FP64 sums
    assert O.normwise_rel_err(S.split_block_f64(p, 0, 0, p.M, p.N, "bf16x6"), exact) < 1e-15


def test_representation_error_on_normal_inputs():
    # N(0,1) operands, K = 4096: each two-part residual contributes about
    # 2.4e-6 and the dropped lo*lo about 2.8e-6, about 4.4e-6 together
    # (below the 5e-6 bound); the three-part split leaves terms near 2^-25
    p = W.sgemm_problem(256, 256, 4096, seed=8, alpha=1.0, beta=0.0)
    ref = O.sgemm_f64(p)
    e3 = O.normwise_rel_err(S.split_block_f64(p, 0, 0, 256, 256, "bf16x3"), ref)
    e6 = O.normwise_rel_err(S.split_block_f64(p, 0, 0, 256, 256, "bf16x6"), ref)
    assert 4.0e-6 <= e3 <= 4.8e-6, e3
    assert e6 <= 3e-8, e6


def test_lognormal_rows_need_three_parts():
    # the FP8 workload's inputs (per-row log-normal(0, 2) magnitudes) at
    # 4096: a few large rows and columns dominate the norm of the first
    # block, and the two-part representation alone puts BF16x3 above 5e-6
    # there; BF16x6 stays near 1e-8
    p = W.fp8_problem(4096)
    ref = O.sgemm_block_f64(p, 0, 0, 256, 256)
    e3 = O.normwise_rel_err(S.split_block_f64(p, 0, 0, 256, 256, "bf16x3"), ref)
    e6 = O.normwise_rel_err(S.split_block_f64(p, 0, 0, 256, 256, "bf16x6"), ref)
    assert e3 > 5e-6, e3
    assert e6 <= 5e-8, e6


def test_small_products_can_exceed_the_bound_in_exact_arithmetic():
    # A 24 x 16 product with K = 16 (the chain's small copy): 384 outputs of
    # 16-term dot products. The normwise error of BF16x3's three products is
    # about 4.4e-6 on average but spreads with so few terms: over 400 seeded
    # N(0,1) draws it exceeds 5e-6 in several; at 128 x 128 with K = 128 it
    # stays near 4.4e-6.
    def err(a, b):
        ah, al = (t.astype(np.float64) for t in Q.split_bf16(a))
        bh, bl = (t.astype(np.float64) for t in Q.split_bf16(b))
        ex = a.astype(np.float64) @ b.astype(np.float64).T
        return np.linalg.norm(ah @ bh.T + ah @ bl.T + al @ bh.T - ex) / np.linalg.norm(ex)
    rng = np.random.default_rng(9)
    small = [err(rng.standard_normal((24, 16)).astype(np.float32),
                 (rng.standard_normal((16, 16)) / 4).astype(np.float32)) for _ in range(400)]
    assert np.median(small) < 5e-6 and sum(e > 5e-6 for e in small) >= 5
    big = [err(rng.standard_normal((128, 128)).astype(np.float32),
               (rng.standard_normal((128, 128)) / np.sqrt(128)).astype(np.float32)) for _ in range(10)]
    assert max(big) < 4.8e-6
