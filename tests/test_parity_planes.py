"""The operand plane cache (HPVM_LAUNCH_CACHE_* / REUSE_*) on the GPU.

A stage that caches op(A) / op(B) converts them into the context's cache; a
later stage that reuses them skips the conversion kernels and computes the
same product bit for bit (the same planes through the same leaf). Reuse on
another stream waits for the conversion; refreshing a cached operand takes
its new values; one matrix used as both operands is converted once.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import sgemm as O
from paper_1611_00860_gb300 import _lib as H
from paper_1611_00860_gb300.sgemm import SgemmDFG

pytestmark = pytest.mark.gpu

TOL = {H.HPVM_TIER_BF16X3: 5e-6, H.HPVM_TIER_BF16: 1e-2, H.HPVM_TIER_FP8: 6e-2}
CACHE = H.HPVM_LAUNCH_CACHE_A | H.HPVM_LAUNCH_CACHE_B
REUSE = H.HPVM_LAUNCH_REUSE_A | H.HPVM_LAUNCH_REUSE_B


@pytest.fixture()
def dfg(cuda_device):
    d = SgemmDFG(0)
    yield d
    d.close()


def _launch(dfg, p, A, B, C, tier, flags, stream=None):
    a = dfg.args_for(p.M, p.N, p.K, A, p.lda, B, p.ldb, C, p.ldc, p.alpha, p.beta, p.transA,
                     p.transB, tier=tier, flags=flags)
    g = dfg.launch(a, stream)
    kernels = H.hpvm_graph_info(g).kernels
    dfg.wait(g, 60000)
    return kernels


@pytest.mark.parametrize("tier", list(TOL))
def test_cache_then_reuse_skips_conversion(dfg, tier):
    p = W.sgemm_problem(300, 260, 200, seed=31, alpha=1.5, beta=0.0, pad=2)
    A, B = p.A.cuda(), p.B.cuda()
    C1 = torch.zeros_like(p.C, device="cuda")
    C2 = torch.zeros_like(p.C, device="cuda")
    assert _launch(dfg, p, A, B, C1, tier, CACHE) == 3        # two conversions + the leaf
    assert H.hpvm_plane_cache_bytes(dfg.ctx) > 0
    assert _launch(dfg, p, A, B, C2, tier, REUSE) == 1        # the leaf alone
    torch.cuda.synchronize()
    assert torch.equal(C1.view(torch.int32), C2.view(torch.int32))
    got = W.col_major(C2.cpu(), p.M, p.N, p.ldc).double().numpy()
    assert O.normwise_rel_err(got, O.sgemm_f64(p)) <= TOL[tier]
    H.hpvm_drop_planes(dfg.ctx)
    assert H.hpvm_plane_cache_bytes(dfg.ctx) == 0


def test_reuse_without_cache_converts_once(dfg):
    # REUSE of an operand the cache does not hold yet converts and caches it
    p = W.sgemm_problem(200, 180, 150, seed=32)
    A, B = p.A.cuda(), p.B.cuda()
    C = torch.zeros_like(p.C, device="cuda")
    assert _launch(dfg, p, A, B, C, H.HPVM_TIER_BF16X3, H.HPVM_LAUNCH_REUSE_A) == 3
    assert _launch(dfg, p, A, B, C, H.HPVM_TIER_BF16X3, H.HPVM_LAUNCH_REUSE_A) == 2


def test_refresh_takes_new_values_and_reuse_keeps_old(dfg):
    p = W.sgemm_problem(256, 200, 128, seed=33, beta=0.0)
    A, B = p.A.cuda(), p.B.cuda()
    C = torch.zeros_like(p.C, device="cuda")
    _launch(dfg, p, A, B, C, H.HPVM_TIER_BF16X3, H.HPVM_LAUNCH_CACHE_A)
    old = O.sgemm_f64(p)
    A.mul_(2.0)
    p2 = W.SgemmProblem(**{**p.__dict__, "A": p.A * 2.0})
    new = O.sgemm_f64(p2)
    # reuse: the cached planes hold the old A (the caller's contract was broken)
    _launch(dfg, p, A, B, C, H.HPVM_TIER_BF16X3, H.HPVM_LAUNCH_REUSE_A)
    got = W.col_major(C.cpu(), p.M, p.N, p.ldc).double().numpy()
    assert O.normwise_rel_err(got, old) <= 5e-6
    # cache again: the new values
    _launch(dfg, p, A, B, C, H.HPVM_TIER_BF16X3, H.HPVM_LAUNCH_CACHE_A)
    got = W.col_major(C.cpu(), p.M, p.N, p.ldc).double().numpy()
    assert O.normwise_rel_err(got, new) <= 5e-6


def test_reuse_on_another_stream_waits_for_the_conversion(dfg):
    # a large conversion on stream 1, the reuse queued at once on stream 2
    n = 2048
    p = W.sgemm_problem(n, n, n, seed=34, beta=0.0)
    A, B = p.A.cuda(), p.B.cuda()
    C1 = torch.zeros_like(p.C, device="cuda")
    C2 = torch.zeros_like(p.C, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    for t in (A, B, C1, C2):
        t.record_stream(s1)
        t.record_stream(s2)
    a1 = dfg.args_for(n, n, n, A, n, B, n, C1, n, 1.0, 0.0, False, True, tier=H.HPVM_TIER_BF16X3,
                      flags=CACHE)
    a2 = dfg.args_for(n, n, n, A, n, B, n, C2, n, 1.0, 0.0, False, True, tier=H.HPVM_TIER_BF16X3,
                      flags=REUSE)
    dfg.ensure_workspace(a1)
    g1 = dfg.launch(a1, s1)
    g2 = dfg.launch(a2, s2)
    assert H.hpvm_graph_info(g2).kernels == 1
    dfg.wait(g1, 60000)
    dfg.wait(g2, 60000)
    torch.cuda.synchronize()
    assert torch.equal(C1.view(torch.int32), C2.view(torch.int32))
    blocks = W.sample_blocks(n, n, bs=128, count=3, seed=5)
    for i0, j0 in blocks:
        want = O.sgemm_block_f64(p, i0, j0, 128, 128)
        got = W.col_major(C2.cpu(), n, n, n)[i0:i0 + 128, j0:j0 + 128].double().numpy()
        assert O.normwise_rel_err(got, want) <= 5e-6


def test_one_matrix_as_both_operands(dfg):
    # C = A A^T: op(A) = A and op(B) = B^T with B the same buffer, ld and
    # shape, so both operands share one cache entry, converted once
    M, K = 192, 160
    g = torch.Generator().manual_seed(35)
    A = torch.randn(M * K, generator=g)
    p = W.SgemmProblem(M=M, N=M, K=K, A=A, lda=M, B=A, ldb=M, C=torch.zeros(M * M), ldc=M,
                       alpha=1.0, beta=0.0, transA=False, transB=True)
    Ad = A.cuda()
    C = torch.zeros(M * M, device="cuda")
    assert _launch(dfg, p, Ad, Ad, C, H.HPVM_TIER_BF16X3, CACHE) == 2
    got = W.col_major(C.cpu(), M, M, M).double().numpy()
    assert O.normwise_rel_err(got, O.sgemm_f64(p)) <= 5e-6
    assert _launch(dfg, p, Ad, Ad, C, H.HPVM_TIER_BF16X3, REUSE) == 1
    got2 = W.col_major(C.cpu(), M, M, M).double().numpy()
    assert np.array_equal(got, got2)
