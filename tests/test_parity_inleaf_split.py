"""The BF16x3 leaf writing its own operand planes (GPU).

Where both operands have their rows contiguous (op(A) = A, op(B) = B^T, 16-byte
aligned, leading dimensions multiples of 4) and the first round of pair tiles
reads at most half of the operands' rows, the plain BF16x3 leaf converts the
operands itself: the split kernels convert only the first round's rows, and
the leaf's idle control warps write the rest of the split planes chunk by
chunk while the TMA producer waits for each slab's chunks. The planes are the
same values, so the result must equal the launch with
HPVM_LAUNCH_SEPARATE_SPLIT bit for bit, on ragged shapes (rows, K), with the
tail split, and alpha/beta; and launches that miss a condition fall back to
the separate split. The converting leaf is told apart by its larger shared
memory (its staging buffers).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import sgemm as O
from paper_1611_00860_gb300 import _lib as H
from paper_1611_00860_gb300.sgemm import SgemmDFG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dfg(cuda_device):
    d = SgemmDFG(0)
    yield d
    d.close()


def _run(dfg, p, dev, flags):
    A, B, C0 = dev
    C = C0.clone()
    info = dfg.run_problem(p, H.HPVM_TIER_BF16X3, (A, B, C), flags=flags, timeout_ms=120000)
    torch.cuda.synchronize()
    return C, info


# (M, N, K, alpha, beta): ragged rows of both operands and K with a partial
# last slab, one slab only, B (or A) wholly in the first round (the
# converters then take only the other operand), the last round split in K
# halves
SHAPES = [(8192, 4096, 512, 1.0, 0.0), (6000, 6000, 777, 1.5, -0.5), (8192, 6144, 64, 1.0, 1.0),
          (16384, 2048, 300, 0.75, 0.25), (2048, 16384, 1000, 1.0, 0.5), (8192, 8192, 4096, 1.0, 1.0)]


@pytest.mark.parametrize("M,N,K,alpha,beta", SHAPES)
def test_inleaf_split_equals_separate_split(dfg, M, N, K, alpha, beta):
    p = W.sgemm_problem(M, N, K, seed=M + N + K, alpha=alpha, beta=beta)
    dev = tuple(t.cuda() for t in (p.A, p.B, p.C))
    fused, info_f = _run(dfg, p, dev, 0)
    separate, info_s = _run(dfg, p, dev, H.HPVM_LAUNCH_SEPARATE_SPLIT)
    assert info_f["smem_bytes"] > info_s["smem_bytes"], (info_f, info_s)  # the converting leaf ran
    assert torch.equal(fused, separate)
    # and the result against the oracle on sampled blocks
    blocks = W.sample_blocks(M, N, bs=256, count=6)
    Cv = W.col_major(fused, M, N, p.ldc)
    pairs = [(Cv[i0:i0 + 256, j0:j0 + 256].double().cpu().numpy(), O.sgemm_block_f64(p, i0, j0, 256, 256))
             for (i0, j0) in blocks]
    assert O.block_errors(pairs) <= 5e-6


def test_repeated_launches_are_identical(dfg):
    # the flags and the claim counter are reset for every launch: a second
    # launch (the same workspace) converts again and gives the same bits
    p = W.sgemm_problem(8192, 4096, 1000, seed=3)
    dev = tuple(t.cuda() for t in (p.A, p.B, p.C))
    first, info = _run(dfg, p, dev, 0)
    _, info_s = _run(dfg, p, dev, H.HPVM_LAUNCH_SEPARATE_SPLIT)
    assert info["smem_bytes"] > info_s["smem_bytes"]
    # change A between the launches: the planes must be made from the new values
    dev[0].mul_(-2.0)
    second, _ = _run(dfg, p, dev, 0)
    assert torch.equal(second, -2.0 * first)
    third, _ = _run(dfg, p, dev, 0)
    assert torch.equal(second, third)


@pytest.mark.parametrize("case", ["unaligned_ld", "transposed_A", "first_round_is_most", "beta_nan_c"])
def test_fallback_and_conditions(dfg, case):
    if case == "unaligned_ld":   # lda = M + 1: the FP32 rows cannot be TMA-read
        p = W.sgemm_problem(8192, 4096, 300, seed=4, pad=1)
        fused = False
    elif case == "transposed_A":  # op(A) = A^T: rows of op(A) are not contiguous
        p = W.sgemm_problem(8192, 4096, 300, seed=5, transA=True)
        fused = False
    elif case == "first_round_is_most":  # 4096^2: the first round reads over half of the rows
        p = W.sgemm_problem(4096, 4096, 300, seed=6)
        fused = False
    else:                        # beta = 0 never reads C (NaN there stays out)
        p = W.sgemm_problem(8192, 4096, 300, seed=7, beta=0.0)
        p.C.fill_(float("nan"))
        fused = True
    dev = tuple(t.cuda() for t in (p.A, p.B, p.C))
    C, info = _run(dfg, p, dev, 0)
    _, info_s = _run(dfg, p, dev, H.HPVM_LAUNCH_SEPARATE_SPLIT)
    assert (info["smem_bytes"] > info_s["smem_bytes"]) == fused, (info, info_s)
    got = W.col_major(C, p.M, p.N, p.ldc)
    assert torch.isfinite(got).all()
    blocks = W.sample_blocks(p.M, p.N, bs=256, count=4)
    pairs = [(got[i0:i0 + 256, j0:j0 + 256].double().cpu().numpy(), O.sgemm_block_f64(p, i0, j0, 256, 256))
             for (i0, j0) in blocks]
    assert O.block_errors(pairs) <= 5e-6


@pytest.mark.slow
def test_large_workload_equals_separate_split(dfg):
    # the benchmark's launch: M = N = K = 8192, beta = 1
    p = W.large_dfg_problem(8192)
    dev = tuple(t.cuda() for t in (p.A, p.B, p.C))
    fused, info_f = _run(dfg, p, dev, 0)
    separate, info_s = _run(dfg, p, dev, H.HPVM_LAUNCH_SEPARATE_SPLIT)
    assert info_f["smem_bytes"] > info_s["smem_bytes"]
    assert torch.equal(fused, separate)
