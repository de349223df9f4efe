"""The allocation-free BF16x3 entry point (GPU).

hpvm_sgemm_bf16x3_noalloc serves callers that cannot allocate device memory
at call time (code inside another framework's memory pool, latency-critical
threads where cudaMalloc may synchronise the device). It keeps the split
planes in a fixed array inside the library instead of a workspace. These
tests call it through the C-ABI and compare its C with the C that the
regular entry point (hpvm_launch, BF16X3 tier, with a workspace) computes
from the same inputs, within the BF16x3 tolerance (normwise 5e-6), on two
calls in a row with different problems, and check that an oversized problem
is refused. This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import sgemm as O
from paper_1611_00860_gb300 import _lib as H
from paper_1611_00860_gb300.sgemm import SgemmDFG

pytestmark = pytest.mark.gpu

TOL = 5e-6


def _regular(dfg, p, A, B, C):
    dfg.run_problem(p, H.HPVM_TIER_BF16X3, (A, B, C))
    torch.cuda.synchronize()
    return W.col_major(C.cpu(), p.M, p.N, p.ldc).double().numpy()


def _noalloc(p, A, B, C, status):
    s = torch.cuda.current_stream()
    H.hpvm_sgemm_bf16x3_noalloc(p.M, p.N, p.K, p.alpha, A.data_ptr(), p.lda, B.data_ptr(), p.ldb,
                                p.beta, C.data_ptr(), p.ldc, p.transA, p.transB,
                                status.data_ptr(), s.cuda_stream)
    torch.cuda.synchronize()
    return W.col_major(C.cpu(), p.M, p.N, p.ldc).double().numpy()


def test_noalloc_matches_regular_entry_point_two_calls(cuda_device):
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    dfg = SgemmDFG(0)
    try:
        problems = [
            W.sgemm_problem(300, 200, 100, seed=31, alpha=1.5, beta=0.5, pad=3),
            W.sgemm_problem(1024, 768, 2048, seed=32, transA=True, transB=False,
                            alpha=-0.75, beta=1.25),
        ]
        for p in problems:  # two calls in a row, different shapes and contents
            A, B, C0 = (t.cuda() for t in (p.A, p.B, p.C))
            want = _regular(dfg, p, A, B, C0.clone())
            got = _noalloc(p, A, B, C0.clone(), status)
            assert int(status.item()) == 0
            assert np.isfinite(got).all()
            assert O.normwise_rel_err(got, want) <= TOL
            # and both stay within the tier's bound of the FP64 definition
            assert O.normwise_rel_err(got, O.sgemm_f64(p)) <= TOL
    finally:
        dfg.close()


def test_noalloc_refuses_problems_beyond_its_scratch(cuda_device):
    # 4*(M+N)*Kp bytes of planes: 8192 x 8192 x 1024 needs 64 MiB + padding > 64 MiB
    A = torch.zeros(16, device="cuda")
    with pytest.raises(H.HpvmError) as e:
        H.hpvm_sgemm_bf16x3_noalloc(8192, 8192, 1032, 1.0, A.data_ptr(), 8192, A.data_ptr(), 8192,
                                    0.0, A.data_ptr(), 8192, False, True, None,
                                    torch.cuda.current_stream().cuda_stream)
    assert e.value.code == H.HPVM_ERR_SHAPE
    assert "scratch" in str(e.value)


@pytest.mark.parametrize("M,N,K", [(2560, 2304, 520), (2560, 2560, 3000)])
def test_noalloc_with_a_split_tail(cuda_device, M, N, K):
    # Shapes whose last round of pair tiles splits in K halves on a 152-SM
    # GB300 (90 and 100 pair tiles for 76 pairs). In the first the array
    # also holds the split's partial sums; in the second the planes alone
    # take 61 MB of the 64 MiB, so the call is accepted (the planes fit) and
    # runs whole tiles. Both agree with the regular entry point.
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    dfg = SgemmDFG(0)
    try:
        p = W.sgemm_problem(M, N, K, seed=M + K, alpha=1.25, beta=-0.5)
        A, B, C0 = (t.cuda() for t in (p.A, p.B, p.C))
        want = _regular(dfg, p, A, B, C0.clone())
        got = _noalloc(p, A, B, C0.clone(), status)
        assert int(status.item()) == 0
        assert np.isfinite(got).all()
        assert O.normwise_rel_err(got, want) <= TOL
    finally:
        dfg.close()
