"""Two contexts on two devices in one process, launches alternating (GPU).

The leaves' per-device state (the dynamic shared-memory opt-in of each
kernel, the cluster occupancy, the SM count) is cached per device: a launch
on device 1 after one on device 0 must not reuse device 0's settings. Each
device runs BF16x3 (CTA pairs, the converting leaf at 4096 x 4096 x 512),
FP8 (single CTAs) and BF16x3 through the allocation-free entry point, and
every result is checked against the oracle. Needs two visible GPUs; skipped
otherwise.
"""
import pytest
import torch

import workloads as W
from oracle import fp8 as F
from oracle import sgemm as O
from paper_1611_00860_gb300 import _lib as H
from paper_1611_00860_gb300.sgemm import SgemmDFG

pytestmark = pytest.mark.gpu

CASES = [(H.HPVM_TIER_BF16X3, (4096, 4096, 512), 5e-6), (H.HPVM_TIER_FP8, (1024, 768, 640), 1e-5),
         (H.HPVM_TIER_BF16X3, (1000, 700, 300), 5e-6)]


@pytest.fixture(scope="module")
def two_devices():
    if not torch.cuda.is_available() or torch.cuda.device_count() < 2:
        pytest.skip("needs two visible CUDA devices")
    ds = [SgemmDFG(0), SgemmDFG(1)]
    yield ds
    for d in ds:
        d.close()


def _check(dev, dfg, tier, shape, tol, seed):
    M, N, K = shape
    p = W.sgemm_problem(M, N, K, seed=seed, alpha=1.0, beta=0.5)
    A, B, C = (t.to(f"cuda:{dev}") for t in (p.A, p.B, p.C))
    with torch.cuda.device(dev):
        dfg.run_problem(p, tier, (A, B, C))
        torch.cuda.synchronize(dev)
    Cv = W.col_major(C.cpu(), M, N, p.ldc)
    blocks = W.sample_blocks(M, N, bs=256, count=2)
    ref = F.fp8_sgemm_block_f64 if tier == H.HPVM_TIER_FP8 else O.sgemm_block_f64
    pairs = [(Cv[i0:i0 + 256, j0:j0 + 256].double().numpy(), ref(p, i0, j0, min(256, M - i0), min(256, N - j0)))
             for i0, j0 in blocks]
    assert O.block_errors(pairs) <= tol, (dev, tier, shape)


def test_launches_alternate_between_devices(two_devices):
    for rep in range(2):
        for i, (tier, shape, tol) in enumerate(CASES):
            for dev in (0, 1):  # device 0 first, then device 1 with device 0's caches warm
                _check(dev, two_devices[dev], tier, shape, tol, seed=100 * rep + 10 * i + dev)


def test_allocation_free_entry_point_per_device(two_devices):
    M, N, K = 512, 384, 256
    for dev in (1, 0, 1):
        p = W.sgemm_problem(M, N, K, seed=7 + dev, alpha=1.0, beta=0.0)
        A, B, C = (t.to(f"cuda:{dev}") for t in (p.A, p.B, p.C))
        with torch.cuda.device(dev):
            H.hpvm_sgemm_bf16x3_noalloc(M, N, K, p.alpha, A.data_ptr(), p.lda, B.data_ptr(), p.ldb, p.beta,
                                        C.data_ptr(), p.ldc, p.transA, p.transB, None,
                                        torch.cuda.current_stream(dev).cuda_stream)
            torch.cuda.synchronize(dev)
        got = W.col_major(C.cpu(), M, N, p.ldc).double().numpy()
        assert O.normwise_rel_err(got, O.sgemm_f64(p)) <= 5e-6
