"""Leaves whose bounded waits run out in the middle of a tile (GPU).

hpvm_set_wait_limit makes every wait of the producer, MMA and converter
roles give up after a few microseconds, so the real waits of a normal launch
run out while copies and MMAs are in flight: nothing is broken and nothing
faults, the waits just end early. The leaf must then stop every role, drain
what it started (the TMA loads of both CTAs of a pair, the MMAs, the
converters' loads), free its tensor memory and return; hpvm_wait reports
HPVM_ERR_DEVICE_FAULT with the status bits of the waits that gave up and
without ST_DRAIN (every drain wait completed). The context must stay usable:
with the default limit restored, the same launch gives the oracle's result.

Cases: the BF16x3 leaf on CTA pairs (separate split: the epilogue's first
wait spans a tile's whole main loop), the FP8 leaf on single CTAs (K = 256:
each tile's MMAs take well under a microsecond and its C traffic several, so
the MMA and producer roles wait on the epilogue with loads in flight), the
BF16x3 leaf converting its own operands (8192 x 4096: flag waits and
converter warps) and the BF16 leaf on CTA pairs.
"""
import re
import time

import pytest
import torch

import workloads as W
from oracle import sgemm as O
from paper_1611_00860_gb300 import _lib as H
from paper_1611_00860_gb300.sgemm import SgemmDFG

pytestmark = pytest.mark.gpu

ST_DRAIN = 8
CASES = [
    ("bf16x3_pairs", H.HPVM_TIER_BF16X3, (2048, 2048, 2048), H.HPVM_LAUNCH_SEPARATE_SPLIT),
    ("fp8_single", H.HPVM_TIER_FP8, (8192, 8192, 256), 0),
    ("bf16x3_inleaf", H.HPVM_TIER_BF16X3, (8192, 4096, 512), 0),
    ("bf16_pairs", H.HPVM_TIER_BF16, (4096, 2048, 1024), 0),
]
TOL = {H.HPVM_TIER_BF16X3: 5e-6, H.HPVM_TIER_BF16: 1e-2}


@pytest.fixture(scope="module")
def dfg(cuda_device):
    d = SgemmDFG(0)
    yield d
    d.close()


def _status_bits(err: H.HpvmError) -> int:
    m = re.search(r"status bits 0x([0-9a-f]+)", str(err))
    assert m, str(err)
    return int(m.group(1), 16)


@pytest.mark.parametrize("name,tier,shape,flags", CASES, ids=[c[0] for c in CASES])
def test_waits_that_run_out_mid_tile_drain_and_return(dfg, name, tier, shape, flags):
    M, N, K = shape
    p = W.sgemm_problem(M, N, K, seed=M + K, alpha=1.0, beta=0.5)
    A, B, C0 = (t.cuda() for t in (p.A, p.B, p.C))
    try:
        for _ in range(2):  # twice in a row: the context stays usable between
            H.hpvm_set_wait_limit(dfg.ctx, 1)
            C = C0.clone()
            t0 = time.perf_counter()
            with pytest.raises(H.HpvmError) as e:
                dfg(M, N, K, A, p.lda, B, p.ldb, C, p.ldc, p.alpha, p.beta, p.transA, p.transB,
                    tier=tier, flags=flags, timeout_ms=60000)
            dt = time.perf_counter() - t0
            assert e.value.code == H.HPVM_ERR_DEVICE_FAULT, str(e.value)
            bits = _status_bits(e.value)
            assert bits != 0 and not (bits & ST_DRAIN), hex(bits)
            assert dt < 1.5, dt  # gave up early; no drain wait ran to its 2 s bound
        torch.cuda.synchronize()
    finally:
        H.hpvm_set_wait_limit(dfg.ctx, 0)
    # the default limit again: the same launch computes the product
    C = C0.clone()
    dfg(M, N, K, A, p.lda, B, p.ldb, C, p.ldc, p.alpha, p.beta, p.transA, p.transB, tier=tier, flags=flags,
        timeout_ms=60000)
    torch.cuda.synchronize()
    Cv = W.col_major(C, M, N, p.ldc)
    blocks = W.sample_blocks(M, N, bs=256, count=3)
    if tier == H.HPVM_TIER_FP8:
        from oracle import fp8 as F
        pairs = [(Cv[i0:i0 + 256, j0:j0 + 256].double().cpu().numpy(), F.fp8_sgemm_block_f64(p, i0, j0, 256, 256))
                 for (i0, j0) in blocks]
        assert O.block_errors(pairs) <= 1e-5
    else:
        pairs = [(Cv[i0:i0 + 256, j0:j0 + 256].double().cpu().numpy(), O.sgemm_block_f64(p, i0, j0, 256, 256))
                 for (i0, j0) in blocks]
        assert O.block_errors(pairs) <= TOL[tier]



def test_batch_waits_that_run_out_drain_and_return(cuda_device):
    # The grouped leaves drain too: single CTAs, CTA pairs (whose stages carry
    # bytes that differ from tile to tile) and pairs converting their own
    # operands. The autotuner runs every policy with a 1 us limit and reports
    # the context's status at its end; then, with the default limit, each
    # kind of leaf computes the oracle's product.
    from paper_1611_00860_gb300.batch import BatchDFG
    shapes = W.batched_shapes(48, 64, 512, seed=9)
    probs = [W.sgemm_problem(m, n, k, seed=900 + i, alpha=1.0, beta=0.0) for i, (m, n, k) in enumerate(shapes)]
    dev = [tuple(t.cuda() for t in (p.A, p.B, p.C)) for p in probs]
    refs = [O.sgemm_f64(p) for p in probs]
    b = BatchDFG(0)
    try:
        b.prepare(probs, dev, tier=H.HPVM_TIER_BF16X3, policy=4)
        H.hpvm_set_wait_limit(b.ctx, 1)
        t0 = time.perf_counter()
        with pytest.raises(H.HpvmError) as e:
            b.autotune(reps=1)
        dt = time.perf_counter() - t0
        assert e.value.code == H.HPVM_ERR_DEVICE_FAULT, str(e.value)
        bits = _status_bits(e.value)
        assert bits != 0 and not (bits & ST_DRAIN), hex(bits)
        assert dt < 5.0, dt
        torch.cuda.synchronize()
        H.hpvm_set_wait_limit(b.ctx, 0)
        for policy in (1, 4, 8):
            b.prepare(probs, dev, tier=H.HPVM_TIER_BF16X3, policy=policy)
            b.run()
            torch.cuda.synchronize()
            for p, (_, _, C), ref in zip(probs, dev, refs):
                got = W.col_major(C.cpu(), p.M, p.N, p.ldc).double().numpy()
                assert O.normwise_rel_err(got, ref) <= 5e-6, (policy, p.M, p.N, p.K)
    finally:
        H.hpvm_set_wait_limit(b.ctx, 0)
        b.close()
