"""The tail split of the pair leaves (GPU), through the C-ABI.

A persistent launch whose last round of 256 x 256 pair tiles would leave
more than half of the pairs idle runs each tile of that round as two K
halves on two pairs; the second half to finish adds the other's partial
sums and writes C. The shapes here are picked for the GPU at hand (tile
count modulo the pairs it runs at once: nonzero and at most half of them),
with ragged M, N and K. Checked: C against the FP64 oracle at the tier's
tolerance and, on integer inputs, bit for bit; the same C bit for bit from
launch to launch (the sum of the two halves does not depend on which one
finishes first); the workspace size, which holds the split's partial sums
and counters; and a merged tanh stage equal to the unmerged one bit for bit
(the unmerged leaf splits exactly where the merged leaf does).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import sgemm as O
from paper_1611_00860_gb300 import _lib as H
from paper_1611_00860_gb300.chain import ChainEngine, _rm_product_args
from paper_1611_00860_gb300.sgemm import SgemmDFG

pytestmark = pytest.mark.gpu

TOL = {H.HPVM_TIER_BF16X3: 5e-6, H.HPVM_TIER_BF16: 1e-2}
EPI_WARPS, ACC = 8, 128


def _al(x):
    return (x + 255) // 256 * 256


def _units():
    return torch.cuda.get_device_properties(0).multi_processor_count // 2


def _tail_shape():
    """(tiles_m, tiles_n, split tiles) with 10 row tiles and a split tail."""
    u = _units()
    for tn in range(1, 64):
        T = 10 * tn
        if T >= u and 0 < T % u <= u // 2:
            return 10, tn, T % u
    pytest.skip("no tail-split shape with 10 row tiles on this GPU")


@pytest.fixture(scope="module")
def dfg(cuda_device):
    d = SgemmDFG(0)
    yield d
    d.close()


def _run(dfg, p, tier):
    A, B, C = (t.cuda() for t in (p.A, p.B, p.C))
    dfg.run_problem(p, tier, (A, B, C))
    torch.cuda.synchronize()
    return C.cpu()


@pytest.mark.parametrize("tier", [H.HPVM_TIER_BF16X3, H.HPVM_TIER_BF16])
@pytest.mark.parametrize("transA,transB", [(False, True), (True, False)])
def test_tail_split_matches_oracle_and_repeats(dfg, tier, transA, transB):
    tm, tn, n = _tail_shape()
    M, N, K = 256 * tm - 37, 256 * tn - 5, 520  # ragged tiles, 9 K slabs (halves of 4 and 5)
    p = W.sgemm_problem(M, N, K, seed=tn, transA=transA, transB=transB, alpha=1.25, beta=-0.5, pad=3)
    C1 = _run(dfg, p, tier)
    C2 = _run(dfg, p, tier)
    assert torch.equal(C1.view(N, p.ldc)[:, :M], C2.view(N, p.ldc)[:, :M])  # (the slack is NaN)
    got = W.col_major(C1, M, N, p.ldc).double().numpy()
    assert np.isfinite(got).all()
    assert O.normwise_rel_err(got, O.sgemm_f64(p)) <= TOL[tier]
    # the leading-dimension slack of C is never written
    assert torch.isnan(C1.view(N, p.ldc)[:, M:]).all()
    # the workspace: the planes, then the split's partial sums and counters
    A, B, C = (t.cuda() for t in (p.A, p.B, p.C))
    a = dfg.args_for(M, N, K, A, p.lda, B, p.ldb, C, p.ldc, tier=tier, transA=transA, transB=transB)
    planes = (2 if tier == H.HPVM_TIER_BF16X3 else 1) * (_al(M * 520 * 2) + _al(N * 520 * 2))
    region = _al(n * 2 * 2 * EPI_WARPS * ACC * 32 * 4) + _al(n * 2 * EPI_WARPS * 4)
    if tier == H.HPVM_TIER_BF16X3:  # the in-leaf conversion's flags, counts and counter (last)
        blocks = -(-M // 128) + -(-N // 128)
        region += _al(4 * (blocks * ((-(-K // 64) + 3) // 4 * 4) + blocks + 1))
    assert H.hpvm_workspace_size(dfg.ctx, dfg.nodes["root"], a) == planes + region


@pytest.mark.parametrize("tier", [H.HPVM_TIER_BF16X3, H.HPVM_TIER_BF16])
def test_tail_split_integer_inputs_exact(dfg, tier):
    tm, tn, _ = _tail_shape()
    p = W.sgemm_problem(256 * tm, 256 * tn - 100, 300, seed=2, alpha=2.0, beta=0.5, dist="int8")
    got = W.col_major(_run(dfg, p, tier), p.M, p.N, p.ldc).double().numpy()
    assert np.array_equal(got, O.sgemm_f64(p))


@pytest.mark.parametrize("tier", [H.HPVM_TIER_BF16X3, H.HPVM_TIER_BF16])
@pytest.mark.parametrize("kind", [H.HPVM_NODE_TANH_LEAF, H.HPVM_NODE_TANH_GRAD_LEAF])
def test_merged_equals_unmerged_at_a_split_tail(cuda_device, tier, kind):
    tm, tn, _ = _tail_shape()
    rows, w_out, k = 256 * tn - 9, 256 * tm, 520  # C: w_out x rows (column-major)
    g = torch.Generator().manual_seed(11)
    Hm = torch.randn(rows, k, generator=g).cuda()
    Wt = (torch.randn(k, w_out, generator=g) / 23).cuda()
    Haux = torch.tanh(torch.randn(rows, w_out, generator=g)).cuda()
    outs = []
    for fuse in (True, False):
        eng = ChainEngine(1, tier=tier, fuse=fuse)
        try:
            out = torch.empty(rows, w_out, device="cuda")
            a = _rm_product_args(out, Hm, Wt, tier, eng.flags)
            if kind == H.HPVM_NODE_TANH_GRAD_LEAF:
                a.aux, a.bytesAux, a.ldaux = Haux.data_ptr(), Haux.numel() * 4, w_out
                eng._run(eng.stage_dtanh, a)
            else:
                eng._run(eng.stage_tanh, a)
            eng._drain()
            outs.append(out.cpu())
        finally:
            eng.close()
    assert torch.equal(outs[0], outs[1])
    ref = Hm.double().cpu() @ Wt.double().cpu()
    ref = torch.tanh(ref) if kind == H.HPVM_NODE_TANH_LEAF else ref * (1 - Haux.double().cpu() ** 2)
    assert O.normwise_rel_err(outs[0].double().numpy(), ref.numpy()) <= TOL[tier]
