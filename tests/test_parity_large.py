"""Parity at the large workload (M = N = K = 8192, the launch configuration
the benchmark times), on sampled 256 x 256 output blocks that the FP64 oracle
computes one by one: 16 seeded block positions plus the first and the last,
and two more inside the last round of pair tiles (row tiles 27-31 of column
tiles 24-31 in the grouped tile order), which the leaf runs in K halves on a
152-SM GB300 (tail split). Also the column-scaled variant (column p of
op(A) scaled by 2^u, u ~ U[-20,20]).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import sgemm as O
from paper_1611_00860_gb300 import _lib as H
from paper_1611_00860_gb300.sgemm import SgemmDFG

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 8192
TOL = {H.HPVM_TIER_FP32: 5e-6, H.HPVM_TIER_BF16X3: 5e-6, H.HPVM_TIER_BF16: 1e-2,
       H.HPVM_TIER_BF16X6: 5e-6}


@pytest.fixture(scope="module")
def dfg(cuda_device):
    d = SgemmDFG(0)
    yield d
    d.close()


@pytest.fixture(scope="module", params=[False, True], ids=["normal", "colscale"])
def problem(request, cuda_device):
    p = W.large_dfg_problem(N, colscale=request.param)
    blocks = W.sample_blocks(p.M, p.N, bs=256, count=16) + [(7424, 6400), (7168, 7936)]
    refs = [O.sgemm_block_f64(p, i0, j0, 256, 256) for (i0, j0) in blocks]
    dev = tuple(t.cuda() for t in (p.A, p.B, p.C))
    yield p, blocks, refs, dev
    del dev
    torch.cuda.empty_cache()


@pytest.mark.parametrize("tier", list(TOL))
def test_large_sampled_blocks(dfg, problem, tier):
    p, blocks, refs, (A, B, C0) = problem
    C = C0.clone()
    info = dfg.run_problem(p, tier, (A, B, C))
    torch.cuda.synchronize()
    Cv = W.col_major(C, p.M, p.N, p.ldc)
    pairs = [(Cv[i0:i0 + 256, j0:j0 + 256].double().cpu().numpy(), r)
             for (i0, j0), r in zip(blocks, refs)]
    err = O.block_errors(pairs)
    print(f"tier {tier} blocks={len(blocks)} err={err:.3e} info={info}")
    assert np.isfinite(err)
    assert err <= TOL[tier], err
    # every block on its own stays within the bound too
    for got, ref in pairs:
        assert O.normwise_rel_err(got, ref) <= TOL[tier]
