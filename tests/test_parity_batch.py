"""Batches of independent sgemm DFG instances on the GPU (one batched split
pre-pass launch and one persistent grouped leaf launch), through the C-ABI:
every instance against the FP64 oracle for every policy (four tile-width
rules, on single CTAs with 128-row tiles, on CTA pairs with 256-row tiles,
and on CTA pairs converting the operands inside the leaf), the batch against
one launch per instance (bit for bit, on either tile height and with the
in-leaf conversion), a CUDA-graph replay against a direct run, and the
autotuner."""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import sgemm as O
from paper_1611_00860_gb300 import _lib as H
from paper_1611_00860_gb300.batch import BatchDFG
from paper_1611_00860_gb300.sgemm import SgemmDFG

pytestmark = pytest.mark.gpu

TOL = {H.HPVM_TIER_BF16X3: 5e-6, H.HPVM_TIER_BF16: 1e-2}


def _problems(count, lo, hi, seed, trans=True):
    shapes = W.batched_shapes(count, lo, hi, seed=seed)
    probs = []
    for i, (m, n, k) in enumerate(shapes):
        ta, tb = (False, True) if not trans else [(False, True), (True, False), (False, False), (True, True)][i % 4]
        probs.append(W.sgemm_problem(m, n, k, seed=seed * 1000 + i, transA=ta, transB=tb,
                                     alpha=1.0 + 0.25 * (i % 3), beta=0.5 * (i % 2), pad=i % 3))
    return probs


def _device(probs):
    return [tuple(t.cuda() for t in (p.A, p.B, p.C)) for p in probs]


def _result(p, C):
    return W.col_major(C.cpu(), p.M, p.N, p.ldc).double().numpy()


@pytest.fixture(scope="module")
def small_batch():
    probs = _problems(40, 16, 300, seed=7)
    refs = [O.sgemm_f64(p) for p in probs]
    return probs, refs


@pytest.mark.parametrize("tier", [H.HPVM_TIER_BF16X3, H.HPVM_TIER_BF16])
@pytest.mark.parametrize("policy", range(12))
def test_every_instance_matches_oracle(cuda_device, small_batch, tier, policy):
    if policy >= 8 and tier != H.HPVM_TIER_BF16X3:
        pytest.skip("in-leaf conversion takes the BF16x3 tier")
    probs, refs = small_batch
    dev = _device(probs)
    b = BatchDFG(0)
    try:
        b.prepare(probs, dev, tier=tier, policy=policy)
        info = b.info()
        assert info["count"] == 40 and info["policy"] == policy and info["tiles"] > 0
        assert info["tile_m"] == (256 if policy >= 4 else 128)
        b.run()
        torch.cuda.synchronize()
        for p, (_, _, C), ref in zip(probs, dev, refs):
            got = _result(p, C)
            assert np.isfinite(got).all()
            assert O.normwise_rel_err(got, ref) <= TOL[tier]
    finally:
        b.close()


@pytest.mark.parametrize("policy", [0, 4, 8])
def test_batch_equals_one_launch_per_instance(cuda_device, small_batch, policy):
    probs, _ = small_batch
    dev_b = _device(probs)
    dev_s = _device(probs)
    b = BatchDFG(0)
    s = SgemmDFG(0)
    try:
        # 256-wide tiles as the single leaf's, 128 rows a CTA (0) or 256 a
        # CTA pair (4, as the single leaf; 8 with the planes made in the leaf)
        b.prepare(probs, dev_b, tier=H.HPVM_TIER_BF16X3, policy=policy)
        b.run()
        for p, t in zip(probs, dev_s):
            s.run_problem(p, H.HPVM_TIER_BF16X3, t)
        torch.cuda.synchronize()
        for p, (_, _, Cb), (_, _, Cs) in zip(probs, dev_b, dev_s):
            # bit for bit, NaN slack of the leading dimension included (these
            # single launches have fewer pair tiles than the GPU has pairs, so
            # none splits its last round in K halves, which would round
            # differently from the batch's whole tiles)
            assert torch.equal(Cb.cpu().view(torch.int32), Cs.cpu().view(torch.int32))
    finally:
        b.close()
        s.close()


def test_graph_replay_equals_direct_run(cuda_device, small_batch):
    probs, refs = small_batch
    dev = _device(probs)
    C0 = [t[2].clone() for t in dev]
    b = BatchDFG(0)
    try:
        b.prepare(probs, dev, tier=H.HPVM_TIER_BF16X3, policy=2)
        graph = b.capture()  # one warm-up run happened during capture set-up
        for (_, _, C), c0 in zip(dev, C0):
            C.copy_(c0)
        graph.replay()
        torch.cuda.synchronize()
        replayed = [t[2].cpu().clone() for t in dev]
        for (_, _, C), c0 in zip(dev, C0):
            C.copy_(c0)
        b.run()
        torch.cuda.synchronize()
        for r, (_, _, C), p, ref in zip(replayed, dev, probs, refs):
            assert torch.equal(r.view(torch.int32), C.cpu().view(torch.int32))
            assert O.normwise_rel_err(_result(p, C), ref) <= 5e-6
    finally:
        b.close()


def test_autotune_picks_a_policy_and_keeps_results_right(cuda_device, small_batch):
    probs, refs = small_batch
    dev = _device(probs)
    C0 = [t[2].clone() for t in dev]
    b = BatchDFG(0)
    try:
        b.prepare(probs, dev, tier=H.HPVM_TIER_BF16X3, policy=0)
        best, ms = b.autotune(reps=2)
        assert best in range(12) and ms > 0
        assert b.info()["policy"] == best
        # a new batch of the same shapes starts from the tuned policy
        b.prepare(probs, dev, tier=H.HPVM_TIER_BF16X3, policy=-1)
        assert b.info()["policy"] == best
        for (_, _, C), c0 in zip(dev, C0):
            C.copy_(c0)
        b.run()
        torch.cuda.synchronize()
        for p, (_, _, C), ref in zip(probs, dev, refs):
            assert O.normwise_rel_err(_result(p, C), ref) <= 5e-6
    finally:
        b.close()


@pytest.mark.slow
@pytest.mark.parametrize("policy", [2, 6, 10])
def test_batched_workload_512_instances(cuda_device, policy):
    # the batched workload: 512 instances, M, N, K log-uniform in [32, 2048]
    shapes = W.batched_shapes()
    probs = [W.sgemm_problem(m, n, k, seed=20000 + i, alpha=1.0, beta=0.0) for i, (m, n, k) in enumerate(shapes)]
    dev = _device(probs)
    b = BatchDFG(0)
    try:
        b.prepare(probs, dev, tier=H.HPVM_TIER_BF16X3, policy=policy)
        b.run()
        torch.cuda.synchronize()
        worst = 0.0
        for p, (_, _, C) in zip(probs, dev):
            # the largest instances on sampled blocks, the rest whole
            if p.M * p.N * p.K > 2 ** 30:
                pairs = [(_result(p, C)[i0:i0 + 256, j0:j0 + 256], O.sgemm_block_f64(p, i0, j0, 256, 256))
                         for (i0, j0) in W.sample_blocks(p.M, p.N, bs=256, count=2)]
                err = O.block_errors(pairs)
            else:
                err = O.normwise_rel_err(_result(p, C), O.sgemm_f64(p))
            worst = max(worst, err)
        print(f"512-instance batch: worst normwise error {worst:.3e}; {b.info()}")
        assert worst <= 5e-6 and math.isfinite(worst)
    finally:
        b.close()


def test_in_leaf_conversion_needs_bf16x3(cuda_device, small_batch):
    probs, _ = small_batch
    dev = _device(probs)
    b = BatchDFG(0)
    try:
        with pytest.raises(H.HpvmError) as e:
            b.prepare(probs, dev, tier=H.HPVM_TIER_BF16, policy=8)
        assert e.value.code == H.HPVM_ERR_INVALID_ARG
    finally:
        b.close()


def test_in_leaf_conversion_repeats_bit_for_bit(cuda_device, small_batch):
    # the converters claim chunks in whatever order the CTAs reach them; the
    # planes, and so C, must not depend on it
    probs, _ = small_batch
    dev = _device(probs)
    C0 = [t[2].clone() for t in dev]
    b = BatchDFG(0)
    try:
        b.prepare(probs, dev, tier=H.HPVM_TIER_BF16X3, policy=10)
        outs = []
        for _ in range(3):
            for (_, _, C), c0 in zip(dev, C0):
                C.copy_(c0)
            b.run()
            torch.cuda.synchronize()
            outs.append([t[2].cpu().view(torch.int32).clone() for t in dev])
        for later in outs[1:]:
            assert all(torch.equal(x, y) for x, y in zip(outs[0], later))
    finally:
        b.close()
