"""Parity of the CUDA leaves with the FP64 oracle, through the C-ABI (GPU).

Tolerances are the normwise relative errors ||C_gpu - C_ref||_F / ||C_ref||_F
fixed for each tier: 5e-6 for FP32 and the split BF16x3 and BF16x6 tiers,
1e-2 for plain BF16.
Integer-valued inputs, where every tier is exact, must match bit for bit.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from oracle import sgemm as O
from paper_1611_00860_gb300 import _lib as H
from paper_1611_00860_gb300.sgemm import SgemmDFG, build_sgemm_graph, make_args

pytestmark = pytest.mark.gpu

TOL = {H.HPVM_TIER_FP32_DFG: 5e-6, H.HPVM_TIER_FP32: 5e-6,
       H.HPVM_TIER_BF16X3: 5e-6, H.HPVM_TIER_BF16: 1e-2, H.HPVM_TIER_BF16X6: 5e-6}
TIERS = list(TOL)
TRANS = [(False, True), (False, False), (True, False), (True, True)]


@pytest.fixture(scope="module")
def dfg(cuda_device):
    d = SgemmDFG(0)
    yield d
    d.close()


def run(dfg, p, tier):
    A, B, C = (t.cuda() for t in (p.A, p.B, p.C))
    block = grid = None
    if tier == H.HPVM_TIER_FP32_DFG:
        block = (16, 16)
        grid = (max(1, -(-p.M // 16)), max(1, -(-p.N // 16)))
    info = dfg.run_problem(p, tier, (A, B, C), block=block, grid=grid)
    torch.cuda.synchronize()
    Cf = C.cpu()
    return W.col_major(Cf, p.M, p.N, p.ldc).double().numpy(), info, Cf


@pytest.mark.parametrize("tier", TIERS)
def test_small_workload(dfg, tier):
    p = W.small_dfg_problem()
    got, info, _ = run(dfg, p, tier)
    err = O.normwise_rel_err(got, O.sgemm_f64(p))
    assert err <= TOL[tier], err
    if tier == H.HPVM_TIER_FP32_DFG:
        # Section 3.4 mapping: internal grid 8 x 6 = CTAs, 16 x 16 leaf = threads,
        # the Allocation's two 16 x 16 FP32 tiles = 2 KB of shared memory
        assert (info["grid_x"], info["grid_y"], info["block_threads"]) == (8, 6, 256)
        assert info["smem_bytes"] == 2 * 16 * 16 * 4 and info["literal"] == 1


@pytest.mark.parametrize("tier", TIERS)
@pytest.mark.parametrize("transA,transB", TRANS)
def test_integer_inputs_exact(dfg, tier, transA, transB):
    p = W.sgemm_problem(150, 270, 70, seed=21, transA=transA, transB=transB,
                        alpha=2.0, beta=0.5, dist="int8", pad=2)
    got, _, _ = run(dfg, p, tier)
    ref = O.sgemm_f64(p)
    assert np.array_equal(got, ref)


SHAPES = [(1, 1, 1), (129, 257, 33), (300, 200, 100), (255, 513, 17), (64, 40, 0),
          (17, 300, 520), (384, 256, 64)]


@pytest.mark.parametrize("tier", TIERS)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("transA,transB", TRANS[:2] + TRANS[3:])
def test_ragged_shapes(dfg, tier, shape, transA, transB):
    M, N, K = shape
    p = W.sgemm_problem(M, N, K, seed=M + 7 * N + 13 * K, transA=transA,
                        transB=transB, alpha=1.25, beta=-0.75, dist="normal", pad=3)
    got, _, Cf = run(dfg, p, tier)
    ref = O.sgemm_f64(p)
    assert np.isfinite(got).all()
    assert O.normwise_rel_err(got, ref) <= TOL[tier]
    # the leading-dimension slack of C (NaN) is never written
    slack = Cf.view(N, p.ldc)[:, M:] if N else Cf[:0]
    assert torch.isnan(slack).all()


@pytest.mark.parametrize("tier", TIERS)
def test_beta_zero_does_not_read_c(dfg, tier):
    p = W.sgemm_problem(200, 300, 50, seed=5, beta=0.0, alpha=3.0)
    p.C.fill_(float("nan"))
    got, _, _ = run(dfg, p, tier)
    assert np.isfinite(got).all()
    assert O.normwise_rel_err(got, O.sgemm_f64(p)) <= TOL[tier]


@pytest.mark.parametrize("tier", TIERS)
def test_empty_result_is_a_no_op(dfg, tier):
    for M, N in [(0, 5), (5, 0)]:
        p = W.sgemm_problem(M, N, 8, seed=1)
        run(dfg, p, tier)


def test_literal_mapping_other_leaf_sizes(dfg):
    for bs in (4, 8, 32):
        p = W.sgemm_problem(70, 45, 37, seed=bs, alpha=0.5, beta=2.0)
        A, B, C = (t.cuda() for t in (p.A, p.B, p.C))
        info = dfg.run_problem(p, H.HPVM_TIER_FP32_DFG, (A, B, C), block=(bs, bs),
                               grid=(-(-70 // bs), -(-45 // bs)))
        got = W.col_major(C.cpu(), p.M, p.N, p.ldc).double().numpy()
        assert info["block_threads"] == bs * bs
        assert O.normwise_rel_err(got, O.sgemm_f64(p)) <= 5e-6


@pytest.mark.parametrize("tier", [H.HPVM_TIER_FP32, H.HPVM_TIER_BF16X3])
def test_memory_tracker_host_buffers(cuda_device, tier):
    # host arrays registered with track_mem; the launch copies them in, and
    # request_mem brings C back (Section 2.3)
    p = W.sgemm_problem(260, 190, 75, seed=9, alpha=1.5, beta=0.5)
    ref = O.sgemm_f64(p)
    A, B, C = (t.clone().pin_memory() for t in (p.A, p.B, p.C))
    ctx = H.hpvm_init(0)
    try:
        nodes = build_sgemm_graph(ctx)
        for t in (A, B, C):
            H.hpvm_track_mem(ctx, t.data_ptr(), t.numel() * 4)
        a = make_args(p.M, p.N, p.K, A.data_ptr(), A.numel() * 4, p.lda, B.data_ptr(),
                      B.numel() * 4, p.ldb, C.data_ptr(), C.numel() * 4, p.ldc,
                      p.alpha, p.beta, p.transA, p.transB, tier)
        g = H.hpvm_launch(ctx, nodes["root"], a)
        info = H.hpvm_graph_info(g).as_dict()
        H.hpvm_wait(g, 60000)
        assert info["h2d_bytes"] == (A.numel() + B.numel() + C.numel()) * 4
        H.hpvm_request_mem(ctx, C.data_ptr(), C.numel() * 4)
        got = W.col_major(C, p.M, p.N, p.ldc).double().numpy()
        assert O.normwise_rel_err(got, ref) <= TOL[tier]
        # a second launch without re-tracking reuses the device copies of A, B
        # and C (C's latest copy is on the device)
        g = H.hpvm_launch(ctx, nodes["root"], a)
        assert H.hpvm_graph_info(g).h2d_bytes == 0
        H.hpvm_wait(g, 60000)
        for t in (A, B, C):
            H.hpvm_untrack_mem(ctx, t.data_ptr())
    finally:
        H.hpvm_cleanup(ctx)


def test_memory_tracker_two_contexts_alternating(cuda_device):
    # the double-buffered loop of the end-to-end benchmark: two contexts,
    # each with its own pinned A, B, C and stream; step i+1 is launched
    # before step i's C is read back (hpvm_request_mem waits for the launch
    # that wrote C, not for the device). Every step's C against the oracle.
    ctxs, sets = [], []
    try:
        for j in range(2):
            ctx = H.hpvm_init(0)
            ctxs.append(ctx)
            nodes = build_sgemm_graph(ctx)
            st = torch.cuda.Stream()
            probs = [W.sgemm_problem(300, 260, 140, seed=40 + 2 * i + j, alpha=1.5, beta=0.5) for i in range(2)]
            sets.append((ctx, nodes, st, probs))
        pending = []
        for i in range(2):
            for j, (ctx, nodes, st, probs) in enumerate(sets):
                p = probs[i]
                A, B, C = (t.clone().pin_memory() for t in (p.A, p.B, p.C))
                for t in (A, B, C):
                    H.hpvm_track_mem(ctx, t.data_ptr(), t.numel() * 4)
                a = make_args(p.M, p.N, p.K, A.data_ptr(), A.numel() * 4, p.lda, B.data_ptr(), B.numel() * 4,
                              p.ldb, C.data_ptr(), C.numel() * 4, p.ldc, p.alpha, p.beta, p.transA, p.transB,
                              H.HPVM_TIER_BF16X3)
                g = H.hpvm_launch(ctx, nodes["root"], a, False, st.cuda_stream)
                pending.append((ctx, g, p, (A, B, C)))
                if len(pending) == 2:  # read back the previous step while this one runs
                    pctx, pg, pp, (pA, pB, pC) = pending.pop(0)
                    H.hpvm_wait(pg, 60000)
                    H.hpvm_request_mem(pctx, pC.data_ptr(), pC.numel() * 4)
                    got = W.col_major(pC, pp.M, pp.N, pp.ldc).double().numpy()
                    assert O.normwise_rel_err(got, O.sgemm_f64(pp)) <= TOL[H.HPVM_TIER_BF16X3]
                    for t in (pA, pB, pC):
                        H.hpvm_untrack_mem(pctx, t.data_ptr())
        for pctx, pg, pp, (pA, pB, pC) in pending:
            H.hpvm_wait(pg, 60000)
            H.hpvm_request_mem(pctx, pC.data_ptr(), pC.numel() * 4)
            got = W.col_major(pC, pp.M, pp.N, pp.ldc).double().numpy()
            assert O.normwise_rel_err(got, O.sgemm_f64(pp)) <= TOL[H.HPVM_TIER_BF16X3]
    finally:
        for ctx in ctxs:
            H.hpvm_cleanup(ctx)


def test_untracked_host_pointer_rejected(cuda_device):
    p = W.sgemm_problem(16, 16, 16, seed=1)
    ctx = H.hpvm_init(0)
    try:
        nodes = build_sgemm_graph(ctx)
        buf = (ctypes.c_float * 256)()
        dev = torch.zeros(256, device="cuda")
        a = make_args(16, 16, 16, ctypes.addressof(buf), 1024, 16, dev.data_ptr(), 1024, 16,
                      dev.data_ptr(), 1024, 16, 1.0, 0.0, False, True, H.HPVM_TIER_FP32)
        with pytest.raises(H.HpvmError) as e:
            H.hpvm_launch(ctx, nodes["root"], a)
        assert e.value.code == H.HPVM_ERR_INVALID_ARG
        del p
    finally:
        H.hpvm_cleanup(ctx)


def test_wait_timeout_leaves_handle_valid(dfg):
    n = 4096
    A = torch.randn(n * n, device="cuda")
    B = torch.randn(n * n, device="cuda")
    C = torch.zeros(n * n, device="cuda")
    args = dfg.args_for(n, n, n, A, n, B, n, C, n, tier=H.HPVM_TIER_FP32_DFG,
                        block=(16, 16), grid=(n // 16, n // 16))
    g = dfg.launch(args)
    try:
        H.hpvm_wait(g, 0)
        finished_early = True
    except H.HpvmError as e:
        assert e.code == H.HPVM_ERR_TIMEOUT
        finished_early = False
    if not finished_early:
        H.hpvm_wait(g, 120000)
    torch.cuda.synchronize()


def test_bounded_wait_gives_up_and_context_survives(cuda_device):
    # a wait nothing satisfies: the bounded wait must expire after ~200 ms,
    # be reported as a device fault, and leave the context usable
    import time
    ctx = H.hpvm_init(0)
    try:
        t0 = time.perf_counter()
        with pytest.raises(H.HpvmError) as e:
            H.hpvm_selftest_wait_timeout(ctx, 200)
        dt = time.perf_counter() - t0
        assert e.value.code == H.HPVM_ERR_DEVICE_FAULT
        assert 0.19 <= dt < 10.0
        # the status word was cleared by the report: a real launch now succeeds
        nodes = build_sgemm_graph(ctx)
        p = W.sgemm_problem(64, 48, 32, seed=3)
        A, B, C = (t.cuda() for t in (p.A, p.B, p.C))
        a = make_args(p.M, p.N, p.K, A.data_ptr(), A.numel() * 4, p.lda, B.data_ptr(), B.numel() * 4, p.ldb,
                      C.data_ptr(), C.numel() * 4, p.ldc, p.alpha, p.beta, p.transA, p.transB,
                      H.HPVM_TIER_BF16X3)
        ws = torch.empty(H.hpvm_workspace_size(ctx, nodes["root"], a), dtype=torch.uint8, device="cuda")
        H.hpvm_set_workspace(ctx, ws.data_ptr(), ws.numel())
        H.hpvm_wait(H.hpvm_launch(ctx, nodes["root"], a), 60000)
        got = W.col_major(C.cpu(), p.M, p.N, p.ldc).double().numpy()
        assert O.normwise_rel_err(got, O.sgemm_f64(p)) <= 5e-6
    finally:
        H.hpvm_cleanup(ctx)


@pytest.mark.parametrize("tier,tile_m,tile_n", [(H.HPVM_TIER_BF16, 256, 256), (H.HPVM_TIER_BF16X3, 256, 256),
                                                (H.HPVM_TIER_FP8, 128, 256)])
def test_tile_mapping_per_tier(dfg, tier, tile_m, tile_n):
    # plain BF16 and BF16x3 run on clusters of two CTAs (a 256 x 256 tile
    # per pair), FP8 on single CTAs (128 x 256); the grid never exceeds the
    # tiles (or their CTAs) and pairs launch an even grid
    M, N, K = 700, 600, 96
    p = W.sgemm_problem(M, N, K, seed=4, alpha=1.0, beta=0.5)
    got, info, _ = run(dfg, p, tier)
    assert info["tile_m"] == tile_m and info["tile_n"] == tile_n
    tiles = -(-M // tile_m) * -(-N // tile_n)
    per_tile = tile_m // 128
    assert info["grid_x"] == min(tiles * per_tile, info["grid_x"]) and info["grid_x"] % per_tile == 0
    assert info["grid_x"] <= tiles * per_tile
    tol = 6e-2 if tier == H.HPVM_TIER_FP8 else TOL[tier]
    assert O.normwise_rel_err(got, O.sgemm_f64(p)) <= tol
