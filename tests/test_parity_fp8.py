"""Parity of the tensor-core operand preparation and of the block-scaled FP8
leaf with the oracle (GPU).

* The BF16 split and the FP8 quantiser are integer-valued decisions taken in
  FP32 on both sides: their outputs must equal the oracle's bit for bit.
* The FP8 leaf's definition is the product of the dequantised operands
  (oracle/fp8.py): the GPU result must match it to FP32-accumulation accuracy
  (normwise 1e-5), and the unquantised FP64 product within the FP8 tier's
  bound (normwise 6e-2) on the FP8 workload.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import fp8 as F
from oracle import quant as Q
from oracle import sgemm as O
from paper_1611_00860_gb300 import _lib as H
from paper_1611_00860_gb300.sgemm import SgemmDFG

pytestmark = pytest.mark.gpu

TIGHT = 1e-5
FP8_TOL = 6e-2


@pytest.fixture(scope="module")
def dfg(cuda_device):
    d = SgemmDFG(0)
    yield d
    d.close()


def _operand(rows, K, kcontig, seed, lognormal=False):
    g = torch.Generator().manual_seed(seed)
    Y = torch.randn(rows, K, generator=g)
    if lognormal:
        Y = Y * torch.exp(2 * torch.randn(rows, 1, generator=g))
    # column-major buffer holding Y (kcontig == 0) or Y^T (kcontig == 1)
    X = Y.t().contiguous().view(-1) if not kcontig else Y.contiguous().view(-1)
    ld = rows if not kcontig else K
    return Y.numpy(), X, ld


@pytest.mark.parametrize("kcontig", [False, True])
@pytest.mark.parametrize("rows,K", [(300, 500), (64, 8), (129, 257)])
def test_split_bf16_bit_exact(kcontig, rows, K):
    Y, X, ld = _operand(rows, K, kcontig, seed=rows + K)
    Kp = (K + 7) // 8 * 8
    hi = torch.zeros(rows * Kp, dtype=torch.bfloat16, device="cuda")
    lo = torch.zeros_like(hi)
    Xd = X.cuda()
    H.hpvm_split_bf16(Xd.data_ptr(), ld, kcontig, rows, K, hi.data_ptr(), lo.data_ptr(),
                      torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    want_hi, want_lo = Q.split_bf16(Y)
    got_hi = hi.float().cpu().numpy().reshape(rows, Kp)
    got_lo = lo.float().cpu().numpy().reshape(rows, Kp)
    assert np.array_equal(got_hi[:, :K], want_hi) and not got_hi[:, K:].any()
    assert np.array_equal(got_lo[:, :K], want_lo) and not got_lo[:, K:].any()


@pytest.mark.parametrize("kcontig", [False, True])
@pytest.mark.parametrize("rows,K", [(300, 500), (128, 128), (17, 33)])
def test_quant_fp8_bit_exact(kcontig, rows, K):
    Y, X, ld = _operand(rows, K, kcontig, seed=7 * rows + K, lognormal=True)
    Y[:5, :7] = 0.0  # part of a block at zero
    X = torch.from_numpy(np.ascontiguousarray(Y.T if not kcontig else Y)).reshape(-1)
    Kq = (K + 15) // 16 * 16
    nkb, nrb = -(-K // 128), -(-rows // 128)
    q = torch.zeros(rows * Kq, dtype=torch.uint8, device="cuda")
    s = torch.zeros(nrb * nkb, dtype=torch.float32, device="cuda")
    H.hpvm_quant_fp8(X.cuda().data_ptr(), ld, kcontig, rows, K, q.data_ptr(), s.data_ptr(),
                     torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    codes, scales = Q.fp8_block_quant(Y)
    got_codes = q.view(torch.float8_e4m3fn).float().cpu().numpy().reshape(rows, Kq)
    assert np.array_equal(s.cpu().numpy().reshape(nrb, nkb), scales)
    assert np.array_equal(got_codes[:, :K], codes) and not got_codes[:, K:].any()


def _e4m3_midpoints():
    """Every point halfway between two consecutive non-negative E4M3 values
    (where rounding x / s to E4M3 depends on the last bit of the FP32
    quotient), as float64."""
    vals = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).double()
    v = np.unique(vals[torch.isfinite(vals) & (vals >= 0)].numpy())
    return (v[:-1] + v[1:]) / 2


@pytest.mark.parametrize("kcontig", [False, True])
def test_quant_fp8_rounding_midpoints_bit_exact(kcontig):
    # Each 128 x 128 block gets its own scale s (one element 448 t sets
    # amax), and values x = RN(m s) and their FP32 neighbours for every E4M3
    # midpoint m (both signs): x / s lies within an ulp of m, so the E4M3
    # code depends on the quotient being rounded exactly as IEEE division
    # rounds it. Scales span 2^-60 .. 2^60, and two blocks take scales
    # near 2^-100 and 2^90 (outside the quantiser's reciprocal path, where
    # it divides). The codes must equal the oracle's (numpy FP32 division).
    rows, K = 256, 384
    g = np.random.default_rng(11)
    Y = (g.standard_normal((rows, K)) * 0.01).astype(np.float32)
    mids = _e4m3_midpoints()
    mids = mids[mids < 416]
    for bi in range(rows // 128):
        for bj in range(K // 128):
            t = np.float32(2.0 ** g.uniform(-60, 60) * g.uniform(1, 2))
            if (bi, bj) == (0, 0):
                t = np.float32(2.0 ** -100 * 1.37)
            if (bi, bj) == (1, 2):
                t = np.float32(2.0 ** 90 * 1.11)
            amax = np.float32(np.float32(448) * t)
            s = np.float32(amax / np.float32(448))
            x = (mids * np.float64(s)).astype(np.float32)
            xs = np.concatenate([x, np.nextafter(x, np.float32(np.inf)), np.nextafter(x, np.float32(0))])
            xs = np.concatenate([xs, -xs])
            blk = Y[bi * 128:(bi + 1) * 128, bj * 128:(bj + 1) * 128]
            blk *= np.float32(t)  # the random fill scaled with the block (below amax)
            flat = blk.reshape(-1)
            flat[1:1 + xs.size] = xs
            flat[0] = amax
            Y[bi * 128:(bi + 1) * 128, bj * 128:(bj + 1) * 128] = flat.reshape(128, 128)
    X = torch.from_numpy(np.ascontiguousarray(Y.T if not kcontig else Y)).reshape(-1)
    ld = rows if not kcontig else K
    q = torch.zeros(rows * K, dtype=torch.uint8, device="cuda")
    sc = torch.zeros((rows // 128) * (K // 128), dtype=torch.float32, device="cuda")
    H.hpvm_quant_fp8(X.cuda().data_ptr(), ld, kcontig, rows, K, q.data_ptr(), sc.data_ptr(),
                     torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    codes, scales = Q.fp8_block_quant(Y)
    assert np.array_equal(sc.cpu().numpy().reshape(rows // 128, K // 128), scales)
    got = q.view(torch.float8_e4m3fn).float().cpu().numpy().reshape(rows, K)
    assert np.array_equal(got, codes), np.argwhere(got != codes)[:5]


SHAPES = [(128, 256, 128), (300, 200, 260), (129, 257, 33), (1, 1, 1), (500, 130, 1024), (64, 40, 0)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("transA,transB", [(False, True), (True, False), (False, False), (True, True)])
def test_fp8_leaf_matches_dequantised_product(dfg, shape, transA, transB):
    M, N, K = shape
    p = W.sgemm_problem(M, N, K, seed=M + 3 * N + 5 * K, transA=transA, transB=transB,
                        alpha=1.25, beta=-0.5, pad=2)
    A, B, C = (t.cuda() for t in (p.A, p.B, p.C))
    dfg.run_problem(p, H.HPVM_TIER_FP8, (A, B, C))
    torch.cuda.synchronize()
    got = W.col_major(C.cpu(), M, N, p.ldc).double().numpy()
    want = F.fp8_sgemm_block_f64(p, 0, 0, M, N)
    assert np.isfinite(got).all()
    assert O.normwise_rel_err(got, want) <= TIGHT


def test_fp8_integer_case_exact(dfg):
    from tests.test_oracle_fp8 import _int_problem
    M, N, K = 140, 130, 260
    p, opA, opBt, Cm = _int_problem(M, N, K, False, True, seed=3)
    A, B, C = (t.cuda() for t in (p.A, p.B, p.C))
    dfg.run_problem(p, H.HPVM_TIER_FP8, (A, B, C))
    torch.cuda.synchronize()
    got = W.col_major(C.cpu(), M, N, p.ldc).double().numpy()
    exact = 2 * (opA.astype(np.int64) @ opBt.astype(np.int64).T) + 0.5 * Cm.astype(np.float64)
    assert np.array_equal(got, exact)


@pytest.mark.slow
def test_fp8_workload_sampled_blocks(dfg):
    # the FP8 workload: M = N = K = 16384, per-row log-normal(0, 2) magnitudes, beta = 0
    p = W.fp8_problem(16384)
    A, B, C = (t.cuda() for t in (p.A, p.B, p.C))
    info = dfg.run_problem(p, H.HPVM_TIER_FP8, (A, B, C), timeout_ms=120000)
    torch.cuda.synchronize()
    Cv = W.col_major(C, p.M, p.N, p.ldc)
    blocks = W.sample_blocks(p.M, p.N, bs=256, count=16)
    pairs = []
    for (i0, j0) in blocks:
        pairs.append((Cv[i0:i0 + 256, j0:j0 + 256].double().cpu().numpy(),
                      O.sgemm_block_f64(p, i0, j0, 256, 256)))
    err = O.block_errors(pairs)
    print(f"fp8 16384: normwise vs unquantised FP64 {err:.3e} over {len(blocks)} blocks; {info}")
    assert err <= FP8_TOL
    # the tight check on a few blocks (the dequantised reference is slower)
    for (i0, j0), (got, _) in list(zip(blocks, pairs))[:3]:
        want = F.fp8_sgemm_block_f64(p, i0, j0, 256, 256)
        assert O.normwise_rel_err(got, want) <= TIGHT
