"""The streamed differentiable chain on the GPU, through the C-ABI.

* MergeDependentNodes: a stage whose tanh leaf is merged into the sgemm
  epilogue equals the same stage with the tanh leaf run as its own kernel,
  bit for bit (both evaluate tanhf on the same FP32 value).
* Forward (one launch of the chain graph, and items pushed through it as a
  streaming graph) against the FP64 chain definition of the oracle.
* Every product of a training step (forward, recomputed forward, input and
  weight adjoints) against the oracle's product of exactly the FP32 inputs
  the GPU consumed, at the tier's bound; each stage's output equals its
  product followed by its elementwise leaf (the unmerged stage, bit for
  bit), and the elementwise kernel matches the FP64 function of the GPU's
  own product.
* Gradients of sum(Y * G) from torch.autograd through ChainFunction (the
  adjoint sgemm and tanh leaves, activations recomputed) against the
  oracle's FP64 gradients, which finite differences pin.

Tolerances (normwise relative): each product within its tier's bound, 1e-2
for BF16 operands and 5e-6 for BF16x3. The chain's outputs compose several
products through tanh leaves: for BF16x3 their bound is the first-order
bound the oracle derives from the chain's Jacobians (``oracle.adjoint.
chain_grad_error_bound`` / ``chain_forward_error_bound``) with every product
and elementwise leaf within 6e-6 (the product's 5e-6 plus 1e-6 for the FP32
tanh and tanh-adjoint evaluations); for BF16 the tier's 1e-2.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as J
from oracle import sgemm as O
from paper_1611_00860_gb300 import _lib as H
from paper_1611_00860_gb300.chain import ChainEngine, chain_apply, _rm_product_args
from paper_1611_00860_gb300.sgemm import make_args

pytestmark = pytest.mark.gpu

TOL = {H.HPVM_TIER_BF16: 1e-2, H.HPVM_TIER_BF16X3: 5e-6}  # per product
STAGE_EPS = {H.HPVM_TIER_BF16: 1e-2, H.HPVM_TIER_BF16X3: 6e-6}  # product + elementwise leaf
ELEMENTWISE_TOL = 1e-6  # FP32 tanh / (1 - h^2) against FP64 on the same product


def _oracle_rm(Am, Bm):
    """Row-major FP32 Am (m x k) times Bm (k x n) in FP64 through the oracle's
    sgemm definition, as the column-major product C^T = Bm^T Am^T."""
    from types import SimpleNamespace
    Am = torch.as_tensor(Am, dtype=torch.float32).contiguous()
    Bm = torch.as_tensor(Bm, dtype=torch.float32).contiguous()
    m, k = Am.shape
    n = Bm.shape[1]
    prob = SimpleNamespace(M=n, N=m, K=k, transA=False, transB=False, alpha=1.0, beta=0.0,
                           A=Bm.reshape(-1), lda=n, B=Am.reshape(-1), ldb=k,
                           C=torch.zeros(1), ldc=n)
    return O.sgemm_f64(prob).T


def _split_rm(Am, Bm):
    """The same product as _oracle_rm, as BF16x3's three split products in
    exact arithmetic (oracle.split): what the tier computes without its
    FP32 accumulation error."""
    from types import SimpleNamespace
    from oracle import split as S
    Am = torch.as_tensor(Am, dtype=torch.float32).contiguous()
    Bm = torch.as_tensor(Bm, dtype=torch.float32).contiguous()
    m, k = Am.shape
    n = Bm.shape[1]
    prob = SimpleNamespace(M=n, N=m, K=k, transA=False, transB=False, alpha=1.0, beta=0.0,
                           A=Bm.reshape(-1), lda=n, B=Am.reshape(-1), ldb=k,
                           C=torch.zeros(1), ldc=n)
    return S.split_block_f64(prob, 0, 0, n, m, "bf16x3").T


# A product with at least this many outputs is held to the BF16x3 bound
# against FP64 directly; below it the normwise error of the method itself
# (its three products in exact arithmetic) spreads past 5e-6 for some
# inputs (a 24 x 16 product with K = 16 does so for about 6% of N(0,1)
# draws; tests/test_oracle_split.py pins one), and such a product is held
# to the method's exact value instead (ACC_TOL, the accumulation error).
MIN_OUTPUTS_FOR_FP64_BOUND = 16384
ACC_TOL = 1e-6


def _plain(eng, a):
    """Run one record through the plain sgemm stage and wait."""
    eng._run(eng.stage_plain, a)
    eng._drain()


def _inputs(items, rows, w, layers, seed):
    g = torch.Generator().manual_seed(seed)
    X = torch.randn(items, rows, w, generator=g)
    Ws = [torch.randn(w, w, generator=g) / w ** 0.5 for _ in range(layers)]
    G = torch.randn(items, rows, w, generator=g)
    return X, Ws, G


@pytest.mark.parametrize("tier", [H.HPVM_TIER_BF16, H.HPVM_TIER_BF16X3])
@pytest.mark.parametrize("kind", [H.HPVM_NODE_TANH_LEAF, H.HPVM_NODE_TANH_GRAD_LEAF])
def test_merged_equals_unmerged(cuda_device, tier, kind):
    fused = ChainEngine(1, tier=tier, fuse=True)
    plain = ChainEngine(1, tier=tier, fuse=False)
    try:
        g = torch.Generator().manual_seed(1)
        Hm = torch.randn(300, 160, generator=g).cuda()
        W = (torch.randn(160, 200, generator=g) / 12).cuda()
        Haux = torch.tanh(torch.randn(300, 200, generator=g)).cuda()
        outs = []
        for eng in (fused, plain):
            out = torch.empty(300, 200, device="cuda")
            a = _rm_product_args(out, Hm, W, tier, eng.flags)
            if kind == H.HPVM_NODE_TANH_GRAD_LEAF:
                a.aux, a.bytesAux, a.ldaux = Haux.data_ptr(), Haux.numel() * 4, 200
                eng._run(eng.stage_dtanh, a)
            else:
                eng._run(eng.stage_tanh, a)
            eng._drain()
            outs.append(out.cpu())
        assert torch.equal(outs[0], outs[1])
        # the product within the tier's bound (a plain leaf on the same
        # inputs: the same kernel up to the epilogue), and the elementwise
        # leaf applied to that product
        prod = torch.empty(300, 200, device="cuda")
        _plain(plain, _rm_product_args(prod, Hm, W, tier))
        prod = prod.cpu()
        ref = _oracle_rm(Hm.cpu(), W.cpu())
        assert O.normwise_rel_err(prod.double().numpy(), ref) <= TOL[tier]
        P = prod.double()
        want = torch.tanh(P) if kind == H.HPVM_NODE_TANH_LEAF else P * (1 - Haux.double().cpu() ** 2)
        assert O.normwise_rel_err(outs[0].double().numpy(), want.numpy()) <= ELEMENTWISE_TOL
    finally:
        fused.close()
        plain.close()


@pytest.mark.parametrize("tier", [H.HPVM_TIER_BF16, H.HPVM_TIER_BF16X3])
@pytest.mark.parametrize("rows,w", [(300, 264), (77, 260)])
def test_forwarded_planes_equal_converted(cuda_device, tier, rows, w):
    # One launch of the chain graph: with the stages merged, each stage's
    # epilogue writes the planes of its result that the next stage reads as
    # B (the streaming edge lowered into the producer), so only X's planes
    # and the weights' are converted. The unmerged launch converts every B
    # from the FP32 result. Both round the same FP32 values: every stage's
    # output must match bit for bit (w = 260: plane rows padded to 264).
    layers = 4
    X, Ws, _ = _inputs(1, rows, w, layers, seed=rows)
    Xd = X[0].cuda()
    Wd = [W.cuda() for W in Ws]
    got, kernels = [], []
    for fuse in (True, False):
        eng = ChainEngine(layers, tier=tier, fuse=fuse)
        try:
            Y, Hs = eng.forward(Xd, Wd, keep=True)
            kernels.append(H.hpvm_graph_info(eng._pending[-1]).kernels)
            eng._drain()
            got.append([t.cpu() for t in Hs + [Y]])
        finally:
            eng.close()
    for a, b in zip(*got):
        assert torch.equal(a, b)
    # merged: 4 leaves + 4 weight conversions + X's; unmerged: 4 leaves,
    # 3 tanh kernels, 4 + 4 conversions
    assert kernels == [2 * layers + 1, 2 * layers + (layers - 1) + layers]


@pytest.mark.parametrize("tier", [H.HPVM_TIER_BF16, H.HPVM_TIER_BF16X3])
@pytest.mark.parametrize("rows,w", [(300, 264), (77, 260), (520, 136)])
def test_cached_result_planes_equal_converted(cuda_device, tier, rows, w):
    # HPVM_LAUNCH_CACHE_C: the recomputing stages' and the adjoint stages'
    # epilogues also write the planes of H_l and dZ_l in the layout the
    # weight adjoints read (rows of the result as operand rows, K = rows of
    # the batch: 300, 77 and 520 are ragged against the 64-wide K slabs,
    # w = 260 pads each plane row). The weight adjoints then convert only G
    # and X: 2 (L - 1) conversions fewer, and every gradient bit for bit
    # the same as with each operand converted from its FP32 values.
    layers = 4
    X, Ws, G = _inputs(1, rows, w, layers, seed=rows + 3 * w)
    Xd, Gd = X[0].cuda(), G[0].cuda()
    Wd = [W.cuda() for W in Ws]
    got, kernels, cache = [], [], []
    for cached in (True, False):
        eng = ChainEngine(layers, tier=tier, cache_results=cached)
        try:
            for _ in range(2):  # the second step refills the entries the first made
                eng.forward(Xd, Wd)
                k0 = eng.kernels
                dX, dWs = eng.backward(Xd, Wd, Gd)
                eng._drain()
            kernels.append(eng.kernels - k0)
            cache.append(H.hpvm_plane_cache_bytes(eng.ctx))
            got.append([t.cpu() for t in [dX] + dWs])
        finally:
            eng.close()
    for a, b in zip(*got):
        assert torch.equal(a, b)
    assert kernels[1] - kernels[0] == 2 * (layers - 1)
    # the cache holds the 2 (L - 1) result entries besides the weights' and X's
    kp = -(-rows // 8) * 8
    entry = -(-w * kp * 2 // 256) * 256 * (2 if tier == H.HPVM_TIER_BF16X3 else 1)
    assert cache[0] - cache[1] == 2 * (layers - 1) * entry
    # (the products' accuracy is the subject of test_every_product_on_its_inputs;
    # here a sanity check of dX at the loosest tier bound)
    ref = J.chain_backward(X[0].double().numpy(), [W.double().numpy() for W in Ws], G[0].double().numpy())
    assert O.normwise_rel_err(got[0][0].double().numpy(), ref[0]) <= 1e-2


@pytest.mark.parametrize("tier", [H.HPVM_TIER_BF16, H.HPVM_TIER_BF16X3])
def test_cache_c_on_a_stage_without_merged_leaf_drops_the_entry(cuda_device, tier):
    # A tanh stage with CACHE_C fills C's row-plane entry; a plain stage (no
    # merged leaf: it cannot write planes) that overwrites C with CACHE_C
    # must drop that entry, so a later REUSE_A over C converts the new values.
    eng = ChainEngine(1, tier=tier)
    try:
        g = torch.Generator().manual_seed(5)
        Hm = torch.randn(200, 96, generator=g).cuda()
        W1 = (torch.randn(96, 136, generator=g) / 10).cuda()
        W2 = (torch.randn(96, 136, generator=g) / 10).cuda()
        V = torch.randn(200, 72, generator=g).cuda()
        out = torch.empty(200, 136, device="cuda")  # C: 136 x 200 column-major
        eng._run(eng.stage_tanh, _rm_product_args(out, Hm, W1, tier, H.HPVM_LAUNCH_CACHE_C))
        eng._run(eng.stage_plain, _rm_product_args(out, Hm, W2, tier, H.HPVM_LAUNCH_CACHE_C))

        def consume(flags):
            # P = C V^T over the column-major C (136 x 200): op(A) = A, K = 200
            P = torch.empty(72, 136, device="cuda")
            eng._run(eng.stage_plain, make_args(136, 72, 200, out.data_ptr(), out.numel() * 4, 136,
                                                V.data_ptr(), V.numel() * 4, 72, P.data_ptr(), P.numel() * 4,
                                                136, 1.0, 0.0, False, True, tier, flags=flags))
            eng._drain()
            return P.cpu()
        assert torch.equal(consume(H.HPVM_LAUNCH_REUSE_A), consume(0))
        # and with the tanh stage last, the entry it fills is the one REUSE_A reads
        eng._run(eng.stage_tanh, _rm_product_args(out, Hm, W1, tier, H.HPVM_LAUNCH_CACHE_C))
        k0 = eng.kernels
        reused = consume(H.HPVM_LAUNCH_REUSE_A)
        assert eng.kernels - k0 == 2  # the leaf and V's conversion only
        assert torch.equal(reused, consume(0))
    finally:
        eng.close()


@pytest.mark.parametrize("tier", [H.HPVM_TIER_BF16, H.HPVM_TIER_BF16X3])
def test_planes_only_skips_the_intermediate_results(cuda_device, tier):
    # HPVM_LAUNCH_PLANES_ONLY on every stage but the last of one chain launch:
    # the intermediate results are read only through the planes forwarded
    # to the next stage, so their FP32 buffers keep their old contents (NaN
    # here) while Y equals the launch that stores them, bit for bit.
    layers, rows, w = 3, 300, 264
    X, Ws, _ = _inputs(1, rows, w, layers, seed=17)
    Xd, Wd = X[0].cuda(), [W.cuda() for W in Ws]
    eng = ChainEngine(layers, tier=tier)
    try:
        got = []
        for mid in (H.HPVM_LAUNCH_PLANES_ONLY, 0):
            outs = [torch.full((rows, w), float("nan"), device="cuda") for _ in range(layers)]
            eng._run(eng.chain, eng.chain_records(Xd, Wd, outs, mid_flags=mid))
            eng._drain()
            got.append([o.cpu() for o in outs])
        planes_only, stored = got
        assert torch.equal(planes_only[-1], stored[-1])
        for l in range(layers - 1):
            assert torch.isnan(planes_only[l]).all()
            assert torch.isfinite(stored[l]).all()
        # forward() without keep uses the flag: the same Y as with keep
        assert torch.equal(eng.forward(Xd, Wd).cpu(), eng.forward(Xd, Wd, keep=True)[0].cpu())
        eng._drain()
    finally:
        eng.close()


@pytest.mark.parametrize("tier", [H.HPVM_TIER_BF16, H.HPVM_TIER_BF16X3])
def test_planes_only_is_ignored_where_no_planes_are_written(cuda_device, tier):
    # a single tanh stage writes no planes of its result (no forwarding, no
    # CACHE_C), and beta != 0 reads C: in both cases C is stored as usual
    eng = ChainEngine(1, tier=tier)
    try:
        g = torch.Generator().manual_seed(3)
        Hm = torch.randn(200, 96, generator=g).cuda()
        Wt = (torch.randn(96, 136, generator=g) / 10).cuda()
        out = torch.full((200, 136), float("nan"), device="cuda")
        eng._run(eng.stage_tanh, _rm_product_args(out, Hm, Wt, tier, H.HPVM_LAUNCH_PLANES_ONLY))
        stored = torch.empty(200, 136, device="cuda")
        eng._run(eng.stage_tanh, _rm_product_args(stored, Hm, Wt, tier))
        eng._drain()
        assert torch.equal(out.cpu(), stored.cpu())
        # beta != 0 with CACHE_C: the row planes are written, but C is read and stored
        C0 = torch.randn(200, 136, generator=g).cuda()
        outs = []
        for flags in (H.HPVM_LAUNCH_PLANES_ONLY | H.HPVM_LAUNCH_CACHE_C, 0):
            out2 = C0.clone()
            a = _rm_product_args(out2, Hm, Wt, tier, flags)
            a.beta = 0.5
            eng._run(eng.stage_tanh, a)
            eng._drain()
            outs.append(out2.cpu())
        assert torch.equal(outs[0], outs[1]) and not torch.equal(outs[0], C0.cpu())
    finally:
        eng.close()


FWD_CASES = [(H.HPVM_TIER_BF16, 3, 24, 16, 4), (H.HPVM_TIER_BF16, 2, 300, 256, 4),
             (H.HPVM_TIER_BF16, 1, 7, 5, 2), (H.HPVM_TIER_BF16X3, 3, 24, 16, 4),
             (H.HPVM_TIER_BF16X3, 1, 7, 5, 2), (H.HPVM_TIER_BF16X3, 1, 40, 24, 4)]


@pytest.mark.parametrize("tier,items,rows,w,layers", FWD_CASES)
def test_forward_and_streaming_match_oracle(cuda_device, tier, items, rows, w, layers):
    X, Ws, _ = _inputs(items, rows, w, layers, seed=rows + w)
    eng = ChainEngine(layers, tier=tier)
    try:
        Xd = X.cuda()
        Wd = [W.cuda() for W in Ws]
        Y = eng.forward(Xd.reshape(-1, w), Wd).reshape(items, rows, w).cpu()
        streamed = eng.stream_forward([Xd[i] for i in range(items)], Wd)
        Wn = [W.double().numpy() for W in Ws]
        for i in range(items):
            _, _, ref = J.chain_forward(X[i].double().numpy(), Wn)
            bound = TOL[tier] if tier == H.HPVM_TIER_BF16 else \
                J.chain_forward_error_bound(X[i].double().numpy(), Wn, STAGE_EPS[tier])
            err = O.normwise_rel_err(Y[i].double().numpy(), ref)
            print(f"forward item {i}: {err:.3e} (bound {bound:.3e})")
            assert err <= bound
            # an item pushed alone through the streaming graph gives the
            # result of the same rows in the batched launch
            assert O.normwise_rel_err(streamed[i].cpu().double().numpy(), Y[i].double().numpy()) <= 1e-6
    finally:
        eng.close()


GRAD_CASES = [(H.HPVM_TIER_BF16, 1, 24, 16), (H.HPVM_TIER_BF16, 2, 64, 128),
              (H.HPVM_TIER_BF16X3, 1, 24, 16), (H.HPVM_TIER_BF16X3, 2, 24, 32)]


@pytest.mark.parametrize("tier,items,rows,w", GRAD_CASES)
def test_gradients_match_oracle(cuda_device, tier, items, rows, w):
    layers = 4
    X, Ws, G = _inputs(items, rows, w, layers, seed=7 * rows + w)
    eng = ChainEngine(layers, tier=tier)
    try:
        Xd = X.cuda().requires_grad_(True)
        Wd = [W.cuda().requires_grad_(True) for W in Ws]
        Y = chain_apply(eng, Xd, Wd)
        (Y * G.cuda()).sum().backward()
        Xf = X.reshape(-1, w).double().numpy()
        Wn = [W.double().numpy() for W in Ws]
        Gf = G.reshape(-1, w).double().numpy()
        dX, dW = J.chain_backward(Xf, Wn, Gf)
        if tier == H.HPVM_TIER_BF16:
            bx, bw = TOL[tier], [TOL[tier]] * layers
        else:
            bx, bw = J.chain_grad_error_bound(Xf, Wn, Gf, STAGE_EPS[tier])
        ex = O.normwise_rel_err(Xd.grad.reshape(-1, w).double().cpu().numpy(), dX)
        print(f"dX: {ex:.3e} (bound {bx:.3e})")
        assert ex <= bx
        for l in range(layers):
            assert O.normwise_rel_err(Wd[l].grad.double().cpu().numpy(), dW[l]) <= bw[l]
    finally:
        eng.close()


@pytest.mark.parametrize("tier", [H.HPVM_TIER_BF16, H.HPVM_TIER_BF16X3])
@pytest.mark.parametrize("items,rows,w", [(1, 24, 16), (2, 64, 128), (1, 300, 264)])
def test_every_product_on_its_inputs(cuda_device, tier, items, rows, w):
    # One training step (forward keeping the activations, backward with the
    # FP32 intermediates stored: cache_results=False, whose products equal
    # the cached path's bit for bit, see the test above). Every product is
    # then checked against the oracle's product of the very FP32 inputs the
    # GPU consumed, at the tier's bound; a product followed by an
    # elementwise leaf is checked as (1) the plain leaf's product on the
    # same inputs, (2) the stage's output equal, bit for bit, to the
    # unmerged stage, (3) the elementwise kernel within ELEMENTWISE_TOL of
    # the FP64 function of the GPU's own product.
    layers = 4
    X, Ws, G = _inputs(items, rows, w, layers, seed=5 * rows + w)
    n = items * rows
    dev = torch.device("cuda:0")
    Xd, Gd = X.reshape(n, w).cuda(), G.reshape(n, w).cuda()
    Wd = [W.cuda() for W in Ws]
    eng = ChainEngine(layers, tier=tier, cache_results=False)
    unm = ChainEngine(1, tier=tier, fuse=False)
    try:
        Y, Hf = eng.forward(Xd, Wd, keep=True)
        dX, dWs = eng.backward(Xd, Wd, Gd)
        eng._drain()
        Hr = [eng._buf(("H", l), (n, w), dev) for l in range(layers - 1)]   # recomputed H_1..H_{L-1}
        dZb = {l: eng._buf(("dH", l), (n, w), dev) for l in range(1, layers)}  # dZ_{l-1}
        Hin = [Xd] + list(Hf)  # H_0 = X, H_l = tanh(Z_{l-1})
        errs = []

        def check_product(prod, a_in, b_in, what):
            # prod = a_in @ b_in (row-major), the inputs the GPU consumed
            a_in = torch.as_tensor(a_in).cpu()
            b_in = torch.as_tensor(b_in).cpu()
            got = prod.double().cpu().numpy()
            ref = _oracle_rm(a_in, b_in)
            e = O.normwise_rel_err(got, ref)
            errs.append((what, e))
            if tier == H.HPVM_TIER_BF16X3:
                ex3 = _split_rm(a_in, b_in)
                acc = float(np.linalg.norm(got - ex3) / np.linalg.norm(ref))
                assert acc <= ACC_TOL, (what, acc)
                if ref.size >= MIN_OUTPUTS_FOR_FP64_BOUND:
                    assert e <= TOL[tier], (what, e)
                else:
                    errs.append((what + "-method", O.normwise_rel_err(ex3, ref)))
            else:
                assert e <= TOL[tier], (what, e)

        # forward and recomputed forward: Z_l = H_l W_l
        for l in range(layers):
            a_in, out = Hin[l], (Hf[l] if l + 1 < layers else Y)
            prod = torch.empty(n, w, device=dev)
            _plain(unm, _rm_product_args(prod, a_in, Wd[l], tier))
            check_product(prod, a_in, Ws[l], f"Z{l}")
            if l + 1 < layers:
                assert torch.equal(Hr[l], Hf[l])  # the recomputation gives the same H
                ref_out = torch.empty(n, w, device=dev)
                unm._run(unm.stage_tanh, _rm_product_args(ref_out, a_in, Wd[l], tier, unm.flags))
                unm._drain()
                assert torch.equal(out.cpu(), ref_out.cpu())
                assert O.normwise_rel_err(out.double().cpu().numpy(),
                                          torch.tanh(prod.double().cpu()).numpy()) <= ELEMENTWISE_TOL
            else:
                assert torch.equal(out.cpu(), prod.cpu())
        # input adjoints: dH_l = dZ_l W_l^T (op(A) = A^T of W), then for l > 0
        # the merged tanh adjoint dZ_{l-1} = dH_l (1 - H_l^2)
        for l in range(layers - 1, -1, -1):
            dZ = Gd if l == layers - 1 else dZb[l + 1]
            W = Wd[l]
            prod = torch.empty(n, w, device=dev)
            a = make_args(w, n, w, W.data_ptr(), W.numel() * 4, w, dZ.data_ptr(), dZ.numel() * 4, w,
                          prod.data_ptr(), prod.numel() * 4, w, 1.0, 0.0, True, False, tier)
            _plain(unm, a)
            check_product(prod, dZ, Ws[l].t(), f"dH{l}")
            if l > 0:
                Hl = Hf[l - 1]
                ref_out = torch.empty(n, w, device=dev)
                a = make_args(w, n, w, W.data_ptr(), W.numel() * 4, w, dZ.data_ptr(), dZ.numel() * 4, w,
                              ref_out.data_ptr(), ref_out.numel() * 4, w, 1.0, 0.0, True, False, tier,
                              flags=unm.flags)
                a.aux, a.bytesAux, a.ldaux = Hl.data_ptr(), Hl.numel() * 4, w
                unm._run(unm.stage_dtanh, a)
                unm._drain()
                assert torch.equal(dZb[l].cpu(), ref_out.cpu())
                want = prod.double().cpu() * (1 - Hl.double().cpu() ** 2)
                assert O.normwise_rel_err(dZb[l].double().cpu().numpy(), want.numpy()) <= ELEMENTWISE_TOL
            else:
                assert torch.equal(dX.cpu(), prod.cpu())
        # weight adjoints: dW_l = H_l^T dZ_l
        for l in range(layers):
            dZ = Gd if l == layers - 1 else dZb[l + 1]
            check_product(dWs[l], Hin[l].t(), dZ, f"dW{l}")
        print(" ".join(f"{k}={v:.2e}" for k, v in errs))
    finally:
        eng.close()
        unm.close()


def test_pop_without_push_and_push_without_stream(cuda_device):
    eng = ChainEngine(2)
    try:
        X = torch.randn(8, 16, device="cuda")
        Ws = [torch.randn(16, 16, device="cuda") for _ in range(2)]
        outs = [torch.empty(8, 16, device="cuda") for _ in range(2)]
        rec = eng.chain_records(X, Ws, outs)
        g = H.hpvm_launch(eng.ctx, eng.chain, rec, True, 0)
        with pytest.raises(H.HpvmError) as e:
            H.hpvm_pop(g, None, 1000)
        assert e.value.code == H.HPVM_ERR_INVALID_ARG
        H.hpvm_push(g, rec)
        H.hpvm_pop(g, None, 60000)
        H.hpvm_wait(g, 60000)
        g2 = H.hpvm_launch(eng.ctx, eng.chain, rec, False, 0)
        with pytest.raises(H.HpvmError):
            H.hpvm_push(g2, rec)
        H.hpvm_wait(g2, 60000)
        torch.cuda.synchronize()
        _, _, ref = J.chain_forward(X.double().cpu().numpy(), [W.double().cpu().numpy() for W in Ws])
        assert O.normwise_rel_err(outs[-1].double().cpu().numpy(), ref) <= 1e-2
    finally:
        eng.close()


def test_push_revalidates_a_graph_changed_after_launch(cuda_device):
    # A streaming graph is validated at launch; pushes skip the validation
    # while no node, edge or binding has been added since. A binding added
    # after the launch that feeds a stage input twice makes the graph
    # invalid, and the next push must refuse it.
    from paper_1611_00860_gb300.chain import _add_stage
    eng = ChainEngine(1)
    try:
        root = H.hpvm_create_node(eng.ctx, None, H.HPVM_NODE_INTERNAL)
        st = _add_stage(eng.ctx, root, 0, H.HPVM_NODE_TANH_LEAF, b_from_edge=False)
        H.hpvm_bind_output(st, 0, 0, stream=True)
        X = torch.randn(8, 16, device="cuda")
        W = torch.randn(16, 16, device="cuda") / 4
        out = torch.empty(8, 16, device="cuda")
        rec = eng.chain_records(X, [W], [out])
        g = H.hpvm_launch(eng.ctx, root, rec, True, 0)
        for _ in range(2):
            H.hpvm_push(g, rec)
            H.hpvm_pop(g, None, 60000)
        torch.cuda.synchronize()
        assert O.normwise_rel_err(out.double().cpu().numpy(),
                                  np.tanh(X.double().cpu().numpy() @ W.double().cpu().numpy())) <= 1e-2
        H.hpvm_bind_input(st, 0, 0)  # input 0 of the stage is now fed twice
        with pytest.raises(H.HpvmError) as e:
            H.hpvm_push(g, rec)
        assert e.value.code == H.HPVM_ERR_INVALID_GRAPH
        H.hpvm_wait(g, 60000)
    finally:
        eng.close()


@pytest.mark.slow
def test_chain_workload_sampled_rows(cuda_device):
    # the chain workload: 64 items of 256 x 4096, four 4096 x 4096 weights,
    # BF16 operands; rows are independent, so the oracle checks the forward
    # output and the input gradient of 32 sampled rows of one item
    import workloads as W
    X, Ws, G = W.chain_inputs()
    eng = ChainEngine(4, tier=H.HPVM_TIER_BF16)
    try:
        Xd = X.cuda().requires_grad_(True)
        Wd = [w.cuda().requires_grad_(True) for w in Ws]
        Y = chain_apply(eng, Xd, Wd)
        (Y * G.cuda()).sum().backward()
        rows = torch.arange(0, 256, 8)
        Xs = X[5, rows].double().numpy()
        Wn = [w.double().numpy() for w in Ws]
        _, _, ref = J.chain_forward(Xs, Wn)
        assert O.normwise_rel_err(Y[5, rows].double().detach().cpu().numpy(), ref) <= 1e-2
        dX, _ = J.chain_backward(Xs, Wn, G[5, rows].double().numpy())
        assert O.normwise_rel_err(Xd.grad[5, rows].double().cpu().numpy(), dX) <= 1e-2
        assert np.isfinite(Wd[0].grad.cpu().numpy()).all()
    finally:
        eng.close()


@pytest.mark.parametrize("tier", [H.HPVM_TIER_BF16, H.HPVM_TIER_BF16X3])
@pytest.mark.parametrize("coalesce", [2, 3, 4])
@pytest.mark.parametrize("adjacent", [False, True])
def test_coalesced_streaming_equals_item_by_item(cuda_device, tier, coalesce, adjacent):
    # Items of one streaming graph run several at a time as one launch
    # (hpvm_stream_coalesce): 7 items, so the last group is short, of
    # differing rows (the columns of one item do not start on a tile
    # boundary). Each output must equal the item pushed alone, bit for bit
    # (these launches are too small to split a last round), pops come back
    # in push order, and a pop of a queued item launches the queue.
    layers, w = 3, 264
    rows = [256, 100, 256, 77, 300, 256, 128]
    g = torch.Generator().manual_seed(coalesce)
    if adjacent:  # views of one tensor, item after item: used in place
        whole = torch.randn(sum(rows), w, generator=g).cuda()
        starts = [sum(rows[:i]) for i in range(len(rows) + 1)]
        items = [whole[starts[i]:starts[i + 1]] for i in range(len(rows))]
    else:         # separate tensors: gathered into the workspace
        items = [torch.randn(r, w, generator=g).cuda() for r in rows]
    Ws = [(torch.randn(w, w, generator=g) / w ** 0.5).cuda() for _ in range(layers)]
    eng = ChainEngine(layers, tier=tier)
    try:
        one = eng.stream_forward(items, Ws, coalesce=1)
        many = eng.stream_forward(items, Ws, coalesce=coalesce)
        torch.cuda.synchronize()
        for a, b in zip(one, many):
            assert torch.equal(a, b)
        if tier == H.HPVM_TIER_BF16:  # (the item-by-item results are checked against the oracle above)
            _, _, ref = J.chain_forward(items[1].double().cpu().numpy(), [W.double().cpu().numpy() for W in Ws])
            assert O.normwise_rel_err(many[1].double().cpu().numpy(), ref) <= TOL[tier]
        # pop before the queue is full: the queued item is launched by the pop
        outs = [torch.full((rows[0], w), float("nan"), device="cuda") for _ in range(layers)]
        rec = eng.chain_records(items[0], Ws, outs)
        gr = H.hpvm_launch(eng.ctx, eng.chain, rec, True, 0)
        H.hpvm_stream_coalesce(gr, 8)
        H.hpvm_push(gr, rec)
        H.hpvm_pop(gr, None, 60000)
        H.hpvm_wait(gr, 60000)
        torch.cuda.synchronize()
        assert torch.equal(outs[-1], one[0])
    finally:
        eng.close()


def test_coalescing_falls_back_for_items_that_differ(cuda_device):
    # an item whose weights differ from the others' runs on its own, with
    # the same result as when every item runs alone
    layers, w, r = 2, 136, 64
    g = torch.Generator().manual_seed(9)
    Ws = [(torch.randn(w, w, generator=g) / w ** 0.5).cuda() for _ in range(layers)]
    W2 = [(torch.randn(w, w, generator=g) / w ** 0.5).cuda() for _ in range(layers)]
    X = [torch.randn(r, w, generator=g).cuda() for _ in range(4)]
    eng = ChainEngine(layers, tier=H.HPVM_TIER_BF16)
    try:
        outs = [[torch.empty(r, w, device="cuda") for _ in range(layers)] for _ in range(4)]
        ref = [[torch.empty(r, w, device="cuda") for _ in range(layers)] for _ in range(4)]
        for coalesce, dst in ((4, outs), (1, ref)):
            gr = H.hpvm_launch(eng.ctx, eng.chain, eng.chain_records(X[0], Ws, dst[0]), True, 0)
            H.hpvm_stream_coalesce(gr, coalesce)
            for i in range(4):
                H.hpvm_push(gr, eng.chain_records(X[i], W2 if i == 2 else Ws, dst[i]))
            for _ in range(4):
                H.hpvm_pop(gr, None, 60000)
            H.hpvm_wait(gr, 60000)
        torch.cuda.synchronize()
        for a, b in zip(outs, ref):
            assert torch.equal(a[-1], b[-1])
    finally:
        eng.close()
