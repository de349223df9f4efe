"""The differentiable streamed chain: sgemm stages joined by tanh leaves.

Row-major items X (rows x w) flow through L weights W_l (w x w):
Z_0 = X W_0, Z_l = tanh(Z_{l-1}) W_l, Y = Z_{L-1}. In the dataflow graph
each stage is a tile grid holding the sgemm example's Allocation and
SgemmLeaf plus, between stages, a TanhLeaf joined to the SgemmLeaf by
one-to-one edges (merged into the leaf's epilogue, MergeDependentNodes);
stages are joined by streaming all-to-all edges that carry the result
matrix (Sections 2.1, 3.5, 4.1).

A row-major matrix is a column-major matrix of the transposed shape, so
Z = H W is computed as the column-major sgemm Z^T = W^T H^T (M = w_out,
N = rows, K = w_in, op(A) = A, op(B) = B), and the adjoint products of the
sgemm leaf are sgemm leaves with the roles reversed:
    dW^T = dZ^T H     (M = w_out, N = w_in, K = rows, op(B) = B^T)
    dH^T = W dZ^T     (M = w_in,  N = rows, K = w_out, op(A) = A^T)
and the adjoint of the tanh leaf is the TanhGradLeaf, dZ_{l-1} =
dH_l * (1 - H_l^2), merged into the dH product's epilogue.

Results that go on only as operand planes are not stored in FP32: the
forward's intermediates (the backward recomputes them) and the adjoint
results dZ_l, whose planes the next adjoint stage and the weight adjoints
read (HPVM_LAUNCH_PLANES_ONLY with the forwarded and cached planes).

Argument marshalling only: every product and elementwise leaf runs in the
library's kernels through the C-ABI. PyTorch provides memory and streams.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as H
from .sgemm import make_args

REC = H.HPVM_RECORD_PORTS  # root ports per stage record


def _add_stage(ctx: int, root: int, base: int, ew_kind: int | None, b_from_edge: bool):
    """One tile-grid stage under ``root`` whose inputs are root ports
    base + field (see hpvm_sgemm_root_args). Returns the stage node."""
    st = H.hpvm_create_node(ctx, root, H.HPVM_NODE_INTERNAL,
                            (H.HPVM_DIM_FROM_INPUT(base + 14), H.HPVM_DIM_FROM_INPUT(base + 15)))
    # stage inputs: 0..19 = the record fields 0..13, 16..19 as in the sgemm
    # internal node; 20..22 = aux, bytesAux, ldaux
    for p in range(14):
        if b_from_edge and p in (3, 4):
            continue  # B and bytesB arrive over the streaming edge
        H.hpvm_bind_input(st, base + p, p)
    for q in range(4):
        H.hpvm_bind_input(st, base + 16 + q, 14 + q)
    if ew_kind == H.HPVM_NODE_TANH_GRAD_LEAF:
        for q in range(3):
            H.hpvm_bind_input(st, base + 20 + q, 18 + q)
    alloc = H.hpvm_create_node(ctx, st, H.HPVM_NODE_ALLOCATION)
    leaf = H.hpvm_create_node(ctx, st, H.HPVM_NODE_SGEMM_LEAF,
                              (H.HPVM_DIM_FROM_INPUT(12), H.HPVM_DIM_FROM_INPUT(13)))
    for sp, dp in ((0, 12), (1, 13), (2, 14), (3, 15)):
        H.hpvm_create_edge(alloc, leaf, H.HPVM_ALL_TO_ALL, sp, dp)
    for p in range(12):
        H.hpvm_bind_input(leaf, p, p)
    for q in range(4):
        H.hpvm_bind_input(leaf, 14 + q, 16 + q)
    H.hpvm_bind_input(alloc, 12, 0)
    H.hpvm_bind_input(alloc, 13, 1)
    last = leaf
    if ew_kind is not None:
        ew = H.hpvm_create_node(ctx, st, ew_kind,
                                (H.HPVM_DIM_FROM_INPUT(12), H.HPVM_DIM_FROM_INPUT(13)))
        H.hpvm_create_edge(leaf, ew, H.HPVM_ONE_TO_ONE, 0, 0)
        H.hpvm_create_edge(leaf, ew, H.HPVM_ONE_TO_ONE, 1, 1)
        H.hpvm_bind_input(ew, 8, 2)    # ld = ldc
        H.hpvm_bind_input(ew, 14, 3)   # M
        H.hpvm_bind_input(ew, 15, 4)   # N
        if ew_kind == H.HPVM_NODE_TANH_GRAD_LEAF:
            for q in range(3):
                H.hpvm_bind_input(ew, 18 + q, 5 + q)  # H, bytesH, ldh
        last = ew
    H.hpvm_bind_output(last, 0, 0)
    H.hpvm_bind_output(last, 1, 1)
    return st


def build_chain_graph(ctx: int, layers: int, tanh_last: bool = False,
                      ew_kind: int = H.HPVM_NODE_TANH_LEAF) -> int:
    """Root -> ``layers`` stages, an elementwise leaf (tanh, or with
    ``ew_kind`` the tanh adjoint) merged into every stage but the last (into
    the last too with ``tanh_last``: the recomputation of the activations),
    stage l's result streamed into stage l+1's B. Returns the root."""
    root = H.hpvm_create_node(ctx, None, H.HPVM_NODE_INTERNAL)
    prev = None
    for l in range(layers):
        ew = l + 1 < layers or tanh_last
        st = _add_stage(ctx, root, REC * l, ew_kind if ew else None, b_from_edge=prev is not None)
        if prev is not None:
            H.hpvm_create_edge(prev, st, H.HPVM_ALL_TO_ALL, 0, 3, stream=True)
            H.hpvm_create_edge(prev, st, H.HPVM_ALL_TO_ALL, 1, 4, stream=True)
        prev = st
    H.hpvm_bind_output(prev, 0, 0, stream=True)
    H.hpvm_validate(root)
    return root


def build_single_stage_graph(ctx: int, ew_kind: int | None) -> int:
    """Root -> one stage with an optional merged elementwise leaf."""
    root = H.hpvm_create_node(ctx, None, H.HPVM_NODE_INTERNAL)
    st = _add_stage(ctx, root, 0, ew_kind, b_from_edge=False)
    H.hpvm_bind_output(st, 0, 0)
    H.hpvm_validate(root)
    return root


def _rm_product_args(out: torch.Tensor, Hm: torch.Tensor, W: torch.Tensor, tier: int, flags: int = 0):
    """Record for the row-major product out = Hm @ W (out: r x c, Hm: r x k,
    W: k x c) as the column-major sgemm out^T = W^T Hm^T."""
    r, k = Hm.shape
    c = W.shape[1]
    return make_args(c, r, k, W.data_ptr(), W.numel() * 4, c, Hm.data_ptr(), Hm.numel() * 4, k,
                     out.data_ptr(), out.numel() * 4, c, 1.0, 0.0, False, False, tier, flags=flags)


class ChainEngine:
    """The chain's graphs on one device: forward chain, one-stage graphs with
    a merged tanh (recomputation) or tanh adjoint, and the plain sgemm stage
    (weight gradients, input gradient)."""

    def __init__(self, layers: int, device: int = 0, tier: int = H.HPVM_TIER_BF16, fuse: bool = True,
                 cache_results: bool = True):
        self.layers = layers
        self.device = device
        self.tier = tier
        self.flags = 0 if fuse else H.HPVM_LAUNCH_NO_FUSION
        # the backward's weight adjoints read the planes of H_l and dZ_l that
        # the producing stages' epilogues cached (needs fuse)
        self.cache_results = cache_results and fuse
        self.kernels = 0  # kernels launched so far (hpvm_graph_info)
        self.ctx = H.hpvm_init(device)
        self.chain = build_chain_graph(self.ctx, layers)
        # H_1 .. H_{L-1} again in backward: the first L - 1 stages, all with tanh
        self.rechain = build_chain_graph(self.ctx, layers - 1, tanh_last=True) if layers > 1 else None
        # the adjoint chain dH_l^T = W_l dZ_l^T, l = L-1 .. 0, the tanh adjoint
        # merged into every stage but the last (whose result is dX)
        self.adjchain = build_chain_graph(self.ctx, layers, ew_kind=H.HPVM_NODE_TANH_GRAD_LEAF)
        self.stage_tanh = build_single_stage_graph(self.ctx, H.HPVM_NODE_TANH_LEAF)
        self.stage_dtanh = build_single_stage_graph(self.ctx, H.HPVM_NODE_TANH_GRAD_LEAF)
        self.stage_plain = build_single_stage_graph(self.ctx, None)
        self._ws = None
        self._pending: list = []
        self._bufs: dict = {}

    def close(self):
        if self.ctx:
            try:
                self._drain()
            finally:
                H.hpvm_cleanup(self.ctx)
                self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers --------------------------------------------------------------
    def _stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def _run(self, root: int, args) -> None:
        """Launch asynchronously on the current stream. Launches share the
        workspace in stream order; their handles are released once finished
        (``_reap``, which never blocks) or waited for by ``_drain``."""
        need = H.hpvm_workspace_size(self.ctx, root, args)
        if need and (self._ws is None or self._ws.numel() < need):
            self._drain()
            self._ws = torch.empty(need, dtype=torch.uint8, device=f"cuda:{self.device}")
            H.hpvm_set_workspace(self.ctx, self._ws.data_ptr(), self._ws.numel())
        self._reap()
        g = H.hpvm_launch(self.ctx, root, args, False, self._stream())
        self._pending.append(g)
        self.kernels += H.hpvm_graph_info(g).kernels

    def _reap(self) -> None:
        """Release the handles of launches that have finished, oldest first,
        without waiting (a device fault surfaces here or in ``_drain``)."""
        while self._pending:
            try:
                H.hpvm_wait(self._pending[0], 0)
            except H.HpvmError as e:
                if e.code == H.HPVM_ERR_TIMEOUT:
                    return
                self._pending.pop(0)
                raise
            self._pending.pop(0)

    def _buf(self, name, shape, device) -> torch.Tensor:
        """An engine-owned buffer, the same one for every call with this name
        and shape: its pointer is the key of the planes cached for it."""
        key = (name, tuple(shape), str(device))
        t = self._bufs.get(key)
        if t is None:
            t = self._bufs[key] = torch.empty(*shape, device=device)
        return t

    def _drain(self, timeout_ms: int = 600000) -> None:
        pending, self._pending = self._pending, []
        for g in pending:
            H.hpvm_wait(g, timeout_ms)

    def chain_records(self, X: torch.Tensor, Ws, outs, plane_flags: int = 0, x_flags: int = 0,
                      out_flags: int = 0, mid_flags: int = 0):
        """Records of a chain graph of len(Ws) stages: stage l computes
        outs[l] = act(in_l) W_l. plane_flags (HPVM_LAUNCH_CACHE_A / REUSE_A)
        applies to the weights, the stages' A operands; x_flags
        (HPVM_LAUNCH_CACHE_B / REUSE_B) to X, the first stage's B (later
        stages take their B planes from the previous stage's epilogue);
        out_flags (HPVM_LAUNCH_CACHE_C) to every stage's result, mid_flags
        (HPVM_LAUNCH_PLANES_ONLY) to every stage's but the last."""
        arr = (H.RootArgs * len(Ws))()
        for l in range(len(Ws)):
            src = X if l == 0 else outs[l - 1]
            arr[l] = _rm_product_args(outs[l], src, Ws[l], self.tier,
                                      self.flags | plane_flags | out_flags | (x_flags if l == 0 else 0) |
                                      (mid_flags if l < len(Ws) - 1 else 0))
            if l > 0:  # B arrives over the streaming edge
                arr[l].B = None
                arr[l].bytesB = 0
        return arr

    # -- forward ------------------------------------------------------------------
    def forward(self, X: torch.Tensor, Ws, keep: bool = False):
        """Y for row-major X (rows x w). With keep, also the activations
        H_1..H_{L-1} (the tanh outputs, the chain's intermediate buffers)."""
        outs = [torch.empty(X.shape[0], W.shape[1], device=X.device) for W in Ws]
        # the weights' and X's planes are made afresh (they may have changed
        # since the last call) and kept for the recomputation in backward;
        # without keep the intermediate results are read only through the
        # planes forwarded to the next stage, so they are not stored
        mid = 0 if keep else H.HPVM_LAUNCH_PLANES_ONLY
        self._run(self.chain, self.chain_records(X, Ws, outs, H.HPVM_LAUNCH_CACHE_A, H.HPVM_LAUNCH_CACHE_B,
                                                 mid_flags=mid))
        return (outs[-1], outs[:-1]) if keep else outs[-1]

    def recompute(self, X: torch.Tensor, Ws):
        """H_0 = X and H_l = tanh(H_{l-1} W_{l-1}) for l = 1..L-1: one launch
        of the first L - 1 stages, every one with its tanh leaf merged. The
        H_l are engine buffers (valid until the next call), and each stage's
        epilogue also caches their planes for the weight adjoints' op(B)."""
        if self.rechain is None:
            return [X]
        outs = [self._buf(("H", l), (X.shape[0], W.shape[1]), X.device) for l, W in enumerate(Ws[:-1])]
        # autograd guarantees the saved X and weights are unchanged since forward
        self._run(self.rechain, self.chain_records(X, Ws[:-1], outs, H.HPVM_LAUNCH_REUSE_A, H.HPVM_LAUNCH_REUSE_B,
                                                   self._cache_c()))
        return [X] + outs

    def _cache_c(self) -> int:
        return H.HPVM_LAUNCH_CACHE_C if self.cache_results else 0

    # -- backward -----------------------------------------------------------------
    def backward(self, X: torch.Tensor, Ws, G: torch.Tensor):
        """dX and dW_l of sum(Y * G), recomputing the activations.

        The input adjoints run as one launch of the adjoint chain: stage j
        (layer l = L-1-j) computes dH_l^T = W_l dZ_l^T with op(A) = A^T, and
        for l > 0 its merged tanh adjoint gives dZ_{l-1} = dH_l * (1 - H_l^2),
        streamed into stage j+1's B (so its planes come from stage j's
        epilogue). The weight adjoints dW_l^T = dZ_l^T H_l follow, one launch
        each (op(B) = B^T), reading the planes of dZ_l (l < L-1) and of H_l
        (l > 0) that the adjoint and recomputing stages' epilogues cached;
        dZ_l is then read only through planes and its FP32 values are not
        stored (HPVM_LAUNCH_PLANES_ONLY)."""
        Hs = self.recompute(X, Ws)
        L = self.layers
        rows = X.shape[0]
        G = G.contiguous()
        cc = self._cache_c()
        # dH_l: rows x w_in; dH_0 = dX is the caller's, the others engine buffers
        dHs = [torch.empty(rows, W.shape[0], device=X.device) if l == 0 else
               self._buf(("dH", l), (rows, W.shape[0]), X.device) for l, W in enumerate(Ws)]
        recs = (H.RootArgs * L)()
        for j, l in enumerate(range(L - 1, -1, -1)):
            W = Ws[l]
            w_in, w_out = W.shape
            a = make_args(w_in, rows, w_out, W.data_ptr(), W.numel() * 4, w_out,
                          G.data_ptr() if j == 0 else None, G.numel() * 4 if j == 0 else 0, w_out,
                          dHs[l].data_ptr(), dHs[l].numel() * 4, w_in, 1.0, 0.0, True, False, self.tier,
                          flags=self.flags | (cc | (H.HPVM_LAUNCH_PLANES_ONLY if cc else 0) if l > 0 else 0))
            if l > 0:
                a.aux, a.bytesAux, a.ldaux = Hs[l].data_ptr(), Hs[l].numel() * 4, w_in
            recs[j] = a
        self._run(self.adjchain, recs)
        dWs = [None] * L
        for l in range(L - 1, -1, -1):
            W = Ws[l]
            w_in, w_out = W.shape
            dZ = G if l == L - 1 else dHs[l + 1]
            # dW^T = dZ^T H_l: M = w_out, N = w_in, K = rows; A = dZ buffer, B = H_l buffer (B^T)
            dW = torch.empty_like(W)
            reuse = 0
            if cc:
                reuse = (H.HPVM_LAUNCH_REUSE_A if l < L - 1 else 0) | (H.HPVM_LAUNCH_REUSE_B if l > 0 else 0)
            a = make_args(w_out, w_in, rows, dZ.data_ptr(), dZ.numel() * 4, w_out, Hs[l].data_ptr(),
                          Hs[l].numel() * 4, w_in, dW.data_ptr(), dW.numel() * 4, w_out, 1.0, 0.0,
                          False, True, self.tier, flags=self.flags | reuse)
            self._run(self.stage_plain, a)
            dWs[l] = dW
        return dHs[0], dWs

    # -- streaming -----------------------------------------------------------------
    def stream_forward(self, items, Ws, timeout_ms: int = 600000, coalesce: int = 32):
        """Push every item (row-major rows x w) through the chain launched as a
        streaming graph and pop the outputs in order (hpvm_push / hpvm_pop).
        ``coalesce`` items at a time run as one launch (hpvm_stream_coalesce):
        an item alone fills a fraction of the GPU (4096 x 256 results are 16
        tiles of 256 x 256)."""
        L = self.layers
        n = len(items)
        # each stage's results of all items in one tensor (item after item):
        # a coalesced launch writes them in place; item i's rows start at
        # starts[i] (pointers computed, views made only where needed)
        starts = np.zeros(n + 1, dtype=np.int64)
        np.cumsum([X.shape[0] for X in items], out=starts[1:])
        stage_out = [torch.empty(int(starts[-1]), W.shape[1], device=items[0].device) for W in Ws]

        def outs_of(i):
            return [o[int(starts[i]):int(starts[i + 1])] for o in stage_out]

        outs0 = outs_of(0)
        mid = H.HPVM_LAUNCH_PLANES_ONLY  # only the last stage's results are returned
        # every item's records in one array: the first item's converts the
        # weights into the plane cache, later items reuse those planes; items
        # of the first item's shape differ only in X and the stage results
        size = ctypes.sizeof(H.RootArgs) * L
        recs = (H.RootArgs * (L * n))()
        first = self.chain_records(items[0], Ws, outs0, H.HPVM_LAUNCH_CACHE_A, mid_flags=mid)
        reuse = self.chain_records(items[0], Ws, outs0, H.HPVM_LAUNCH_REUSE_A, mid_flags=mid)
        same = np.array([i for i, X in enumerate(items) if i > 0 and X.shape == items[0].shape], dtype=np.int64)
        raw = np.frombuffer(recs, dtype=np.uint8).reshape(n, size)
        if same.size:
            # the template copied to those items at once, then their X (B of
            # stage 0) and stage results (C of every stage) patched in
            raw[same] = np.frombuffer(reuse, dtype=np.uint8)
            b_off, c_off = H.RootArgs.B.offset, H.RootArgs.C.offset
            as_bytes = lambda p: np.ascontiguousarray(p, dtype="<i8").view(np.uint8).reshape(-1, 8)
            raw[same, b_off:b_off + 8] = as_bytes([items[i].data_ptr() for i in same])
            rec_bytes = ctypes.sizeof(H.RootArgs)
            for l in range(L):
                o = l * rec_bytes + c_off
                ptrs = stage_out[l].data_ptr() + starts[same] * (stage_out[l].shape[1] * 4)
                raw[same, o:o + 8] = as_bytes(ptrs)
        for i, X in enumerate(items):
            if i == 0 or X.shape != items[0].shape:
                src = first if i == 0 else self.chain_records(X, Ws, outs_of(i), H.HPVM_LAUNCH_REUSE_A, mid_flags=mid)
                ctypes.memmove(ctypes.addressof(recs) + i * size, ctypes.addressof(src), size)
        g = H.hpvm_launch(self.ctx, self.chain, self.chain_records(items[0], Ws, outs0, mid_flags=mid),
                          True, self._stream())
        try:
            H.hpvm_stream_coalesce(g, coalesce)
            for i in range(len(items)):
                H.hpvm_push(g, (H.RootArgs * L).from_buffer(recs, i * size))
            popped = []
            rec = (H.RootArgs * L)()
            for _ in items:
                H.hpvm_pop(g, rec, timeout_ms)
                popped.append(rec[L - 1].C)
        finally:
            H.hpvm_wait(g, timeout_ms)
        last = stage_out[-1]
        results = [last[int(starts[i]):int(starts[i + 1])] for i in range(n)]
        assert popped == [r.data_ptr() for r in results]
        return results


class ChainFunction(torch.autograd.Function):
    """Y = chain(X; W_0..W_{L-1}) with the library's forward and adjoint
    leaves; the backward recomputes the activations from X."""

    @staticmethod
    def forward(ctx, engine: ChainEngine, X: torch.Tensor, *Ws: torch.Tensor):
        X = X.contiguous()
        Ws = [W.contiguous() for W in Ws]
        ctx.engine = engine
        ctx.save_for_backward(X, *Ws)
        return engine.forward(X, Ws)

    @staticmethod
    def backward(ctx, G: torch.Tensor):
        X, *Ws = ctx.saved_tensors
        dX, dWs = ctx.engine.backward(X, Ws, G.contiguous().float())
        return (None, dX, *dWs)


def chain_apply(engine: ChainEngine, X: torch.Tensor, Ws) -> torch.Tensor:
    """Differentiable chain over X of shape (..., w): leading dimensions are
    the items and their rows, flattened into one product per stage."""
    shape = X.shape
    Y = ChainFunction.apply(engine, X.reshape(-1, shape[-1]), *Ws)
    return Y.reshape(*shape[:-1], Ws[-1].shape[1])


__all__ = ["ChainEngine", "ChainFunction", "chain_apply", "build_chain_graph", "build_single_stage_graph"]
