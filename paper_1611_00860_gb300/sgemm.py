"""The sgemm dataflow graph of Section 6.1, built through the C-ABI, and a
launcher that passes PyTorch CUDA tensors to it.

Argument marshalling only: the graph is built with the intrinsic calls of
``_lib`` and every launch runs the library's kernels. PyTorch provides the
device memory (operands and the workspace) and the CUDA stream.

Port numbering (the listing's ports, extended where it leaves values
implicit):
  SgemmLeaf   0 A, 1 bytesA, 2 lda, 3 B, 4 bytesB, 5 ldb, 6 C, 7 bytesC,
              8 ldc, 9 k, 10 alpha, 11 beta, 12 shB, 13 bytesShB,
              14 shA, 15 bytesShA, 16 M, 17 N, 18 transA, 19 transB
  Internal    0..11 as the leaf, 12 block_x, 13 block_y, 14 M, 15 N,
              16 transA, 17 transB
  Root        the record fields 0..19 (hpvm_sgemm_root_args)
  Allocation  in: 0 block_x, 1 block_y; out: 0 shB, 1 bytesShB, 2 shA, 3 bytesShA
"""
from __future__ import annotations

import torch

from . import _lib as H


def build_sgemm_graph(ctx: int) -> dict:
    """Create SgemmRoot -> SgemmInternal (2-D, grid_x x grid_y) ->
    {Allocation, SgemmLeaf (2-D, block_x x block_y)} under ``ctx``.
    Returns the node handles."""
    root = H.hpvm_create_node(ctx, None, H.HPVM_NODE_INTERNAL)
    # createNode2D(SgemmInternal, grid_x, grid_y): extents are root inputs 14, 15
    inner = H.hpvm_create_node(ctx, root, H.HPVM_NODE_INTERNAL,
                               (H.HPVM_DIM_FROM_INPUT(14), H.HPVM_DIM_FROM_INPUT(15)))
    for p in range(14):
        H.hpvm_bind_input(inner, p, p)
    for q in range(4):  # M, N, transA, transB
        H.hpvm_bind_input(inner, 16 + q, 14 + q)
    alloc = H.hpvm_create_node(ctx, inner, H.HPVM_NODE_ALLOCATION)
    # createNode2D(SgemmLeaf, block_x, block_y): extents are internal inputs 12, 13
    leaf = H.hpvm_create_node(ctx, inner, H.HPVM_NODE_SGEMM_LEAF,
                              (H.HPVM_DIM_FROM_INPUT(12), H.HPVM_DIM_FROM_INPUT(13)))
    for sp, dp in ((0, 12), (1, 13), (2, 14), (3, 15)):
        H.hpvm_create_edge(alloc, leaf, H.HPVM_ALL_TO_ALL, sp, dp)
    for p in range(12):
        H.hpvm_bind_input(leaf, p, p)
    H.hpvm_bind_input(alloc, 12, 0)
    H.hpvm_bind_input(alloc, 13, 1)
    for q in range(4):
        H.hpvm_bind_input(leaf, 14 + q, 16 + q)
    return {"root": root, "internal": inner, "allocation": alloc, "leaf": leaf}


def make_args(M, N, K, A_ptr, bytesA, lda, B_ptr, bytesB, ldb, C_ptr, bytesC, ldc,
              alpha, beta, transA, transB, tier, block=None, grid=None, flags=0) -> H.RootArgs:
    """Pack the root record. ``block``/``grid`` default to the tier's plan."""
    if block is None or grid is None:
        bx, by, gx, gy = H.hpvm_plan_sgemm(tier, M, N, K)
        block = block or (bx, by)
        grid = grid or (gx, gy)
    a = H.RootArgs()
    a.A, a.bytesA, a.lda = A_ptr, int(bytesA), int(lda)
    a.B, a.bytesB, a.ldb = B_ptr, int(bytesB), int(ldb)
    a.C, a.bytesC, a.ldc = C_ptr, int(bytesC), int(ldc)
    a.k, a.alpha, a.beta = int(K), float(alpha), float(beta)
    a.block_x, a.block_y = int(block[0]), int(block[1])
    a.grid_x, a.grid_y = int(grid[0]), int(grid[1])
    a.M, a.N, a.transA, a.transB = int(M), int(N), int(bool(transA)), int(bool(transB))
    a.tier, a.flags = int(tier), int(flags)
    return a


def _nbytes(t: torch.Tensor | None) -> int:
    return 0 if t is None else t.numel() * t.element_size()


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None or t.numel() == 0 else t.data_ptr()


class SgemmDFG:
    """One context, one sgemm graph, and a PyTorch-owned workspace.

    ``launch`` takes flat FP32 CUDA tensors holding column-major matrices
    (see ``workloads``) and enqueues the graph on the current torch stream;
    ``wait`` blocks until it finished. ``__call__`` does both."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        self.ctx = H.hpvm_init(self.device)
        self.nodes = build_sgemm_graph(self.ctx)
        H.hpvm_validate(self.nodes["root"])
        self._ws = None
        self.last_info = None

    def close(self):
        if self.ctx:
            H.hpvm_cleanup(self.ctx)
            self.ctx = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def args_for(self, M, N, K, A, lda, B, ldb, C, ldc, alpha=1.0, beta=0.0,
                 transA=False, transB=True, tier=H.HPVM_TIER_BF16X3, block=None,
                 grid=None, flags=0) -> H.RootArgs:
        for name, t in (("A", A), ("B", B), ("C", C)):
            if t is not None and t.numel():
                if t.dtype != torch.float32:
                    raise TypeError(f"{name} must be float32")
                if not t.is_contiguous():
                    raise ValueError(f"{name} must be a contiguous flat buffer")
        return make_args(M, N, K, _ptr(A), _nbytes(A), lda, _ptr(B), _nbytes(B), ldb,
                         _ptr(C), _nbytes(C), ldc, alpha, beta, transA, transB, tier,
                         block, grid, flags)

    def ensure_workspace(self, args: H.RootArgs) -> None:
        need = H.hpvm_workspace_size(self.ctx, self.nodes["root"], args)
        if need and (self._ws is None or self._ws.numel() < need):
            self._ws = torch.empty(need, dtype=torch.uint8, device=f"cuda:{self.device}")
            H.hpvm_set_workspace(self.ctx, self._ws.data_ptr(), self._ws.numel())

    def launch(self, args: H.RootArgs, stream: torch.cuda.Stream | None = None) -> int:
        self.ensure_workspace(args)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return H.hpvm_launch(self.ctx, self.nodes["root"], args, False, s.cuda_stream)

    def wait(self, graph: int, timeout_ms: int = -1) -> None:
        H.hpvm_wait(graph, timeout_ms)

    def __call__(self, *a, timeout_ms: int = 60000, **kw):
        args = self.args_for(*a, **kw)
        g = self.launch(args)
        self.last_info = H.hpvm_graph_info(g).as_dict()
        self.wait(g, timeout_ms)
        return self.last_info

    def run_problem(self, p, tier, dev_tensors=None, block=None, grid=None, timeout_ms=60000, flags=0):
        """Run a ``workloads.SgemmProblem`` whose A, B, C were moved to the device
        (``dev_tensors`` = (A, B, C) CUDA tensors; C is updated in place)."""
        A, B, C = dev_tensors
        return self(p.M, p.N, p.K, A, p.lda, B, p.ldb, C, p.ldc, p.alpha, p.beta,
                    p.transA, p.transB, tier=tier, block=block, grid=grid,
                    timeout_ms=timeout_ms, flags=flags)
