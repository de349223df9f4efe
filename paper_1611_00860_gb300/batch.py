"""Batches of independent sgemm DFG instances in one persistent launch.

Argument marshalling only: the instances are records of the sgemm example
graph (one per instance); ``hpvm_batch_prepare`` lowers each, takes the
tile height (a CTA or a CTA pair), every instance's tile width and where the
operand planes are made (a split launch, or inside the leaf) from a policy
(or the one ``hpvm_batch_autotune`` measured best), and lays the operand
planes and schedule out on the device; ``hpvm_batch_run`` enqueues the
batched split pre-pass and the grouped persistent leaf. ``capture`` records
a run in a CUDA graph for replay.
"""
from __future__ import annotations

import torch

from . import _lib as H
from .sgemm import build_sgemm_graph, make_args


class BatchDFG:
    """One context and sgemm graph; ``prepare`` a batch from problems whose
    A, B, C are flat float32 CUDA tensors (column-major, see ``workloads``)."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        self.ctx = H.hpvm_init(self.device)
        self.root = build_sgemm_graph(self.ctx)["root"]
        self.batch = None
        self._records = None

    def close(self):
        if self.ctx:
            H.hpvm_cleanup(self.ctx)
            self.ctx = None
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def records(self, problems, tensors, tier):
        arr = (H.RootArgs * len(problems))()
        for i, (p, (A, B, C)) in enumerate(zip(problems, tensors)):
            arr[i] = make_args(p.M, p.N, p.K, A.data_ptr() if A.numel() else None, A.numel() * 4, p.lda,
                               B.data_ptr() if B.numel() else None, B.numel() * 4, p.ldb,
                               C.data_ptr() if C.numel() else None, C.numel() * 4, p.ldc,
                               p.alpha, p.beta, p.transA, p.transB, tier)
        return arr

    def prepare(self, problems, tensors, tier=H.HPVM_TIER_BF16X3, policy: int = -1) -> int:
        if self.batch is not None:
            H.hpvm_batch_free(self.batch)
            self.batch = None
        self._records = self.records(problems, tensors, tier)
        self.batch = H.hpvm_batch_prepare(self.ctx, self.root, self._records, len(problems), policy)
        return self.batch

    def run(self, stream: torch.cuda.Stream | None = None) -> None:
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        H.hpvm_batch_run(self.batch, s.cuda_stream)

    def autotune(self, reps: int = 3) -> tuple[int, float]:
        return H.hpvm_batch_autotune(self.batch, torch.cuda.current_stream(self.device).cuda_stream, reps)

    def info(self) -> dict:
        return H.hpvm_batch_info(self.batch).as_dict()

    def capture(self) -> torch.cuda.CUDAGraph:
        """A CUDA graph holding one run of the batch (replay with .replay())."""
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self.run(side)  # warm-up outside the capture
        torch.cuda.current_stream(self.device).wait_stream(side)
        torch.cuda.synchronize(self.device)
        with torch.cuda.graph(graph):
            H.hpvm_batch_run(self.batch, torch.cuda.current_stream(self.device).cuda_stream)
        return graph
