"""Oracle for the sgemm hierarchical dataflow graph (HPVM, arXiv 1611.00860).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, independent
reference that the CUDA library is checked against. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it. The product package never imports it and has no CPU fallback.
It shares no code, header, table or constant generator with the CUDA path;
the only module both sides use is ``workloads`` (seeded random inputs, no
arithmetic of the method).

Contents
  * ``sgemm``   -- the definition C <- alpha*op(A)*op(B) + beta*C in FP64
                   (plain C triple loop, Section 6.1 SgemmLeaf), whole or on
                   sampled blocks, and the normwise error metric.
  * ``dfg``     -- a small interpreter of the hierarchical dataflow graph
                   (Sections 2.1-2.2, the intrinsics of Table 1) that runs the
                   sgemm example graph node by node, leaf instances in
                   barrier-separated phases.
  * ``quant``   -- round-to-nearest-even FP32->BF16, the two-term BF16 split,
                   FP32->e4m3 saturating, per-128x128-block FP8 scaling.
  * ``adjoint`` -- FP64 gradients of the sgemm leaf and of the tanh chain.

Pins (what ties each function to something other than itself) live in
``tests/test_oracle_*.py``; see each function's docstring for the passage of
the paper it follows.
"""
from .build import build, lib_path  # noqa: F401
