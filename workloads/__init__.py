"""Seeded synthetic inputs for the sgemm dataflow-graph workloads.

This module is shared by the oracle (``oracle/``), the tests, ``bench.py`` and
the package's smoke check. It draws random numbers and nothing else: it holds
no part of the method's arithmetic (no products, no splitting, no
quantisation, no rounding of results). Every generator runs on the CPU with a
seeded ``torch.Generator`` so the oracle and the CUDA path see bit-identical
FP32 inputs.

Storage convention (the paper's sgemm leaf takes BLAS-style ``lda/ldb/ldc``
arguments, Section 6.1): matrices are column-major. A matrix with ``rows`` rows
and ``cols`` columns and leading dimension ``ld >= rows`` is a flat FP32
buffer of ``ld * cols`` elements whose element (r, c) sits at ``r + c * ld``.
The helpers below return such flat buffers together with their shapes.

Workload shapes (the sgemm example of Section 6.1 at the sizes the
measurement plan fixes):
  * small DFG:  M=128, N=96, K=160, alpha=1.5, beta=0.5, A,B,C ~ U[-1,1];
  * large DFG:  M=N=K=8192, A,B,C ~ N(0,1), alpha=beta=1; variant "colscale"
    multiplies column p of A by 2**u_p with u_p ~ U[-20,20];
  * batched:    512 instances, M,N,K each log-uniform in [32,2048];
  * chain:      64 items of 256x4096, four 4096x4096 weights ~ N(0,1/4096);
  * fp8:        M=N=K=16384, A,B ~ N(0,1) times a per-row log-normal(0,2)
    magnitude.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

__all__ = [
    "SgemmProblem",
    "col_major",
    "stored_shape",
    "uniform",
    "normal",
    "sgemm_problem",
    "small_dfg_problem",
    "large_dfg_problem",
    "sample_blocks",
    "batched_shapes",
    "chain_inputs",
    "fp8_problem",
]


def _gen(seed: int) -> torch.Generator:
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return g


def uniform(n: int, lo: float, hi: float, g: torch.Generator) -> torch.Tensor:
    """n FP32 samples from U[lo, hi)."""
    return torch.rand(n, generator=g, dtype=torch.float32) * (hi - lo) + lo


def normal(n: int, g: torch.Generator, std: float = 1.0) -> torch.Tensor:
    """n FP32 samples from N(0, std^2)."""
    x = torch.randn(n, generator=g, dtype=torch.float32)
    if std != 1.0:
        x = x * std
    return x


def stored_shape(rows_op: int, cols_op: int, trans: bool) -> tuple[int, int]:
    """Stored (rows, cols) of a matrix whose op() is rows_op x cols_op.

    op(X) = X when ``trans`` is False, X^T when it is True.
    """
    return (cols_op, rows_op) if trans else (rows_op, cols_op)


def col_major(flat: torch.Tensor, rows: int, cols: int, ld: int) -> torch.Tensor:
    """View a flat column-major buffer as a (rows, cols) tensor (strided)."""
    return flat.as_strided((rows, cols), (1, ld))


@dataclass
class SgemmProblem:
    """One sgemm instance: C <- alpha*op(A)*op(B) + beta*C, column-major."""

    M: int
    N: int
    K: int
    transA: bool
    transB: bool
    alpha: float
    beta: float
    A: torch.Tensor  # flat FP32, lda * cols(A)
    lda: int
    B: torch.Tensor  # flat FP32, ldb * cols(B)
    ldb: int
    C: torch.Tensor  # flat FP32, ldc * N
    ldc: int

    @property
    def a_shape(self) -> tuple[int, int]:
        return stored_shape(self.M, self.K, self.transA)

    @property
    def b_shape(self) -> tuple[int, int]:
        return stored_shape(self.K, self.N, self.transB)

    def flops(self) -> int:
        return 2 * self.M * self.N * self.K


def sgemm_problem(M: int, N: int, K: int, *, seed: int, transA: bool = False,
                  transB: bool = True, alpha: float = 1.0, beta: float = 0.0,
                  dist: str = "normal", pad: int = 0,
                  colscale: bool = False) -> SgemmProblem:
    """A seeded problem. ``dist`` is "normal" (N(0,1)), "uniform" (U[-1,1]) or
    "int8" (integers in [-8, 8], exactly representable everywhere).

    ``pad`` adds that many rows of unused leading-dimension slack to every
    operand (ld = rows + pad), filled with NaN so that a kernel which reads
    outside its operand is caught. ``colscale`` scales column p of op(A) by
    2**u_p, u_p ~ U[-20, 20].
    """
    g = _gen(seed)
    ar, ac = stored_shape(M, K, transA)
    br, bc = stored_shape(K, N, transB)
    lda, ldb, ldc = max(ar, 1) + pad, max(br, 1) + pad, max(M, 1) + pad

    def draw(n: int) -> torch.Tensor:
        if dist == "normal":
            return normal(n, g)
        if dist == "uniform":
            return uniform(n, -1.0, 1.0, g)
        if dist == "int8":
            return torch.randint(-8, 9, (n,), generator=g).to(torch.float32)
        raise ValueError(dist)

    def mat(rows: int, cols: int, ld: int) -> torch.Tensor:
        flat = torch.full((ld * cols,), float("nan"), dtype=torch.float32)
        if rows * cols:
            col_major(flat, rows, cols, ld).copy_(draw(rows * cols).view(cols, rows).t())
        return flat

    A = mat(ar, ac, lda)
    B = mat(br, bc, ldb)
    C = mat(M, N, ldc)
    if colscale and K:
        u = uniform(K, -20.0, 20.0, g).to(torch.float64)
        s = torch.exp2(u).to(torch.float32)  # scale of column p of op(A)
        Av = col_major(A, ar, ac, lda)
        if transA:
            Av.mul_(s.view(K, 1))  # op(A) = A^T: column p of op(A) is row p of A
        else:
            Av.mul_(s.view(1, K))
    return SgemmProblem(M, N, K, transA, transB, float(alpha), float(beta),
                        A, lda, B, ldb, C, ldc)


def small_dfg_problem(seed: int = 0) -> SgemmProblem:
    """The small sgemm DFG: M=128, N=96, K=160, alpha=1.5, beta=0.5, U[-1,1]."""
    return sgemm_problem(128, 96, 160, seed=seed, alpha=1.5, beta=0.5,
                         dist="uniform")


def large_dfg_problem(n: int = 8192, seed: int = 1, colscale: bool = False) -> SgemmProblem:
    """The large sgemm DFG: M=N=K=n, N(0,1), alpha=beta=1 (NT, column-major)."""
    return sgemm_problem(n, n, n, seed=seed, alpha=1.0, beta=1.0,
                         dist="normal", colscale=colscale)


def sample_blocks(M: int, N: int, bs: int = 256, count: int = 16,
                  seed: int = 11) -> list[tuple[int, int]]:
    """Top-left corners of sampled bs x bs output blocks on the bs-aligned block
    grid: ``count`` distinct seeded positions plus the first and the last block.
    Blocks at the ragged edge are clipped by the caller."""
    gm, gn = max(1, math.ceil(M / bs)), max(1, math.ceil(N / bs))
    total = gm * gn
    g = _gen(seed)
    picks = torch.randperm(total, generator=g)[: min(count, total)].tolist()
    picks = sorted(set(picks) | {0, total - 1})
    return [((p % gm) * bs, (p // gm) * bs) for p in picks]


def batched_shapes(count: int = 512, lo: int = 32, hi: int = 2048,
                   seed: int = 2) -> list[tuple[int, int, int]]:
    """(M, N, K) per instance, each log-uniform in [lo, hi], rounded to int."""
    g = _gen(seed)
    u = uniform(3 * count, math.log(lo), math.log(hi), g).to(torch.float64)
    v = torch.exp(u).round().clamp(lo, hi).to(torch.int64).view(count, 3)
    return [tuple(int(x) for x in row) for row in v.tolist()]


def chain_inputs(items: int = 64, rows: int = 256, width: int = 4096,
                 layers: int = 4, seed: int = 3):
    """Streamed chain: ``items`` inputs X_t (rows x width, N(0,1)) and
    ``layers`` weights W_l (width x width, N(0, 1/width)), plus a seeded
    upstream gradient G_t per item (N(0,1)) for the loss sum(Y * G).
    All row-major torch tensors (rows x width)."""
    g = _gen(seed)
    X = normal(items * rows * width, g).view(items, rows, width)
    W = normal(layers * width * width, g, std=1.0 / math.sqrt(width)).view(layers, width, width)
    G = normal(items * rows * width, g).view(items, rows, width)
    return X, W, G


def fp8_problem(n: int = 16384, seed: int = 4, sigma: float = 2.0) -> SgemmProblem:
    """FP8 workload: A, B ~ N(0,1) times exp(sigma*Z_r) per stored row r of A
    (the M side) and per row of B stored N x K (the N side); beta = 0."""
    p = sgemm_problem(n, n, n, seed=seed, alpha=1.0, beta=0.0, dist="normal")
    g = _gen(seed + 1000)
    ra = torch.exp(sigma * normal(n, g).to(torch.float64)).to(torch.float32)
    rb = torch.exp(sigma * normal(n, g).to(torch.float64)).to(torch.float32)
    col_major(p.A, n, n, p.lda).mul_(ra.view(n, 1))
    col_major(p.B, n, n, p.ldb).mul_(rb.view(n, 1))
    return p
