"""Pins of the oracle's dataflow-graph interpreter (CPU only).

The interpreter runs the sgemm example graph node by node. It is pinned to
the paper's listing (graph structure, port numbers, allocation size, record
layout), to the FP64 definition by brute force on tiny graphs, and to the
barrier semantics by a planted mistake (a leaf without its barrier reads a
tile before any instance wrote it).
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import dfg as D
from oracle import sgemm as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sgemm_dfg_listing.txt")


def _golden_records():
    recs = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                recs.append(line.split())
    return recs


def _flat(p):
    return (p.A.double().tolist(), p.B.double().tolist(), p.C.double().tolist())


def test_trace_contains_every_call_of_the_listing():
    p = W.sgemm_problem(8, 8, 8, seed=0, beta=0.5)
    A, B, C = _flat(p)
    _, rt = D.run_sgemm_dfg(p.M, p.N, p.K, A, p.lda, B, p.ldb, C, p.ldc,
                            p.alpha, p.beta, p.transA, p.transB, block=4,
                            return_runtime=True)
    trace = rt.trace
    names = {"block_x": 4, "block_y": 4, "grid_x": 2, "grid_y": 2}
    for rec in _golden_records():
        who, what = rec[0], rec[1]
        if who not in ("SgemmInternal", "SgemmRoot"):
            continue
        if what == "createNode":
            assert ("createNode", rec[2], ()) in trace
        elif what == "createNode2D":
            dims = (names[rec[3]], names[rec[4]])
            assert ("createNode", rec[2], dims) in trace
        elif what == "createEdge":
            want = ("createEdge", rec[2], rec[3], rec[4] == "all_to_all", int(rec[5]), int(rec[6]))
            assert want in trace
        elif what == "bind.input":
            assert ("bind.input", rec[2], int(rec[3]), int(rec[4])) in trace


def test_allocation_size_formula():
    rec = [r for r in _golden_records() if r[0] == "Allocation"][0]
    _, _, alloc, _ = D.make_sgemm_graph()
    mem = D.Memory()
    rt = D.Runtime(mem)
    for bx, by in [(16, 16), (4, 4), (3, 5)]:
        out = alloc(rt, bx, by)
        assert out[1] == bx * by * int(rec[4]) == (bx * by) << 2
        assert len(mem.objs[out[0][0]]) == bx * by


def test_linear_instance_id_is_x_fastest():
    seen = []

    @D.leaf(0)
    def Probe(rt):
        me = rt.getNode()
        x, y = rt.getNodeInstanceID(me, 0), rt.getNodeInstanceID(me, 1)
        nx = rt.getNumNodeInstances(me, 0)
        seen.append((nx * y + x, x, y))
        return ()

    @D.internal(0)
    def Root(rt):
        rt.createNode2D(Probe, 3, 2)

    D.launch(D.Runtime(D.Memory()), Root, [])
    # the interpreter starts instances in linear-id order: id = numX * y + x
    assert [s[0] for s in seen] == list(range(6))
    assert seen[1][1:] == (1, 0) and seen[3][1:] == (0, 1)


@pytest.mark.parametrize("transA,transB", [(False, True), (False, False), (True, False), (True, True)])
@pytest.mark.parametrize("M,N,K,block", [(5, 3, 7, 2), (4, 4, 4, 4), (9, 6, 10, 3), (1, 1, 1, 1), (7, 5, 0, 2)])
def test_interpreter_equals_definition(M, N, K, block, transA, transB):
    p = W.sgemm_problem(M, N, K, seed=M * 100 + N * 10 + K, transA=transA,
                        transB=transB, alpha=1.5, beta=0.5, pad=1)
    A, B, C = _flat(p)
    out = D.run_sgemm_dfg(M, N, K, A, p.lda, B, p.ldb, C, p.ldc, p.alpha,
                          p.beta, transA, transB, block=block)
    got = np.array(out).reshape(N, p.ldc).T[:M, :]
    ref = O.sgemm_f64(p)
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-13)


def test_interpreter_small_workload_shape():
    # the small workload's DFG: 16x16 leaf, 8 x 6 internal grid, M=128, N=96, K=160
    p = W.small_dfg_problem()
    # run a 32 x 32 x 48 corner of it to keep the pure-Python interpreter quick
    M, N, K = 32, 32, 48
    sub = W.sgemm_problem(M, N, K, seed=0, alpha=1.5, beta=0.5, dist="uniform")
    A, B, C = _flat(sub)
    out = D.run_sgemm_dfg(M, N, K, A, sub.lda, B, sub.ldb, C, sub.ldc, 1.5, 0.5,
                          False, True, block=16, grid=(2, 2))
    got = np.array(out).reshape(N, sub.ldc).T[:M, :]
    assert np.allclose(got, O.sgemm_f64(sub), rtol=1e-13, atol=1e-13)
    assert (p.M // 16, p.N // 16) == (8, 6)


def test_barrier_is_needed():
    # planted mistake: a leaf that multiplies right after staging, without the
    # barrier, reads tile slots that other instances have not written yet
    # (malloc fills them with NaN), so the result is wrong.
    _, _, Allocation, Leaf = D.make_sgemm_graph()

    @D.leaf(20)
    def NoBarrierLeaf(rt, *a):
        g = Leaf(rt, *a)
        try:
            while True:
                next(g)  # run through every barrier without yielding
        except StopIteration:
            return ()

    @D.internal(18)
    def Internal(rt, *a):
        alloc = rt.createNode(Allocation)
        sg = rt.createNode2D(NoBarrierLeaf, a[12], a[13])
        for sp, dp in [(0, 12), (1, 13), (2, 14), (3, 15)]:
            rt.createEdge(alloc, sg, True, sp, dp, False)
        for q in range(12):
            rt.bind_input(sg, q, q, False)
        rt.bind_input(alloc, 12, 0, False)
        rt.bind_input(alloc, 13, 1, False)
        for q in range(4):
            rt.bind_input(sg, 14 + q, 16 + q, False)

    @D.internal(20)
    def Root(rt, *a):
        inner = rt.createNode2D(Internal, a[14], a[15])
        for q in range(14):
            rt.bind_input(inner, q, q, False)
        for q in range(4):
            rt.bind_input(inner, 16 + q, 14 + q, False)

    p = W.sgemm_problem(4, 4, 4, seed=1)
    mem = D.Memory()
    pA, pB, pC = (mem.new(x) for x in _flat(p))
    D.launch(D.Runtime(mem), Root, [pA, 64, p.lda, pB, 64, p.ldb, pC, 64, p.ldc, 4,
                                    1.0, 0.0, 2, 2, 2, 2, 4, 4, False, True])
    assert np.isnan(np.array(mem.objs[pC[0]])).any()


def test_graph_rules():
    @D.leaf(1)
    def L(rt, x):
        return (x,)

    @D.internal(1)
    def BadEdge(rt, x):
        a = rt.createNode1D(L, 4)
        b = rt.createNode1D(L, 3)
        rt.createEdge(a, b, False, 0, 0, False)  # one-to-one on unequal grids

    with pytest.raises(D.DFGError):
        D.launch(D.Runtime(D.Memory()), BadEdge, [1])
    with pytest.raises(D.DFGError):
        D.launch(D.Runtime(D.Memory()), L, [1])  # a leaf cannot be the root

    @D.internal(1)
    def Unbound(rt, x):
        rt.createNode(L)  # input 0 never bound

    with pytest.raises(D.DFGError):
        D.launch(D.Runtime(D.Memory()), Unbound, [1])

    @D.internal(1)
    def OneToOne(rt, x):
        a = rt.createNode1D(L, 3)
        b = rt.createNode1D(L, 3)
        rt.bind_input(a, 0, 0, False)
        rt.createEdge(a, b, False, 0, 0, False)

    D.launch(D.Runtime(D.Memory()), OneToOne, [5])
