"""Pins of the interpreter's streamed chain (CPU only): sgemm stages joined
by elementwise tanh leaves over one-to-one edges, stages joined by streaming
all-to-all edges, items pushed and popped in order. Pinned to the FP64 chain
definition of oracle/adjoint.py (itself pinned by finite differences) and to
the plain product for a one-stage chain."""
import numpy as np
import pytest

from oracle import adjoint as J
from oracle import dfg as D


@pytest.mark.parametrize("rows,w,layers,block", [(5, 6, 3, 4), (24, 16, 4, 8), (3, 2, 2, 2)])
def test_chain_equals_definition(rows, w, layers, block):
    rng = np.random.default_rng(rows * 10 + w)
    Ws = [rng.standard_normal((w, w)) / np.sqrt(w) for _ in range(layers)]
    items = [rng.standard_normal((rows, w)) for _ in range(3)]
    outs = D.run_chain(items, Ws, block=block)
    for X, Y in zip(items, outs):
        _, _, ref = J.chain_forward(X, Ws)
        assert np.allclose(Y, ref, rtol=1e-12, atol=1e-12)


def test_single_stage_is_the_product():
    rng = np.random.default_rng(1)
    W = rng.standard_normal((4, 4))
    X = rng.standard_normal((3, 4))
    (Y,) = D.run_chain([X], [W], block=2)
    assert np.allclose(Y, X @ W, rtol=1e-13, atol=1e-13)


def test_pop_order_is_push_order():
    rng = np.random.default_rng(2)
    Ws = [rng.standard_normal((3, 3)) for _ in range(2)]
    items = [np.full((2, 3), float(k)) for k in range(4)]
    outs = D.run_chain(items, Ws, block=2)
    refs = [J.chain_forward(X, Ws)[2] for X in items]
    assert all(np.allclose(a, b) for a, b in zip(outs, refs))
    g = D.StreamingGraph(D.Runtime(D.Memory()), D.make_chain_graph(1))
    with pytest.raises(D.DFGError):
        g.pop()


def test_tanh_leaf_needs_the_same_grid():
    # planted mistake: the elementwise leaf on another grid than the sgemm
    # leaf cannot take a one-to-one edge from it
    _, _, Allocation, SgemmLeaf = D.make_sgemm_graph()

    @D.internal(2)
    def Bad(rt, bx, by):
        sg = rt.createNode2D(SgemmLeaf, bx, by)
        th = rt.createNode2D(D.TanhLeaf, bx, by + 1)
        rt.createEdge(sg, th, False, 0, 0, False)

    with pytest.raises(D.DFGError):
        D.launch(D.Runtime(D.Memory()), Bad, [2, 2])
