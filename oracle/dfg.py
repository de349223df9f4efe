"""A small interpreter of HPVM's hierarchical dataflow graph, and the sgemm
example graph written in it.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Pure Python, meant for
tiny graphs; it is independent of the C-ABI graph builder of the product.

Semantics followed
  * Section 2.1: a program is a hierarchy of nodes; an internal node holds a
    child graph, a leaf node computes. A static node stands for a 1-D/2-D/3-D
    grid of independent dynamic instances. Edges are replicated either
    all-to-all (every source instance feeds every sink instance; it acts as a
    barrier between the groups) or one-to-one (instance i feeds instance i;
    the two grids must have the same rank and extents).
  * Section 2.2 / Table 1: node functions receive their incoming edges as
    arguments and return one value per outgoing edge. Internal node functions
    only call the graph intrinsics createNode{,1D,2D,3D}, createEdge,
    bind.input, bind.output. Leaf functions may use the query intrinsics
    getNode, getParentNode, getNumDims, getNodeInstanceID.[xyz],
    getNumNodeInstances.[xyz], the allocation intrinsic malloc and the
    synchronisation intrinsic barrier, which only orders the dynamic
    instances of the executing leaf that share its parent instance.
  * Section 3.4 (tiling): memory a leaf allocates is private to the instances
    of its sibling leaf created by the same dynamic instance of the parent.

Barriers are modelled by writing leaf functions as Python generators: each
``yield`` is a call to barrier(). The interpreter advances every instance of
a leaf (under one parent instance) to its next barrier before any instance
passes it, i.e. the code between two barriers is one phase.

Readings where the paper is silent (also listed in the design notes):
  * createEdge takes (src, dst, repl, sp, dp, stream), the order of the
    intrinsic list and of the example listing; repl True = all-to-all.
  * An all-to-all edge carries one value to every sink instance: from a
    single-instance source (the example's Allocation node), or from a
    replicated source whose instances all produce the same value (the
    result buffer a tile grid writes, in the chain of sgemm stages).
  * Replication extents may be given as values known to the parent function
    at the time it runs (the example passes its own arguments block_x,
    block_y, grid_x, grid_y).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field
from typing import Any, Callable


class DFGError(Exception):
    """An ill-formed graph or a leaf that breaks the barrier discipline."""


@dataclass(eq=False)
class Node:
    func: Callable
    dims: tuple  # extents, () for a single instance
    parent: "Node | None"
    n_in: int
    children: list = field(default_factory=list)
    edges: list = field(default_factory=list)      # edges among children
    in_binds: list = field(default_factory=list)   # (child, ip, ic, stream)
    out_binds: list = field(default_factory=list)  # (child, oc, op, stream)

    @property
    def is_internal(self) -> bool:
        return getattr(self.func, "hpvm_internal", False)

    def num_instances(self) -> int:
        return int(math.prod(self.dims)) if self.dims else 1


@dataclass
class Edge:
    src: Node
    dst: Node
    all_to_all: bool
    sp: int
    dp: int
    stream: bool


def internal(n_in: int):
    """Mark a Python function as an internal node function with n_in inputs."""
    def deco(f):
        f.hpvm_internal = True
        f.hpvm_n_in = n_in
        return f
    return deco


def leaf(n_in: int):
    """Mark a Python function as a leaf node function with n_in inputs."""
    def deco(f):
        f.hpvm_internal = False
        f.hpvm_n_in = n_in
        return f
    return deco


class Memory:
    """Flat FP64 memory objects named by handles; pointers are (handle, off)."""

    def __init__(self):
        self.objs: dict[int, list] = {}
        self._next = 1

    def new(self, values) -> tuple:
        h = self._next
        self._next += 1
        self.objs[h] = list(values)
        return (h, 0)

    def load(self, ptr, idx: int) -> float:
        h, off = ptr
        return self.objs[h][off + idx]

    def store(self, ptr, idx: int, v: float) -> None:
        h, off = ptr
        self.objs[h][off + idx] = v


class _Instance:
    """The identity of one running dynamic instance (for the query intrinsics)."""

    def __init__(self, node: Node, idx: tuple, parent: "_Instance | None"):
        self.node = node
        self.idx = idx
        self.parent = parent


class Runtime:
    """The intrinsics available to node functions (Table 1)."""

    def __init__(self, memory: Memory):
        self.mem = memory
        self._cur: _Instance | None = None
        self._building: Node | None = None
        self.trace: list = []  # (event, details) for structural tests

    # -- graph intrinsics (internal node functions only) -------------------
    def _child(self, f, dims) -> Node:
        if self._building is None:
            raise DFGError("graph intrinsic called outside an internal node")
        dims = tuple(int(d) for d in dims)
        if any(d <= 0 for d in dims):
            raise DFGError(f"replication extents must be positive: {dims}")
        n = Node(f, dims, self._building, f.hpvm_n_in)
        self._building.children.append(n)
        self.trace.append(("createNode", f.__name__, dims))
        return n

    def createNode(self, f) -> Node:
        return self._child(f, ())

    def createNode1D(self, f, n1) -> Node:
        return self._child(f, (n1,))

    def createNode2D(self, f, n1, n2) -> Node:
        return self._child(f, (n1, n2))

    def createNode3D(self, f, n1, n2, n3) -> Node:
        return self._child(f, (n1, n2, n3))

    def createEdge(self, src: Node, dst: Node, all_to_all: bool, sp: int,
                   dp: int, stream: bool = False) -> Edge:
        if self._building is None or src.parent is not self._building \
                or dst.parent is not self._building:
            raise DFGError("edge endpoints must be children of the current node")
        if not all_to_all and src.dims != dst.dims:
            raise DFGError("one-to-one edge needs identical grids")
        if not 0 <= dp < dst.n_in:
            raise DFGError("destination port out of range")
        e = Edge(src, dst, bool(all_to_all), int(sp), int(dp), bool(stream))
        self._building.edges.append(e)
        self.trace.append(("createEdge", src.func.__name__, dst.func.__name__,
                           bool(all_to_all), int(sp), int(dp)))
        return e

    def bind_input(self, child: Node, ip: int, ic: int, stream: bool = False):
        if self._building is None or child.parent is not self._building:
            raise DFGError("bind.input on a node that is not a child")
        if not 0 <= ic < child.n_in or not 0 <= ip < self._building.n_in:
            raise DFGError("bind.input port out of range")
        self._building.in_binds.append((child, int(ip), int(ic), bool(stream)))
        self.trace.append(("bind.input", child.func.__name__, int(ip), int(ic)))

    def bind_output(self, child: Node, oc: int, op: int, stream: bool = False):
        if self._building is None or child.parent is not self._building:
            raise DFGError("bind.output on a node that is not a child")
        self._building.out_binds.append((child, int(oc), int(op), bool(stream)))

    # -- query intrinsics (leaf node functions) ----------------------------
    def getNode(self) -> _Instance:
        return self._cur

    def getParentNode(self, n: _Instance) -> _Instance:
        return n.parent

    def getNumDims(self, n: _Instance) -> int:
        return len(n.node.dims)

    def getNodeInstanceID(self, n: _Instance, dim: int) -> int:
        return n.idx[dim] if dim < len(n.idx) else 0

    def getNumNodeInstances(self, n: _Instance, dim: int) -> int:
        return n.node.dims[dim] if dim < len(n.node.dims) else 1

    # -- memory -------------------------------------------------------------
    def malloc(self, nbytes: int):
        """Allocation intrinsic: FP32-sized slots, initialised to NaN so a
        read before a write shows up."""
        return self.mem.new([float("nan")] * (int(nbytes) // 4))


def _instances(dims: tuple):
    if not dims:
        return [()]
    # x fastest, matching the linear id x + numX * y of Section 6.1
    return [tuple(reversed(t)) for t in itertools.product(*[range(d) for d in reversed(dims)])]


def _run_node(rt: Runtime, node: Node, inst: _Instance, args: list) -> tuple:
    """Run one dynamic instance of ``node`` with its input values."""
    if node.is_internal:
        # the node function builds its child graph (graph intrinsics only)
        node.children, node.edges, node.in_binds, node.out_binds = [], [], [], []
        saved = rt._building
        rt._building = node
        try:
            node.func(rt, *args)
        finally:
            rt._building = saved
        return _run_child_graph(rt, node, inst, args)
    raise DFGError("leaf instances are run by _run_leaf")


def _topo(children: list, edges: list) -> list:
    order, seen, temp = [], set(), set()

    def visit(n):
        if id(n) in seen:
            return
        if id(n) in temp:
            raise DFGError("cycle among ordinary edges")
        temp.add(id(n))
        for e in edges:
            if e.src is n:
                visit(e.dst)
        temp.discard(id(n))
        seen.add(id(n))
        order.append(n)

    for n in children:
        visit(n)
    return list(reversed(order))


def _run_child_graph(rt: Runtime, parent: Node, pinst: _Instance, pargs: list) -> tuple:
    outs: dict[int, dict] = {}  # id(node) -> {instance idx: outputs tuple}
    results: dict[int, Any] = {}
    for child in _topo(parent.children, parent.edges):
        bound = {ic: pargs[ip] for (c, ip, ic, _s) in parent.in_binds if c is child}
        in_edges = [e for e in parent.edges if e.dst is child]
        per_inst_args = {}
        for idx in _instances(child.dims):
            a = [None] * child.n_in
            for ic, v in bound.items():
                a[ic] = v
            for e in in_edges:
                src_outs = outs[id(e.src)]
                if e.all_to_all:
                    # every source instance feeds every sink instance; the
                    # value carried must be the same from all of them (a
                    # shared buffer, or a single-instance source)
                    vals = [o[e.sp] for o in src_outs.values()]
                    if any(v != vals[0] for v in vals[1:]):
                        raise DFGError("all-to-all edge carries different values from different instances")
                    a[e.dp] = vals[0]
                else:
                    a[e.dp] = src_outs[idx][e.sp]
            if any(v is None for v in a):
                missing = [i for i, v in enumerate(a) if v is None]
                raise DFGError(f"{child.func.__name__}: unbound inputs {missing}")
            per_inst_args[idx] = a
        if child.is_internal:
            outs[id(child)] = {}
            for idx, a in per_inst_args.items():
                ci = _Instance(child, idx, pinst)
                outs[id(child)][idx] = _run_node(rt, child, ci, a) or ()
        else:
            outs[id(child)] = _run_leaf(rt, child, pinst, per_inst_args)
        results[id(child)] = outs[id(child)]
    # bind.output: child output oc -> parent output op (single-instance child)
    out_vals = {}
    for (c, oc, op, _s) in parent.out_binds:
        vals = list(outs[id(c)].values())
        out_vals[op] = vals[0][oc]
    return tuple(out_vals[k] for k in sorted(out_vals))


def _run_leaf(rt: Runtime, node: Node, pinst: _Instance, per_inst_args: dict) -> dict:
    """Run all instances of a leaf under one parent instance, phase by phase."""
    gens, done = {}, {}
    for idx, a in per_inst_args.items():
        inst = _Instance(node, idx, pinst)
        rt._cur = inst
        r = node.func(rt, *a)
        if hasattr(r, "__next__"):
            gens[idx] = (inst, r)
        else:
            done[idx] = tuple(r) if r is not None else ()
    phase = 0
    while gens:
        finished, waiting = [], []
        for idx, (inst, g) in gens.items():
            rt._cur = inst
            try:
                next(g)
                waiting.append(idx)
            except StopIteration as stop:
                done[idx] = tuple(stop.value) if stop.value is not None else ()
                finished.append(idx)
        if finished and waiting:
            raise DFGError(f"barrier mismatch in phase {phase}: some instances "
                           "finished while others wait at a barrier")
        for idx in finished:
            del gens[idx]
        phase += 1
    rt._cur = None
    return done


def launch(rt: Runtime, root_func, args: list) -> tuple:
    """llvm.hpvm.launch + wait: run the graph of a root function (one instance)."""
    if not getattr(root_func, "hpvm_internal", False):
        raise DFGError("the root must be an internal node function")
    root = Node(root_func, (), None, root_func.hpvm_n_in)
    if len(args) != root.n_in:
        raise DFGError("argument count does not match the root function")
    return _run_node(rt, root, _Instance(root, (), None), list(args))


# ---------------------------------------------------------------------------
# The sgemm example (Section 6.1), in this interpreter.
#
# Input ports of the leaf: 0 A, 1 bytesA, 2 lda, 3 B, 4 bytesB, 5 ldb, 6 C,
# 7 bytesC, 8 ldc, 9 k, 10 alpha, 11 beta, 12 shB, 13 bytesShB (as in the
# example), then 14 shA, 15 bytesShA (the A tile of the small workload's
# Allocation), 16 M, 17 N, 18 transA, 19 transB (explicit where the example
# leaves them implicit).
# Internal node: 0..11 as the leaf, 12 block_x, 13 block_y, 14 M, 15 N,
# 16 transA, 17 transB. Root: 0..11, 12 block_x, 13 block_y, 14 grid_x,
# 15 grid_y, 16 M, 17 N, 18 transA, 19 transB.
# ---------------------------------------------------------------------------

def _op(mem, X, ld, trans, r, c):
    return mem.load(X, c + r * ld) if trans else mem.load(X, r + c * ld)


def make_sgemm_graph():
    """The node functions of the sgemm example. The Allocation node returns
    the example's B tile (outputs 0, 1 -> leaf ports 12, 13) and, as the small
    workload asks, an A tile of the same size (outputs 2, 3 -> ports 14, 15)."""

    @leaf(2)
    def Allocation(rt, block_x, block_y):
        nbytes = block_x * block_y * 4  # bytes of one block_x x block_y FP32 tile
        shB = rt.malloc(nbytes)
        shA = rt.malloc(nbytes)
        return (shB, nbytes, shA, nbytes)

    @leaf(20)
    def SgemmLeaf(rt, A, bytesA, lda, B, bytesB, ldb, C, bytesC, ldc, k,
                  alpha, beta, shB, bytesShB, shA, bytesShA, M, N, transA,
                  transB):
        mem = rt.mem
        me = rt.getNode()
        par = rt.getParentNode(me)
        tx, ty = rt.getNodeInstanceID(me, 0), rt.getNodeInstanceID(me, 1)
        bx, by = rt.getNodeInstanceID(par, 0), rt.getNodeInstanceID(par, 1)
        nx, ny = rt.getNumNodeInstances(me, 0), rt.getNumNodeInstances(me, 1)
        if nx != ny:
            raise DFGError("the tiled leaf needs a square instance grid")
        ts = nx  # K extent of one staged tile
        i, j = bx * nx + tx, by * ny + ty
        acc = 0.0
        for t in range((k + ts - 1) // ts):
            # phase 1: this instance stages one element of each tile
            pa = t * ts + ty
            a_val = _op(mem, A, lda, transA, i, pa) if (i < M and pa < k) else 0.0
            pb = t * ts + tx
            b_val = _op(mem, B, ldb, transB, pb, j) if (pb < k and j < N) else 0.0
            mem.store(shA, tx + ty * ts, a_val)  # shA[tx, q=ty] = opA(i, t*ts+ty)
            mem.store(shB, tx + ty * ts, b_val)  # shB[q=tx, ty] = opB(t*ts+tx, j)
            yield  # barrier()
            # phase 2: multiply-accumulate over the staged K slice
            for q in range(ts):
                acc += mem.load(shA, tx + q * ts) * mem.load(shB, q + ty * ts)
            yield  # barrier()
        if i < M and j < N:
            r = alpha * acc
            if beta != 0.0:
                r += beta * mem.load(C, i + j * ldc)
            mem.store(C, i + j * ldc, r)
        # outputs 0, 1: the result matrix, for a dependent elementwise leaf
        return (C, bytesC)

    @internal(18)
    def SgemmInternal(rt, A, bytesA, lda, B, bytesB, ldb, C, bytesC, ldc, k,
                      alpha, beta, block_x, block_y, M, N, transA, transB):
        alloc = rt.createNode(Allocation)
        sg = rt.createNode2D(SgemmLeaf, block_x, block_y)
        rt.createEdge(alloc, sg, True, 0, 12, False)
        rt.createEdge(alloc, sg, True, 1, 13, False)
        rt.createEdge(alloc, sg, True, 2, 14, False)
        rt.createEdge(alloc, sg, True, 3, 15, False)
        for p in range(12):
            rt.bind_input(sg, p, p, False)
        rt.bind_input(alloc, 12, 0, False)
        rt.bind_input(alloc, 13, 1, False)
        for p in range(4):
            rt.bind_input(sg, 14 + p, 16 + p, False)

    @internal(20)
    def SgemmRoot(rt, A, bytesA, lda, B, bytesB, ldb, C, bytesC, ldc, k,
                  alpha, beta, block_x, block_y, grid_x, grid_y, M, N, transA,
                  transB):
        inner = rt.createNode2D(SgemmInternal, grid_x, grid_y)
        for p in range(14):
            rt.bind_input(inner, p, p, False)
        for p in range(4):
            rt.bind_input(inner, 16 + p, 14 + p, False)

    return SgemmRoot, SgemmInternal, Allocation, SgemmLeaf


def run_sgemm_dfg(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, transA, transB,
                  block, grid=None, return_runtime=False):
    """Run the sgemm DFG on plain Python/numpy inputs (flat column-major
    sequences). Returns the resulting C as a flat FP64 list (and the runtime
    when asked, for structural checks)."""
    if grid is None:
        grid = (max(1, -(-M // block)), max(1, -(-N // block)))
    mem = Memory()
    pA = mem.new(float(x) for x in A)
    pB = mem.new(float(x) for x in B)
    pC = mem.new(float(x) for x in C)
    root, *_ = make_sgemm_graph()
    rt = Runtime(mem)
    args = [pA, len(A) * 4, lda, pB, len(B) * 4, ldb, pC, len(C) * 4, ldc, K,
            float(alpha), float(beta), block, block, grid[0], grid[1],
            M, N, bool(transA), bool(transB)]
    launch(rt, root, args)
    out = list(mem.objs[pC[0]])
    return (out, rt) if return_runtime else out


# ---------------------------------------------------------------------------
# Elementwise leaves and the streamed chain.
#
# A chain of sgemm stages joined by elementwise tanh leaves, with items fed
# through streaming edges (Section 2.1 streaming edges; Section 3.5: a
# streaming graph's nodes stay alive and process every item pushed).
# Row-major items X (rows x w_in) and weights W (w_in x w_out) are stored so
# that the column-major sgemm leaf computes Y^T = W^T X^T: M = w_out,
# N = rows, K = w_in, op(A) = the W buffer read as a column-major
# w_out x w_in matrix, op(B) = the X buffer read as a column-major w_in x rows
# matrix. The output buffer, read row-major, is Y = X W.
# ---------------------------------------------------------------------------

@leaf(5)
def TanhLeaf(rt, X, bytesX, ldx, M, N):
    """Instance (tx, ty) of tile (bx, by) applies tanh to element
    (bx*nx + tx, by*ny + ty) of the column-major M x N matrix X."""
    me = rt.getNode()
    par = rt.getParentNode(me)
    nx, ny = rt.getNumNodeInstances(me, 0), rt.getNumNodeInstances(me, 1)
    i = rt.getNodeInstanceID(par, 0) * nx + rt.getNodeInstanceID(me, 0)
    j = rt.getNodeInstanceID(par, 1) * ny + rt.getNodeInstanceID(me, 1)
    if i < M and j < N:
        rt.mem.store(X, i + j * ldx, math.tanh(rt.mem.load(X, i + j * ldx)))
    return (X, bytesX)


def make_chain_graph(layers: int):
    """Node functions of the chain. Stage input ports: 0..19 as the sgemm
    internal node's record (A = W_l, B = X_l, C = Y_l, ...), except that B of
    stages after the first arrives over a streaming edge from the previous
    stage's output 0; ports 20, 21 select tanh (1) or not (0)."""
    _, _, Allocation, SgemmLeaf = make_sgemm_graph()

    def stage_func(with_tanh: bool):
        @internal(20)
        def ChainStage(rt, A, bytesA, lda, B, bytesB, ldb, C, bytesC, ldc, k, alpha, beta,
                       block_x, block_y, M, N, transA, transB, _r0, _r1):
            alloc = rt.createNode(Allocation)
            sg = rt.createNode2D(SgemmLeaf, block_x, block_y)
            for sp, dp in ((0, 12), (1, 13), (2, 14), (3, 15)):
                rt.createEdge(alloc, sg, True, sp, dp, False)
            for p in range(12):
                rt.bind_input(sg, p, p, False)
            rt.bind_input(alloc, 12, 0, False)
            rt.bind_input(alloc, 13, 1, False)
            for q in range(4):
                rt.bind_input(sg, 14 + q, 16 + q, False)
            last = sg
            if with_tanh:
                th = rt.createNode2D(TanhLeaf, block_x, block_y)
                rt.createEdge(sg, th, False, 0, 0, False)  # one-to-one: same grid
                rt.createEdge(sg, th, False, 1, 1, False)
                rt.bind_input(th, 8, 2, False)   # ldc
                rt.bind_input(th, 14, 3, False)  # M
                rt.bind_input(th, 15, 4, False)  # N
                last = th
            rt.bind_output(last, 0, 0, False)
            rt.bind_output(last, 1, 1, False)
        return ChainStage

    stages = [stage_func(l + 1 < layers) for l in range(layers)]
    per = 22  # root ports per stage: the 20 stage inputs + grid_x, grid_y

    @internal(per * layers)
    def ChainRoot(rt, *a):
        nodes = []
        for l in range(layers):
            base = per * l
            node = rt.createNode2D(stages[l], a[base + 20], a[base + 21])
            for p in range(20):
                if l > 0 and p in (3, 4):
                    continue  # B and bytesB come from the previous stage
                rt.bind_input(node, base + p, p, False)
            if l > 0:
                rt.createEdge(nodes[-1], node, True, 0, 3, True)  # streaming
                rt.createEdge(nodes[-1], node, True, 1, 4, True)
            nodes.append(node)
        rt.bind_output(nodes[-1], 0, 0, True)

    return ChainRoot


class StreamingGraph:
    """launch(F, args, Stream=true) / push / pop of Table 1: every pushed
    argument record is one item that flows through the graph; pop returns
    the outputs of the items in the order they were pushed."""

    def __init__(self, rt: Runtime, root_func):
        self.rt = rt
        self.root_func = root_func
        self.queue: list = []

    def push(self, args: list) -> None:
        self.queue.append(launch(self.rt, self.root_func, args))

    def pop(self):
        if not self.queue:
            raise DFGError("pop on an empty stream")
        return self.queue.pop(0)


def run_chain(items, Ws, block: int = 4):
    """Push row-major FP64 items (each rows x w) through the chain of
    weights Ws (w x w each) and pop the outputs, as row-major arrays."""
    import numpy as np

    layers = len(Ws)
    root = make_chain_graph(layers)
    mem = Memory()
    rt = Runtime(mem)
    g = StreamingGraph(rt, root)
    w = Ws[0].shape[0]
    wptr = [mem.new(np.asarray(Wl, np.float64).reshape(-1).tolist()) for Wl in Ws]
    outs = []
    for X in items:
        rows = X.shape[0]
        xp = mem.new(np.asarray(X, np.float64).reshape(-1).tolist())
        bufs = [mem.new([0.0] * (rows * w)) for _ in range(layers)]
        args = []
        for l in range(layers):
            # Y_l^T = W_l^T X_l^T: M = w, N = rows, K = w, A = W_l (lda = w), B = X_l (ldb = w)
            args += [wptr[l], w * w * 8, w, xp if l == 0 else None, rows * w * 8, w,
                     bufs[l], rows * w * 8, w, w, 1.0, 0.0, block, block, w, rows, False, False,
                     0, 0, -(-w // block), -(-rows // block)]
        g.push(args)
        outs.append((bufs[-1], rows))
    results = []
    for buf, rows in outs:
        C = g.pop()[0]
        assert C == buf
        results.append(np.array(mem.objs[buf[0]]).reshape(rows, w))
    return results
