"""The C-ABI on the host (no GPU): library load and exports, record layout,
graph building with the intrinsic calls, validation rules and the errors of
the launch path that are found before any device work."""
import ctypes
import os

import pytest

from paper_1611_00860_gb300 import _lib as H
from paper_1611_00860_gb300.sgemm import build_sgemm_graph, make_args

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sgemm_dfg_listing.txt")


@pytest.fixture()
def ctx():
    c = H.hpvm_init(-1)  # host-only context
    yield c
    H.hpvm_cleanup(c)


def test_library_exports_every_declared_function():
    names = H.declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(H.LIB, n), n
        assert hasattr(H, n), f"no Python binding named {n}"
    assert H.hpvm_version() >= 100


def test_root_record_layout_matches_listing():
    rec = [l.split() for l in open(GOLDEN) if l.startswith("RootIn")]
    fields = [f.split(":")[0] for f in rec[0][2:]]
    size = int(rec[1][2])
    assert [f for f, _ in H.RootArgs._fields_][:16] == fields
    assert H.RootArgs.__dict__["grid_y"].offset + 4 == size == H.HPVM_ROOTIN_PAPER_BYTES
    assert ctypes.sizeof(H.RootArgs) == H.HPVM_SGEMM_ROOT_ARGS_BYTES


def test_sgemm_graph_builds_and_validates(ctx):
    nodes = build_sgemm_graph(ctx)
    H.hpvm_validate(nodes["root"])
    assert H.hpvm_get_parent_node(nodes["leaf"]) == nodes["internal"]
    assert H.hpvm_get_parent_node(nodes["internal"]) == nodes["root"]
    assert H.hpvm_get_parent_node(nodes["root"]) is None
    assert H.hpvm_get_num_dims(nodes["leaf"]) == 2
    assert H.hpvm_get_num_dims(nodes["allocation"]) == 0
    assert H.hpvm_get_num_node_instances(nodes["internal"], 0) == H.HPVM_DIM_FROM_INPUT(14)
    assert H.hpvm_get_num_node_instances(nodes["allocation"], 1) == 1


def test_launch_on_host_context_reaches_the_device_check(ctx):
    nodes = build_sgemm_graph(ctx)
    a = make_args(128, 96, 160, 0x1000, 4 * 128 * 160, 128, 0x2000, 4 * 96 * 160, 96,
                  0x3000, 4 * 128 * 96, 128, 1.5, 0.5, False, True, H.HPVM_TIER_FP32_DFG,
                  block=(16, 16), grid=(8, 6))
    with pytest.raises(H.HpvmError) as e:
        H.hpvm_launch(ctx, nodes["root"], a)
    assert e.value.code == H.HPVM_ERR_NO_DEVICE


@pytest.mark.parametrize("change,code", [
    (dict(lda=100), H.HPVM_ERR_SHAPE),                  # lda < M
    (dict(bytesB=100), H.HPVM_ERR_SHAPE),               # B buffer too small
    (dict(grid_x=7), H.HPVM_ERR_SHAPE),                 # grid does not cover M
    (dict(block_y=8, grid_y=12), H.HPVM_ERR_UNSUPPORTED),  # non-square literal leaf
    (dict(block_x=64, block_y=64, grid_x=2, grid_y=2), H.HPVM_ERR_UNSUPPORTED),  # > 1024 threads
    (dict(tier=9), H.HPVM_ERR_INVALID_ARG),
    (dict(M=-1), H.HPVM_ERR_SHAPE),
])
def test_launch_rejects_bad_records(ctx, change, code):
    nodes = build_sgemm_graph(ctx)
    a = make_args(128, 96, 160, 0x1000, 4 * 128 * 160, 128, 0x2000, 4 * 96 * 160, 96,
                  0x3000, 4 * 128 * 96, 128, 1.5, 0.5, False, True, H.HPVM_TIER_FP32_DFG,
                  block=(16, 16), grid=(8, 6))
    for k, v in change.items():
        setattr(a, k, v)
    with pytest.raises(H.HpvmError) as e:
        H.hpvm_launch(ctx, nodes["root"], a)
    assert e.value.code == code


def test_workspace_size_on_host(ctx):
    nodes = build_sgemm_graph(ctx)
    a = make_args(300, 200, 100, 0x1000, 4 * 300 * 100, 300, 0x2000, 4 * 200 * 100, 200,
                  0x3000, 4 * 300 * 200, 300, 1.0, 0.0, False, True, H.HPVM_TIER_BF16X3)
    kp = 104  # K rounded up to a multiple of 8
    def al(x):
        return (x + 255) // 256 * 256
    # BF16x3: hi and lo planes of both operands, then one flag per 128-row
    # block and 64-element slab of each operand and a counter (the leaf's
    # own conversion of its operands)
    blocks = -(-300 // 128) + -(-200 // 128)
    flags = blocks * 4 + blocks + 1  # 2 slabs, a block's flags padded to 4
    assert H.hpvm_workspace_size(ctx, nodes["root"], a) == 2 * (al(300 * kp * 2) + al(200 * kp * 2)) + al(4 * flags)
    a.tier = H.HPVM_TIER_BF16
    assert H.hpvm_workspace_size(ctx, nodes["root"], a) == al(300 * kp * 2) + al(200 * kp * 2)
    a.tier = H.HPVM_TIER_FP32
    assert H.hpvm_workspace_size(ctx, nodes["root"], a) == 0


def test_plan():
    assert H.hpvm_plan_sgemm(H.HPVM_TIER_FP32_DFG, 128, 96, 160) == (16, 16, 8, 6)
    bx, by, gx, gy = H.hpvm_plan_sgemm(H.HPVM_TIER_BF16X3, 8192, 8192, 8192)
    assert bx * gx >= 8192 and by * gy >= 8192
    assert H.hpvm_plan_sgemm(H.HPVM_TIER_FP32, 0, 0, 0)[2:] == (1, 1)


# ---- graph rules (Sections 2.1-2.2) ------------------------------------------

def test_root_must_be_single_internal(ctx):
    with pytest.raises(H.HpvmError) as e:
        H.hpvm_create_node(ctx, None, H.HPVM_NODE_INTERNAL, (4,))
    assert e.value.code == H.HPVM_ERR_INVALID_GRAPH
    with pytest.raises(H.HpvmError):
        H.hpvm_create_node(ctx, None, H.HPVM_NODE_SGEMM_LEAF)


def test_leaf_cannot_hold_children(ctx):
    root = H.hpvm_create_node(ctx, None, H.HPVM_NODE_INTERNAL)
    leaf = H.hpvm_create_node(ctx, root, H.HPVM_NODE_SGEMM_LEAF, (2, 2))
    with pytest.raises(H.HpvmError) as e:
        H.hpvm_create_node(ctx, leaf, H.HPVM_NODE_ALLOCATION)
    assert e.value.code == H.HPVM_ERR_INVALID_GRAPH


def test_one_to_one_needs_identical_grids(ctx):
    root = H.hpvm_create_node(ctx, None, H.HPVM_NODE_INTERNAL)
    a = H.hpvm_create_node(ctx, root, H.HPVM_NODE_ALLOCATION)
    l1 = H.hpvm_create_node(ctx, root, H.HPVM_NODE_SGEMM_LEAF, (4, 4))
    with pytest.raises(H.HpvmError) as e:
        H.hpvm_create_edge(a, l1, H.HPVM_ONE_TO_ONE, 0, 12)
    assert e.value.code == H.HPVM_ERR_INVALID_GRAPH
    H.hpvm_create_edge(a, l1, H.HPVM_ALL_TO_ALL, 0, 12)  # all-to-all is fine


def test_ports_and_flags_checked(ctx):
    root = H.hpvm_create_node(ctx, None, H.HPVM_NODE_INTERNAL)
    a = H.hpvm_create_node(ctx, root, H.HPVM_NODE_ALLOCATION)
    l1 = H.hpvm_create_node(ctx, root, H.HPVM_NODE_SGEMM_LEAF, (2, 2))
    for bad in [(a, l1, 1, 4, 12), (a, l1, 1, 0, 20), (a, l1, 2, 0, 12), (l1, a, 1, 2, 0)]:
        with pytest.raises(H.HpvmError) as e:
            H.hpvm_create_edge(*bad)
        assert e.value.code == H.HPVM_ERR_INVALID_ARG
    with pytest.raises(H.HpvmError):
        H.hpvm_bind_input(l1, 23 * 16, 0)  # the root has 16 records of 23 ports
    with pytest.raises(H.HpvmError):
        H.hpvm_bind_input(root, 0, 0)  # the root has no parent
    with pytest.raises(H.HpvmError):
        H.hpvm_create_node(ctx, root, H.HPVM_NODE_SGEMM_LEAF, (H.HPVM_DIM_FROM_INPUT(23 * 16), 2))


def test_streaming_edge_inside_a_tile_is_not_lowered(ctx):
    nodes = build_sgemm_graph(ctx)
    # a second, streaming Allocation -> leaf edge would feed port 12 twice;
    # build a fresh tile node whose Allocation edge is streaming instead
    root = H.hpvm_create_node(ctx, None, H.HPVM_NODE_INTERNAL)
    inner = H.hpvm_create_node(ctx, root, H.HPVM_NODE_INTERNAL,
                               (H.HPVM_DIM_FROM_INPUT(14), H.HPVM_DIM_FROM_INPUT(15)))
    for p in range(20):
        H.hpvm_bind_input(inner, p, p)
    alloc = H.hpvm_create_node(ctx, inner, H.HPVM_NODE_ALLOCATION)
    leaf = H.hpvm_create_node(ctx, inner, H.HPVM_NODE_SGEMM_LEAF,
                              (H.HPVM_DIM_FROM_INPUT(12), H.HPVM_DIM_FROM_INPUT(13)))
    for sp, dp in ((0, 12), (1, 13), (2, 14), (3, 15)):
        H.hpvm_create_edge(alloc, leaf, H.HPVM_ALL_TO_ALL, sp, dp, stream=(sp == 0))
    for p in range(12):
        H.hpvm_bind_input(leaf, p, p)
    for q in range(4):
        H.hpvm_bind_input(leaf, 16 + q, 16 + q)
    H.hpvm_bind_input(alloc, 12, 0)
    H.hpvm_bind_input(alloc, 13, 1)
    H.hpvm_validate(root)
    a = make_args(128, 96, 160, 0x1000, 4 * 128 * 160, 128, 0x2000, 4 * 96 * 160, 96,
                  0x3000, 4 * 128 * 96, 128, 1.5, 0.5, False, True, H.HPVM_TIER_BF16X3)
    with pytest.raises(H.HpvmError) as e:
        H.hpvm_workspace_size(ctx, root, a)
    assert e.value.code == H.HPVM_ERR_UNSUPPORTED
    del nodes


def test_unfed_and_twice_fed_inputs(ctx):
    nodes = build_sgemm_graph(ctx)
    H.hpvm_bind_input(nodes["leaf"], 0, 0)  # input 0 now fed twice
    with pytest.raises(H.HpvmError) as e:
        H.hpvm_validate(nodes["root"])
    assert e.value.code == H.HPVM_ERR_INVALID_GRAPH and "fed 2 times" in str(e.value)

    root = H.hpvm_create_node(ctx, None, H.HPVM_NODE_INTERNAL)
    H.hpvm_create_node(ctx, root, H.HPVM_NODE_SGEMM_LEAF, (2, 2))
    with pytest.raises(H.HpvmError) as e:
        H.hpvm_validate(root)
    assert "not fed" in str(e.value)


def test_cycle_rejected(ctx):
    root = H.hpvm_create_node(ctx, None, H.HPVM_NODE_INTERNAL)
    a = H.hpvm_create_node(ctx, root, H.HPVM_NODE_INTERNAL)
    b = H.hpvm_create_node(ctx, root, H.HPVM_NODE_INTERNAL)
    H.hpvm_create_edge(a, b, H.HPVM_ONE_TO_ONE, 0, 0)
    H.hpvm_create_edge(b, a, H.HPVM_ONE_TO_ONE, 0, 0)
    with pytest.raises(H.HpvmError) as e:
        H.hpvm_validate(root)
    assert "cycle" in str(e.value)


def test_unsupported_shapes_named(ctx):
    # a valid graph that is not the sgemm shape: root -> leaf directly
    root = H.hpvm_create_node(ctx, None, H.HPVM_NODE_INTERNAL)
    alloc = H.hpvm_create_node(ctx, root, H.HPVM_NODE_ALLOCATION)
    H.hpvm_bind_input(alloc, 12, 0)
    H.hpvm_bind_input(alloc, 13, 1)
    a = make_args(4, 4, 4, 0x1000, 64, 4, 0x2000, 64, 4, 0x3000, 64, 4, 1, 0, False, True,
                  H.HPVM_TIER_FP32)
    with pytest.raises(H.HpvmError) as e:
        H.hpvm_launch(ctx, root, a)
    assert e.value.code == H.HPVM_ERR_UNSUPPORTED


def test_rewired_ports_resolve_by_meaning(ctx):
    # the same graph with the internal node's ports permuted still lowers:
    # values are found by following bindings up to the root record
    root = H.hpvm_create_node(ctx, None, H.HPVM_NODE_INTERNAL)
    inner = H.hpvm_create_node(ctx, root, H.HPVM_NODE_INTERNAL,
                               (H.HPVM_DIM_FROM_INPUT(14), H.HPVM_DIM_FROM_INPUT(15)))
    perm = {p: 30 + p for p in range(20)}  # root field p -> internal port 30 + p
    for p in range(20):
        H.hpvm_bind_input(inner, p, perm[p])
    alloc = H.hpvm_create_node(ctx, inner, H.HPVM_NODE_ALLOCATION)
    leaf = H.hpvm_create_node(ctx, inner, H.HPVM_NODE_SGEMM_LEAF,
                              (H.HPVM_DIM_FROM_INPUT(perm[12]), H.HPVM_DIM_FROM_INPUT(perm[13])))
    for sp, dp in ((0, 12), (1, 13), (2, 14), (3, 15)):
        H.hpvm_create_edge(alloc, leaf, H.HPVM_ALL_TO_ALL, sp, dp)
    for p in range(12):
        H.hpvm_bind_input(leaf, perm[p], p)
    for q in range(4):
        H.hpvm_bind_input(leaf, perm[16 + q], 16 + q)
    H.hpvm_bind_input(alloc, perm[12], 0)
    H.hpvm_bind_input(alloc, perm[13], 1)
    H.hpvm_validate(root)
    a = make_args(128, 96, 160, 0x1000, 4 * 128 * 160, 128, 0x2000, 4 * 96 * 160, 96,
                  0x3000, 4 * 128 * 96, 128, 1.5, 0.5, False, True, H.HPVM_TIER_BF16X3)
    assert H.hpvm_workspace_size(ctx, root, a) > 0


def test_type_mismatch_is_an_invalid_graph(ctx):
    # the leaf's lda (i32, port 2) fed from the root's pointer field B (port 3)
    root = H.hpvm_create_node(ctx, None, H.HPVM_NODE_INTERNAL)
    inner = H.hpvm_create_node(ctx, root, H.HPVM_NODE_INTERNAL,
                               (H.HPVM_DIM_FROM_INPUT(14), H.HPVM_DIM_FROM_INPUT(15)))
    for p in range(20):
        H.hpvm_bind_input(inner, p, p)
    alloc = H.hpvm_create_node(ctx, inner, H.HPVM_NODE_ALLOCATION)
    leaf = H.hpvm_create_node(ctx, inner, H.HPVM_NODE_SGEMM_LEAF,
                              (H.HPVM_DIM_FROM_INPUT(12), H.HPVM_DIM_FROM_INPUT(13)))
    for sp, dp in ((0, 12), (1, 13), (2, 14), (3, 15)):
        H.hpvm_create_edge(alloc, leaf, H.HPVM_ALL_TO_ALL, sp, dp)
    for p in range(12):
        H.hpvm_bind_input(leaf, 3 if p == 2 else p, p)
    for q in range(4):
        H.hpvm_bind_input(leaf, 16 + q, 16 + q)
    H.hpvm_bind_input(alloc, 12, 0)
    H.hpvm_bind_input(alloc, 13, 1)
    a = make_args(128, 96, 160, 0x1000, 4 * 128 * 160, 128, 0x2000, 4 * 96 * 160, 96,
                  0x3000, 4 * 128 * 96, 128, 1.5, 0.5, False, True, H.HPVM_TIER_BF16X3)
    with pytest.raises(H.HpvmError) as e:
        H.hpvm_workspace_size(ctx, root, a)
    assert e.value.code == H.HPVM_ERR_INVALID_GRAPH


def test_tracker_host_side(ctx):
    buf = (ctypes.c_float * 16)()
    p = ctypes.addressof(buf)
    H.hpvm_track_mem(ctx, p, 64)
    H.hpvm_track_mem(ctx, p, 64)  # re-tracking marks the host copy latest again
    with pytest.raises(H.HpvmError):
        H.hpvm_track_mem(ctx, p + 8, 16)  # overlaps
    H.hpvm_request_mem(ctx, p, 64)  # host copy is current: nothing to do
    with pytest.raises(H.HpvmError):
        H.hpvm_request_mem(ctx, p, 128)
    H.hpvm_untrack_mem(ctx, p)
    with pytest.raises(H.HpvmError):
        H.hpvm_untrack_mem(ctx, p)


def test_chain_graph_lowers_on_host(ctx):
    from paper_1611_00860_gb300.chain import build_chain_graph, build_single_stage_graph
    root = build_chain_graph(ctx, 4)
    w, rows = 64, 48
    arr = (H.RootArgs * 4)()
    for l in range(4):
        arr[l] = make_args(w, rows, w, 0x1000, w * w * 4, w, 0 if l else 0x2000, rows * w * 4, w,
                           0x3000 + 0x10000 * l, rows * w * 4, w, 1.0, 0.0, False, False,
                           H.HPVM_TIER_BF16)
    assert H.hpvm_workspace_size(ctx, root, arr) > 0
    # fewer records than stages: stage 3 reads a record that was not passed
    short = (H.RootArgs * 3)(*arr[:3])
    with pytest.raises(H.HpvmError) as e:
        H.hpvm_workspace_size(ctx, root, short)
    assert e.value.code == H.HPVM_ERR_INVALID_ARG
    g = build_single_stage_graph(ctx, H.HPVM_NODE_TANH_GRAD_LEAF)
    a = make_args(w, rows, w, 0x1000, w * w * 4, w, 0x2000, rows * w * 4, w, 0x3000, rows * w * 4, w,
                  1.0, 0.0, True, False, H.HPVM_TIER_BF16)
    with pytest.raises(H.HpvmError) as e:  # the tanh adjoint needs H
        H.hpvm_workspace_size(ctx, g, a)
    assert e.value.code == H.HPVM_ERR_SHAPE
    a.aux, a.bytesAux, a.ldaux = 0x4000, rows * w * 4, w
    assert H.hpvm_workspace_size(ctx, g, a) > 0


def test_workspace_of_a_tail_split(ctx):
    # 10 x 8 = 80 pair tiles, more than the pairs of the GPU (or of the
    # 148-SM default without one), with a short last round: K = 520 (9 slabs
    # of 64) splits it, and the workspace holds, after the planes, per split
    # tile 2 K halves x 2 CTAs x 8 epilogue warps x 128 x 32 FP32 partial
    # sums (512 KiB) and then 2 x 8 counters per tile (aligned to 256 B).
    # With 3 slabs (K = 192), or 2 x 2 tiles, nothing splits.
    nodes = build_sgemm_graph(ctx)

    def al(x):
        return (x + 255) // 256 * 256

    def ws(M, N, K, tier):
        a = make_args(M, N, K, 0x1000, 4 * M * K, M, 0x2000, 4 * N * K, N, 0x3000, 4 * M * N, M,
                      1.0, 0.0, False, True, tier)
        kp = (K + 7) // 8 * 8
        planes = (2 if tier == H.HPVM_TIER_BF16X3 else 1) * (al(M * kp * 2) + al(N * kp * 2))
        if tier == H.HPVM_TIER_BF16X3:  # the in-leaf conversion's flags, counts and counter (last)
            blocks = -(-M // 128) + -(-N // 128)
            planes += al(4 * (blocks * ((-(-K // 64) + 3) // 4 * 4) + blocks + 1))
        return H.hpvm_workspace_size(ctx, nodes["root"], a) - planes

    for tier in (H.HPVM_TIER_BF16X3, H.HPVM_TIER_BF16):
        extra = ws(2560, 2048, 520, tier)
        n = extra // (2 * 2 * 8 * 128 * 32 * 4)
        assert n >= 1 and extra == n * 2 * 2 * 8 * 128 * 32 * 4 + al(n * 2 * 8 * 4)
        assert ws(2560, 2048, 192, tier) == 0
        assert ws(512, 400, 520, tier) == 0
    # the FP32 tiers use no workspace
    assert ws(2560, 2048, 520, H.HPVM_TIER_FP32) == -(al(2560 * 520 * 2) + al(2048 * 520 * 2))


def test_chain_workspace_holds_forwarded_planes(ctx):
    # A 4-stage chain whose stages read the previous stage's result as B:
    # merged, each stage's epilogue writes the next stage's B planes into one
    # of two regions after the largest stage's planes; unmerged
    # (HPVM_LAUNCH_NO_FUSION) every B is converted and the regions are absent.
    from paper_1611_00860_gb300.chain import build_chain_graph
    root = build_chain_graph(ctx, 4)
    w, rows = 64, 48  # each stage: M = K = 64, N = 48

    def al(x):
        return (x + 255) // 256 * 256

    def records(tier, flags):
        arr = (H.RootArgs * 4)()
        for l in range(4):
            arr[l] = make_args(w, rows, w, 0x1000, w * w * 4, w, 0 if l else 0x2000, rows * w * 4, w,
                               0x3000 + 0x10000 * l, rows * w * 4, w, 1.0, 0.0, False, False, tier,
                               flags=flags)
        return arr

    for tier, planes in ((H.HPVM_TIER_BF16, 1), (H.HPVM_TIER_BF16X3, 2)):
        stage = planes * (al(w * w * 2) + al(rows * w * 2))  # A (64 x 64) and B (48 x 64) planes
        if tier == H.HPVM_TIER_BF16X3:  # the in-leaf conversion's flags (padded to 4 a block), counts, counter
            stage += al(4 * ((1 + 1) * 4 + 2 + 1))
        region = planes * al(rows * w * 2)                    # C as the next B: 48 rows of 64
        assert H.hpvm_workspace_size(ctx, root, records(tier, 0)) == al(stage) + 2 * al(region)
        assert H.hpvm_workspace_size(ctx, root, records(tier, H.HPVM_LAUNCH_NO_FUSION)) == stage


def test_push_pop_need_a_streaming_graph(ctx):
    with pytest.raises(H.HpvmError):
        H.hpvm_pop(0)


def test_plane_cache_on_a_host_only_context(ctx):
    # nothing is cached without a device; dropping the empty cache is fine
    assert H.hpvm_plane_cache_bytes(ctx) == 0
    H.hpvm_drop_planes(ctx)
    assert H.hpvm_plane_cache_bytes(ctx) == 0
    flags = (H.HPVM_LAUNCH_CACHE_A, H.HPVM_LAUNCH_REUSE_A, H.HPVM_LAUNCH_CACHE_B, H.HPVM_LAUNCH_REUSE_B,
             H.HPVM_LAUNCH_CACHE_C, H.HPVM_LAUNCH_PLANES_ONLY)
    assert len(set(flags)) == 6 and all(f & (H.HPVM_LAUNCH_NO_EVENT | H.HPVM_LAUNCH_NO_FUSION) == 0 for f in flags)
    with pytest.raises(H.HpvmError):
        H.hpvm_plane_cache_bytes(None)


def test_wait_limit_bounds():
    # 0 (the default) .. 10^7 microseconds; a host-only context keeps it too
    ctx = H.hpvm_init(-1)
    try:
        for bad in (-1, 10 ** 7 + 1):
            with pytest.raises(H.HpvmError) as e:
                H.hpvm_set_wait_limit(ctx, bad)
            assert e.value.code == H.HPVM_ERR_INVALID_ARG
        H.hpvm_set_wait_limit(ctx, 5)
        H.hpvm_set_wait_limit(ctx, 0)
    finally:
        H.hpvm_cleanup(ctx)


def test_workspace_size_bf16x6_on_host(ctx):
    # three planes (hi, mid, lo) of each operand; no in-leaf conversion region
    nodes = build_sgemm_graph(ctx)
    a = make_args(300, 200, 100, 0x1000, 4 * 300 * 100, 300, 0x2000, 4 * 200 * 100, 200,
                  0x3000, 4 * 300 * 200, 300, 1.0, 0.0, False, True, H.HPVM_TIER_BF16X6)
    def al(x):
        return (x + 255) // 256 * 256
    assert H.hpvm_workspace_size(ctx, nodes["root"], a) == 3 * (al(300 * 104 * 2) + al(200 * 104 * 2))


def _code(fn, *args):
    try:
        fn(*args)
    except H.HpvmError as e:
        return e.code
    return H.HPVM_OK


def test_split3_argument_checks():
    # checked before anything reaches the device
    ok = 0x10000
    assert _code(H.hpvm_split3_bf16, ok, 64, True, 0, 64, ok, ok, ok) == H.HPVM_OK  # nothing to do
    assert _code(H.hpvm_split3_bf16, ok, 64, True, -1, 64, ok, ok, ok) == H.HPVM_ERR_SHAPE
    assert _code(H.hpvm_split3_bf16, None, 64, True, 8, 64, ok, ok, ok) == H.HPVM_ERR_INVALID_ARG
    assert _code(H.hpvm_split3_bf16, ok, 64, True, 8, 64, ok, None, ok) == H.HPVM_ERR_INVALID_ARG
    assert _code(H.hpvm_split3_bf16, ok, 32, True, 8, 64, ok, ok, ok) == H.HPVM_ERR_SHAPE  # ld < K
    assert _code(H.hpvm_split3_bf16, ok, 64, True, 8, 64, ok, ok + 8, ok) == H.HPVM_ERR_ALIGN


def test_stream_coalesce_argument_checks():
    assert _code(H.hpvm_stream_coalesce, None, 4) == H.HPVM_ERR_INVALID_ARG
