"""ctypes binding of the C-ABI in ``include/hpvm.h``.

Argument marshalling only: every function here forwards to the function of
the same name in ``_lib/libhpvm_gb300.so`` and raises ``HpvmError`` when it
returns a negative status. There is no other code path: when the library is
missing, importing this module raises ``ImportError`` (call
``paper_1611_00860_gb300.build.build()`` first).
"""
from __future__ import annotations

import ctypes
import functools
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhpvm_gb300.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "hpvm.h")

# ---- constants of include/hpvm.h -------------------------------------------
HPVM_OK = 0
HPVM_ERR_INVALID_ARG = -1
HPVM_ERR_INVALID_GRAPH = -2
HPVM_ERR_UNSUPPORTED = -3
HPVM_ERR_SHAPE = -4
HPVM_ERR_ALIGN = -5
HPVM_ERR_CUDA = -6
HPVM_ERR_TIMEOUT = -7
HPVM_ERR_DEVICE_FAULT = -8
HPVM_ERR_NO_DEVICE = -9
HPVM_ERR_OUT_OF_MEMORY = -10

HPVM_NODE_INTERNAL = 0
HPVM_NODE_ALLOCATION = 1
HPVM_NODE_SGEMM_LEAF = 2
HPVM_NODE_TANH_LEAF = 3
HPVM_NODE_TANH_GRAD_LEAF = 4

HPVM_ONE_TO_ONE = 0
HPVM_ALL_TO_ALL = 1

HPVM_TIER_FP32_DFG = 0
HPVM_TIER_FP32 = 1
HPVM_TIER_BF16X3 = 2
HPVM_TIER_BF16 = 3
HPVM_TIER_FP8 = 4
HPVM_TIER_BF16X6 = 5

HPVM_LAUNCH_NO_EVENT = 1
HPVM_LAUNCH_NO_FUSION = 2
HPVM_LAUNCH_CACHE_A = 4
HPVM_LAUNCH_REUSE_A = 8
HPVM_LAUNCH_CACHE_B = 16
HPVM_LAUNCH_REUSE_B = 32
HPVM_LAUNCH_CACHE_C = 64
HPVM_LAUNCH_PLANES_ONLY = 128
HPVM_LAUNCH_SEPARATE_SPLIT = 256
HPVM_NOALLOC_SCRATCH_BYTES = 64 * 1024 * 1024
HPVM_ROOTIN_PAPER_BYTES = 88
HPVM_SGEMM_ROOT_ARGS_BYTES = 136
HPVM_RECORD_PORTS = 23


def HPVM_DIM_FROM_INPUT(p: int) -> int:
    return -1 - int(p)


class HpvmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hpvm error {code}: {msg}")
        self.code = code


class RootArgs(ctypes.Structure):
    """hpvm_sgemm_root_args: the paper's packed RootIn record + trailer."""
    _pack_ = 1
    _fields_ = [
        ("A", ctypes.c_void_p), ("bytesA", ctypes.c_int64), ("lda", ctypes.c_int32),
        ("B", ctypes.c_void_p), ("bytesB", ctypes.c_int64), ("ldb", ctypes.c_int32),
        ("C", ctypes.c_void_p), ("bytesC", ctypes.c_int64), ("ldc", ctypes.c_int32),
        ("k", ctypes.c_int32), ("alpha", ctypes.c_float), ("beta", ctypes.c_float),
        ("block_x", ctypes.c_int32), ("block_y", ctypes.c_int32),
        ("grid_x", ctypes.c_int32), ("grid_y", ctypes.c_int32),
        ("M", ctypes.c_int32), ("N", ctypes.c_int32),
        ("transA", ctypes.c_int32), ("transB", ctypes.c_int32),
        ("tier", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("aux", ctypes.c_void_p), ("bytesAux", ctypes.c_int64), ("ldaux", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class LaunchInfo(ctypes.Structure):
    _fields_ = [
        ("tier", ctypes.c_int32), ("kernels", ctypes.c_int32),
        ("grid_x", ctypes.c_int32), ("grid_y", ctypes.c_int32), ("grid_z", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("tile_m", ctypes.c_int32), ("tile_n", ctypes.c_int32), ("tile_k", ctypes.c_int32),
        ("smem_bytes", ctypes.c_int32), ("literal", ctypes.c_int32),
        ("workspace_bytes", ctypes.c_int64),
        ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class BatchInfo(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int32), ("tier", ctypes.c_int32), ("policy", ctypes.c_int32),
        ("tiles", ctypes.c_int32), ("split_tiles", ctypes.c_int32), ("grid", ctypes.c_int32),
        ("tile_width_count", ctypes.c_int32 * 3), ("tile_m", ctypes.c_int32),
        ("workspace_bytes", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["tile_width_count"] = list(self.tile_width_count)
        return d


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()'); there is no fallback path")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, I64, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "hpvm_init": (I, [I, PP]),
        "hpvm_cleanup": (I, [P]),
        "hpvm_create_node": (I, [P, P, I, I, ctypes.POINTER(ctypes.c_int64), PP]),
        "hpvm_create_edge": (I, [P, P, I, I, I, I, PP]),
        "hpvm_bind_input": (I, [P, I, I, I]),
        "hpvm_bind_output": (I, [P, I, I, I]),
        "hpvm_get_parent_node": (I, [P, PP]),
        "hpvm_get_num_dims": (I, [P, ctypes.POINTER(ctypes.c_int)]),
        "hpvm_get_num_node_instances": (I, [P, I, ctypes.POINTER(ctypes.c_int64)]),
        "hpvm_validate": (I, [P]),
        "hpvm_launch": (I, [P, P, P, SZ, I, P, PP]),
        "hpvm_wait": (I, [P, I64]),
        "hpvm_push": (I, [P, P, SZ]),
        "hpvm_pop": (I, [P, P, SZ, I64]),
        "hpvm_graph_info": (I, [P, ctypes.POINTER(LaunchInfo)]),
        "hpvm_stream_coalesce": (I, [P, I]),
        "hpvm_track_mem": (I, [P, P, I64]),
        "hpvm_request_mem": (I, [P, P, I64]),
        "hpvm_untrack_mem": (I, [P, P]),
        "hpvm_workspace_size": (I, [P, P, P, SZ, ctypes.POINTER(ctypes.c_size_t)]),
        "hpvm_set_workspace": (I, [P, P, SZ]),
        "hpvm_plane_cache_bytes": (I, [P, ctypes.POINTER(ctypes.c_int64)]),
        "hpvm_drop_planes": (I, [P]),
        "hpvm_plan_sgemm": (I, [I, I64, I64, I64] + [ctypes.POINTER(ctypes.c_int32)] * 4),
        "hpvm_set_kernel_timing": (I, [P, I]),
        "hpvm_kernel_timing": (I, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
        "hpvm_split_bf16": (I, [P, I64, I, I64, I64, P, P, P]),
        "hpvm_split3_bf16": (I, [P, I64, I, I64, I64, P, P, P, P]),
        "hpvm_quant_fp8": (I, [P, I64, I, I64, I64, P, P, P]),
        "hpvm_sgemm_bf16x3_noalloc": (I, [I64, I64, I64, ctypes.c_float, P, I64, P, I64,
                                          ctypes.c_float, P, I64, I, I, P, P]),
        "hpvm_batch_prepare": (I, [P, P, P, SZ, I, I, PP]),
        "hpvm_batch_run": (I, [P, P]),
        "hpvm_batch_autotune": (I, [P, P, I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
        "hpvm_batch_info": (I, [P, ctypes.POINTER(BatchInfo)]),
        "hpvm_batch_free": (I, [P]),
        "hpvm_batch_plan": (I, [I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.c_int64), I, ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_int32), I64, ctypes.POINTER(ctypes.c_int64)]),
        "hpvm_selftest_wait_timeout": (I, [P, I64, P]),
        "hpvm_set_wait_limit": (I, [P, I64]),
        "hpvm_last_error": (ctypes.c_char_p, []),
        "hpvm_version": (I, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


def declared_functions() -> list[str]:
    """Names of the functions include/hpvm.h declares."""
    with open(HEADER_PATH) as f:
        text = f.read()
    return sorted(set(re.findall(r"HPVM_API\s+[\w\s\*]*?\b(hpvm_\w+)\s*\(", text)))


def _check(rc: int) -> None:
    if rc != HPVM_OK:
        raise HpvmError(rc, LIB.hpvm_last_error().decode())


# ---- the C-ABI, one wrapper per function --------------------------------------
def hpvm_init(device: int) -> int:
    out = ctypes.c_void_p()
    _check(LIB.hpvm_init(int(device), ctypes.byref(out)))
    return out.value


def hpvm_cleanup(ctx: int) -> None:
    _check(LIB.hpvm_cleanup(ctx))


def hpvm_create_node(ctx: int, parent: int | None, kind: int, dims=()) -> int:
    nd = len(dims)
    arr = (ctypes.c_int64 * max(nd, 1))(*[int(d) for d in dims]) if nd else None
    out = ctypes.c_void_p()
    _check(LIB.hpvm_create_node(ctx, parent, int(kind), nd, arr, ctypes.byref(out)))
    return out.value


def hpvm_create_edge(src: int, dst: int, repl: int, sp: int, dp: int, stream: bool = False) -> int:
    out = ctypes.c_void_p()
    _check(LIB.hpvm_create_edge(src, dst, int(repl), int(sp), int(dp), int(bool(stream)), ctypes.byref(out)))
    return out.value


def hpvm_bind_input(child: int, ip: int, ic: int, stream: bool = False) -> None:
    _check(LIB.hpvm_bind_input(child, int(ip), int(ic), int(bool(stream))))


def hpvm_bind_output(child: int, oc: int, op: int, stream: bool = False) -> None:
    _check(LIB.hpvm_bind_output(child, int(oc), int(op), int(bool(stream))))


def hpvm_get_parent_node(node: int) -> int | None:
    out = ctypes.c_void_p()
    _check(LIB.hpvm_get_parent_node(node, ctypes.byref(out)))
    return out.value


def hpvm_get_num_dims(node: int) -> int:
    out = ctypes.c_int()
    _check(LIB.hpvm_get_num_dims(node, ctypes.byref(out)))
    return out.value


def hpvm_get_num_node_instances(node: int, dim: int) -> int:
    out = ctypes.c_int64()
    _check(LIB.hpvm_get_num_node_instances(node, int(dim), ctypes.byref(out)))
    return out.value


def hpvm_validate(root: int) -> None:
    _check(LIB.hpvm_validate(root))


def hpvm_launch(ctx: int, root: int, args, stream_graph: bool = False,
                cuda_stream: int = 0) -> int:
    """``args``: one RootArgs or a ctypes array of them (one per stage)."""
    out = ctypes.c_void_p()
    _check(LIB.hpvm_launch(ctx, root, ctypes.byref(args), ctypes.sizeof(args),
                           int(bool(stream_graph)), cuda_stream or None, ctypes.byref(out)))
    return out.value


def hpvm_push(graph: int, args) -> None:
    _check(LIB.hpvm_push(graph, ctypes.byref(args), ctypes.sizeof(args)))


def hpvm_pop(graph: int, out=None, timeout_ms: int = -1) -> None:
    """Pop the oldest item; ``out`` (RootArgs or array) receives its records."""
    if out is None:
        _check(LIB.hpvm_pop(graph, None, 0, int(timeout_ms)))
    else:
        _check(LIB.hpvm_pop(graph, ctypes.byref(out), ctypes.sizeof(out), int(timeout_ms)))


def hpvm_wait(graph: int, timeout_ms: int = -1) -> None:
    _check(LIB.hpvm_wait(graph, int(timeout_ms)))


def hpvm_stream_coalesce(graph: int, items: int) -> None:
    _check(LIB.hpvm_stream_coalesce(graph, int(items)))


def hpvm_graph_info(graph: int) -> LaunchInfo:
    info = LaunchInfo()
    _check(LIB.hpvm_graph_info(graph, ctypes.byref(info)))
    return info


def hpvm_track_mem(ctx: int, ptr: int, nbytes: int) -> None:
    _check(LIB.hpvm_track_mem(ctx, ptr, int(nbytes)))


def hpvm_request_mem(ctx: int, ptr: int, nbytes: int) -> None:
    _check(LIB.hpvm_request_mem(ctx, ptr, int(nbytes)))


def hpvm_untrack_mem(ctx: int, ptr: int) -> None:
    _check(LIB.hpvm_untrack_mem(ctx, ptr))


def hpvm_workspace_size(ctx: int, root: int, args) -> int:
    out = ctypes.c_size_t()
    _check(LIB.hpvm_workspace_size(ctx, root, ctypes.byref(args), ctypes.sizeof(args), ctypes.byref(out)))
    return out.value


def hpvm_set_workspace(ctx: int, ptr: int | None, nbytes: int) -> None:
    _check(LIB.hpvm_set_workspace(ctx, ptr, int(nbytes)))


def hpvm_plane_cache_bytes(ctx: int) -> int:
    v = ctypes.c_int64()
    _check(LIB.hpvm_plane_cache_bytes(ctx, ctypes.byref(v)))
    return v.value


def hpvm_drop_planes(ctx: int) -> None:
    _check(LIB.hpvm_drop_planes(ctx))


@functools.lru_cache(maxsize=4096)
def hpvm_plan_sgemm(tier: int, M: int, N: int, K: int) -> tuple[int, int, int, int]:
    # a pure function of its arguments: memoised (records are packed per item)
    v = [ctypes.c_int32() for _ in range(4)]
    _check(LIB.hpvm_plan_sgemm(int(tier), int(M), int(N), int(K), *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def hpvm_set_kernel_timing(ctx: int, enable: bool) -> None:
    _check(LIB.hpvm_set_kernel_timing(ctx, int(bool(enable))))


def hpvm_kernel_timing(ctx: int) -> tuple[float, int]:
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(LIB.hpvm_kernel_timing(ctx, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def hpvm_split_bf16(X: int, ld: int, kcontig: bool, rows: int, K: int, hi: int,
                    lo: int | None, cuda_stream: int = 0) -> None:
    _check(LIB.hpvm_split_bf16(X, int(ld), int(bool(kcontig)), int(rows), int(K), hi, lo,
                               cuda_stream or None))


def hpvm_split3_bf16(X: int, ld: int, kcontig: bool, rows: int, K: int, hi: int, mid: int,
                     lo: int, cuda_stream: int = 0) -> None:
    _check(LIB.hpvm_split3_bf16(X, int(ld), int(bool(kcontig)), int(rows), int(K), hi, mid, lo,
                                cuda_stream or None))


def hpvm_quant_fp8(X: int, ld: int, kcontig: bool, rows: int, K: int, q: int, scales: int,
                   cuda_stream: int = 0) -> None:
    _check(LIB.hpvm_quant_fp8(X, int(ld), int(bool(kcontig)), int(rows), int(K), q, scales,
                              cuda_stream or None))


def hpvm_sgemm_bf16x3_noalloc(M: int, N: int, K: int, alpha: float, A: int, lda: int,
                              B: int, ldb: int, beta: float, C: int, ldc: int,
                              transA: bool, transB: bool, dev_status: int | None = None,
                              cuda_stream: int = 0) -> None:
    """The allocation-free BF16x3 leaf: device pointers in, C updated on
    ``cuda_stream`` (asynchronous); see include/hpvm.h."""
    _check(LIB.hpvm_sgemm_bf16x3_noalloc(int(M), int(N), int(K), float(alpha), A, int(lda), B,
                                         int(ldb), float(beta), C, int(ldc), int(bool(transA)),
                                         int(bool(transB)), dev_status, cuda_stream or None))


def hpvm_batch_prepare(ctx: int, root: int, records, count: int, policy: int = -1) -> int:
    """``records``: a ctypes array of ``count`` RootArgs (one per instance)."""
    out = ctypes.c_void_p()
    _check(LIB.hpvm_batch_prepare(ctx, root, ctypes.byref(records), ctypes.sizeof(RootArgs), int(count),
                                  int(policy), ctypes.byref(out)))
    return out.value


def hpvm_batch_run(batch: int, cuda_stream: int = 0) -> None:
    _check(LIB.hpvm_batch_run(batch, cuda_stream or None))


def hpvm_batch_autotune(batch: int, cuda_stream: int = 0, reps: int = 3) -> tuple[int, float]:
    best = ctypes.c_int()
    ms = ctypes.c_double()
    _check(LIB.hpvm_batch_autotune(batch, cuda_stream or None, int(reps), ctypes.byref(best), ctypes.byref(ms)))
    return best.value, ms.value


def hpvm_batch_info(batch: int) -> BatchInfo:
    info = BatchInfo()
    _check(LIB.hpvm_batch_info(batch, ctypes.byref(info)))
    return info


def hpvm_batch_free(batch: int) -> None:
    _check(LIB.hpvm_batch_free(batch))


def hpvm_batch_plan(M, N, K, policy: int):
    """Tile widths and the schedule: one (instance, m0, n0, unit) per slot in
    launch order, instance -1 for an empty slot (policies 4-7: 256-row tiles
    on CTA pairs, the unit a pair)."""
    n = len(M)
    arr = lambda v: (ctypes.c_int64 * max(n, 1))(*[int(x) for x in v])
    Ma, Na, Ka = arr(M), arr(N), arr(K)
    bn = (ctypes.c_int32 * max(n, 1))()
    cnt = ctypes.c_int64()
    _check(LIB.hpvm_batch_plan(n, Ma, Na, Ka, int(policy), bn, None, 0, ctypes.byref(cnt)))
    tiles = (ctypes.c_int32 * max(4 * cnt.value, 1))()
    _check(LIB.hpvm_batch_plan(n, Ma, Na, Ka, int(policy), bn, tiles, cnt.value, ctypes.byref(cnt)))
    return list(bn)[:n], [tuple(tiles[4 * i:4 * i + 4]) for i in range(cnt.value)]


def hpvm_selftest_wait_timeout(ctx: int, limit_ms: int, cuda_stream: int = 0) -> None:
    """Raises HpvmError(HPVM_ERR_DEVICE_FAULT) when the bounded wait gave up, as it must."""
    _check(LIB.hpvm_selftest_wait_timeout(ctx, int(limit_ms), cuda_stream or None))


def hpvm_set_wait_limit(ctx: int, limit_us: int) -> None:
    _check(LIB.hpvm_set_wait_limit(ctx, int(limit_us)))


def hpvm_last_error() -> str:
    return LIB.hpvm_last_error().decode()


def hpvm_version() -> int:
    return LIB.hpvm_version()
