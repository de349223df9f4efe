"""Benchmark of the sgemm dataflow graph on GB300.

Default (``--impl gb300``): one step is one launch of the whole sgemm DFG
through the C-ABI (``hpvm_launch``: the BF16 split pre-pass of A and B, then
the tcgen05 leaf kernel) on the large workload, M = N = K = 8192, op(A) = A,
op(B) = B^T (column-major), A, B, C ~ N(0,1), alpha = beta = 1. Inputs are
resident in HBM when the timed region starts and larger than L2 (768 MiB of
FP32 operands plus 512 MiB of split planes), so no L2 flush is needed.

Printed (rank 0, one JSON line): useful TFLOP/s (2*M*N*K per step) of the
split-BF16x3 DFG; the roofline of its leaf kernel (tensor FLOP = 3 products
x 2*M*N*K, over the kernel's own CUDA-event time, against the measured dense
BF16 peak); the plain FP32 CUDA-core DFG on the same workload; the normwise
error of both against the FP64 oracle on sampled blocks (computed in the
CPU-baseline leg, which times that oracle); the end-to-end figure through
the memory tracker with pinned host buffers (every step copies its A, B, C
in and its C out; two contexts alternate so one step's copies overlap the
other's kernels, and the one-step-at-a-time time is reported beside it);
SM clocks sampled during the timed region; the number of kernels launched.

``--impl reference``: the FP64 oracle timed on the host cores, each step one
256 x 256 output block of the same workload (full K), rank 0 only.

Multi-GPU (torchrun, one rank per GPU): every rank runs its own replica of
the workload (weak scaling, no data exchange); value = FLOP of all ranks /
max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sgemm-DFG TFLOP/s and % of roofline at ≤5e-6 rel. err, split-BF16 vs plain FP32"
WORKLOAD = ("sgemm DFG, M=N=K={n}, op(A)=A, op(B)=B^T column-major, A,B,C ~ N(0,1) seed 1, "
            "alpha=beta=1; leaf = split-BF16x3 tcgen05 (3 products, FP32 accumulate)")
WORKLOAD_REF = ("sgemm DFG, M=N=K={n}, op(A)=A, op(B)=B^T column-major, A,B,C ~ N(0,1) seed 1, "
                "alpha=beta=1; FP64 oracle on the host cores")
N_SIZE = 8192
TILE_BLOCK = 256


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--size", type=int, default=N_SIZE, help="M = N = K of the headline workload")
    ap.add_argument("--fp32-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp8", action="store_true", help="skip the 16384 FP8 workload section")
    ap.add_argument("--fp8-n", type=int, default=16384)
    ap.add_argument("--no-chain", action="store_true", help="skip the streamed chain section")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-instances section")
    ap.add_argument("--batch-count", type=int, default=512,
                    help="instances of the batched workload (a smaller batch for profiling)")
    ap.add_argument("--only", choices=["chain", "batch", "fp8"], default=None,
                    help="run one workload section alone and print its JSON (for profiling); "
                         "no headline line")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms: float, device: str) -> float:
    """The slowest rank's time (every rank gets it); the local time when the
    job has one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(flop_per_rank: float, world: int, ms: float) -> float:
    """Whole-job TFLOP/s: the work of all ranks over the slowest rank's time
    (weak scaling: every rank runs its own replica)."""
    return flop_per_rank * world / (ms * 1e-3) / 1e12


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0, "_source": "fallback"}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("tc_leaf.cu", "internal.h"):
        with open(os.path.join(ROOT, "paper_1611_00860_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_from_profiles(src_hash: str, name: str = "sgemm_tc_bf16x3_8192.md",
                          what: str = "per launch"):
    """DRAM bytes (read + write) from a committed ncu summary, if it was
    taken on the current kernel source: per launch of the headline leaf, or
    per run of the batch (split pre-pass and grouped leaf)."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"kernel source sha256\[:16\]:\s*`?([0-9a-f]{16})", text)
    m_bytes = re.search(r"dram bytes " + re.escape(what) + r" \(read \+ write\)\W*([0-9.eE+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != src_hash:
        return None
    return float(m_bytes.group(1))


def gpu_id(local: int) -> str:
    """nvidia-smi --id of the CUDA device `local` (its UUID when torch knows it)."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(local).uuid)
        if u and u != "None":
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    parts = [x for x in vis.split(",") if x.strip()]
    return parts[local] if local < len(parts) else str(local)


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"hpvm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def cpu_oracle_leg(p, seconds: float):
    """Time the oracle (as it stands) on sampled 256 x 256 blocks of the
    workload for about ``seconds``: first the 16 seeded positions plus the
    first and last block (whose FP64 values are returned for the error
    check), then further seeded positions until the time is used."""
    import workloads as W
    from oracle import sgemm as O
    check = W.sample_blocks(p.M, p.N, bs=TILE_BLOCK, count=16)
    extra = [b for b in W.sample_blocks(p.M, p.N, bs=TILE_BLOCK, count=4096, seed=12) if b not in check]
    refs, t0, done = [], time.perf_counter(), 0
    flops = 0
    for idx, (i0, j0) in enumerate(check + extra):
        blk = O.sgemm_block_f64(p, i0, j0, TILE_BLOCK, TILE_BLOCK)
        if idx < len(check):
            refs.append(((i0, j0), blk))
        done += 1
        flops += 2 * min(TILE_BLOCK, p.M - i0) * min(TILE_BLOCK, p.N - j0) * p.K
        if idx + 1 >= len(check) and time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": O.num_threads(),
            "kind": "oracle",
            "sample": f"{done} sampled {TILE_BLOCK}x{TILE_BLOCK} output blocks of the "
                      f"{p.M}x{p.N}x{p.K} workload (full K), FP64 triple loop, {dt:.1f} s"}, refs


def block_error(C_dev, p, refs):
    import workloads as W
    from oracle import sgemm as O
    Cv = W.col_major(C_dev, p.M, p.N, p.ldc)
    pairs = [(Cv[i0:i0 + TILE_BLOCK, j0:j0 + TILE_BLOCK].double().cpu().numpy(), r)
             for (i0, j0), r in refs]
    return O.block_errors(pairs)


def fp8_section(args, dfg, H, W, torch, local, peaks, world, rank, barrier):
    """FP8 block-scaled DFG on its workload, with BF16x3, BF16x6 and FP32 on
    the same inputs; error of each against the FP64 oracle on sampled blocks
    (rank 0, one GPU: the CPU-baseline leg's oracle), and the error BF16x3's
    three products have on those blocks in exact arithmetic (its
    representation floor)."""
    n = args.fp8_n
    p = W.fp8_problem(n)
    flop = 2.0 * n * n * n
    A, B = p.A.to(f"cuda:{local}"), p.B.to(f"cuda:{local}")
    stream = torch.cuda.current_stream(local)
    out = {"workload": f"M=N=K={n}, A,B ~ N(0,1) x exp(2 Z) per row, beta=0, seed 4",
           "unit": "TFLOP/s"}
    blocks = W.sample_blocks(n, n, bs=TILE_BLOCK, count=4)
    outputs = {}
    for name, tier, steps in (("fp8", H.HPVM_TIER_FP8, 20), ("bf16x3", H.HPVM_TIER_BF16X3, 5),
                              ("bf16x6", H.HPVM_TIER_BF16X6, 3), ("fp32", H.HPVM_TIER_FP32, 2)):
        C = torch.zeros(n * n, dtype=torch.float32, device=f"cuda:{local}")
        a = dfg.args_for(n, n, n, A, n, B, n, C, n, 1.0, 0.0, False, True, tier=tier)
        dfg.ensure_workspace(a)
        dfg.wait(dfg.launch(a), 600000)
        barrier()
        H.hpvm_set_kernel_timing(dfg.ctx, True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        gs = [dfg.launch(a) for _ in range(steps)]
        ev1.record(stream)
        barrier()
        H.hpvm_set_kernel_timing(dfg.ctx, False)
        kms, kn = H.hpvm_kernel_timing(dfg.ctx)
        for g in gs:
            dfg.wait(g)
        ms = max_over_ranks(ev0.elapsed_time(ev1) / steps, f"cuda:{local}")
        ent = {"value": flop * world / (ms * 1e-3) / 1e12, "ms_per_step": ms, "steps": steps,
               "leaf_ms": kms / max(1, kn)}
        if name == "fp8":
            peak8 = 2.0 * peaks["bf16_tflops"]
            ach = flop / (ent["leaf_ms"] * 1e-3) / 1e12
            ent["roofline"] = {"bound": "tensor", "achieved": ach, "peak": peak8, "unit": "TFLOP/s",
                               "frac": ach / peak8,
                               "peak_source": f"{peaks['_source']} dense BF16 burst x 2 (nominal FP8/BF16 ratio 4.5/2.25)"}
        out[name] = ent
        Cv = W.col_major(C, n, n, n)
        outputs[name] = [Cv[i0:i0 + TILE_BLOCK, j0:j0 + TILE_BLOCK].double().cpu().numpy()
                         for (i0, j0) in blocks]
        del C
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import sgemm as O
        refs = [O.sgemm_block_f64(p, i0, j0, TILE_BLOCK, TILE_BLOCK) for (i0, j0) in blocks]
        from oracle import split as S
        out["rel_err"] = {k: O.block_errors(list(zip(v, refs))) for k, v in outputs.items()}
        exact3 = [S.split_block_f64(p, i0, j0, TILE_BLOCK, TILE_BLOCK, "bf16x3") for (i0, j0) in blocks]
        out["rel_err"]["bf16x3_exact_arithmetic"] = O.block_errors(list(zip(exact3, refs)))
        out["rel_err"]["blocks"] = len(blocks)
        out["rel_err"]["tolerance"] = {"fp8": 6e-2, "bf16x3": 5e-6, "bf16x6": 5e-6, "fp32": 5e-6}
        out["rel_err"]["note"] = ("bf16x3_exact_arithmetic: the sum of BF16x3's three products in FP64 "
                                  "(oracle.split) on the same blocks; above 5e-6, BF16x3 cannot meet the "
                                  "bound on these inputs, and BF16x6 is the split tier that does")
    del A, B
    torch.cuda.empty_cache()
    return out


def chain_section(args, H, W, torch, local, world, barrier):
    """The streamed chain: 64 items of 256 x 4096 through four 4096 x 4096
    weights with tanh between (BF16 operands, FP32 accumulate).
    (a) a training step of the whole batch through ChainFunction: forward
        chain launch, recomputed activations, adjoint leaves;
    (b) the forward of the 64 items pushed one by one through the chain
        launched as a streaming graph (hpvm_push / hpvm_pop)."""
    from paper_1611_00860_gb300.chain import ChainEngine, chain_apply
    X, Ws, G = W.chain_inputs()
    items, rows, w = X.shape
    L = len(Ws)
    dev = f"cuda:{local}"
    Xd, Gd = X.to(dev), G.to(dev)
    Wd = [x.to(dev).requires_grad_(True) for x in Ws]
    eng = ChainEngine(L, device=local, tier=H.HPVM_TIER_BF16)
    stream = torch.cuda.current_stream(local)
    n = items * rows
    prod = 2.0 * n * w * w                      # one stage's product
    fwd, bwd, recompute = L * prod, 2 * L * prod, (L - 1) * prod
    out = {"workload": f"{items} items x {rows} x {w}, {L} weights {w}x{w} ~ N(0,1/{w}), tanh between, "
                       "BF16 operands, FP32 accumulate, seed 3", "unit": "TFLOP/s"}

    def step():
        Xr = Xd.requires_grad_(True)
        Y = chain_apply(eng, Xr, Wd)
        (Y * Gd).sum().backward()
        Xd.grad = None
        for x in Wd:
            x.grad = None

    steps = 5
    step()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        step()
    ev1.record(stream)
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / steps, dev)
    executed = (fwd + bwd + recompute) / (ms * 1e-3) / 1e12  # per GPU
    peaks = load_peaks()
    out["train_step"] = {"value": (fwd + bwd) * world / (ms * 1e-3) / 1e12, "ms_per_step": ms, "steps": steps,
                         "executed_tflop_per_step": (fwd + bwd + recompute) / 1e12,
                         "executed_rate": executed * world,
                         "note": "value counts forward + backward products; the recomputed forward "
                                 "of the activations is in executed_rate",
                         "roofline": {"bound": "tensor", "achieved": executed, "peak": peaks["bf16_tflops"],
                                      "unit": "TFLOP/s", "frac": executed / peaks["bf16_tflops"],
                                      "algorithmic": "15 products of 2*16384*4096*4096 FLOP per step (4 forward, "
                                                     "3 recomputed, 8 adjoint), whole step incl. operand "
                                                     "conversion and PyTorch's loss",
                                      "peak_source": f"{peaks['_source']} dense BF16 burst (MEASURED_PEAKS.json)"}}
    with torch.no_grad():
        Wn = [x.detach() for x in Wd]
        xs = [Xd[i] for i in range(items)]
        eng.stream_forward(xs, Wn)
        barrier()
        t0 = time.perf_counter()
        eng.stream_forward(xs, Wn)
        barrier()
        dt = time.perf_counter() - t0
    dt = max_over_ranks(dt * 1e3, dev) * 1e-3
    out["streamed_forward"] = {"value": fwd * world / dt / 1e12, "ms_per_batch": dt * 1e3,
                               "items": items, "path": "hpvm_launch(stream_graph=1) + hpvm_stream_coalesce(32) + 64 x hpvm_push + 64 x hpvm_pop"}
    eng.close()
    del Xd, Gd, Wd
    torch.cuda.empty_cache()
    return out


def batch_section(args, H, W, torch, local, world, rank, barrier):
    """512 independent sgemm DFG instances (M, N, K log-uniform in [32, 2048],
    BF16x3 leaves): one autotuned batch (batched split pre-pass + grouped
    persistent leaf) replayed from a CUDA graph, against one hpvm_launch per
    instance on the same inputs."""
    from paper_1611_00860_gb300.batch import BatchDFG
    from paper_1611_00860_gb300.sgemm import SgemmDFG
    shapes = W.batched_shapes(args.batch_count)
    probs = [W.sgemm_problem(m, n, k, seed=20000 + i, alpha=1.0, beta=0.0) for i, (m, n, k) in enumerate(shapes)]
    flop = sum(2.0 * m * n * k for m, n, k in shapes)
    dev = [tuple(t.to(f"cuda:{local}") for t in (p.A, p.B, p.C)) for p in probs]
    stream = torch.cuda.current_stream(local)
    b = BatchDFG(local)
    b.prepare(probs, dev, tier=H.HPVM_TIER_BF16X3, policy=-1)
    best, tuned_ms = b.autotune(3)
    graph = b.capture()
    reps = 20
    graph.replay()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(reps):
        graph.replay()
    ev1.record(stream)
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / reps, f"cuda:{local}")
    # the grouped leaf's own time (runtime's CUDA events around it), the rest
    # of a batch being the batched split pre-pass
    H.hpvm_set_kernel_timing(b.ctx, True)
    for _ in range(reps):
        b.run(stream)
    barrier()
    H.hpvm_set_kernel_timing(b.ctx, False)
    leaf_total, leaf_n = H.hpvm_kernel_timing(b.ctx)
    leaf_ms = leaf_total / max(1, leaf_n)
    peaks = load_peaks()
    algo_bytes = sum(4.0 * (m * k + n * k + m * n) for m, n, k in shapes)
    achieved = algo_bytes / (ms * 1e-3) / 1e9
    out = {"workload": f"{args.batch_count} sgemm DFG instances, M,N,K log-uniform in [32,2048] (seed 2), N(0,1), "
                       "alpha=1, beta=0, BF16x3 leaves", "unit": "TFLOP/s",
           "useful_tflop": flop / 1e12, "batch": {
               "value": flop * world / (ms * 1e-3) / 1e12, "ms_per_batch": ms,
               "launches": 2, "path": "hpvm_batch_prepare + hpvm_batch_autotune, hpvm_batch_run captured "
                                      "in a CUDA graph, replayed",
               "autotuned_policy": best, "info": b.info(),
               "leaf_ms": leaf_ms, "split_ms": ms - leaf_ms,
               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": achieved / peaks["hbm_gbs"],
                            "traffic": traffic_from_profiles(kernel_source_hash(), "launches_batch_512.md",
                                                             "per batch") if args.batch_count == 512 else None,
                            "algorithmic": "4*(M*K + N*K + M*N) bytes per instance: FP32 A and B read once, "
                                           "C written once (beta = 0); the split planes are extra traffic",
                            "peak_source": f"{peaks['_source']} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}}}
    # one launch per instance (each: split of A, split of B, leaf)
    s = SgemmDFG(local)
    args_list = [s.args_for(p.M, p.N, p.K, A, p.lda, B, p.ldb, C, p.ldc, p.alpha, p.beta, p.transA,
                            p.transB, tier=H.HPVM_TIER_BF16X3) for p, (A, B, C) in zip(probs, dev)]
    for a in args_list:
        s.ensure_workspace(a)
    for a in args_list:
        s.wait(s.launch(a))
    barrier()
    t0 = time.perf_counter()
    ev0.record(stream)
    gs = [s.launch(a) for a in args_list]
    ev1.record(stream)
    barrier()
    wall = (time.perf_counter() - t0) * 1e3
    for g in gs:
        s.wait(g)
    ms1 = max_over_ranks(ev0.elapsed_time(ev1), f"cuda:{local}")
    out["one_launch_per_instance"] = {"value": flop * world / (ms1 * 1e-3) / 1e12, "ms_per_batch": ms1,
                                      "host_ms": wall, "launches": 3 * len(probs)}
    out["speedup"] = ms1 / ms
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import sgemm as O
        # error of the batch on the 32 smallest instances (the oracle computes them whole)
        order = sorted(range(len(probs)), key=lambda i: probs[i].M * probs[i].N * probs[i].K)[:32]
        for (_, _, C) in dev:
            C.zero_()
        graph.replay()
        torch.cuda.synchronize()
        worst = 0.0
        for i in order:
            p = probs[i]
            got = W.col_major(dev[i][2].cpu(), p.M, p.N, p.ldc).double().numpy()
            worst = max(worst, O.normwise_rel_err(got, O.sgemm_f64(p)))
        out["rel_err_worst_of_32_smallest"] = worst
    s.close()
    b.close()
    del dev
    torch.cuda.empty_cache()
    return out


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import workloads as W
    from oracle import sgemm as O
    p = W.large_dfg_problem(args.size)
    blocks = W.sample_blocks(p.M, p.N, bs=TILE_BLOCK, count=max(16, args.steps + args.warmup))
    seq = [blocks[i % len(blocks)] for i in range(args.steps + args.warmup)]
    for (i0, j0) in seq[:args.warmup]:
        O.sgemm_block_f64(p, i0, j0, TILE_BLOCK, TILE_BLOCK)
    t0 = time.perf_counter()
    flops = 0
    for (i0, j0) in seq[args.warmup:]:
        O.sgemm_block_f64(p, i0, j0, TILE_BLOCK, TILE_BLOCK)
        flops += 2 * min(TILE_BLOCK, p.M - i0) * min(TILE_BLOCK, p.N - j0) * p.K
    dt = time.perf_counter() - t0
    v = flops / dt / 1e12
    sample = (f"each step one {TILE_BLOCK}x{TILE_BLOCK} output block of the {p.M}x{p.N}x{p.K} "
              "workload (full K), FP64 triple loop on the host cores")
    print(json.dumps({
        "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD_REF.format(n=p.M), "M": p.M, "N": p.N, "K": p.K},
        "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": O.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import workloads as W
    from paper_1611_00860_gb300 import _lib as H
    from paper_1611_00860_gb300.sgemm import SgemmDFG

    peaks = load_peaks()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(local)

    if args.only:
        out = None
        if args.only == "chain":
            out = chain_section(args, H, W, torch, local, world, barrier)
        elif args.only == "batch":
            out = batch_section(args, H, W, torch, local, world, rank, barrier)
        else:
            dfg = SgemmDFG(local)
            out = fp8_section(args, dfg, H, W, torch, local, peaks, world, rank, barrier)
            dfg.close()
        if rank == 0:
            print(json.dumps({"section": args.only, **out}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    n = args.size
    p = W.large_dfg_problem(n)
    flop = 2.0 * p.M * p.N * p.K
    A, B, C0 = (t.to(f"cuda:{local}") for t in (p.A, p.B, p.C))
    C = C0.clone()
    dfg = SgemmDFG(local)
    stream = torch.cuda.current_stream(local)

    def launch_args(tier, Cbuf):
        return dfg.args_for(p.M, p.N, p.K, A, p.lda, B, p.ldb, Cbuf, p.ldc, p.alpha, p.beta,
                            p.transA, p.transB, tier=tier)

    def timed(tier, steps, warmup, Cbuf, clocks=False):
        a = launch_args(tier, Cbuf)
        dfg.ensure_workspace(a)
        for _ in range(warmup):
            dfg.wait(dfg.launch(a))
        barrier()
        sampler = ClockSampler(gpu_id(local)) if clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.3)  # let the sampler start before the load
        H.hpvm_set_kernel_timing(dfg.ctx, True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        graphs, kernels = [], 0
        for _ in range(steps):
            g = dfg.launch(a)
            kernels += H.hpvm_graph_info(g).kernels
            graphs.append(g)
        ev1.record(stream)
        barrier()
        H.hpvm_set_kernel_timing(dfg.ctx, False)
        kms, klaunch = H.hpvm_kernel_timing(dfg.ctx)
        for g in graphs:
            dfg.wait(g)
        clk = sampler.stop() if sampler else None
        ms = ev0.elapsed_time(ev1)
        return max_over_ranks(ms, f"cuda:{local}"), kms / max(1, klaunch), kernels, clk

    # 1) correctness run of both tiers on a fresh C (checked below against the oracle)
    C_bf = C0.clone()
    dfg.wait(dfg.launch(launch_args(H.HPVM_TIER_BF16X3, C_bf)))
    C_fp = C0.clone()
    dfg.wait(dfg.launch(launch_args(H.HPVM_TIER_FP32, C_fp)))
    C_b6 = C0.clone()
    dfg.wait(dfg.launch(launch_args(H.HPVM_TIER_BF16X6, C_b6)))

    # 2) timed split-BF16x3 DFG (headline)
    ms_total, kern_ms, launches, clocks = timed(H.HPVM_TIER_BF16X3, args.steps, args.warmup, C, True)
    ms_step = ms_total / args.steps
    value = job_rate(flop * args.steps, world, ms_total)
    tensor_flop = 3 * flop
    achieved = tensor_flop / (kern_ms * 1e-3) / 1e12
    src_hash = kernel_source_hash()
    traffic = traffic_from_profiles(src_hash)
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_tflops"],
                "unit": "TFLOP/s", "frac": achieved / peaks["bf16_tflops"], "traffic": traffic,
                "peak_source": f"{peaks['_source']} dense BF16 burst (MEASURED_PEAKS.json bf16_tflops)",
                "frac_of_sustained": achieved / peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]),
                "kernel": "sgemm_tc<3>", "kernel_ms": kern_ms,
                "algorithmic": "3 x 2*M*N*K tensor FLOP per launch", "kernel_source": src_hash}

    # 3) plain FP32 CUDA-core DFG on the same workload
    fp_total, fp_kern_ms, fp_launches, _ = timed(H.HPVM_TIER_FP32, args.fp32_steps, 2, C)
    props = torch.cuda.get_device_properties(local)
    fp32_peak = props.multi_processor_count * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    fp32 = {"value": flop * world * args.fp32_steps / (fp_total * 1e-3) / 1e12, "unit": "TFLOP/s",
            "ms_per_step": fp_total / args.fp32_steps, "steps": args.fp32_steps,
            "kernel_frac_of_fp32_peak": flop / (fp_kern_ms * 1e-3) / 1e12 / fp32_peak,
            "fp32_peak_tflops": fp32_peak,
            "fp32_peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x max SM clock"}

    # 3b) the three-part split (BF16x6: six products) on the same workload
    b6_total, b6_kern_ms, _, _ = timed(H.HPVM_TIER_BF16X6, args.fp32_steps, 2, C)
    b6_ach = 6 * flop / (b6_kern_ms * 1e-3) / 1e12
    bf16x6 = {"value": flop * world * args.fp32_steps / (b6_total * 1e-3) / 1e12, "unit": "TFLOP/s",
              "ms_per_step": b6_total / args.fp32_steps, "steps": args.fp32_steps, "kernel_ms": b6_kern_ms,
              "kernel_tensor_tflops": b6_ach, "kernel_frac": b6_ach / peaks["bf16_tflops"],
              "algorithmic": "6 x 2*M*N*K tensor FLOP per launch"}

    # 4) end to end through the memory tracker with pinned host buffers: two
    # contexts alternate, each with its own pinned A, B, C and its own
    # stream. Every step copies its A, B, C in and its C back out; step i+1
    # is launched (copies and kernels enqueued) before step i's result is
    # waited for and read back, so the host link carries one step while the
    # GPU computes the other (double buffering, as a serving loop would).
    from paper_1611_00860_gb300.sgemm import SgemmDFG, make_args
    dfg2 = SgemmDFG(local)
    sets = []
    for j, d in enumerate((dfg, dfg2)):
        hA, hB, hC = (t.pin_memory() for t in (p.A, p.B, p.C))
        for t in (hA, hB, hC):
            H.hpvm_track_mem(d.ctx, t.data_ptr(), t.numel() * 4)
        ha = make_args(p.M, p.N, p.K, hA.data_ptr(), hA.numel() * 4, p.lda, hB.data_ptr(),
                       hB.numel() * 4, p.ldb, hC.data_ptr(), hC.numel() * 4, p.ldc, p.alpha, p.beta,
                       p.transA, p.transB, H.HPVM_TIER_BF16X3)
        d.ensure_workspace(ha)
        sets.append((d, (hA, hB, hC), ha, torch.cuda.Stream(local)))

    def e2e_launch(j, st=None):
        d, hs, ha, own = sets[j]
        for t in hs:
            H.hpvm_track_mem(d.ctx, t.data_ptr(), t.numel() * 4)  # the step's inputs: host copy is the latest
        return H.hpvm_launch(d.ctx, d.nodes["root"], ha, False, (st or own).cuda_stream)

    def e2e_finish(j, g):
        d, (_, _, hC), _, _ = sets[j]
        H.hpvm_wait(g, 60000)
        H.hpvm_request_mem(d.ctx, hC.data_ptr(), hC.numel() * 4)

    def e2e_run(n):
        g = e2e_launch(0)
        h2d = H.hpvm_graph_info(g).h2d_bytes
        for i in range(n):
            nxt = e2e_launch((i + 1) % 2) if i + 1 < n else None
            e2e_finish(i % 2, g)
            g = nxt
        return h2d

    def e2e_serial(n):  # one step at a time on the launch stream (for comparison)
        for _ in range(n):
            g = e2e_launch(0, stream)
            e2e_finish(0, g)

    e2e_run(2)
    barrier()
    t0 = time.perf_counter()
    h2d = e2e_run(args.e2e_steps)
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps * 1e3, f"cuda:{local}") * 1e-3
    t0 = time.perf_counter()
    e2e_serial(args.e2e_steps)
    barrier()
    serial_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps * 1e3, f"cuda:{local}") * 1e-3
    for d, hs, _, _ in sets:
        for t in hs:
            H.hpvm_untrack_mem(d.ctx, t.data_ptr())
    dfg2.close()
    sets.clear()
    e2e = {"value": flop * world / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(p.C.numel() * 4), "ms_per_step": e2e_s * 1e3,
           "serial_ms_per_step": serial_s * 1e3,
           "path": "two contexts alternating, each with its own pinned A, B, C and stream: hpvm_track_mem(A,B,C) "
                   "+ hpvm_launch of step i+1, then hpvm_wait + hpvm_request_mem(C) of step i"}

    # 5) CPU baseline (the oracle, timed) and the error of the runs of step 1
    cpu, err = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, refs = cpu_oracle_leg(p, args.cpu_seconds)
        err = {"bf16x3": block_error(C_bf, p, refs), "fp32": block_error(C_fp, p, refs),
               "bf16x6": block_error(C_b6, p, refs),
               "blocks": len(refs), "metric": "normwise ||C-C_ref||_F/||C_ref||_F over sampled blocks",
               "tolerance": 5e-6}

    # 6) batches of independent instances, and the streamed chain
    batch = None
    if not args.no_batch:
        batch = batch_section(args, H, W, torch, local, world, rank, barrier)
    chain = None
    if not args.no_chain:
        chain = chain_section(args, H, W, torch, local, world, barrier)

    # 7) the FP8 workload: M = N = K = 16384, per-row log-normal(0,2)
    # magnitudes, beta = 0; FP8 block-scaled leaf vs BF16x3 vs plain FP32 on
    # the same inputs and GPU
    fp8 = None
    if not args.no_fp8:
        del A, B, C0, C, C_bf, C_fp, C_b6, hA, hB, hC
        torch.cuda.empty_cache()
        fp8 = fp8_section(args, dfg, H, W, torch, local, peaks, world, rank, barrier)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3", "data": "synthetic",
            "config": {"workload": WORKLOAD.format(n=p.M), "M": p.M, "N": p.N, "K": p.K, "transA": "N",
                       "transB": "T", "tier": "bf16x3", "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (768 MiB FP32 operands + 512 MiB split planes); no flush"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches, "rel_err": err, "fp32_cuda_core": fp32, "bf16x6_split": bf16x6,
            "fp8_workload": fp8, "chain_workload": chain, "batched_workload": batch,
        }
        print(json.dumps(line), flush=True)
    dfg.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
