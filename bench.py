"""Benchmark of the two-stage Householder orthogonalization on GB300.

One step = one orthogonalization (Algorithm 1, second choice of P, every
phase from the QR of V_{1:k0,:} to the explicit Q) of a resident synthetic
problem.  Default workload: complex128, n = 2^22, k0 = 128, k = 32, half of
A numerically in Range(V) (the n = 2^22 configuration of the headline metric).

Metric: GB/s of algorithmic bytes B_alg = s n (3 k0 + 4 k) per orthogonalization
(s = 16 bytes for complex128, 8 for real): three sweeps over V and A forced by
the three global reductions of Algorithm 1 (W^* A, the trailing QR's R, and
W^* [0; Qbar]), plus the write of Q.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3|c3-fp32|c2|c1]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Multi-GPU (torchrun): replicas only -- every rank orthogonalizes its own
independent problem (block Krylov solvers issue independent orthogonalizations);
there is no collective on the data path.  value = total bytes of all ranks /
the slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "two-stage HHQR GB/s (% HBM roof) at n=2^22; batched & fwd+bwd vs looped plain"
UNIT = "GB/s"
# FP64 FMA peak of one GB300 (roofline denominator of the FP64 path), from the unit
# count and clock, checked against a one-off probe (profiles/fp64_peak_probe.md):
# 2 FP64 FMA / clk / SM x 152 SMs x 2.07 GHz = 1.259 TFLOP/s (nominal 1.25); the probe reads
# 1.04 (DFMA chains) and the streaming kernels sustain 1.23.  The FP64 kernels issue DFMA.
FP64_PEAK_TFLOPS = 1.259
FP32_PEAK_TFLOPS = 78.4
HBM_GBS_FALLBACK = 6795.1

WORKLOADS = {
    # name: (config id, n, k0, k, dtype name, precision mode, description)
    # precision 0: FP64 arithmetic; 1: FP32-bulk variant; 2: FP64-accurate split-n
    # products on bf16 tensor cores (same tolerances as 0; the QR of the leaves,
    # the TSQR tree and the small solves stay FP64).
    "c3": (3, 1 << 22, 128, 32, "complex128", 2,
           "complex128 n=4194304 k0=128 k=32, A=[V C1 + 1e-14 G1, G2] (numerically rank deficient); "
           "FP64-accurate, split-n products on bf16 tensor cores"),
    "c3-native": (3, 1 << 22, 128, 32, "complex128", 0,
                  "complex128 n=4194304 k0=128 k=32, A=[V C1 + 1e-14 G1, G2], FP64 arithmetic throughout"),
    "c3-fp32": (3, 1 << 22, 128, 32, "complex128", 1,
                "complex128 n=4194304 k0=128 k=32, FP32-bulk variant"),
    "c2": (2, 1 << 20, 64, 16, "float64", 2,
           "real n=1048576 k0=64 k=16, A=V C + 1e-10 G (cond ~1e10); FP64-accurate, products on bf16 tensor cores"),
    "c2-native": (2, 1 << 20, 64, 16, "float64", 0, "real n=1048576 k0=64 k=16, A=V C + 1e-10 G, FP64 arithmetic"),
    "c1": (1, 4096, 16, 4, "float64", 0, "real n=4096 k0=16 k=4, A=N(0,1)"),
    "c5": (5, 1 << 20, 64, 16, "float64", 0,
           "differentiation: real n=1048576 k0=64 k=16, A=N(0,1), dQ=N(0,1); fused forward+adjoint vs "
           "autograd through a GPU torch-ops composition of Algorithm 1"),
    "c4": (4, 0, 0, 0, "float64", 0,
           "batched: 256 real problems, n log-uniform in [16384, 262144], k0 in {8..128}, k in {4..32}, "
           "one graph replay vs 256 looped tho_orth calls"),
    "blocks": (6, 1 << 20, 0, 16, "float64", 2,
               "Algorithm 3 (block Householder-QR): real n=2^20, eight blocks of 16 columns, block-Krylov input "
               "A_{i+1} = D A_i (cond > 1e12); FP64-accurate products on bf16 tensor cores"),
    "c4-emu": (4, 0, 0, 0, "float64", 2,
               "batched: the 256 real problems of c4 with FP64-accurate products on bf16 tensor cores, "
               "one graph replay vs 256 looped tho_orth calls"),
}
CPU_SAMPLE_ROWS = {"c3": 65536, "c3-native": 65536, "c3-fp32": 65536, "c2": 131072, "c2-native": 131072, "c1": 4096}
REF_STEP_ROWS = {"c3": 16384, "c3-native": 16384, "c3-fp32": 16384, "c2": 32768, "c2-native": 32768, "c1": 4096}

# Algorithmic real flops per trailing row of each streaming phase (x4 for complex).
# FP64 arithmetic (precision 0 and the FP32-bulk variant):
#   gram: V_2^* A_2 (2 k0 k); leaf: A' = A + V_2 Z (2 k0 k), Householder QR
#   (2 k^2) and explicit leaf Q (2 k^2); apply: Q_leaf F (2 k^2) and V_2^* Qbar
#   (2 k0 k); update_q: V_2 Z2 (2 k0 k).
# With the products on tensor cores (precision 2) the leaf kernel keeps only
# the Householder QR of its leaves (compact WY form, no explicit leaf Q): over
# nb leaves of the m trailing rows, 2 m k^2 - nb (2/3) k^3 flops (real count;
# x4 complex); A' moves to update_a.
PHASE_FLOPS_PER_ROW = {
    "gram": lambda k0, k: 2 * k0 * k,
    "leaf": lambda k0, k: 2 * k0 * k + 4 * k * k,
    "apply": lambda k0, k: 2 * k * k + 2 * k0 * k,
    "update_q": lambda k0, k: 2 * k0 * k,
}
LEAF_WY_QR_FLOPS = lambda m, k, nb: 2 * m * k * k - nb * (2.0 / 3.0) * k ** 3
# bf16 tensor-core flops per trailing row of one emulated rank-k0 update (36
# slice pairs of a real-embedded (rows x 2k0) times (2k0 x 2k) product; real: k0, k).
EMU_UPDATE_MMA_FLOPS_PER_ROW = lambda k0, k, cplx: 2 * 36 * (2 * k0 if cplx else k0) * (2 * k if cplx else k)
BF16_MMA_SYNC_PEAK_TFLOPS = 607.0  # mma.sync m16n8k16 bf16, measured once by a probe (profiles/fp64_peak_probe.md; legacy path)


def _bf16_peak():
    """Dense bf16 tensor peak for a kernel timed inside a long step: the
    sustained cuBLAS figure of MEASURED_PEAKS.json (the tcgen05 products run
    on the same tensor cores), else the profiling fallback of 1.7 PFLOP/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback 1.7 PFLOP/s sustained (of fallback)"

def b_alg(n, k0, k, cplx):
    return (16 if cplx else 8) * n * (3 * k0 + 4 * k)


def f_alg(n, k0, k, cplx):
    return n * (8 * k0 * k + 4 * k * k) * (4 if cplx else 1)


def max_over_ranks(x: float, device=None) -> float:
    """Largest value over all ranks (the slowest rank's time); identity on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(bytes_per_step: float, steps: int, world_size: int, elapsed_ms: float) -> float:
    """GB/s of the whole job: every rank ran `steps` independent problems."""
    return bytes_per_step * world_size * steps / (elapsed_ms * 1e-3) / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: str):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.index, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except ValueError:
                continue
            for nm, v in zip(names, r[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json"
    except (OSError, KeyError, ValueError):
        return HBM_GBS_FALLBACK, "fallback"


# Source files each streaming kernel is built from (its own file and the
# helpers it includes): a traffic record stays valid while these are unchanged.
_KERNEL_FILES = {
    "k_gram": ("tho_scalar.cuh", "tho_plan.h", "tho_kernels.cuh"),
    "k_leaf": ("tho_scalar.cuh", "tho_plan.h", "tho_kernels.cuh"),
    "k_apply_gram": ("tho_scalar.cuh", "tho_plan.h", "tho_kernels.cuh"),
    "k_update_q": ("tho_scalar.cuh", "tho_plan.h", "tho_kernels.cuh"),
    "k_gram_emu": ("tho_scalar.cuh", "tho_plan.h", "tho_kernels.cuh", "tho_emu.cuh"),
    "k_update_emu": ("tho_scalar.cuh", "tho_plan.h", "tho_kernels.cuh", "tho_emu.cuh"),
    "k_apply_emu": ("tho_scalar.cuh", "tho_plan.h", "tho_kernels.cuh", "tho_emu.cuh"),
    "k_leaf_emu": ("tho_scalar.cuh", "tho_plan.h", "tho_kernels.cuh", "tho_emu.cuh"),
    "k_gram_umma": ("tho_scalar.cuh", "tho_plan.h", "tho_kernels.cuh", "tho_emu.cuh", "tho_umma.cuh"),
    "k_update_umma": ("tho_scalar.cuh", "tho_plan.h", "tho_kernels.cuh", "tho_emu.cuh", "tho_umma.cuh"),
    "k_tree_up": ("tho_scalar.cuh", "tho_plan.h", "tho_kernels.cuh", "tho_tree.cuh"),
    "k_tree_down": ("tho_scalar.cuh", "tho_plan.h", "tho_kernels.cuh", "tho_tree.cuh"),
    "k_tree_down_w": ("tho_scalar.cuh", "tho_plan.h", "tho_kernels.cuh", "tho_tree.cuh"),
}


def kernel_source_hash(kernel: str) -> str:
    """sha256[:16] of the sources `kernel` is built from, with comments and
    blank lines removed so that documentation edits keep it."""
    import hashlib
    import re
    d = os.path.join(ROOT, "paper_2602_14449_gb300", "csrc")
    h = hashlib.sha256()
    for f in _KERNEL_FILES[kernel.split("@")[0]]:
        for line in open(os.path.join(d, f)):
            code = re.sub(r"//.*", "", line).strip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def _traffic_for(kernel: str):
    """DRAM bytes per trailing row of `kernel` from the committed ncu summary,
    or None when the kernel's sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        h = kernel_source_hash(kernel)
        for line in open(path):
            f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
            if f.get("kernel") == kernel and f.get("src") == h:
                return float(f["bytes_per_row"])
    except OSError:
        pass
    return None


def _oracle_sample(job):
    """One oracle call on a seeded sample of a workload (run in a spawned worker
    process): returns (algorithmic bytes, seconds of the oracle call alone)."""
    import torch
    import oracle
    from paper_2602_14449_gb300 import inputs
    wl, rows = job
    cid, _, k0, k, dt, _, _ = WORKLOADS[wl]
    torch.set_num_threads(1)
    p = inputs.config_problem(cid, n=rows, dtype=getattr(torch, dt))
    V, A = p.V.numpy(), p.A.numpy()
    t0 = time.perf_counter()
    oracle.two_stage(V, A)
    return b_alg(rows, k0, k, dt == "complex128"), time.perf_counter() - t0


def cpu_baseline(wl: str, rows: int):
    """The CPU oracle, as it stands (one thread per call), on `rows` rows of the
    workload: once on one core, then as one call per allowed core at once (each
    on its own sample, in processes started with spawn); the N-core value is the
    bytes of all calls over the slowest call."""
    import multiprocessing as mp
    nb, t1 = _oracle_sample((wl, rows))
    out = {"value": nb / t1 / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{rows} rows of the same workload (same k0, k, structure), one call, {t1:.2f} s"}
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    if cores > 1:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_sample, [(wl, rows)] * cores)
        slow = max(t for _, t in res)
        out["n_core"] = {"value": sum(b for b, _ in res) / slow / 1e9, "unit": UNIT, "cores": cores,
                         "kind": "oracle",
                         "sample": f"{cores} concurrent oracle calls (one per core, spawned processes), each on "
                                   f"{rows} rows; bytes of all calls / slowest call ({slow:.2f} s)"}
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if ws > 1 and rank != 0:
        return 0
    if args.workload in ("c4", "c4-emu", "c5", "blocks"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle reference arm covers the single-problem "
                          "workloads c1, c2, c3"}), flush=True)
        return 0
    import oracle
    import torch
    from paper_2602_14449_gb300 import inputs
    wl = args.workload
    cid, n, k0, k, dt, prec, desc = WORKLOADS[wl]
    rows = REF_STEP_ROWS[wl]
    p = inputs.config_problem(cid, n=rows, dtype=getattr(torch, dt))
    V, A = p.V.numpy(), p.A.numpy()
    for _ in range(args.warmup):
        oracle.two_stage(V, A)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.two_stage(V, A)
    el = time.perf_counter() - t0
    cplx = dt == "complex128"
    val = b_alg(rows, k0, k, cplx) * args.steps / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128" if cplx else "f64",
        "data": "synthetic",
        "config": {"workload": desc, "reference_sample_rows": rows, "oracle": "CPU oracle (plain C++ loops), 1 thread"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: one oracle call on {rows} rows of the workload"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_blocks(args):
    """Algorithm 3: tho_orth_blocks over eight blocks of 16 columns (k0 = 0, 16,
    ..., 112 in its eight Algorithm 1 steps) on a block-Krylov matrix."""
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2602_14449_gb300 import inputs, tho
    tho.load()
    _, n, _, k, _, prec, desc = WORKLOADS["blocks"]
    if args.rows:
        n = args.rows
    nb = 8
    g = torch.Generator().manual_seed(1449 + 6)
    d = torch.exp(torch.linspace(0.0, 4.0, n, dtype=torch.float64))
    blocks = [torch.randn(n, k, generator=g, dtype=torch.float64)]
    for _ in range(nb - 1):
        blocks.append(d[:, None] * blocks[-1])
    A = inputs.colmajor(torch.cat(blocks, dim=1)).to(dev)
    del blocks
    K = k * nb
    blk = tho.Blocks(n, [k] * nb, torch.float64, prec)
    Q = torch.empty_strided((n, K), (1, n), dtype=torch.float64, device=dev)
    R = torch.empty_strided((K, K), (1, K), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(3, args.warmup)):
        blk.orth(A, Q, R)
    torch.cuda.synchronize(dev)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    smi_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(dev.index)).split(",")[0] if ws == 1 else str(local)
    sampler = ClockSampler(smi_index)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        blk.orth(A, Q, R)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dev) / args.steps
    B = sum(b_alg(n, i * k, k, False) for i in range(nb))
    F = sum(f_alg(n, i * k, k, False) for i in range(nb))
    I = torch.eye(K, dtype=torch.float64, device=dev)
    check = {"loo": float(torch.linalg.matrix_norm(Q.T @ Q - I, ord=2)),
             "resid_fro": float(torch.linalg.norm(A - Q @ R) / torch.linalg.norm(A))}
    if rank == 0:
        line = {
            "metric": METRIC, "value": B * ws / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (fp64-accurate; products on bf16 tensor cores)", "data": "synthetic",
            "config": {"workload": desc, "n": n, "blocks": [k] * nb, "B_alg": B, "F_alg": F,
                       "l2": "inputs larger than L2", "parallelism": "replicas" if ws > 1 else "single GPU"},
            "tflops": F / (ms * 1e-3) / 1e12, "clocks": clocks, "check": check,
            "gpu_launches": blk.kernel_launches * args.steps,
        }
        print(json.dumps(line), flush=True)
    return 0


def c4_compare(dev, prec, steps, warmup, tune=True, ws=1):
    """C4: the 256-problem batch as one tho_orth_batched graph replay, against
    the same problems looped through tho_orth (one plan each).  Returns a dict
    with both times, the speed-up, the launches and the tuning (search untimed)."""
    import torch
    from paper_2602_14449_gb300 import inputs, tho
    shapes = inputs.batched_shapes()
    probs = inputs.batched_problems(shapes, device=dev)
    pairs = [(p.V, p.A) for p in probs]
    outs = [(torch.empty_strided((n, k), (1, n), dtype=torch.float64, device=dev),
             torch.empty_strided((k, k), (1, k), dtype=torch.float64, device=dev),
             torch.empty_strided((k0, k), (1, k0), dtype=torch.float64, device=dev)) for (n, k0, k) in shapes]
    # Partition of the batch plan from the autotuner (untimed; synthetic
    # operands of the same shapes); the looped comparator keeps the defaults.
    tuning, tune_info = None, {"autotuned": False}
    if tune:
        t0 = time.time()
        tuning, tune_ms = tho.autotune(shapes, torch.float64, prec)
        tune_info = {"autotuned": True, "search_s": round(time.time() - t0, 2), "search_ms_per_call": tune_ms}
    bplan = tho.Plan(shapes, torch.float64, prec, tuning=tuning)
    tune_info.update(zip(("leaf_rows", "split_chunks", "balance"), bplan.tuning))
    lplans = [tho.Plan([s], torch.float64, prec) for s in shapes]
    stream = torch.cuda.current_stream(dev)

    def batched():
        tho.orth_batched(pairs, prec=prec, plan=bplan, outs=outs)

    def looped():
        for (V, A), pl, (Q, R, S) in zip(pairs, lplans, outs):
            tho.orth(V, A, prec=prec, plan=pl, Q=Q, R=R, S=S)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(e0.elapsed_time(e1), dev) / steps

    smi_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(dev.index)).split(",")[0] if ws == 1 else str(dev.index)
    sampler = ClockSampler(smi_index)
    sampler.start()
    ms_b = timed(batched)
    clocks = sampler.stop()
    ms_l = timed(looped)
    B = sum(b_alg(n, k0, k, False) for (n, k0, k) in shapes)
    F = sum(f_alg(n, k0, k, False) for (n, k0, k) in shapes)
    res = {"problems": len(shapes), "rows_total": sum(s[0] for s in shapes), "B_alg": B, "F_alg": F,
           "precision": "fp64" if prec == 0 else "fp64-accurate (products on bf16 tensor cores)",
           "batched": {"ms": ms_b, "gbs": B / (ms_b * 1e-3) / 1e9, "tflops": F / (ms_b * 1e-3) / 1e12,
                       "launches": bplan.kernel_launches, "tuning": tune_info},
           "looped": {"ms": ms_l, "gbs": B / (ms_l * 1e-3) / 1e9, "tflops": F / (ms_l * 1e-3) / 1e12,
                      "launches": sum(p.kernel_launches for p in lplans)},
           "speedup_batched_vs_looped": ms_l / ms_b, "clocks": clocks,
           "timing": f"CUDA events, {warmup} warm-up and {steps} timed repetitions of each form"}
    for pl in lplans:
        pl.close()
    bplan.close()
    return res


def run_batched(args):
    """C4 as its own bench line (batched vs looped)."""
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2602_14449_gb300 import tho
    tho.load()
    prec = WORKLOADS[args.workload][5]
    r = c4_compare(dev, prec, args.steps, args.warmup, tune=not args.no_tune, ws=ws)
    ms_b = r["batched"]["ms"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": r["B_alg"] * ws / (ms_b * 1e-3) / 1e9, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == 0 else "f64 (fp64-accurate; products on bf16 tensor cores)",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][6], "problems": r["problems"],
                       "rows_total": r["rows_total"], "B_alg": r["B_alg"], "F_alg": r["F_alg"],
                       "l2": "inputs larger than L2", "parallelism": "replicas" if ws > 1 else "single GPU"},
            "batched": r["batched"], "looped": r["looped"],
            "speedup_batched_vs_looped": r["speedup_batched_vs_looped"],
            "clocks": r["clocks"], "gpu_launches": r["batched"]["launches"] * args.steps,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _torch_composition(V, A):
    """Algorithm 1 (choice 2 of P) as plain differentiable torch ops on the GPU:
    the comparator of the fused forward+adjoint (autograd through every step)."""
    import torch
    n, k0 = V.shape

    def hh(X):
        m, k = X.shape
        R, vs, bs = X, [], []
        for j in range(k):
            x = R[j:, j]
            alpha = torch.sqrt((x * x).sum())
            sg = torch.where(x[0] < 0, -1.0, 1.0)
            v = torch.cat([x[:1] + sg * alpha, x[1:]])
            b = 2.0 / (v * v).sum()
            R = torch.cat([R[:j], R[j:] - b * torch.outer(v, v @ R[j:])], 0)
            vs.append(v)
            bs.append(b)
        Qx = torch.eye(m, k, dtype=X.dtype, device=X.device)
        for j in reversed(range(k)):
            Qx = torch.cat([Qx[:j], Qx[j:] - bs[j] * torch.outer(vs[j], vs[j] @ Qx[j:])], 0)
        d = torch.where(torch.diagonal(R[:k]) < 0, -1.0, 1.0)
        return Qx * d, d[:, None] * torch.triu(R[:k])

    def solve_tri(Tm, B, lower):
        rows = [None] * Tm.shape[0]
        order = range(Tm.shape[0]) if lower else range(Tm.shape[0] - 1, -1, -1)
        for i in order:
            s = B[i]
            for j in (range(i) if lower else range(i + 1, Tm.shape[0])):
                s = s - Tm[i, j] * rows[j]
            rows[i] = s / Tm[i, i]
        return torch.stack(rows, 0)

    Q1, R1 = hh(V[:k0])
    T = torch.eye(k0, dtype=V.dtype, device=V.device) + R1.T
    W = torch.cat([-Q1, torch.zeros(n - k0, k0, dtype=V.dtype, device=V.device)], 0) - V
    Z = solve_tri(T.T, W.T @ A, lower=False)
    Ap = A - W @ Z
    Qb, _ = hh(Ap[k0:])
    E = torch.cat([torch.zeros(k0, A.shape[1], dtype=A.dtype, device=A.device), Qb], 0)
    Z2 = solve_tri(T, W.T @ E, lower=True)
    return E - W @ Z2


def _unfused_backward(V, A, Q, dQ):
    """Comparator of the fused adjoint: the same reverse-mode formulas (the
    derivative of Algorithm 1's map, second choice of P) as separate plain torch
    operations -- cuBLAS products over the n rows, the k0 x k0 and k x k
    factorizations, inverses and solves on the CPU.  Returns (dV, dA)."""
    import torch
    dev = V.device
    n, k0 = V.shape
    I0 = torch.eye(k0, dtype=V.dtype)
    Q1, R1 = torch.linalg.qr(V[:k0].cpu())
    sg = torch.where(torch.diagonal(R1) < 0, -1.0, 1.0).to(V.dtype)
    Q1, R1 = Q1 * sg, sg[:, None] * R1          # diag(R1) >= 0
    T = I0 + R1.T                              # lower triangular
    Wt = -Q1 - V[:k0].cpu()
    tt = lambda B: torch.linalg.solve_triangular(T.T, B, upper=True)   # T^{-T} B
    t1 = lambda B: torch.linalg.solve_triangular(T, B, upper=False)    # T^{-1} B
    V2, A1, A2, Qt, Q2, dQ1, dQ2 = V[k0:], A[:k0], A[k0:], Q[:k0], Q[k0:], dQ[:k0], dQ[k0:]
    Z = tt(Wt.T @ A1.cpu() - (V2.T @ A2).cpu())
    Z2 = tt(Q1.T @ Qt.cpu())                   # Q_1 = -Wtop Z2
    Y = tt(Wt.T @ dQ1.cpu() - (V2.T @ dQ2).cpu())
    Zd, Z2d, Yd = Z.to(dev), Z2.to(dev), Y.to(dev)
    Ap2 = A2 + V2 @ Zd                          # A'_2
    Qbar = Q2 - V2 @ Z2d                        # E_2
    R = torch.triu((Qbar.T @ Ap2).cpu())
    Xb = dQ2 + V2 @ Yd                          # (dQ - W Y)_2
    M = -(Xb.T @ Qbar).cpu()
    C = torch.tril(M) + torch.tril(M, -1).T    # copyltu
    Rinv = torch.linalg.solve_triangular(R, torch.eye(R.shape[0], dtype=R.dtype), upper=True)
    Abar = (Xb + Qbar @ C.to(dev)) @ Rinv.T.to(dev)
    Gb = t1((V2.T @ Abar).cpu())
    Gbd = Gb.to(dev)
    dA = torch.empty_like(A)
    dA[:k0] = (Wt @ Gb).to(dev)
    dA[k0:] = Abar - V2 @ Gbd
    dV = torch.empty_like(V)
    dV[k0:] = dQ2 @ Z2d.T + Qbar @ Yd.T + Abar @ Zd.T - A2 @ Gbd.T
    Wb = -dQ1.cpu() @ Z2.T + A1.cpu() @ Gb.T
    R1b = torch.triu((Y @ Z2.T - Z @ Gb.T).T)
    M1 = R1 @ R1b.T + Wb.T @ Q1                 # R1 R1bar^T - Q1bar^T Q1, Q1bar = -Wbar_top
    C1 = torch.tril(M1) + torch.tril(M1, -1).T
    R1inv = torch.linalg.solve_triangular(R1, I0, upper=True)
    dV[:k0] = (-Wb + (-Wb + Q1 @ C1) @ R1inv.T).to(dev)
    return dV, dA


def c5_compare(dev, steps, warmup):
    """C5 (n = 2^20, k0 = 64, k = 16): the fused forward + hand-written adjoint
    through the C ABI (autograd.Function) against (a) the plain tho_orth forward
    plus the same adjoint unfused into separate torch operations and (b)
    autograd through a torch-ops composition of Algorithm 1 on the same GPU."""
    import torch
    from paper_2602_14449_gb300 import inputs, tho
    from paper_2602_14449_gb300.autograd import two_stage_orth
    cid, n, k0, k, dt, prec, desc = WORKLOADS["c5"]
    p = inputs.config_problem(5, device=dev)
    V0, A0, dQ = p.V, p.A, p.dQ
    stream = torch.cuda.current_stream(dev)
    plan = tho.get_plan([(n, k0, k)], torch.float64)

    def fused():
        V = V0.detach().requires_grad_()
        A = A0.detach().requires_grad_()
        two_stage_orth(V, A).backward(dQ)
        return V.grad, A.grad

    def unfused():
        Q, _, _ = tho.orth(V0, A0, plan=plan, want_R=False, want_S=False)
        return _unfused_backward(V0, A0, Q, dQ)

    def composed():
        V = V0.detach().clone().requires_grad_()
        A = A0.detach().clone().requires_grad_()
        _torch_composition(V, A).backward(dQ)
        return V.grad, A.grad

    def timed(fn, nsteps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nsteps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / nsteps

    smi_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(dev.index)).split(",")[0]
    sampler = ClockSampler(smi_index)
    sampler.start()
    ms_f = timed(fused, steps, warmup)
    clocks = sampler.stop()
    ms_fwd = timed(lambda: tho.orth(V0, A0, plan=plan), steps, 1)
    ms_u = timed(unfused, steps, 1)
    ms_c = timed(composed, 1, 1)
    gVf, gAf = fused()
    gVu, gAu = unfused()
    gVc, gAc = composed()
    rel = lambda a, b: float((a - b).abs().max() / b.abs().max())
    B = b_alg(n, k0, k, False)
    return {"workload": desc, "n": n, "k0": k0, "k": k, "B_alg": B,
            "fused_fwd_bwd_ms": ms_f, "forward_only_ms": ms_fwd, "backward_ms": ms_f - ms_fwd,
            "plain_fwd_unfused_bwd_ms": ms_u, "speedup_fused_vs_unfused": ms_u / ms_f,
            "torch_composition_fwd_bwd_ms": ms_c, "speedup_fused_vs_composition": ms_c / ms_f,
            "grad_rel_diff_fused_vs_unfused": max(rel(gVf, gVu), rel(gAf, gAu)),
            "grad_rel_diff_fused_vs_composition": max(rel(gVf, gVc), rel(gAf, gAc)),
            "clocks": clocks, "launches_fused": plan.kernel_launches + 9,
            "timing": f"CUDA events, {warmup} warm-up and {steps} timed repetitions (composition: 1)"}


def run_adjoint(args):
    """C5 as its own bench line."""
    import torch
    ws, rank, local = _dist()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2602_14449_gb300 import tho
    tho.load()
    r = c5_compare(dev, args.steps, args.warmup)
    ms_f = r["fused_fwd_bwd_ms"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": r["B_alg"] / (ms_f * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_f, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": r["workload"], "n": r["n"], "k0": r["k0"], "k": r["k"],
                       "value_is": "B_alg of one forward / (forward+backward time)"},
            "gpu_launches": r["launches_fused"] * args.steps,
        }
        line.update({k: v for k, v in r.items() if k not in ("workload", "n", "k0", "k", "B_alg", "launches_fused")})
        print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2602_14449_gb300 import inputs, tho
    tho.load()
    wl = args.workload
    cid, n, k0, k, dt, prec, desc = WORKLOADS[wl]
    if args.rows:
        n = args.rows
        desc = desc.replace(f"n={WORKLOADS[wl][1]}", f"n={n}")
    cplx = dt == "complex128"
    p = inputs.config_problem(cid, n=n, device=dev)
    V, A = p.V, p.A
    tuning, tune_info = None, {"autotuned": False}
    if args.tune:  # untimed partition search on synthetic operands of this shape
        t0 = time.time()
        tuning, tune_ms = tho.autotune([(n, k0, k)], V.dtype, prec)
        tune_info = {"autotuned": True, "search_s": round(time.time() - t0, 2), "search_ms_per_call": tune_ms}
    plan = tho.Plan([(n, k0, k)], V.dtype, prec, 0, tuning=tuning)
    tune_info.update(zip(("leaf_rows", "split_chunks", "balance"), plan.tuning))
    Q = torch.empty_strided((n, k), (1, n), dtype=V.dtype, device=dev)
    R = torch.empty_strided((k, k), (1, k), dtype=V.dtype, device=dev)
    S = torch.empty_strided((k0, k), (1, k0), dtype=V.dtype, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        tho.orth(V, A, prec=prec, plan=plan, Q=Q, R=R, S=S)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    smi_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(dev.index)).split(",")[0] if ws == 1 else str(local)
    sampler = ClockSampler(smi_index)
    plan.set_phase_timing(True)
    plan.read_phase_timing()
    barrier()
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    barrier()
    el_ms = e0.elapsed_time(e1)
    phases = plan.read_phase_timing()
    plan.set_phase_timing(False)
    el_ms = max_over_ranks(el_ms, dev)
    ms_step = el_ms / args.steps
    B = b_alg(n, k0, k, cplx)
    value = replica_throughput(B, args.steps, ws, el_ms)

    # Roofline of the dominant kernel, from the live CUDA-event phase times.
    m = n - k0
    kernel_of = {"gram": "k_gram", "leaf": "k_leaf", "apply": "k_apply_gram", "update_q": "k_update_q"}
    if prec == 2:
        # Complex panels of k >= 24 take the leaf kernel with tensor-core trailing updates.
        kernel_of["leaf"] = "k_leaf_emu" if (cplx and k >= 24) else "k_leaf"
        dom = "leaf"
        nb = -(-m // plan.leaf_rows)
        flops_launch = LEAF_WY_QR_FLOPS(m, k, nb) * (4 if cplx else 1)
    else:
        dom = max(PHASE_FLOPS_PER_ROW, key=lambda ph: phases[ph][0])
        flops_launch = PHASE_FLOPS_PER_ROW[dom](k0, k) * m * (4 if cplx else 1)
    dom_ms, dom_groups = phases[dom]
    achieved = flops_launch / (dom_ms / dom_groups * 1e-3) / 1e12
    peak = FP32_PEAK_TFLOPS if prec == 1 else FP64_PEAK_TFLOPS
    tr_row = _traffic_for(kernel_of[dom] + ("@emu" if prec == 2 else ""))
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": (tr_row * m if tr_row is not None else None), "kernel": kernel_of[dom],
                "share_of_step": dom_ms / args.steps / ms_step,
                "peak_source": ("2 DFMA/clk/SM x 152 SMs x 2.07 GHz (nominal; probe 1.04, k_gram sustains 1.23)"
                                if prec != 1 else "FP32 FFMA measured by a one-off probe (of measured)")}
    roofline_tensor = None
    if prec == 2 and phases["update_q"][1] > 0:
        t_ms, t_groups = phases["update_q"]
        mma = EMU_UPDATE_MMA_FLOPS_PER_ROW(k0, k, cplx) * m / (t_ms / t_groups * 1e-3) / 1e12
        tpk, tsrc = _bf16_peak()
        roofline_tensor = {"bound": "tensor", "kernel": "k_update_umma", "achieved": mma,
                           "peak": tpk, "unit": "TFLOP/s (bf16 tcgen05)", "frac": mma / tpk,
                           "traffic": (lambda t: t * m if t is not None else None)(_traffic_for("k_update_umma@emu")),
                           "peak_source": tsrc}
    hbm, hbm_src = _hbm_peak()
    step_tflops = f_alg(n, k0, k, cplx) / (ms_step * 1e-3) / 1e12

    # End to end through the C ABI with host buffers (pinned), copies in the timed
    # region: tho_orth_host stages each call's problem in device buffers (two
    # sets, used alternately) and copies the outputs back; consecutive calls
    # overlap the copies with the previous computation.
    e2e = None
    if not args.no_e2e:
        hV = torch.empty_like(V, device="cpu").pin_memory()
        hA = torch.empty_like(A, device="cpu").pin_memory()
        hV.copy_(V)
        hA.copy_(A)
        hQ = torch.empty_strided((n, k), (1, n), dtype=V.dtype).pin_memory()
        hR = torch.empty_strided((k, k), (1, k), dtype=V.dtype).pin_memory()
        hS = torch.empty_strided((k0, k), (1, k0), dtype=V.dtype).pin_memory()
        ne2e = max(1, args.steps)

        def e2e_step():
            tho.orth_host(hV, hA, hQ, hR, hS, prec=prec, plan=plan)

        e2e_step()  # allocates the staging sets
        tho.orth_host_wait(plan)
        torch.cuda.synchronize(dev)
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(ne2e):
            e2e_step()
        tho.orth_host_wait(plan)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = max_over_ranks(f0.elapsed_time(f1), dev)
        esz = V.element_size()
        e2e = {"value": replica_throughput(B, ne2e, ws, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int((V.numel() + A.numel()) * esz),
               "d2h_bytes_per_step": int((n * k + k * k + k0 * k) * esz), "steps": ne2e,
               "ms_per_step": e2e_ms / ne2e, "api": "tho_orth_host (pinned host buffers)"}
        # The last call's outputs against the device result of the same inputs.
        e2e["max_abs_diff_vs_device_Q"] = float((hQ.to(dev) - tho.orth(V, A, prec=prec, plan=plan)[0]).abs().max())
        del hV, hA

    # Accuracy of the benchmarked output (outside the timed region).
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    check = {}
    try:
        import gpu_metrics
        Qc, Rc, Sc = tho.orth(V, A, prec=prec, plan=plan)
        check = {"loo": gpu_metrics.loo(V, Qc), "resid_fro": gpu_metrics.resid_fro(V, A, Qc, Rc, Sc)}
    except Exception as ex:  # the metric helper is optional for the bench line
        check = {"error": str(ex)}

    # The same workload with FP64 arithmetic throughout, in the same run.
    native = None
    if prec == 2 and not args.no_native:
        nplan = tho.Plan([(n, k0, k)], V.dtype, 0, 0)
        nplan.set_phase_timing(True)
        for _ in range(2):
            tho.orth(V, A, prec=0, plan=nplan, Q=Q, R=R, S=S)
        torch.cuda.synchronize(dev)
        nplan.read_phase_timing()
        nsteps = max(1, min(args.steps, 3))
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(nsteps):
            tho.orth(V, A, prec=0, plan=nplan, Q=Q, R=R, S=S)
        g1.record(stream)
        torch.cuda.synchronize(dev)
        nms = g0.elapsed_time(g1) / nsteps
        nph = nplan.read_phase_timing()
        lms, lgr = nph["leaf"]
        nleaf = PHASE_FLOPS_PER_ROW["leaf"](k0, k) * (n - k0) * (4 if cplx else 1) / (lms / lgr * 1e-3) / 1e12
        native = {"ms_per_step": nms, "value": B * ws / (nms * 1e-3) / 1e9, "unit": UNIT, "steps": nsteps,
                  "fp64_tflops": f_alg(n, k0, k, cplx) / (nms * 1e-3) / 1e12,
                  "roofline": {"bound": "alu", "kernel": "k_leaf", "achieved": nleaf, "peak": FP64_PEAK_TFLOPS,
                               "unit": "TFLOP/s", "frac": nleaf / FP64_PEAK_TFLOPS,
                               "traffic": (lambda t: t * (n - k0) if t is not None else None)(_traffic_for("k_leaf"))},
                  "phases_ms_per_step": {ph: v[0] / nsteps for ph, v in nph.items()}}
        nplan.close()

    # The benchmark spec's other two comparisons, on the same GPU in the same run
    # (headline workload only, one GPU): the batched form against looped
    # tho_orth calls (C4, in the headline's precision, autotuned partition with
    # the search untimed) and the fused forward + adjoint against the plain
    # forward plus the unfused adjoint and against a torch-ops composition (C5).
    extras = {}
    if ws == 1 and wl == "c3" and not args.no_extras and not args.rows:
        del Q, R, S
        extras["batched_c4"] = c4_compare(dev, prec, max(3, min(args.steps, 5)), 3, tune=True)
        extras["fwd_bwd_c5"] = c5_compare(dev, max(3, min(args.steps, 5)), 3)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, CPU_SAMPLE_ROWS[wl])

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": ("c128" if cplx else "f64") + {0: "", 1: " (fp32-bulk)", 2: " (fp64-accurate; products on bf16 tensor cores)"}[prec],
            "data": "synthetic",
            "config": {"workload": desc, "n": n, "k0": k0, "k": k,
                       "l2": f"inputs larger than L2 ({(V.numel() + A.numel()) * V.element_size() / 1e9:.1f} GB)",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": roofline, "roofline_tensor": roofline_tensor,
            "fp64_native": native,
            "hbm_roof": {"peak_gbs": hbm, "source": hbm_src, "frac_of_hbm": value / ws / hbm},
            "fp64_flop_roof": {"F_alg": f_alg(n, k0, k, cplx), "B_alg": B,
                               "t_roof_ms": max(f_alg(n, k0, k, cplx) / (FP64_PEAK_TFLOPS * 1e12),
                                                B / (hbm * 1e9)) * 1e3,
                               "step_over_roof_time": ms_step / (max(f_alg(n, k0, k, cplx) / (FP64_PEAK_TFLOPS * 1e12),
                                                                    B / (hbm * 1e9)) * 1e3),
                               "note": "t_roof = max(F_alg / FP64 peak, B_alg / HBM): the roof of an FP64-arithmetic "
                                       "path; the emulated products run on tensor cores, so their step can be "
                                       "shorter than this roof (ratio < 1)",
                               "f_alg_rate_tflops": step_tflops},
            "columns_per_s": k * ws * args.steps / (el_ms * 1e-3),
            "phases_ms_per_step": {ph: v[0] / args.steps for ph, v in phases.items()},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, **extras,
            "gpu_launches": plan.kernel_launches * args.steps, "check": check, "tuning": tune_info,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--rows", type=int, default=0, help="override n (smaller problem of the same structure)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-native", action="store_true", help="skip the FP64-arithmetic comparison run")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline line without the batched (C4) and forward+backward (C5) comparisons")
    ap.add_argument("--tune", action="store_true",
                    help="single-problem workloads: time the autotuned partition instead of the default")
    ap.add_argument("--no-tune", action="store_true", help="batched workloads: time the default partition")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("c4", "c4-emu"):
        return run_batched(args)
    if args.workload == "blocks":
        return run_blocks(args)
    if args.workload == "c5":
        return run_adjoint(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
