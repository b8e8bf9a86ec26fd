#!/usr/bin/env python
"""Benchmark of GB300 CholeskyQR2 (Hutter & Solomonik, arXiv 1710.08471).

Default workload (one step = one CholeskyQR2 factorization, Algorithm CQR2):
FP64 A = G diag(sigma) V with m = 2^23, n = 128, sigma log-spaced 1 .. 1e-6
(kappa ~ 1e6), fused pass-1 Q-form / pass-2 Gram. The metric is TFLOP/s at
the paper's nominal 4 m n^2 + 5 n^3 / 3 flops (Section IV), with the roofline
fraction of the dominant kernel and the three error norms against the CPU
FP64 oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload tall|small|square|wide512] [--variant fused|plain]

Timing: inputs (8.6 GB) are larger than L2 (129 MB), so L2 is not flushed.
Device time comes from CUDA events on the plan's stream; the end-to-end
number goes through the host-buffer C entry point with pinned buffers. With
N > 1 (torchrun) each rank factors its own matrix (replicas, weak scaling);
the timed region is bracketed by barriers and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOADS = {
    # name: (m, n, kappa, seed, description)
    "tall": (1 << 23, 128, 1e6, 1, "FP64 CholeskyQR2, m=2^23 n=128 (8.6 GB), A=G diag(sigma) V, kappa=1e6"),
    "small": (4096, 64, None, 0, "FP64 CholeskyQR2, m=4096 n=64, iid N(0,1), kappa~1.3"),
    "square": (65536, 8192, 1e4, 2, "FP64 CholeskyQR2, m=65536 n=8192 (4.3 GB), kappa=1e4"),
    "wide512": (1 << 21, 512, 1e6, 3, "FP64 CholeskyQR2, m=2^21 n=512 (8.6 GB), kappa=1e6"),
    # profiling size: larger than L2, a few GB on the device
    "mid": (1 << 20, 128, 1e6, 1, "FP64 CholeskyQR2, m=2^20 n=128 (1.07 GB), kappa=1e6"),
    # many small problems in one grouped launch (one step = one batch call)
    "batch": (4096, 32, None, 5, "grouped batch: 1024 FP64 CholeskyQR2 problems, m=4096 n=32 each (1.07 GB), "
                                 "iid N(0,1)"),
}
BATCH_COUNT = 1024

# GB300 FP64: 2 DFMA per clock per SM (one warp instruction every 16 clocks
# per SM partition), 152 SMs, 2 flops per FMA, at the maximum SM clock.
FP64_FMA_PER_CLK_PER_SM = 2
GB300_SMS = 152

# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu
# capture (`profiles/`), keyed by kernel, workload and a hash of the kernel's
# source file, so that an entry lapses (null) once the kernel changes. The
# "tall" entries were captured on "mid" (2^20 of the 2^23 rows) and scaled by
# the row count: these kernels stream their operands once per launch.
NCU_TRAFFIC = {
    "k_qform_gram_small@mid@32201450a5426255": 2145473280,
    "k_qform_gram_small@tall@32201450a5426255": 17163786240,
    "k_ozaki_gemm<7,QFORM>@mid@f33dc9b14d75de37": 2938640128,
    "k_ozaki_gemm<7,QFORM>@tall@f33dc9b14d75de37": 23509121024,
    "k_ozaki_gemm<7,GRAM>@mid@f33dc9b14d75de37": 1892780800,
    "k_ozaki_gemm<7,GRAM>@tall@f33dc9b14d75de37": 15142246400,
    "k_cqr2_small_batched@batch@c56aa36f0d944e5a": 5306968320,
}


def nominal_flops(m: int, n: int) -> float:
    return 4.0 * m * n * n + 5.0 * n ** 3 / 3.0


def src_sha(name: str) -> str:
    p = os.path.join(ROOT, "paper_1710_08471_gb300", "csrc", name)
    with open(p, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


# ------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ helpers

def make_input(m: int, n: int, kappa, seed: int, pinned: bool):
    import torch

    if pinned:
        t = torch.empty((n, m), dtype=torch.float64, pin_memory=True)
        A = t.numpy().T  # Fortran-ordered (m, n) view of pinned memory
    else:
        t = None
        A = np.empty((m, n), dtype=np.float64, order="F")
    synth.make_matrix(m, n, kappa, seed, out=A)
    return A, t


def pinned_colmajor(m: int, n: int):
    import torch

    t = torch.empty((n, m), dtype=torch.float64, pin_memory=True)
    return t.numpy().T, t


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def allreduce_max(x: float, ws: int) -> float:
    """Largest value over the ranks (host-side timing aggregation only; the
    factorizations themselves exchange nothing)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ws: int, flops_per_replica: float, ms_local: float) -> tuple[float, float]:
    """Whole-job TFLOP/s of ws independent replicas timed by the slowest rank:
    (value, ms_per_step)."""
    ms = allreduce_max(ms_local, ws)
    return ws * flops_per_replica / (ms * 1e-3) / 1e12, ms


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def cpu_cores() -> int:
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        v = os.environ.get(var)
        if v and v.isdigit():
            return int(v)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle_sample(A_full: np.ndarray, budget_rows: int):
    """Time the CPU oracle on the first `budget_rows` rows of the workload."""
    import oracle

    ms = min(A_full.shape[0], budget_rows)
    As = np.asfortranarray(A_full[:ms]) if ms < A_full.shape[0] else A_full
    t0 = time.perf_counter()
    Q, R = oracle.cqr2(As)
    dt = time.perf_counter() - t0
    return ms, dt, Q, R


# ------------------------------------------------------------- arms

def workload_config(args, ws: int) -> dict:
    """The bench line's config, the same for both arms."""
    m, n, kappa, seed, desc = WORKLOADS[args.workload]
    fused = args.variant == "fused" and args.precision == "fp64"
    return {"workload": desc, "m": m, "n": n, "kappa": kappa, "precision": args.precision,
            "variant": "fused" if fused else "plain", "inverse_depth": args.inverse_depth, "graph": args.graph,
            "parallelism": f"replicas{ws}" if ws > 1 else "single",
            "l2": ("512 MB buffer rewritten between steps (outside the timed events)" if needs_flush(m, n)
                   else f"inputs {m * n * 8 / 1e9:.1f} GB > 129 MB L2 (no flush)")}


def needs_flush(m: int, n: int) -> bool:
    """An input that fits in L2 (129 MB) would stay there from one step to
    the next: such workloads rewrite a 512 MB buffer between timed steps."""
    return m * n * 8 <= 129 * 2**20


def bench_reference(args, ws, rank):
    """The CPU FP64 oracle on the host cores (the reference arm)."""
    m, n, kappa, seed, desc = WORKLOADS[args.workload]
    if rank != 0:
        return
    if args.workload == "batch":
        return bench_reference_batch(args, ws)
    rows = min(m, args.oracle_rows or (1 << 21))
    A, _ = make_input(rows, n, kappa, seed, pinned=False)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        import oracle

        oracle.cqr2(A)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    fl = nominal_flops(rows, n)
    val = fl / (ms * 1e-3) / 1e12
    sample = f"first {rows} of {m} rows of the workload ({desc}); numpy FP64 oracle"
    line = {
        "impl": "reference", "metric": "CQR2 TFLOP/s (nominal 4mn^2+5n^3/3)", "value": val, "unit": "TFLOP/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(args, ws), sampled_rows=rows),
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_config(args, ws: int) -> dict:
    m, n, kappa, seed, desc = WORKLOADS["batch"]
    return {"workload": desc, "m": m, "n": n, "count": BATCH_COUNT, "precision": "fp64", "variant": "grouped",
            "parallelism": f"replicas{ws}" if ws > 1 else "single",
            "l2": f"inputs {BATCH_COUNT * m * n * 8 / 1e9:.2f} GB > 129 MB L2 (no flush)"}


def bench_reference_batch(args, ws):
    """The oracle on a bounded sample of the batch's problems."""
    import oracle

    m, n, kappa, seed, desc = WORKLOADS["batch"]
    count = min(BATCH_COUNT, args.oracle_rows or 64)  # problems per step
    A = synth.make_matrix(count * m, n, kappa, seed)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for p in range(count):
            oracle.cqr2(np.asfortranarray(A[p * m:(p + 1) * m]))
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    val = count * nominal_flops(m, n) / (ms * 1e-3) / 1e12
    sample = f"{count} of the {BATCH_COUNT} problems per step ({desc}); numpy FP64 oracle, one problem at a time"
    line = {
        "impl": "reference", "metric": "CQR2 TFLOP/s (nominal 4mn^2+5n^3/3)", "value": val, "unit": "TFLOP/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(batch_config(args, ws), sampled_problems=count),
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bench_batch(args, ws, rank, local):
    """The batch workload as the bench line."""
    out = measure_batch(args.steps, args.warmup, ws, rank, local, args.quick)
    if rank == 0:
        print(json.dumps(out), flush=True)


def measure_batch(steps: int, warmup: int, ws: int, rank: int, local: int, quick: bool) -> dict:
    """One step = one cqr2_batch_factor call over BATCH_COUNT problems, all
    routed to the persistent grouped kernel, replayed from a captured graph."""
    import torch

    import paper_1710_08471_gb300 as cq

    m, n, kappa, seed, desc = WORKLOADS["batch"]
    count = BATCH_COUNT
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hA, hA_t = make_input(count * m, n, kappa, seed + 1000 * rank, pinned=True)
    A = cq.empty_colmajor(count * m, n, device=dev)
    A.t().copy_(hA_t.to(dev, non_blocking=True))
    Q = cq.empty_colmajor(count * m, n, device=dev)
    R = cq.empty_colmajor(n, count * n, device=dev)
    probs = [(A[i * m:(i + 1) * m], Q[i * m:(i + 1) * m], R[:, i * n:(i + 1) * n]) for i in range(count)]
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    batch = cq.Batch(count, stream=stream, graph=True, small_work_limit=m * n * n)
    desc_arr = batch.descriptors(probs)
    infos = batch.factor(desc_arr)
    if any(i.status != 0 for i in infos):
        raise SystemExit("batch factorization failed")
    for _ in range(warmup):
        batch.factor(desc_arr, sync=False)
    batch.info()
    torch.cuda.synchronize()
    barrier(ws)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = cq.cqr2_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        batch.factor(desc_arr, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = cq.cqr2_launch_count() - l0
    barrier(ws)
    ms_local = e0.elapsed_time(e1) / steps
    flops = count * nominal_flops(m, n)
    value, ms_step = replica_throughput(ws, flops, ms_local)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    fp64_pk = FP64_FMA_PER_CLK_PER_SM * 2 * GB300_SMS * sm_max * 1e6 / 1e12
    achieved = flops / (ms_local * 1e-3) / 1e12
    out = {
        "metric": "CQR2 TFLOP/s (nominal 4mn^2+5n^3/3)", "value": value, "unit": "TFLOP/s", "n_gpus": ws,
        "steps": steps, "warmup": warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": batch_config(None, ws),
        "gpu_launches": launches,
        "qr_per_s": ws * count / (ms_step * 1e-3),
        "roofline": {"bound": "alu", "kernel": "k_cqr2_small_batched", "stage": "batch", "achieved": achieved,
                     "peak": fp64_pk, "unit": "TFLOP/s", "frac": achieved / fp64_pk,
                     "traffic": NCU_TRAFFIC.get(f"k_cqr2_small_batched@batch@{src_sha('batched.cu')}"),
                     "peak_note": f"derived FP64 DFMA peak: {FP64_FMA_PER_CLK_PER_SM} FMA/clk/SM x 152 SMs x 2 "
                                  f"flops x {sm_max:.0f} MHz; work = nominal flops of every problem"},
        "clocks": clk,
    }
    if rank == 0 and not quick:
        import oracle

        # errors on a sample of problems against the oracle, and the CPU baseline
        sample = list(range(0, count, count // 8))
        errs = []
        t_cpu = 0.0
        for i in sample:
            Ai = np.asfortranarray(hA[i * m:(i + 1) * m])
            Qi = probs[i][1].cpu().numpy()
            Ri = probs[i][2].cpu().numpy()
            t0 = time.perf_counter()
            Qo, Ro = oracle.cqr2(Ai)
            t_cpu += time.perf_counter() - t0
            errs.append({"orthogonality": oracle.orthogonality(Qi), "residual": oracle.residual(Ai, Qi, Ri),
                         "R_rel_vs_oracle": oracle.rel_error(np.asfortranarray(Ri), Ro)})
        out["errors"] = {k: max(e[k] for e in errs) for k in errs[0]}
        out["errors"]["problems_checked"] = len(sample)
        out["cpu_baseline"] = {"value": len(sample) * nominal_flops(m, n) / t_cpu / 1e12, "unit": "TFLOP/s",
                               "cores": cpu_cores(), "kind": "oracle", "seconds": t_cpu,
                               "sample": f"{len(sample)} of the {count} problems ({desc}); numpy FP64 oracle"}
        # end to end: every problem's A in from pinned host memory, Q and R
        # back, around the same batch call
        hQ_t = torch.empty((n, count * m), dtype=torch.float64, pin_memory=True)
        hR_t = torch.empty((count * n, n), dtype=torch.float64, pin_memory=True)
        times = []
        for _ in range(max(2, steps // 2)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                A.t().copy_(hA_t, non_blocking=True)
                batch.factor(desc_arr, sync=False)
                hQ_t.copy_(Q.t(), non_blocking=True)
                hR_t.copy_(R.t(), non_blocking=True)
            stream.synchronize()
            times.append(time.perf_counter() - t0)
        batch.info()
        e2e_ms = 1e3 * statistics.median(times)
        out["e2e"] = {"value": flops / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": e2e_ms,
                      "h2d_bytes_per_step": count * m * n * 8, "d2h_bytes_per_step": count * (m * n + n * n) * 8,
                      "api": "cqr2_batch_factor with pinned host copies on the batch stream"}
    batch.close()
    return out


PRECISIONS = {"fp64": 0, "ozaki": 1, "ozaki6": 2}
SLICES = {"fp64": 0, "ozaki": 7, "ozaki6": 6}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16": float(d["bf16_tflops"]),
                "bf16_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "src": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "src": "fallback"}


def stage_work(m: int, n: int, precision: str, fused: bool) -> dict:
    """Algorithmic work per stage instance: FP64 flops (native) or BF16
    tensor-core flops of the kept slice products (split precision)."""
    S = SLICES[precision]
    tri = m * n * (n + 1)  # one Syrk or one triangular Q-form, 2 flops per FMA
    if S == 0:
        return {"gram1": tri, "qform1": 2 * tri if fused else tri, "gram2": 0 if fused else tri, "qform2": tri,
                "cholinv1": 2 * n ** 3 / 3, "cholinv2": 2 * n ** 3 / 3, "trmm": n ** 3 / 3}
    P = S * (S + 1) // 2
    ntj = -(-n // 64)
    np_ = ntj * 64
    ntiles = sum(ntj - 2 * i for i in range(ntj) if 2 * i < ntj)
    gram = ntiles * 2 * 128 * 64 * m * P
    qform = 2 * 128 * 64 * P * (-(-m // 128)) * sum(min(64 * (j + 1), np_) for j in range(ntj))
    return {"gram1": gram, "gram2": gram, "qform1": qform, "qform2": qform}


def fp64_peak(clk: dict) -> float:
    """Derived FP64 peak in TFLOP/s at the sampled maximum SM clock."""
    sm_max = clk.get("sm_max_mhz") or 2070.0
    return FP64_FMA_PER_CLK_PER_SM * 2 * GB300_SMS * sm_max * 1e6 / 1e12


def roofline_of(per_stage: dict, m: int, n: int, precision: str, fz: bool, clk: dict, workload: str,
                peaks: dict) -> dict:
    """Roofline of the dominant stage: its algorithmic work per launch over
    its CUDA-event time, against the FP64 peak (native) or the sustained BF16
    tensor peak (split precision)."""
    work = stage_work(m, n, precision, fz)
    cands = {k: v for k, v in per_stage.items() if k in work and work[k] > 0}
    dom = max(cands, key=cands.get)
    achieved = work[dom] / (per_stage[dom] * 1e-3) / 1e12
    if SLICES[precision] == 0:
        sm_max = clk.get("sm_max_mhz") or 2070.0
        peak = fp64_peak(clk)
        if n <= 256:
            kern = {"qform1": "k_qform_gram_small" if fz else "k_qform_small", "gram1": "k_gram_tile",
                    "gram2": "k_gram_tile", "qform2": "k_qform_small"}.get(dom, dom)
        else:
            kern = {"qform1": "k_gemm_f64", "qform2": "k_gemm_f64", "gram1": "k_gram_tile",
                    "gram2": "k_gram_tile"}.get(dom, dom)
        kfile = {"k_gemm_f64": "gemm.cu", "k_gram_tile": "gram.cu"}.get(kern, "qform.cu")
        note = f"derived FP64 DFMA peak: {FP64_FMA_PER_CLK_PER_SM} FMA/clk/SM x 152 SMs x 2 flops x {sm_max:.0f} MHz"
        bound = "alu"
    else:
        peak = peaks["bf16_sustained"]
        kern = "k_ozaki_gemm<%d,%s>" % (SLICES[precision], "GRAM" if dom.startswith("gram") else "QFORM")
        kfile = "ozaki.cu"
        note = f"{peaks['src']} sustained bf16 tensor peak; work = BF16 flops of the kept slice products"
        bound = "tensor"
    traffic = NCU_TRAFFIC.get(f"{kern}@{workload}@{src_sha(kfile)}")
    return {"bound": bound, "kernel": kern, "stage": dom, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic, "peak_note": note}


def step_roofline(m: int, n: int, precision: str, fz: bool, ms_step: float, clk: dict, peaks: dict) -> dict:
    """The whole step against its roofline: max(compulsory bytes / HBM,
    work / the pipes' peaks) over the measured time. Compulsory bytes: the 4
    trips of an m x n FP64 matrix (32mn: A in and Q out, twice). Work:
    nominal FP64 flops at the FP64 peak, or, for split precision, the kept
    slice products at the sustained BF16 peak plus CholInv and R2 R1 (FP64)
    at the FP64 peak."""
    fp64 = fp64_peak(clk) * 1e12
    t_bw = 32.0 * m * n / (peaks["hbm_gbs"] * 1e9) * 1e3
    if SLICES[precision] == 0:
        t_fl = nominal_flops(m, n) / fp64 * 1e3
        pipe = "fp64"
    else:
        tensor = sum(stage_work(m, n, precision, fz).values())
        t_fl = (tensor / (peaks["bf16_sustained"] * 1e12) + (4 * n ** 3 / 3 + n ** 3 / 3) / fp64) * 1e3
        pipe = "bf16 tensor + fp64"
    rt = max(t_bw, t_fl)
    return {"t_hbm_ms": t_bw, "t_compute_ms": t_fl, "compute_pipe": pipe,
            "bound": "hbm" if t_bw >= t_fl else "compute", "roofline_ms": rt, "frac": rt / ms_step,
            "peaks": peaks["src"]}


def timed_plan(pl, A, Q, R, stream, steps: int, warmup: int, profile: bool, ws: int = 1, flush=None):
    """CUDA-event time per factorization on the plan's stream (ms), kernel
    launches in the timed region, and per-stage ms when profiling. With
    `flush` (a device buffer larger than L2) every step is timed alone with
    the buffer rewritten between steps, outside the timed events."""
    import torch

    import paper_1710_08471_gb300 as cq

    info = pl.factor(A, Q, R, sync=True)[2]
    if info.status != 0:
        raise SystemExit(f"factorization failed: status {info.status}")
    for _ in range(max(3, warmup)):
        pl.factor(A, Q, R, sync=False)
    torch.cuda.synchronize()
    barrier(ws)
    pl.set_profiling(profile)
    l0 = cq.cqr2_launch_count()
    if flush is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            pl.factor(A, Q, R, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
    else:
        evs = []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.add_(1.0)  # rewrite a buffer larger than L2
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pl.factor(A, Q, R, sync=False)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    launches = cq.cqr2_launch_count() - l0
    barrier(ws)
    st = pl.stage_times() if profile else None
    pl.set_profiling(False)
    # per step: a stage that runs several times in one factorization (the
    # split-precision slicing) is summed over its occurrences
    return ms, launches, {k: v[0] / steps for k, v in st.items() if v[1] > 0} if st else {}


def oracle_seconds_one_core(m: int, n: int, kappa, seed: int, repeats: int = 5) -> float | None:
    """Median seconds of the CPU oracle's CQR2 on one core (a child process
    with one BLAS thread), or None if that could not be run."""
    code = ("import sys, time, statistics; sys.path.insert(0, %r); import synth, oracle; "
            "A = synth.make_matrix(%d, %d, %r, %d, threads=1); ts = []\n"
            "for _ in range(%d):\n t0 = time.perf_counter(); oracle.cqr2(A); ts.append(time.perf_counter() - t0)\n"
            "print(statistics.median(ts))") % (ROOT, m, n, kappa, seed, repeats)
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300, env=env)
        return float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        return None


def fp64_gemm_probe(dev) -> dict:
    """A measured FP64 reference beside the derived DFMA peak: cuBLAS DGEMM
    (torch.matmul, float64) on 8192 x 8192 operands, best of 3 after one
    warm-up, CUDA events."""
    import torch

    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    torch.cuda.empty_cache()
    return {"cublas_dgemm_tflops": 2.0 * n ** 3 / (best * 1e-3) / 1e12, "n": n, "ms": best}


def bench_configs(steps: int, warmup: int, local: int, peaks: dict, clk: dict, serving_pool=None) -> dict:
    """The other configurations of the benchmark plan, measured in the same
    run (device-timed with CUDA events, errors against the CPU oracle):
    - small (4096 x 64, the latency-bound case), replayed from a CUDA graph,
      L2 rewritten between steps (its 2 MB input fits in L2);
    - wide512 (2^21 x 512, kappa 1e6), native FP64 and split precision (S = 7)
      at the same shape;
    - 8192 x 4096 (kappa 1e4), plain CholeskyQR2 against column panels of 512;
    - batch (1024 problems of 4096 x 32 in one grouped launch per step);
    - the 20,000-request least-squares stream at 2000 requests/s, split
      precision, continuous batching against one request at a time."""
    import torch

    import oracle
    import paper_1710_08471_gb300 as cq

    dev = torch.device("cuda", local)
    out = {}

    def errs(hA, Q, R, Ro):
        hQ = np.asfortranarray(Q.cpu().numpy())
        hR = np.asfortranarray(R.cpu().numpy())
        e = {"orthogonality": oracle.orthogonality(hQ), "residual": oracle.residual(hA, hQ, hR)}
        if Ro is not None:
            e["R_rel_vs_oracle"] = oracle.rel_error(hR, Ro)
        return e

    # ---- small: 4096 x 64, FP64, fused, graph-replayed
    try:
        m, n, kappa, seed, desc = WORKLOADS["small"]
        hA = synth.make_matrix(m, n, kappa, seed)
        A = cq.colmajor(torch.from_numpy(np.ascontiguousarray(hA.T)).to(dev).t())
        Q, R = cq.empty_colmajor(m, n, device=dev), cq.empty_colmajor(n, n, device=dev)
        stream = torch.cuda.Stream(device=dev)
        flush = torch.zeros(64 << 20, dtype=torch.float64, device=dev)  # 512 MB > L2
        res = {"workload": desc, "m": m, "n": n, "precision": "fp64", "variant": "fused", "graph": True,
               "l2": "512 MB buffer rewritten between steps (outside the timed events)"}
        with cq.Plan(m, n, fused=True, stream=stream, graph=True) as pl:
            ms, launches, _ = timed_plan(pl, A, Q, R, stream, max(20, steps), warmup, False, flush=flush)
            with cq.Plan(m, n, fused=True, stream=stream) as pe:
                ms_eager, _, st = timed_plan(pe, A, Q, R, stream, max(20, steps), warmup, True, flush=flush)
        del flush
        t0 = time.perf_counter()
        Qo, Ro = oracle.cqr2(hA)
        fl = nominal_flops(m, n)
        pk = fp64_peak(clk)
        res.update({"ms_per_step": ms, "tflops": fl / (ms * 1e-3) / 1e12, "gpu_launches_per_step": launches / max(20, steps),
                    "eager_ms_per_step": ms_eager, "eager_stages_ms": {k: round(v, 4) for k, v in st.items()},
                    "roofline": {"bound": "alu", "achieved": fl / (ms * 1e-3) / 1e12, "peak": pk, "unit": "TFLOP/s",
                                 "frac": fl / (ms * 1e-3) / 1e12 / pk,
                                 "note": "nominal flops of the whole step over the derived FP64 peak; the step is "
                                         "latency-bound (two one-CTA CholInv base cases on its critical path)"},
                    "errors": dict(errs(hA, Q, R, Ro), oracle_orthogonality=oracle.orthogonality(Qo))})
        ts = []
        for _ in range(5):
            t0 = time.perf_counter()
            oracle.cqr2(hA)
            ts.append(time.perf_counter() - t0)
        t1 = oracle_seconds_one_core(m, n, kappa, seed)
        res["cpu_baseline"] = {"value": fl / statistics.median(ts) / 1e12, "unit": "TFLOP/s", "cores": cpu_cores(),
                               "kind": "oracle", "sample": "full workload, median of 5",
                               "one_core_tflops": fl / t1 / 1e12 if t1 else None}
        out["small"] = res
    except Exception as ex:  # a configuration must not cost the main line
        out["small"] = {"error": repr(ex)}
    torch.cuda.empty_cache()

    # ---- wide512: 2^21 x 512, kappa 1e6, native FP64 against split precision
    try:
        m, n, kappa, seed, desc = WORKLOADS["wide512"]
        hA = synth.make_matrix(m, n, kappa, seed)
        A = cq.colmajor(torch.from_numpy(np.ascontiguousarray(hA.T)).to(dev).t())
        Q, R = cq.empty_colmajor(m, n, device=dev), cq.empty_colmajor(n, n, device=dev)
        stream = torch.cuda.current_stream()
        res = {"workload": desc, "m": m, "n": n, "kappa": kappa, "l2": "inputs 8.6 GB > 129 MB L2 (no flush)"}
        fl = nominal_flops(m, n)
        runs = {}
        for name, prec, nsteps in (("fp64", "fp64", 3), ("ozaki7", "ozaki", max(5, steps))):
            with cq.Plan(m, n, precision=PRECISIONS[prec], stream=stream) as pl:
                ms, launches, st = timed_plan(pl, A, Q, R, stream, nsteps, warmup, True)
            runs[name] = {"ms_per_step": ms, "tflops": fl / (ms * 1e-3) / 1e12, "steps": nsteps,
                          "stages_ms": {k: round(v, 4) for k, v in st.items()},
                          "roofline": roofline_of(st, m, n, prec, False, clk, "wide512", peaks),
                          "step_roofline": step_roofline(m, n, prec, False, ms, clk, peaks),
                          "errors": errs(hA, Q, R, None)}
        t0 = time.perf_counter()
        Qo, Ro = oracle.cqr2(hA)
        dt = time.perf_counter() - t0
        for name, prec in (("fp64", "fp64"), ("ozaki7", "ozaki")):
            with cq.Plan(m, n, precision=PRECISIONS[prec], stream=stream) as pl:
                pl.factor(A, Q, R, sync=True)
            hR = np.asfortranarray(R.cpu().numpy())
            runs[name]["errors"]["R_rel_vs_oracle"] = oracle.rel_error(hR, Ro)
        runs["oracle"] = {"orthogonality": oracle.orthogonality(Qo), "residual": oracle.residual(hA, Qo, Ro)}
        del Qo
        res.update(runs)
        res["split_speedup_vs_fp64"] = runs["fp64"]["ms_per_step"] / runs["ozaki7"]["ms_per_step"]
        res["cpu_baseline"] = {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                               "sample": "full workload, one run", "seconds": dt}
        out["wide512"] = res
        del A, Q, R, hA
    except Exception as ex:
        out["wide512"] = {"error": repr(ex)}
    torch.cuda.empty_cache()

    # ---- near-square: 8192 x 4096, plain CholeskyQR2 against panels of 512
    try:
        m, n, kappa, b = 8192, 4096, 1e4, 512
        hA = synth.make_matrix(m, n, kappa, 6)
        A = cq.colmajor(torch.from_numpy(np.ascontiguousarray(hA.T)).to(dev).t())
        Q, R = cq.empty_colmajor(m, n, device=dev), cq.empty_colmajor(n, n, device=dev)
        stream = torch.cuda.current_stream()
        fl = nominal_flops(m, n)
        res = {"workload": "FP64 CholeskyQR2, m=8192 n=4096 (268 MB), kappa=1e4, plain and on column panels",
               "m": m, "n": n, "kappa": kappa, "panel_width": b,
               "l2": "inputs 268 MB > 129 MB L2 (no flush)"}
        t0 = time.perf_counter()
        Qo, Ro = oracle.panel_cqr2(hA, b)
        res["cpu_baseline"] = {"value": fl / (time.perf_counter() - t0) / 1e12, "unit": "TFLOP/s",
                               "cores": cpu_cores(), "kind": "oracle", "sample": "full workload, panels, one run"}
        for name, width in (("plain", 0), ("panels", b)):
            with cq.Plan(m, n, stream=stream) as pl:
                pl.set_panel_width(width)
                ms, launches, st = timed_plan(pl, A, Q, R, stream, max(3, min(steps, 5)), warmup, True)
            e = errs(hA, Q, R, Ro)
            res[name] = {"ms_per_step": ms, "tflops": fl / (ms * 1e-3) / 1e12,
                         "vs_fp64_peak": fl / (ms * 1e-3) / 1e12 / fp64_peak(clk),
                         "stages_ms": {k: round(v, 3) for k, v in st.items()}, "errors": e}
        res["oracle"] = {"orthogonality": oracle.orthogonality(Qo), "residual": oracle.residual(hA, Qo, Ro)}
        res["panel_speedup"] = res["plain"]["ms_per_step"] / res["panels"]["ms_per_step"]
        out["panels"] = res
        del A, Q, R, hA, Qo
    except Exception as ex:
        out["panels"] = {"error": repr(ex)}
    torch.cuda.empty_cache()

    # ---- batch: 1024 problems of 4096 x 32 per grouped launch
    try:
        out["batch"] = measure_batch(max(5, steps), warmup, 1, 0, local, False)
    except Exception as ex:
        out["batch"] = {"error": repr(ex)}
    torch.cuda.empty_cache()

    # ---- the full request stream of the serving configuration
    try:
        from paper_1710_08471_gb300 import serving

        pool = serving_pool or serving.InputPool(262144, (16, 32, 64, 128, 256), seed=100)
        sv = {"requests": 20000, "rate_per_s": 2000.0, "precision": "split (S = 7)",
              "inputs": "per-request kappa served from a 21-value grid 1..1e5 (within x1.33 of the draw)"}
        sv["continuous"] = serving.run_workload(20000, 2000.0, 100, 1, 8, 64e9, pool=pool, group_max=64)
        sv["one_at_a_time"] = serving.run_workload(20000, 2000.0, 100, 1, 1, 64e9, pool=pool, group_max=1)
        out["serving_20000"] = sv
    except Exception as ex:
        out["serving_20000"] = {"error": repr(ex)}
    return out


def bench_ours(args, ws, rank, local):
    import torch

    import paper_1710_08471_gb300 as cq

    m, n, kappa, seed, desc = WORKLOADS[args.workload]
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fused = args.variant == "fused" and args.precision == "fp64"
    peaks = measured_peaks()
    # inputs: generated on the host (seed + rank), kept pinned for the e2e leg
    hA, hA_t = make_input(m, n, kappa, seed + 1000 * rank, pinned=True)
    A = cq.empty_colmajor(m, n, device=dev)
    A.t().copy_(hA_t.to(dev, non_blocking=True))
    Q = cq.empty_colmajor(m, n, device=dev)
    R = cq.empty_colmajor(n, n, device=dev)
    torch.cuda.synchronize()
    # a graph needs a stream of its own (not the legacy default stream)
    stream = torch.cuda.Stream(device=dev) if args.graph else torch.cuda.current_stream()

    def make_plan(precision, fz, depth=0, graph=False):
        pl = cq.Plan(m, n, precision=PRECISIONS[precision], fused=fz, stream=stream, graph=graph)
        if depth:
            pl.set_inverse_depth(depth)
        return pl

    flush = torch.zeros(64 << 20, dtype=torch.float64, device=dev) if needs_flush(m, n) else None

    def timed(pl, steps, warmup, profile):
        return timed_plan(pl, A, Q, R, stream, steps, warmup, profile, ws, flush=flush)

    plan = make_plan(args.precision, fused, args.inverse_depth, graph=args.graph)
    clocks = ClockSampler(local)
    clocks.start()
    if args.graph:
        # stage timers run eagerly (they bypass the graph); the step time is
        # the graph replay's
        _, _, per_stage = timed(plan, max(2, args.steps // 2), 1, True)
        ms_local, launches, _ = timed(plan, args.steps, args.warmup, False)
    else:
        ms_local, launches, per_stage = timed(plan, args.steps, args.warmup, True)
    clk = clocks.stop()
    flops = nominal_flops(m, n)
    value, ms_step = replica_throughput(ws, flops, ms_local)
    fp64_pk = fp64_peak(clk)

    out = {
        "metric": "CQR2 TFLOP/s (nominal 4mn^2+5n^3/3)", "value": value, "unit": "TFLOP/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "bf16-slices->f64",
        "data": "synthetic",
        "config": workload_config(args, ws),
        "gpu_launches": launches,
        "roofline": roofline_of(per_stage, m, n, args.precision, fused, clk, args.workload, peaks),
        "vs_fp64_peak": {"achieved": value / ws, "peak": fp64_pk, "frac": value / ws / fp64_pk},
        "step_roofline": step_roofline(m, n, args.precision, fused, ms_local, clk, peaks),
        "stages_ms": {k: round(v, 4) for k, v in per_stage.items()},
        "clocks": clk,
    }
    if rank == 0 and not args.quick:
        import oracle

        try:
            probe = fp64_gemm_probe(dev)
            probe["frac_of_derived_peak"] = probe["cublas_dgemm_tflops"] / fp64_pk
            out["fp64_reference"] = probe
            out["vs_fp64_peak"]["frac_of_cublas_dgemm"] = value / ws / probe["cublas_dgemm_tflops"]
        except Exception as ex:  # a reference probe must not cost the main line
            out["fp64_reference"] = {"error": repr(ex)}
        hQ, hQ_t = pinned_colmajor(m, n)
        hR, hR_t = pinned_colmajor(n, n)
        # End to end through the host-buffer C entry point, before the CPU
        # legs below: after the oracle and the error checks the same process
        # copied pinned memory at a fraction of its rate (210 -> 11 GB/s in
        # one run). The plain host-copy rate (pinned A to the device and back)
        # is reported beside it.
        def copy_rate():
            torch.cuda.synchronize()
            c0 = time.perf_counter()
            A.t().copy_(hA_t, non_blocking=True)
            torch.cuda.synchronize()
            c1 = time.perf_counter()
            hQ_t.copy_(A.t(), non_blocking=True)
            torch.cuda.synchronize()
            c2 = time.perf_counter()
            return {"h2d_gbs": m * n * 8 / (c1 - c0) / 1e9, "d2h_gbs": m * n * 8 / (c2 - c1) / 1e9}

        probe_before = copy_rate()
        plan.factor_host(hA, hQ, hR)  # allocates staging
        times = []
        for _ in range(max(2, args.steps // 2)):
            t0 = time.perf_counter()
            plan.factor_host(hA, hQ, hR)
            times.append(time.perf_counter() - t0)
        e2e_ms = 1e3 * statistics.median(times)
        # one more call with the stage timers on, for the copy bandwidths
        plan.set_profiling(True)
        plan.factor_host(hA, hQ, hR)
        st_e = plan.stage_times()
        plan.set_profiling(False)
        h2d_ms, d2h_ms = st_e["h2d"][0], st_e["d2h"][0]
        out["e2e"] = {"value": flops / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": e2e_ms,
                      "h2d_bytes_per_step": m * n * 8, "d2h_bytes_per_step": m * n * 8 + n * n * 8,
                      "h2d_ms": h2d_ms, "d2h_ms": d2h_ms,
                      "h2d_gbs": m * n * 8 / (h2d_ms * 1e-3) / 1e9 if h2d_ms else None,
                      "d2h_gbs": (m * n * 8 + n * n * 8) / (d2h_ms * 1e-3) / 1e9 if d2h_ms else None,
                      "api": "cqr2_factor_host (pinned host buffers)",
                      "plain_copy_probe": {"before": probe_before, "after": copy_rate()}}
        # the same probe at the top level of the line as well: the pinned
        # host<->device copy rate of this machine bounds the end-to-end figure
        out["copy_probe"] = dict(out["e2e"]["plain_copy_probe"], bytes=m * n * 8,
                                 note="one cudaMemcpyAsync of pinned A to the device and back, GB/s")
        # CPU FP64 oracle of the same workload: errors and the CPU baseline
        rows, dt, Qo, Ro = run_oracle_sample(hA, args.oracle_rows or m)
        sample = (f"full workload ({desc})" if rows == m else f"first {rows} of {m} rows of the workload ({desc})")
        out["cpu_baseline"] = {"value": nominal_flops(rows, n) / dt / 1e12, "unit": "TFLOP/s", "cores": cpu_cores(),
                               "kind": "oracle", "sample": sample + "; numpy FP64 oracle, one run",
                               "seconds": dt}
        ref = {"oracle_orthogonality": oracle.orthogonality(Qo), "oracle_residual": oracle.residual(hA, Qo, Ro)}
        del Qo

        def errors():
            hQ_t.copy_(Q.t())
            hR_t.copy_(R.t())
            torch.cuda.synchronize()
            e = {"orthogonality": oracle.orthogonality(hQ), "residual": oracle.residual(hA, hQ, hR)}
            if rows == m:
                e["R_rel_vs_oracle"] = oracle.rel_error(np.asfortranarray(hR), Ro)
            return e

        plan.factor(A, Q, R, sync=True)
        out["errors"] = dict(errors(), **ref)
        # other variants of the same factorization at the same size
        variants = {}
        todo = [("fp64", not fused), ("ozaki", False), ("ozaki6", False)] if args.precision == "fp64" else \
            [("fp64", True)] + [(p, False) for p in ("ozaki", "ozaki6") if p != args.precision]
        for prec, fz in todo:
            if SLICES[prec] and n > 16384:
                continue
            name = prec + ("_fused" if fz and prec == "fp64" else "")
            try:
                pl = make_plan(prec, fz)
                ms_v, _, st_v = timed(pl, max(2, args.steps // 2), 1, True)
                variants[name] = {"ms_per_step": ms_v, "tflops": flops / (ms_v * 1e-3) / 1e12,
                                  "speedup_vs_main": ms_step / ms_v,
                                  "stages_ms": {k: round(v, 4) for k, v in st_v.items()},
                                  "roofline": roofline_of(st_v, m, n, prec, fz, clk, args.workload, peaks),
                                  "step_roofline": step_roofline(m, n, prec, fz, ms_v, clk, peaks),
                                  "errors": errors()}
                pl.close()
            except Exception as ex:  # a variant must not cost the main line
                variants[name] = {"error": repr(ex)}
        out["variants"] = variants
    plan.close()
    pool = None
    if rank == 0 and not args.quick and args.serving_requests > 0:
        # serving leg: a bounded stream of least-squares requests (Poisson
        # arrivals, m in [1024, 262144], n in {16..256}, kappa in [1, 1e5])
        # under a 64 GB HBM budget: continuous batching over 8 stream slots
        # with small requests grouped into one launch, the same without
        # grouping, and one request at a time
        del A, Q, R
        torch.cuda.empty_cache()
        from paper_1710_08471_gb300 import serving

        pool = serving.InputPool(262144, (16, 32, 64, 128, 256), seed=100)
        # warm-up, not reported: the first serving run in a process pays for
        # the caching allocator's first device allocations and first kernel
        # loads (measured: 0.66 s more over 1000 requests)
        serving.run_workload(min(300, args.serving_requests), 2000.0, 99, 1, 8, 64e9, pool=pool)
        sv = {}
        # at the offered 2000 requests/s (overload: latency is queueing), and
        # at rates each precision sustains (latency is service time)
        nreq = args.serving_requests
        for name, prec, slots, gmax, rate, count in (
                ("ozaki_continuous", 1, 8, 64, 2000.0, nreq), ("ozaki_continuous_ungrouped", 1, 8, 1, 2000.0, nreq),
                ("ozaki_one_at_a_time", 1, 1, 1, 2000.0, nreq), ("fp64_continuous", 0, 8, 64, 2000.0, nreq),
                ("fp64_one_at_a_time", 0, 1, 1, 2000.0, nreq),
                ("ozaki_continuous_at_800_per_s", 1, 8, 64, 800.0, nreq),
                ("fp64_continuous_at_100_per_s", 0, 8, 64, 100.0, max(1, nreq // 2))):
            try:
                sv[name] = serving.run_workload(count, rate, 100, prec, slots, 64e9, pool=pool, group_max=gmax)
            except Exception as ex:  # a serving leg must not cost the main line
                sv[name] = {"error": repr(ex)}
        out["serving"] = sv
    if rank == 0 and not args.quick and args.configs:
        # the plan's other configurations, each with its own timing and errors
        if "A" in locals():
            del A, Q, R
        torch.cuda.empty_cache()
        out["configs"] = bench_configs(args.steps, args.warmup, local, peaks, clk, serving_pool=pool)
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="tall")
    ap.add_argument("--variant", choices=["fused", "plain"], default="fused")
    ap.add_argument("--inverse-depth", type=int, default=0,
                    help="FP64, n > 256: CholInv levels without the off-diagonal inverse (block substitution)")
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="fp64",
                    help="fp64: native FP64; ozaki / ozaki6: BF16 tensor-core slices (7 / 6 per entry)")
    ap.add_argument("--oracle-rows", type=int, default=None,
                    help="rows of the workload the CPU oracle runs on (default: all for the error check, "
                         "2^21 for --impl reference)")
    ap.add_argument("--quick", action="store_true", help="device timing only (no e2e / oracle legs)")
    ap.add_argument("--graph", action="store_true",
                    help="replay the factorization from a captured CUDA graph (CQR2_GRAPH); for launch-bound sizes")
    ap.add_argument("--serving-requests", type=int, default=1000,
                    help="requests in the serving leg (0 = skip)")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the other configurations (small, wide512, batch, the 20,000-request stream)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        if ws > 1 and rank != 0:
            return
        bench_reference(args, ws, rank)
        return
    if ws > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    try:
        if args.workload == "batch":
            bench_batch(args, ws, rank, local)
        else:
            bench_ours(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
