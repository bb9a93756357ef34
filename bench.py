"""Throughput of the full HPM force solve (tree build + all solve stages).

Default workload: 2^21 particles from a truncated Plummer sphere, adaptive
tree (> 32 splits, depth <= 12), 4^3 gridlets, eps = 1e-4, on one GPU.
One step = hpm_build_tree + hpm_solve on device-resident inputs. Prints one
JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the paper's FFT algorithm, plain
C with OpenMP) on the host cores instead, on a bounded sample of the same
workload. Multi-GPU runs (torchrun) solve one independent problem per rank
(replicas: the method has no exchange between problems).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1906_10734_gb300 import inputs as I  # noqa: E402

METRIC = "particles/s for full HPM force solve at stated force error; p50/p99 latency"
UNIT = "particles/s"
P2P_FLOP_PER_PAIR = 20     # the usual N-body count (Kahan compensation not counted)


def m2l_flops_per_target(ng: int) -> float:
    """Nominal FFT-convolution work per target: forward r2c + inverse c2r of P^3 points at
    2.5 n log2 n each, plus the real Green product on the half spectrum (P = 8 Ng)."""
    P = 8 * ng
    return 5.0 * P ** 3 * math.log2(P ** 3) + 2.0 * P * P * (P // 2 + 1)


def dense_flop_per_parent(ng: int) -> int:
    """Executed tensor work of the dense source-to-target product per parent: three FP16
    products (hi*hi, hi*lo, lo*hi) x 2 x rows x K, rows = 8 Ng^3 padded to 128-row blocks,
    K = 216 slots x Ng^3 nodes padded to 16 (Ng = 4: 512 x 13824; Ng = 6: 1792 x 48384)."""
    m3 = ng ** 3
    rows = -(-8 * m3 // 128) * 128
    k = 216 * (-(-m3 // 16) * 16)
    return 3 * 2 * rows * k


DENSE_FLOP_PER_PARENT = dense_flop_per_parent(4)


def alu_peaks() -> dict:
    """FP32 / FP64 FMA and rsqrt peaks of this GPU from the committed microbenchmark summary
    (profiles/alu_peaks_gb300.md, written by hpm_measure_alu_peaks); {} if absent."""
    try:
        text = open(os.path.join(ROOT, "profiles", "alu_peaks_gb300.md")).read()
    except OSError:
        return {}
    out = {}
    for key in ("fp32_tflops", "fp64_tflops", "rsqrt_gops"):
        m = re.search(key + r":\s*([0-9.eE+]+)", text)
        if m:
            out[key] = float(m.group(1))
    return out


def fp32_peak(live: dict | None) -> tuple[float, str]:
    """Measured FP32 FFMA peak (TFLOP/s) and where it comes from: the committed summary,
    else this run's own measurement."""
    p = alu_peaks().get("fp32_tflops")
    if p:
        return p, "profiles/alu_peaks_gb300.md fp32_tflops (hpm_measure_alu_peaks on GB300) of measured"
    if live and live.get("fp32_tflops"):
        return live["fp32_tflops"], "hpm_measure_alu_peaks in this run, of measured"
    return float("nan"), "no measured FP32 peak"


def roofline_of(stats_steps, ng, n_targets, traffic_src, live_peaks=None, tile_n=None):
    """Roofline object of the source-to-target kernel of the last steps.

    `achieved` is the ALGORITHMIC work: the nominal FFT-convolution count per target
    (5 P^3 log2 P^3 + 2 P^2 (P/2+1), P = 8 Ng) times the targets, per launch duration.
    Ng = 4 default path (dense product on the tensor cores): over the kernel's own
    CUDA-event time, against the measured dense bf16 burst peak (FP16 has the bf16
    tensor rate); the executed dense work (three FP16 products per term) is reported
    beside it. FFT-form and any-order kernels: over the stage time, against the measured
    FP32 FFMA peak."""
    peaks = measured_peaks()
    stage_ms = statistics.mean(s["ms_m2l"] for s in stats_steps)
    nominal_flop = m2l_flops_per_target(ng) * n_targets
    parents = stats_steps[-1].get("m2l_parents", 0)
    if parents:
        kms = statistics.mean(s["ms_m2l_kernel"] for s in stats_steps)
        achieved = nominal_flop / (kms / 1e3) / 1e12
        executed = dense_flop_per_parent(ng) * parents / (kms / 1e3) / 1e12
        peak = peaks.get("bf16_tflops", 1900.0)
        return {"kernel": f"k_m2l_tc<{ng}>: source-to-target as a dense FP16-pair tcgen05 product per parent block",
                "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": profile_traffic(traffic_src, tile_n) if traffic_src else None, "ms_per_launch": kms,
                "launches_per_step": 1, "flop_per_target": m2l_flops_per_target(ng),
                "targets_per_launch": n_targets,
                "flop_basis": "nominal FFT convolution work per target x targets (algorithmic)",
                "peak_basis": "MEASURED_PEAKS.json bf16_tflops (dense, burst) of measured; FP16 has the bf16 tensor rate",
                "executed": {"achieved": executed, "frac": executed / peak, "flop_per_parent": dense_flop_per_parent(ng),
                             "parents_per_launch": parents,
                             "basis": "3 FP16 products (hi*hi, hi*lo, lo*hi) x 2 x rows x K per parent, rows and K "
                                      "padded as the kernel runs them"},
                "stage": {"ms": stage_ms, "achieved": nominal_flop / (stage_ms / 1e3) / 1e12,
                          "frac": nominal_flop / (stage_ms / 1e3) / 1e12 / peak,
                          "basis": "same nominal work over the whole source-to-target stage (preparation "
                                   "kernels k_level_amax, k_split, k_col_exp included)"}}
    peak, basis = fp32_peak(live_peaks)
    achieved = nominal_flop / (stage_ms / 1e3) / 1e12
    return {"kernel": "source-to-target FFT convolution (k_m2l4)" if ng == 4 else
                      "source-to-target convolution, x-transform or any-order kernel (k_m2l_xdft / k_m2l_generic)",
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": profile_traffic(traffic_src) if traffic_src else None, "ms_per_launch": stage_ms,
            "launches_per_step": 1, "flop_per_target": m2l_flops_per_target(ng), "targets_per_launch": n_targets,
            "flop_basis": "nominal FFT convolution work per target x targets (algorithmic)", "peak_basis": basis}


def p2p_roofline(stats_steps, live_peaks=None) -> dict:
    """Near field: 20 FLOP per near-zone pair over the near-field stage time against the
    measured FP32 FFMA peak, and pairs per second against the measured rsqrt rate (one
    reciprocal square root per pair)."""
    pairs = stats_steps[-1].get("p2p_pairs", 0)
    ms = statistics.mean(s["ms_p2p"] for s in stats_steps)
    if not pairs or not ms:
        return {}
    peak, basis = fp32_peak(live_peaks)
    achieved = P2P_FLOP_PER_PAIR * pairs / (ms / 1e3) / 1e12
    out = {"kernel": "k_p2p (+ k_p2p_combine): Kahan-compensated FP32 near field", "bound": "alu",
           "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "pairs": pairs,
           "ms": ms, "flop_basis": f"{P2P_FLOP_PER_PAIR} FLOP per near-zone pair (j != i)", "peak_basis": basis}
    rs = alu_peaks().get("rsqrt_gops") or (live_peaks or {}).get("rsqrt_gops")
    if rs:
        out["rsqrt_frac"] = pairs / (ms / 1e3) / (rs * 1e9)
    return out


def workload_for(rank: int, n_override: int | None = None, kind: str = "plummer", ng: int = 4) -> I.Workload:
    if kind == "uniform":
        n = n_override or (1 << 24)
        w = I.uniform_16m_depth7(ng=ng, n=n)
        if rank:
            w.pos = I.uniform_cube(n, 3 + 1000 * rank)
        return w
    n = n_override or (1 << 21)
    w = I.plummer_2m_adaptive(ng=4, n=n) if rank == 0 else I.Workload(
        f"plummer{n}_adaptive32_depth12_rank{rank}", I.plummer_sphere(n, 2 + 1000 * rank),
        I.equal_masses(n), max_depth=12, leaf_max=32, ng=4, eps=1e-4)
    return w


def config_of(n: int, max_depth=12, leaf_max=32, ng=4, eps=1e-4, extra=None) -> dict:
    desc = (f"uniform cube N={n}, uniform tree depth {max_depth}, gridlet {ng}^3, eps={eps:g}" if leaf_max == 0 else
            f"plummer sphere N={n} (a=0.05, r<=0.5), adaptive tree >{leaf_max}/leaf, depth<={max_depth}, "
            f"gridlet {ng}^3, eps={eps:g}")
    c = {"workload": desc,
         "n": n, "max_depth": max_depth, "leaf_max": leaf_max, "gridlet_order": ng, "eps": eps,
         "stated_force_error": "FP32 solve within 1e-5 rel RMS of the FP64 HPM (parity tests)"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for k, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(k)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def profile_traffic(kernel_src: str, tile_n: int | None = None) -> float | None:
    """DRAM bytes per full launch from the committed ncu summary, if it was taken on the
    kernel source as it is now (its sha256 matches); else None. With tile_n, the figure
    of that tile width (`dram_bytes_per_full_launch_tn<N>:`) where the summary has one."""
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for fn in sorted(os.listdir(pdir)):
        if not fn.startswith("m2l_") or not fn.endswith(".md"):
            continue
        text = open(os.path.join(pdir, fn)).read()
        m_sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
        if not m_sha or m_sha.group(1) != h:
            continue
        m_tn = re.search(rf"dram_bytes_per_full_launch_tn{tile_n}:\s*([0-9.eE+]+)", text) if tile_n else None
        m_tr = m_tn or re.search(r"dram_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
        if m_tr:
            return float(m_tr.group(1))
    return None


def reduce_over_ranks(total_ms: float, n_local: int, device=None):
    """Replica aggregation: the job time is the slowest rank's, the work is every rank's
    particles (weak scaling, no data-path collective; this is bookkeeping only)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return total_ms, n_local
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    n = torch.tensor([n_local], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


# ---------------------------------------------------------------------------
def run_gpu(args) -> None:
    import torch
    import torch.distributed as dist
    from paper_1906_10734_gb300 import hpm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1906_10734_gb300 import build as B
    B.build()

    w = workload_for(rank, args.n, args.workload, args.ng)
    stream = torch.cuda.current_stream(dev)
    pos = torch.from_numpy(w.pos).to(dev)
    mass = torch.from_numpy(w.mass).to(dev)
    phi = torch.empty(w.n, dtype=torch.float32, device=dev)
    acc = torch.empty((w.n, 3), dtype=torch.float32, device=dev)
    m2l_flag = {"tensor": 0, "fft": hpm.HPM_FLAG_FFT_M2L, "xtransform": hpm.HPM_FLAG_XTRANSFORM_M2L}[args.m2l]
    plan = hpm.hpm_plan((0.0, 0.0, 0.0), 1.0, w.max_depth, w.ng, w.eps, w.leaf_max, flags=1 | m2l_flag)
    l2_flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def step():
        hpm.hpm_build_tree(plan, pos, w.n, stream)
        hpm.hpm_solve(plan, pos, mass, phi, acc, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    # launch shapes picked by the library's autotuner on this input (untimed;
    # results are the same for every shape)
    tuning = hpm.hpm_tune(plan, pos, mass, stream) if not args.no_tune else hpm.hpm_get_tuning(plan)
    step()
    torch.cuda.synchronize(dev)
    info = hpm.hpm_get_lists_info(plan)
    live_peaks = hpm.hpm_measure_alu_peaks(stream) if rank == 0 else None   # untimed
    torch.cuda.synchronize(dev)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats_steps, launches = [], 0
    stage_keys = ("ms_tree", "ms_p2g", "ms_m2m", "ms_m2l", "ms_l2l", "ms_g2p", "ms_p2p")
    stage_sum = {k: 0.0 for k in stage_keys}
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            l2_flush.fill_(k & 0xff)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            st = hpm.hpm_get_stats(plan)       # waits for this step's last event
            stats_steps.append(st)
            for key in stage_keys:
                stage_sum[key] += st[key]
            launches += st["launches"]
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms, n_all = reduce_over_ranks(sum(step_ms), w.n, dev)
    clocks = clk.summary()

    # end to end through the host-memory entry point: pinned inputs in, results out
    hp = torch.from_numpy(w.pos).pin_memory()
    hm = torch.from_numpy(w.mass).pin_memory()
    hphi = torch.empty(w.n, dtype=torch.float32).pin_memory()
    hacc = torch.empty((w.n, 3), dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    hpm.hpm_solve_host(plan, hp.numpy(), hm.numpy(), hphi.numpy(), hacc.numpy(), stream)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        hpm.hpm_solve_host(plan, hp.numpy(), hm.numpy(), hphi.numpy(), hacc.numpy(), stream)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    hpm.hpm_destroy(plan)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    n_total = n_all
    ms_per_step = total_ms / args.steps
    value = n_total * args.steps / (total_ms / 1e3)
    csrc = os.path.join(ROOT, "paper_1906_10734_gb300", "csrc")
    traffic_src = None
    if args.workload == "plummer" and w.ng == 4:
        traffic_src = os.path.join(csrc, "m2l_tc.cu" if args.m2l == "tensor" else "m2l.cu")
    roofline = roofline_of(stats_steps, w.ng, info["n_targets"], traffic_src, live_peaks,
                           tuning.get("m2l_tile_parents") or 256)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of(w.n, w.max_depth, w.leaf_max, w.ng, w.eps, {"parallelism": "replicas" if world > 1 else "single",
                                "l2": "flushed between steps (256 MiB write outside the timed events)",
                                "tuning": tuning,
                                "cells": info["n_cells"], "targets": info["n_targets"],
                                "leaves": info["n_leaves"], "boxes": info["n_boxes"],
                                "depth_reached": info["depth_reached"]}),
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "min": min(step_ms), "max": max(step_ms)},
        "e2e": {"value": n_total / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 32 * w.n,
                "d2h_bytes_per_step": 16 * w.n, "api": "hpm_solve_host (pinned host buffers)"},
        "gpu_launches": int(launches),
        "stages_ms": {k[3:]: v / args.steps for k, v in stage_sum.items()},
        "roofline": roofline,
        "rooflines_other": {"p2p": p2p_roofline(stats_steps, live_peaks)},
        "alu_peaks_this_run": live_peaks,
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batch(args) -> None:
    """256 independent problems (N log-uniform in [1e3, 1e6], Plummer or uniform by coin
    flip, adaptive <= 32, Ng = 4, eps = 1e-4): one batched solve per step, and the same
    problems solved one after another with the same plan for comparison."""
    import torch
    from paper_1906_10734_gb300 import build as B, hpm
    B.build()
    dev = torch.device("cuda", 0)
    P = args.problems
    ws = [I.batch_problem(k) for k in range(P)]
    bufs = [(torch.from_numpy(w.pos).to(dev), torch.from_numpy(w.mass).to(dev),
             torch.zeros(w.n, dtype=torch.float32, device=dev), torch.zeros((w.n, 3), dtype=torch.float32, device=dev))
            for w in ws]
    n_total = sum(w.n for w in ws)
    plan = hpm.hpm_plan((0.0, 0.0, 0.0), 1.0, 12, 4, 1e-4, 32, flags=1)
    stream = torch.cuda.current_stream(dev)
    l2_flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        hpm.hpm_solve_batch(plan, bufs, stream)
    torch.cuda.synchronize(dev)
    step_ms, stats_steps, launches = [], [], 0
    with ClockSampler(0) as clk:
        for k in range(args.steps):
            l2_flush.fill_(k & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            hpm.hpm_solve_batch(plan, bufs, stream)
            b.record(stream)
            b.synchronize()
            st = hpm.hpm_get_stats(plan)
            stats_steps.append(st)
            launches += st["launches"]
            step_ms.append(a.elapsed_time(b))
    info = hpm.hpm_get_lists_info(plan)
    # the same problems one by one with the same plan
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for (pos, mass, phi, acc) in bufs:
        hpm.hpm_build_tree(plan, pos, pos.shape[0], stream)
        hpm.hpm_solve(plan, pos, mass, phi, acc, stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    loop_ms = a.elapsed_time(b)
    hpm.hpm_destroy(plan)
    total = sum(step_ms)
    value = n_total * args.steps / (total / 1e3)
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch of {P} problems, N log-uniform in [1e3, 1e6] (sum {n_total}), Plummer or "
                               "uniform by coin flip, adaptive <=32/leaf, depth<=12, gridlet 4^3, eps=1e-4",
                   "problems": P, "n": n_total, "targets": info["n_targets"],
                   "l2": "flushed between steps (256 MiB write outside the timed events)"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "per_problem_loop": {"value": n_total / (loop_ms / 1e3), "ms": loop_ms,
                             "speedup_of_batch": loop_ms / (total / args.steps)},
        "gpu_launches": int(launches),
        "roofline": roofline_of(stats_steps, 4, info["n_targets"], None),
        "clocks": clk.summary()}), flush=True)


def run_serve(args) -> None:
    """Poisson request stream (mean rate --rate req/s) of solves with N log-uniform in
    [1e4, 4e6], Plummer or uniform by coin flip, through the continuous-batching server.
    Requests reuse a pool of --pool seeded payloads held in pinned host memory."""
    import torch
    from paper_1906_10734_gb300 import build as B, hpm
    B.build()
    pool = []
    for k in range(args.pool):
        w = I.batch_problem(k, 1e4, 4e6, seed=5)
        pool.append((torch.from_numpy(w.pos).pin_memory(), torch.from_numpy(w.mass).pin_memory(),
                     torch.zeros(w.n, dtype=torch.float32).pin_memory(),
                     torch.zeros((w.n, 3), dtype=torch.float32).pin_memory()))
    rng = np.random.default_rng(5)
    sv = hpm.Server(max_depth=12, gridlet_order=4, eps=1e-4, leaf_max=32, workers=args.workers,
                    max_batch=args.max_batch, hbm_budget_bytes=150 << 30,
                    max_batch_particles=args.max_batch_particles)

    def drive(seconds):
        t0 = time.perf_counter()
        t_next = t0
        tickets = []
        offered = 0
        while True:
            t_next += rng.exponential(1.0 / args.rate)
            if t_next - t0 > seconds:
                break
            now = time.perf_counter()
            if t_next > now:
                time.sleep(t_next - now)
            k = int(rng.integers(len(pool)))
            tickets.append(sv.submit(*pool[k]))
            offered += pool[k][0].shape[0]
        for t in tickets:
            sv.wait(t, 600000)
        return offered, time.perf_counter() - t0, len(tickets)

    drive(args.serve_warmup_s)
    sv.reset_stats()
    with ClockSampler(0) as clk:
        offered, span, nreq = drive(args.serve_seconds)
    st = sv.stats()
    sv.close()
    print(json.dumps({
        "metric": METRIC, "value": st["particles_per_s"], "unit": UNIT, "n_gpus": 1, "steps": nreq,
        "warmup": int(args.serve_warmup_s), "ms_per_step": st["mean_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"Poisson requests, mean {args.rate}/s, N log-uniform in [1e4, 4e6] (pool of "
                               f"{args.pool} seeded payloads, Plummer or uniform), adaptive <=32/leaf, depth<=12, "
                               "gridlet 4^3, eps=1e-4, pinned host buffers in and out",
                   "workers": args.workers, "max_batch": args.max_batch, "hbm_budget_gb": 150,
                   "max_batch_particles": args.max_batch_particles,
                   "seconds": args.serve_seconds},
        "latency_ms": {"p50": st["p50_ms"], "p99": st["p99_ms"], "mean": st["mean_ms"]},
        "offered_particles_per_s": offered / args.serve_seconds, "requests": st["completed"],
        "batches": st["batches"],
        "admission": {"bytes_per_particle_measured": st["bytes_per_particle"],
                      "estimate": "1.25 x measured bytes per particle x N + 8 MiB per request"},
        "clocks": clk.summary()}), flush=True)


def run_pointsource(args) -> None:
    """The accuracy test of Sec. 3.2: a point mass at (1, 1, 1) and the cells of a patch grid
    (8^3 cells per patch; --geometry uniform4, uniform5 or mixed) as zero-mass targets,
    Newtonian kernel. For each gridlet order of --orders: device time of build + solve per step
    (inputs resident, L2 flushed between steps) and the relative error of the accelerations
    against the analytic field (L2 and LMAX, as in Sec. 3.2): the shape of the paper's
    time-versus-accuracy curve for HPM."""
    import torch
    from paper_1906_10734_gb300 import build as B, hpm
    B.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    l2_flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sweep = []
    with ClockSampler(0) as clk:
        for ng in [int(x) for x in args.orders.split(",")]:
            w = I.point_source_patch_grid(args.geometry, ng=ng)
            print(f"pointsource {args.geometry} Ng={ng}: {w.n - 1} cells", file=sys.stderr, flush=True)
            pos = torch.from_numpy(w.pos).to(dev)
            mass = torch.from_numpy(w.mass).to(dev)
            phi = torch.empty(w.n, dtype=torch.float32, device=dev)
            acc = torch.empty((w.n, 3), dtype=torch.float32, device=dev)
            plan = hpm.hpm_plan((0.0, 0.0, 0.0), 1.0, w.max_depth, ng, 0.0, w.leaf_max, flags=1,
                                green=hpm.Green.newton())

            def step():
                hpm.hpm_build_tree(plan, pos, w.n, stream)
                hpm.hpm_solve(plan, pos, mass, phi, acc, stream)

            for _ in range(args.warmup):
                step()
            ms = []
            for k in range(args.steps):
                l2_flush.fill_(k & 0xff)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                step()
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            st = hpm.hpm_get_stats(plan)
            hpm.hpm_destroy(plan)
            print(f"  {statistics.mean(ms):.2f} ms per step", file=sys.stderr, flush=True)
            got = acc.cpu().numpy().astype(np.float64)[1:]
            d = w.pos[0][None, :] - w.pos[1:]
            an = d / np.linalg.norm(d, axis=1)[:, None] ** 3
            err = np.linalg.norm(got - an, axis=1) / np.linalg.norm(an, axis=1)
            sweep.append({"ng": ng, "ms_per_step": statistics.mean(ms), "ms_m2l": st["ms_m2l"],
                          "cells_per_s": (w.n - 1) / (statistics.mean(ms) / 1e3),
                          "l2": float(np.sqrt(np.sum(np.linalg.norm(got - an, axis=1) ** 2) /
                                              np.sum(np.linalg.norm(an, axis=1) ** 2))),
                          "lmax": float(err.max())})
    best = sweep[-1]
    print(json.dumps({
        "metric": METRIC, "value": best["cells_per_s"], "unit": "cells/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": best["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"point source at (1,1,1) on patch grid '{args.geometry}' (8^3 cells per patch), "
                               "Newtonian kernel, cells as zero-mass targets",
                   "geometry": args.geometry, "cells": int(w.n - 1),
                   "l2": "flushed between steps (256 MiB write outside the timed events)"},
        "sweep": sweep, "clocks": clk.summary()}), flush=True)


def oracle_step(n: int):
    """One timed oracle solve on a reduced Plummer problem of the same recipe."""
    import oracle as O
    w = I.small_plummer(n, 2, leaf_max=32, max_depth=12, ng=4, eps=1e-4)
    t0 = time.perf_counter()
    tr = O.Tree(w.pos, max_depth=w.max_depth, leaf_max=w.leaf_max)
    O.solve_fft(tr, w.mass, w.ng, w.eps)
    return time.perf_counter() - t0, w.n


def cpu_baseline(args) -> dict:
    import oracle as O
    n = args.cpu_sample
    oracle_step(n // 8)                      # load and warm the library
    times = [oracle_step(n)[0] for _ in range(2)]
    t = min(times)
    return {"value": n / t, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle, paper's FFT algorithm (solve_fft), Plummer N={n} same recipe "
                      f"(adaptive >32, depth<=12, 4^3, eps=1e-4), best of 2, {t:.2f} s per solve"}


def run_reference(args) -> None:
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    n = args.ref_sample
    for _ in range(args.warmup):
        oracle_step(max(1024, n // 8))
    times = []
    for _ in range(args.steps):
        dt, _ = oracle_step(n)
        times.append(dt)
    total = sum(times)
    value = n * args.steps / total
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": config_of(args.n or (1 << 21), extra={
               "sample": f"each step solves a Plummer N={n} problem of the same recipe on the host"}),
           "latency_ms": {"p50": float(np.percentile(times, 50)) * 1e3,
                          "p99": float(np.percentile(times, 99)) * 1e3},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                            "sample": f"FP64 oracle (paper's FFT algorithm), Plummer N={n} per step"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="plummer", choices=["plummer", "uniform", "batch", "serve", "pointsource"])
    ap.add_argument("--geometry", default="mixed", choices=["uniform4", "uniform5", "mixed"],
                    help="patch grid of the point-source workload")
    ap.add_argument("--orders", default="2,4,6,8", help="gridlet orders of the point-source sweep")
    ap.add_argument("--ng", type=int, default=4, help="gridlet order of the uniform workload")
    ap.add_argument("--m2l", default="tensor", choices=["tensor", "fft", "xtransform"],
                    help="Ng = 4 source-to-target kernel: register FFT or x-transform + direct (y, z)")
    ap.add_argument("--problems", type=int, default=256)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--pool", type=int, default=32)
    ap.add_argument("--workers", type=int, default=2)
    ap.add_argument("--max-batch", type=int, default=32)
    ap.add_argument("--max-batch-particles", type=int, default=1 << 20,
                    help="serving: particles per batch; larger requests run alone, one at a time (0: FIFO)")
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    ap.add_argument("--serve-warmup-s", type=float, default=3.0)
    ap.add_argument("--n", type=int, default=None, help="particles per problem (default 2^21)")
    ap.add_argument("--cpu-sample", type=int, default=1 << 15)
    ap.add_argument("--ref-sample", type=int, default=1 << 14)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shapes (no autotuner)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "pointsource":
        run_pointsource(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
