#!/usr/bin/env python
"""Benchmark of the multilevel NMF hot path on GB300.

One step = one complete multilevel solve through the C ABI: restriction of M
to every level, the V-cycle schedule of HALS sweeps (pre-smoothing,
restriction of V, coarse cycle, prolongation, post-smoothing) and the final
||M - VW||_F, on the 19 x 19-grid workload (m = 361 pixels, n = 2429 images,
r = 49; the CBCL face-database shape) with L = 3 levels and sweep budget
K = 500 (1250 sweeps over the three levels).  Inputs are synthetic (seeded
generator, paper_1009_0881_gb300/synth.py).

  value  sweeps per second (all levels) with inputs resident in HBM
  e2e    the same through nmf_solve on pinned host buffers (H2D + D2H timed)

Also reported: time to reach (1 + 1e-3) times the FP64 oracle's final
objective, the plain single-level FP32 path, a roofline of the dominant
kernel (CUDA events per launch, live), the CPU oracle's speed, SM clocks.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-3 rel objective & sweeps/s vs plain FP32; served p50/p99 latency"
WORKLOAD = "grid19_n2429_r49"
L2_BYTES = 129 * 1024 * 1024


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--algo", default="hals")
    ap.add_argument("--levels", type=int, default=3)
    ap.add_argument("--iters", type=int, default=500)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision-form", action="store_true")
    ap.add_argument("--no-batched-form", action="store_true")
    ap.add_argument("--no-serving-form", action="store_true")
    ap.add_argument("--no-time-to-target-table", action="store_true")
    ap.add_argument("--no-sequence-table", action="store_true", help="skip the image-sequence (column coarsening) table")
    ap.add_argument("--no-analysis", action="store_true",
                    help="skip everything after the timed steps (for profiler launch lists)")
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-rate-low", type=float, default=40.0)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-precisions", default="fp32,bf16,bf16_fp32_finish,auto")
    ap.add_argument("--serve-max-batches", default="16,1")
    ap.add_argument("--_oracle_sample", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm): run in a single-threaded child
# ---------------------------------------------------------------------------
def oracle_sample_child(args):
    import numpy as np  # noqa: F401

    from oracle import nmf_oracle as o
    from paper_1009_0881_gb300 import synth

    gh, gw, n, r, sigma = synth.WORKLOADS[args.workload]
    p = synth.make_problem(gh, gw, n, r, sigma=sigma)
    sweeps = sum(_schedule_py(args.levels, args.iters))
    t0 = time.perf_counter()
    o.solve(p.M, gh, gw, p.V, p.W, args.algo, levels=args.levels, K=args.iters)
    dt = time.perf_counter() - t0
    print(json.dumps({"sweeps": sweeps, "seconds": dt}))


def _schedule_py(L, K):
    counts = [0] * L
    for lvl in range(L - 1):
        counts[lvl] = K // 4 + K // 2
    counts[L - 1] = K
    return counts


def workload_config(args, world=1, iters=None, gpu=True):
    """The `config` object of a bench line: the workload each step runs (iters = the sweep
    budget K actually run; the GPU arm also states how L2 is flushed between steps)."""
    from paper_1009_0881_gb300 import synth

    K = args.iters if iters is None else iters
    gh, gw, n, r, _ = synth.WORKLOADS[args.workload]
    sched = _schedule_py(args.levels, K)
    cfg = {"workload": f"{args.workload}: {gh}x{gw} grid, m={gh * gw}, n={n}, r={r}; {args.algo} V-cycle "
                       f"L={args.levels} K={K} ({sum(sched)} sweeps) + final error",
           "algo": args.algo, "levels": args.levels, "iters": K,
           "sweeps_per_step": sum(sched), "sweeps_per_level": sched,
           "parallelism": "replicas" if world > 1 else "single GPU"}
    if gpu:
        cfg["l2"] = "inputs (3.5 MB) fit in L2: a 258 MB buffer is written between timed steps"
    return cfg


def run_oracle_sample(args, K=None, levels=None, threads=1):
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--_oracle_sample", "--workload", args.workload, "--algo",
           args.algo, "--levels", str(levels or args.levels), "--iters", str(K or args.iters)]
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, check=True).stdout.strip().splitlines()[-1]
    return json.loads(out)


# sweep budget K of one reference-arm step (a bounded sample of the K = 500 workload)
REFERENCE_ITERS = 40


def host_cpu():
    """CPU model and logical core count of this host (for the CPU-baseline records)."""
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
            else:
                f.seek(0)
                for line in f:
                    if line.startswith("CPU part"):
                        model = "Arm CPU part " + line.split(":", 1)[1].strip()
                        break
    except OSError:
        pass
    return f"{model}, nproc {os.cpu_count()}"


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    samples = []
    for _ in range(args.warmup):
        run_oracle_sample(args, K=REFERENCE_ITERS)
    for _ in range(args.steps):
        samples.append(run_oracle_sample(args, K=REFERENCE_ITERS))
    sweeps = sum(s["sweeps"] for s in samples)
    secs = sum(s["seconds"] for s in samples)
    value = sweeps / secs
    desc = (f"FP64 numpy oracle, single thread; each step a bounded sample of the workload: {args.workload} "
            f"{args.algo} V-cycle L={args.levels} with K={REFERENCE_ITERS} ({samples[0]['sweeps']} sweeps) instead "
            f"of K={args.iters}, throughput in sweeps/s; host {host_cpu()}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, world, iters=REFERENCE_ITERS, gpu=False),
        "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        import tempfile

        self.path = os.path.join(tempfile.gettempdir(), f"nmf_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = list(csv.reader(io.StringIO(open(self.path).read())))
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in rows:
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                smax = float(row[2])
            except ValueError:
                continue
            for nm, v in zip(names, row[5:9]):
                if v.strip().lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main_ours(args):
    import numpy as np
    import torch

    from paper_1009_0881_gb300 import native, replicas, synth

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # CPU baseline before any GPU work (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = run_oracle_sample(args)
        ncores = os.cpu_count() or 1
        sa = run_oracle_sample(args, threads=ncores)
        cpu = {"value": s["sweeps"] / s["seconds"], "unit": "sweeps/s", "cores": 1, "kind": "oracle",
               "sample": (f"the whole step once: FP64 numpy oracle, one thread, {args.workload} {args.algo} "
                          f"V-cycle L={args.levels} K={args.iters} ({s['sweeps']} sweeps in {s['seconds']:.1f} s)"),
               "host": host_cpu(),
               "all_cores": {"value": sa["sweeps"] / sa["seconds"], "unit": "sweeps/s", "cores": ncores,
                             "sample": (f"the same step with numpy's BLAS on all {ncores} host threads "
                                        f"({sa['sweeps']} sweeps in {sa['seconds']:.1f} s)")}}

    from paper_1009_0881_gb300 import build
    build.build()
    gh, gw, n, r, sigma = synth.WORKLOADS[args.workload]
    # independent problem per rank (replicas): weak scaling
    prob = synth.make_problem(gh, gw, n, r, sigma=sigma, data_seed=replicas.replica_seed(rank))
    m = gh * gw
    sched = native.schedule("vcycle", args.levels, args.iters)
    sweeps_per_step = sum(sched)

    h = native.Handle(local)
    stream = torch.cuda.current_stream(dev)
    h.set_stream(stream.cuda_stream)
    Md = torch.from_numpy(prob.M).to(dev)
    V0d = torch.from_numpy(prob.V).to(dev)
    W0d = torch.from_numpy(prob.W).to(dev)
    Vd = torch.empty_like(V0d)
    Wd = torch.empty_like(W0d)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    err = {}

    def step():
        Vd.copy_(V0d)
        Wd.copy_(W0d)
        h.solve(Md, gh, gw, Vd, Wd, args.algo, levels=args.levels, iters=args.iters)
        err["f"] = h.error(Md, Vd, Wd)

    launches_per_step = 0
    for _ in range(args.warmup):
        step()
    step()
    launches_per_step = h.last_launch_count()  # error call
    Vd.copy_(V0d)
    Wd.copy_(W0d)
    h.solve(Md, gh, gw, Vd, Wd, args.algo, levels=args.levels, iters=args.iters)
    launches_per_step += h.last_launch_count()

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    total_ms = sum(times)
    clk = clocks.stop()
    value, total_ms = replicas.aggregate_throughput(sweeps_per_step * args.steps, total_ms, world, dev)
    ms_per_step = total_ms / args.steps

    # --- e2e through nmf_solve on pinned host buffers -----------------------
    Mh = torch.from_numpy(prob.M).pin_memory()
    Vh = torch.empty(prob.V.shape, dtype=torch.float32).pin_memory()
    Wh = torch.empty(prob.W.shape, dtype=torch.float32).pin_memory()
    V0h = torch.from_numpy(prob.V)
    W0h = torch.from_numpy(prob.W)

    def e2e_step():
        Vh.copy_(V0h)
        Wh.copy_(W0h)
        h.solve(Mh, gh, gw, Vh, Wh, args.algo, levels=args.levels, iters=args.iters)
        err["fh"] = h.error(Mh, Vh, Wh)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e2e_times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        e1.synchronize()
        e2e_times.append(e0.elapsed_time(e1))
    e2e_ms = sum(e2e_times) / args.steps
    h2d = 2 * (prob.M.nbytes + prob.V.nbytes + prob.W.nbytes)  # solve + error each stage M, V, W
    d2h = prob.V.nbytes + prob.W.nbytes + 8

    extra = {}
    if rank == 0 and not args.no_analysis:
        extra = analysis(args, h, prob, Md, V0d, W0d, Vd, Wd, stream, sched, err, gh, gw, m, n, r)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded generator, CBCL-shaped 19x19 images)",
            "config": workload_config(args, world),
            "e2e": {"value": world * sweeps_per_step / (e2e_ms / 1e3), "unit": "sweeps/s",
                    "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
        }
        line.update(extra)
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def analysis(args, h, prob, Md, V0d, W0d, Vd, Wd, stream, sched, err, gh, gw, m, n, r):
    """Time-to-target, the plain single-level path, and the roofline of the dominant kernel."""
    import numpy as np
    import torch

    from paper_1009_0881_gb300 import native

    out = {}
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "objectives.json")))
    key = f"grid19_{args.algo}_L{args.levels}_K{args.iters}"
    fstar = golden.get(key, {}).get("objective") if args.workload == WORKLOAD else None
    out["objective"] = {"gpu": err["f"], "oracle_fp64": fstar,
                        "rel_diff": None if fstar is None else abs(err["f"] - fstar) / fstar}
    if fstar is not None:
        target = (1 + 1e-3) * fstar
        Vd.copy_(V0d)
        Wd.copy_(W0d)
        cap = sched[0]
        tr = h.solve(Md, gh, gw, Vd, Wd, args.algo, levels=args.levels, iters=args.iters, trace_len=cap)
        hit = np.nonzero(tr <= target)[0]
        ttt = None
        if len(hit):
            # schedule position of that fine-level sweep: all coarse sweeps precede the post-smoothing
            s_fine = int(hit[0]) + 1
            pre = args.iters // 4
            stop = s_fine if s_fine <= pre else s_fine + sum(sched[1:])
            ms = []
            for _ in range(args.warmup + args.steps):
                Vd.copy_(V0d)
                Wd.copy_(W0d)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.solve(Md, gh, gw, Vd, Wd, args.algo, levels=args.levels, iters=args.iters, stop_after=stop)
                f = h.error(Md, Vd, Wd)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            assert f <= target * (1 + 1e-12), (f, target)
            ttt = {"ms": statistics.median(ms[args.warmup:]), "sweeps": stop, "fine_sweeps": s_fine}
        out["time_to_target"] = {"target": "(1+1e-3) x FP64 oracle objective of the same cycle",
                                 "objective_target": target, "multilevel": ttt}
        # plain single-level FP32 path with the same sweep budget K
        plain = {}
        ms = []
        for _ in range(2 + 3):
            Vd.copy_(V0d)
            Wd.copy_(W0d)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tr1 = h.solve(Md, gh, gw, Vd, Wd, args.algo, levels=1, iters=args.iters, trace_len=args.iters)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        plain["sweeps_per_s_with_trace"] = args.iters / (statistics.median(ms[2:]) / 1e3)
        Vd.copy_(V0d)
        Wd.copy_(W0d)
        ms = []
        for _ in range(2 + 3):
            Vd.copy_(V0d)
            Wd.copy_(W0d)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.solve(Md, gh, gw, Vd, Wd, args.algo, levels=1, iters=args.iters)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        plain["sweeps_per_s"] = args.iters / (statistics.median(ms[2:]) / 1e3)
        plain["ms_per_solve"] = statistics.median(ms[2:])
        plain["final_objective"] = float(tr1[-1])
        hit1 = np.nonzero(tr1 <= target)[0]
        plain["reaches_target_after_sweeps"] = int(hit1[0]) + 1 if len(hit1) else None
        # the single-level path for the wall time of the whole multilevel solve (the paper
        # compares the methods at equal time)
        ms = []
        for _ in range(2 + 3):
            Vd.copy_(V0d)
            Wd.copy_(W0d)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.solve(Md, gh, gw, Vd, Wd, args.algo, levels=args.levels, iters=args.iters)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        ml_ms = statistics.median(ms[2:])
        k_eq = max(1, int(ml_ms / (plain["ms_per_solve"] / args.iters)))
        Vd.copy_(V0d)
        Wd.copy_(W0d)
        tr2 = h.solve(Md, gh, gw, Vd, Wd, args.algo, levels=1, iters=k_eq, trace_len=k_eq)
        hit2 = np.nonzero(tr2 <= target)[0]
        plain["equal_wall_time"] = {"multilevel_ms": ml_ms, "sweeps": k_eq, "objective": float(tr2[-1]),
                                    "multilevel_objective": err["f"],
                                    "reaches_target_after_sweeps": int(hit2[0]) + 1 if len(hit2) else None}
        out["plain_fp32_single_level"] = plain

    out["roofline"], out["kernel_times_per_step_ms"] = roofline(args, h, Md, gh, gw, n, r, sched)
    if args.workload == WORKLOAD:
        out["other_algorithms"] = other_algorithms(args, h, Md, V0d, W0d, Vd, Wd, stream, golden, gh, gw)
        if not args.no_time_to_target_table:
            out["time_to_target_table"] = time_to_target_table(args, h, Md, V0d, W0d, Vd, Wd, stream, golden, gh, gw)
        if not args.no_sequence_table:
            out["image_sequence"] = sequence_table(h, stream, golden)
        out["time_split_vcycle"] = {a: time_split_vcycle(args, h, Md, V0d, W0d, Vd, Wd, stream, golden, gh, gw, a)
                                    for a in ("hals", "mu", "anls")}
    if not args.no_precision_form:
        out["precision_form"] = precision_form(args)
    if not args.no_batched_form:
        out["oracle_sample_forms"] = oracle_sample_forms(_sample_pool())
    if not (args.no_batched_form and args.no_serving_form):
        pool = batched_problems(BATCH_COUNT)
        if not args.no_batched_form:
            out["batched_form"] = batched_form(args, pool)
        if not args.no_serving_form:
            out["serving_form"] = serving_form(args, pool)
    return out


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture,
# valid while the kernel's sources hash to `src`; the captures and their commands are
# summarised under profiles/.
TRAFFIC = {
    "half_sweep_kernel": {"bytes": 0.5 * (4.969728e6 + 4.232192e6), "src": "a16cd947a6743266",
                          "files": ("fused.cu", "fused.cuh", "rowupdate.cuh", "ptx.cuh", "nmf_internal.cuh"),
                          "scope": "mean of the finest-level V-step (64-row tiles) and W-step (32-row tiles) launches, 19x19 grid n=2429 r=49"},
    "tc_gemm_kernel": {"bytes": 268.110080e6 + 12.589056e6, "src": "77970ec086c9a0b9",
                       "files": ("tc_gemm.cu", "tc_gemm.cuh", "ptx.cuh", "nmf_internal.cuh"),
                       "scope": "finest-level V-step product, 256x256 grid n=2000 r=64"},
}


def _traffic(kernel):
    """Captured DRAM bytes per launch, or None if the kernel changed since the capture."""
    import hashlib

    t = TRAFFIC[kernel]
    hsh = hashlib.sha256()
    for f in t["files"]:
        with open(os.path.join(ROOT, "paper_1009_0881_gb300", "csrc", f), "rb") as fh:
            hsh.update(fh.read())
    return t["bytes"] if hsh.hexdigest()[:16] == t["src"] else None


def time_to_target(h, Md, V0d, W0d, Vd, Wd, stream, gh, gw, algo, L, K, fstar, reps=3, warm=1, cols=False,
                   level_sweeps=None):
    """Wall time of a V-cycle solve (device-resident inputs, CUDA events) until the finest-level
    objective first reaches (1 + 1e-3) f*, f* the FP64 oracle's final objective for the same
    (algo, L, K): the per-sweep trace locates that sweep, then solves stopped right after it
    are timed.  None if the schedule never reaches the target.  cols: the V-cycle coarsens
    the columns of M too."""
    import numpy as np
    import torch

    from paper_1009_0881_gb300 import native

    if level_sweeps is None:
        sched = native.schedule("vcycle", L, K)
        pre = K // 4 if L > 1 else K
    else:
        pre_c, coarse_c, post_c = level_sweeps
        sched = [pre_c[0] + post_c[0]] + [pre_c[l] + post_c[l] for l in range(1, L - 1)] + [coarse_c]
        pre = pre_c[0]
    target = (1 + 1e-3) * fstar
    Vd.copy_(V0d)
    Wd.copy_(W0d)
    kw = {"level_sweeps": level_sweeps} if level_sweeps is not None else {}
    tr = h.solve(Md, gh, gw, Vd, Wd, algo, levels=L, iters=K, trace_len=sched[0], coarsen_columns=cols, **kw)
    hit = np.nonzero(tr <= target)[0]
    res = {"algo": algo, "levels": L, "iters": K, "oracle_fp64": fstar, "objective_target": target,
           "final_objective_gpu": float(tr[-1]) if len(tr) else None}
    if not len(hit):
        res["ms"] = None
        return res
    s_fine = int(hit[0]) + 1
    stop = s_fine if s_fine <= pre else s_fine + sum(sched[1:])
    ms = []
    for it in range(warm + reps):
        Vd.copy_(V0d)
        Wd.copy_(W0d)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.solve(Md, gh, gw, Vd, Wd, algo, levels=L, iters=K, stop_after=stop, coarsen_columns=cols, **kw)
        e1.record(stream)
        e1.synchronize()
        if it >= warm:
            ms.append(e0.elapsed_time(e1))
    f = h.error(Md, Vd, Wd)
    res.update(ms=statistics.median(ms), sweeps=stop, fine_sweeps=s_fine, objective_at_stop=f,
               reached=bool(f <= target * (1 + 1e-12)))
    return res


def _solve_ms(h, Md, V0d, W0d, Vd, Wd, stream, gh, gw, algo, L, K, reps=3, **kw):
    """Median CUDA-event time of a solve from the initial iterate (one untimed run first)."""
    import torch

    ms = []
    for it in range(reps + 1):
        Vd.copy_(V0d)
        Wd.copy_(W0d)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.solve(Md, gh, gw, Vd, Wd, algo, levels=L, iters=K, **kw)
        e1.record(stream)
        e1.synchronize()
        if it:
            ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def time_split_vcycle(args, h, Md, V0d, W0d, Vd, Wd, stream, golden, gh, gw, algo="hals"):
    """Algorithm V-cycle with its time budgets taken as time (T/4 before, T/4 to the coarser
    cycle, T/2 after): the per-sweep cost of each level is measured here, inside solves with
    explicit counts (100 extra sweeps on one level against a one-sweep-per-run cycle, median of
    three), the budget is the time of the single-level run's K sweeps, and nmf_time_schedule
    turns both into counts.  Reported: the counts, the time and objective of that V-cycle, the
    single-level run's, and the V-cycle's time to the single-level run's target."""
    from paper_1009_0881_gb300 import native

    L, K, extra = args.levels, args.iters, 100
    base = ([1] * (L - 1), 1, [1] * (L - 1))
    t0 = _solve_ms(h, Md, V0d, W0d, Vd, Wd, stream, gh, gw, algo, L, K, level_sweeps=base)
    costs = []
    for lvl in range(L):
        pre, coarse, post = [list(x) if isinstance(x, list) else x for x in base]
        if lvl == L - 1:
            coarse += extra
        else:
            post[lvl] += extra
        t = _solve_ms(h, Md, V0d, W0d, Vd, Wd, stream, gh, gw, algo, L, K, level_sweeps=(pre, coarse, post))
        costs.append(max(t - t0, 1e-6) / extra)
    budget = K * costs[0]
    counts = native.time_schedule(budget, costs)
    ms_ml = _solve_ms(h, Md, V0d, W0d, Vd, Wd, stream, gh, gw, algo, L, K, level_sweeps=counts)
    f_ml = h.error(Md, Vd, Wd)
    ms_sl = _solve_ms(h, Md, V0d, W0d, Vd, Wd, stream, gh, gw, algo, 1, K)
    f_sl = h.error(Md, Vd, Wd)
    out = {"algo": algo, "levels": L, "budget_fine_sweeps": K, "sweep_cost_ms_per_level": costs,
           "level_sweeps": {"pre": counts[0], "coarse": counts[1], "post": counts[2]},
           "multilevel": {"ms": ms_ml, "objective": f_ml}, "single_level": {"ms": ms_sl, "objective": f_sl}}
    g = golden.get(f"grid19_{algo}_timed_L3", {})
    if args.workload == WORKLOAD and g.get("level_sweeps") and [list(x) if isinstance(x, list) else x
                                                                for x in g["level_sweeps"]] == list(counts):
        out["multilevel"]["oracle_fp64"] = g["objective"]
        out["multilevel"]["rel_diff"] = abs(f_ml - g["objective"]) / g["objective"]
    f1 = golden.get(f"grid19_{algo}_L1_K{K}", {}).get("objective") if args.workload == WORKLOAD else None
    if f1 is not None:
        t = time_to_target(h, Md, V0d, W0d, Vd, Wd, stream, gh, gw, algo, L, K, f1, level_sweeps=counts)
        out["multilevel_to_single_level_target"] = {k: t.get(k) for k in ("objective_target", "ms", "sweeps",
                                                                         "fine_sweeps", "reached")}
    return out


def time_to_target_table(args, h, Md, V0d, W0d, Vd, Wd, stream, golden, gh, gw):
    """Time to (1 + 1e-3) f* for HALS, MU and ANLS (active set and block pivoting), multilevel
    (L = 3) and single-level (L = 1), K = 500, on the 19 x 19 workload; f* is the FP64
    oracle's objective of each (algo, L).  ANLS with block pivoting uses the active-set
    oracle's f* (the two reach the same NNLS solutions)."""
    out = {}
    for algo in ("hals", "mu", "anls", "anls_bpp"):
        for L in (3, 1):
            key = f"grid19_{'anls' if algo == 'anls_bpp' else algo}_L{L}_K{args.iters}"
            fstar = golden.get(key, {}).get("objective")
            name = f"{algo}_L{L}"
            if fstar is None:
                out[name] = {"ms": None, "note": f"no FP64 oracle value stored for {key}"}
                continue
            slow = algo.startswith("anls")
            out[name] = time_to_target(h, Md, V0d, W0d, Vd, Wd, stream, gh, gw, algo, L, args.iters, fstar,
                                       reps=1 if slow else 3, warm=0 if slow else 1)
            f1 = golden.get(f"grid19_{'anls' if algo == 'anls_bpp' else algo}_L1_K{args.iters}", {}).get("objective")
            if L > 1 and f1 is not None:
                # the same run against the single-level run's target (one objective for both)
                t1 = time_to_target(h, Md, V0d, W0d, Vd, Wd, stream, gh, gw, algo, L, args.iters, f1,
                                    reps=1 if slow else 3, warm=0 if slow else 1)
                out[name]["single_level_target"] = {k: t1.get(k) for k in ("objective_target", "ms", "sweeps",
                                                                            "fine_sweeps", "reached")}
    return out


def sequence_table(h, stream, golden):
    """Image sequences (32 x 32 frames, n = 4096, r = 16): time for the single-level run, the
    pixel-only V-cycle and the V-cycle that also coarsens the columns to reach (1 + 1e-3) f*,
    f* the FP64 oracle's single-level objective (the weakest of the three, so every run can
    reach it), and the wall time of the whole solve; HALS with K = 100 and ANLS with K = 20."""
    import torch

    from paper_1009_0881_gb300 import synth

    gh, gw, n, r, sigma = synth.SEQUENCE_WORKLOADS["seq32_n4096_r16"]
    p = synth.make_problem(gh, gw, n, r, sigma=sigma, sequence=True)
    dev = torch.device("cuda", 0)
    Md = torch.from_numpy(p.M).to(dev)
    V0d = torch.from_numpy(p.V).to(dev)
    W0d = torch.from_numpy(p.W).to(dev)
    Vd, Wd = V0d.clone(), W0d.clone()
    out = {"workload": "seq32_n4096_r16 (32x32 frames, n=4096, r=16, smooth along the sequence)"}
    for algo, K in (("hals", 100), ("anls", 20)):
        fstar = golden.get(f"seq32_{algo}_L1_K{K}", {}).get("objective")
        tab = {"K": K, "target": None if fstar is None else (1 + 1e-3) * fstar}
        for name, L, cols in (("L1", 1, False), ("L3", 3, False), ("L3_cols", 3, True)):
            key = f"seq32_{algo}_{'cols_' if cols else ''}L{L}_K{K}"
            res = {"ms_to_target": None}
            if fstar is not None:
                t = time_to_target(h, Md, V0d, W0d, Vd, Wd, stream, gh, gw, algo, L, K, fstar, cols=cols)
                res = {"ms_to_target": t["ms"], "sweeps_to_target": t.get("sweeps"),
                       "fine_sweeps_to_target": t.get("fine_sweeps")}
            ms = []
            for it in range(3):
                Vd.copy_(V0d)
                Wd.copy_(W0d)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.solve(Md, gh, gw, Vd, Wd, algo, levels=L, iters=K, coarsen_columns=cols)
                e1.record(stream)
                e1.synchronize()
                if it:
                    ms.append(e0.elapsed_time(e1))
            f = h.error(Md, Vd, Wd)
            fo = golden.get(key, {}).get("objective")
            res.update(ms_whole_solve=statistics.median(ms), objective=f, oracle_fp64=fo,
                       rel_diff=None if fo is None else abs(f - fo) / fo)
            tab[name] = res
        out[algo] = tab
    return out


def other_algorithms(args, h, Md, V0d, W0d, Vd, Wd, stream, golden, gh, gw):
    """MU and ANLS on the same workload, multilevel (L = 3) next to single-level, same sweep
    budget; objective against the FP64 oracle's stored value where one exists."""
    import torch

    from paper_1009_0881_gb300 import native

    out = {}
    for algo in ("mu", "anls", "anls_bpp"):
        for L in (3, 1):
            sweeps = sum(native.schedule("vcycle", L, args.iters))
            ms = []
            for it in range(2):
                Vd.copy_(V0d)
                Wd.copy_(W0d)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.solve(Md, gh, gw, Vd, Wd, algo, levels=L, iters=args.iters)
                e1.record(stream)
                e1.synchronize()
                if it:
                    ms.append(e0.elapsed_time(e1))
            f = h.error(Md, Vd, Wd)
            fstar = golden.get(f"grid19_{'anls' if algo == 'anls_bpp' else algo}_L{L}_K{args.iters}", {}).get("objective")
            out[f"{algo}_L{L}"] = {"ms_per_solve": ms[0], "sweeps": sweeps, "sweeps_per_s": sweeps / (ms[0] / 1e3),
                                   "objective": f, "oracle_fp64": fstar,
                                   "rel_diff": None if fstar is None else abs(f - fstar) / fstar}
    return out


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def roofline(args, h, Md, gh, gw, n, r, sched):
    """Per-kernel CUDA-event timing at each level's size, weighted by the sweep schedule.

    The FP32 path runs one fused kernel per half-sweep (products, reduction and
    factor update) and, on coarse levels whose V has at most 32 rows, all sweeps of
    a run in one persistent kernel.  Algorithmic flops per sweep (Appendix A.1
    accounting, multiply-add = 2): F_l = 4 m_l n r + 4 (m_l + n) r^2, i.e. the two
    products with M plus the Gram matrices W W^T, V^T V and the update terms
    V (W W^T), (V^T V) W.  The roofline line reports the kernel with the larger
    share of the step.
    """
    import torch

    peaks = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sms, _ = h.device_info()
    fp32_peak = n_sms * 128 * 2 * sm_mhz * 1e6  # FFMA lanes x 2 flops x clock
    dev = Md.device
    Ml = Md
    hh, ww = gh, gw
    hs = "half_sweep_kernel (fused products + update)"
    cr = "coarse_run_kernel (persistent coarse-level sweeps)"
    kinds = {hs: [0.0, 0.0, 0], cr: [0.0, 0.0, 0], "error_tile_kernel": [0.0, 0.0, 0]}
    g = torch.Generator(device="cpu").manual_seed(0)
    W = torch.rand(r, n, generator=g).to(dev)
    L = len(sched)
    for lvl, count in enumerate(sched):
        ml = hh * ww
        V = torch.rand(ml, r, generator=g).to(dev)
        # Appendix A.1 accounting of one sweep (multiply-add = 2): 4 m_l n r for the two
        # products with M, 4 (m_l + n) r^2 for the Gram matrices and the r^2 update terms
        flv = 2 * ml * n * r + 2 * (ml + n) * r * r
        flw = 2 * ml * n * r + 2 * (ml + n) * r * r
        tc = h.profile_coarse(Ml, V, W, args.algo, sweeps=100) if lvl > 0 else None
        if tc is not None:
            kinds[cr][0] += count * tc
            kinds[cr][1] += count * (flv + flw)
            kinds[cr][2] += 1 if lvl == L - 1 else 2  # one run per visit of the level (V-cycle)
        else:
            t = h.profile_sweep(Ml, V, W, args.algo, reps=50)
            kinds[hs][0] += count * (t[0] + t[2])
            kinds[hs][1] += count * (flv + flw)
            kinds[hs][2] += 2 * count
        if lvl == 0:
            t0 = h.profile_sweep(Ml, V, W, args.algo, reps=5) if tc is not None else t
            kinds["error_tile_kernel"] = [t0[4], 2 * ml * n * r, 1]
        if lvl + 1 < len(sched):
            hc, wc = (hh + 1) // 2, (ww + 1) // 2
            Mc = torch.empty(hc * wc, n, device=dev)
            h.restrict(Ml, hh, ww, Mc)
            Ml, hh, ww = Mc, hc, wc
    times = {k: v[0] for k, v in kinds.items() if v[2] > 0}
    top = hs if kinds[hs][0] >= kinds[cr][0] else cr
    ms, flops, launches = kinds[top]
    achieved = flops / (ms / 1e3) / 1e12
    peak = fp32_peak / 1e12
    roof = {"kernel": top, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": _traffic("half_sweep_kernel") if top == hs else None,
            "traffic_scope": TRAFFIC["half_sweep_kernel"]["scope"] if top == hs else None,
            "launches_per_step": launches, "mean_launch_us": 1e3 * ms / launches,
            "peak_basis": f"FP32 FFMA: {n_sms} SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz (derived)",
            "share_of_step": {k: v[0] / sum(x[0] for x in kinds.values()) for k, v in kinds.items() if v[2] > 0}}
    return roof, times


PRECISION_WORKLOADS = [("grid112x92_n400_r40", 3, 100), ("grid256_n2000_r64", 3, 100)]


def precision_form(args, reps=3):
    """BF16 operands on the tensor cores (tcgen05, FP32 accumulation) next to the plain FP32
    path on the precision-form workloads; objective against the FP64 oracle's (stored) value."""
    import torch

    from paper_1009_0881_gb300 import native, synth

    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "objectives.json")))
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    stream = torch.cuda.current_stream()
    out = {}
    for wl, L, K in PRECISION_WORKLOADS:
        gh, gw, n, r, sigma = synth.WORKLOADS[wl]
        p = synth.make_problem(gh, gw, n, r, sigma=sigma)
        m = gh * gw
        Md = torch.from_numpy(p.M).cuda()
        V0 = torch.from_numpy(p.V).cuda()
        W0 = torch.from_numpy(p.W).cuda()
        sweeps = sum(native.schedule("vcycle", L, K))
        key = f"{wl.split('_')[0]}_hals_L{L}_K{K}"
        fstar = golden.get(key, {}).get("objective")
        res = {"levels": L, "iters": K, "sweeps": sweeps, "m": m, "n": n, "r": r}
        for label, prec in (("bf16_tcgen05", native.NMF_BF16), ("bf16_fp32_finish", native.NMF_BF16_FP32),
                            ("fp32", native.NMF_FP32)):
            with native.Handle(0, precision=prec) as hh:
                hh.set_stream(stream.cuda_stream)
                V = V0.clone()
                W = W0.clone()
                ms = []
                for it in range(1 + reps):
                    V.copy_(V0)
                    W.copy_(W0)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    hh.solve(Md, gh, gw, V, W, "hals", levels=L, iters=K)
                    e1.record(stream)
                    e1.synchronize()
                    if it:
                        ms.append(e0.elapsed_time(e1))
                f = hh.error(Md, V, W)
                t = statistics.median(ms)
                entry = {"ms_per_solve": t, "sweeps_per_s": sweeps / (t / 1e3), "objective": f,
                         "rel_diff_vs_fp64_oracle": None if fstar is None else (f - fstar) / fstar}
                if fstar is not None:
                    # time to (1 + 1e-3) f*: the float32 path from its trace; the BF16 forms
                    # reach it only at the end of the solve if at all (their last sweeps decide)
                    if prec == native.NMF_FP32:
                        Vt, Wt = V0.clone(), W0.clone()
                        tt = time_to_target(hh, Md, V0, W0, Vt, Wt, stream, gh, gw, "hals", L, K, fstar)
                        entry["time_to_1e-3_ms"] = tt["ms"]
                    else:
                        entry["time_to_1e-3_ms"] = t if f <= (1 + 1e-3) * fstar else None
                if prec == native.NMF_BF16:
                    # tcgen05 product of the V-step at the finest level: HBM roofline
                    g = torch.Generator(device="cpu").manual_seed(1)
                    Vr = torch.rand(m, r, generator=g).cuda()
                    tt = hh.profile_sweep(Md, Vr, W0, "hals", reps=20)
                    # algorithmic bytes: read bf16 M and W once, write the FP32 product once
                    bytes_v = m * n * 2 + r * n * 2 + m * r * 4
                    ach = bytes_v / (tt[0] / 1e3) / 1e9
                    entry["kernel_ms"] = {"tc_gemm V-step": tt[0], "gram+rows V": tt[1], "tc_gemm W-step": tt[2],
                                          "gram+rows W": tt[3]}
                    # DRAM traffic was captured on the 256 x 256 workload only
                    captured = wl == "grid256_n2000_r64"
                    entry["roofline"] = {"kernel": "tc_gemm_kernel (V-step, A = M W^T, finest level)",
                                         "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                                         "frac": ach / hbm, "peak_basis": "measured (MEASURED_PEAKS.json hbm_gbs)",
                                         "traffic": _traffic("tc_gemm_kernel") if captured else None,
                                         "traffic_scope": TRAFFIC["tc_gemm_kernel"]["scope"] if captured
                                         else "not captured on this workload",
                                         "algorithmic_bytes": bytes_v}
                res[label] = entry
        res["oracle_fp64_objective"] = fstar
        a, b = res["bf16_fp32_finish"].get("time_to_1e-3_ms"), res["fp32"].get("time_to_1e-3_ms")
        res["bf16_fp32_finish_speedup_to_1e-3"] = (b / a) if (a and b) else None
        out[wl] = res
    return out


# Batched and serving forms: 64 problems of uneven size (side in {16,19,32,64,92,128},
# n ~ U[200,4000], r ~ U[5,64], data seeds 0..63), multilevel HALS L = 3 with the
# device-side stopping rule |f_{t-1} - f_t| <= 1e-3 f_t on the finest-level sweeps.
BATCH_COUNT = 64
BATCH_LEVELS = 3
BATCH_ITERS = {"hals": 200, "mu": 200, "anls": 20}
# serving: per-request sweep caps (the 1e-3 relative-change rule ends most requests earlier;
# ANLS sweeps are exact block minimisations, far costlier, and converge in few sweeps)
SERVE_ITERS = {"hals": 100, "mu": 100, "anls": 8}
BATCH_TOL = 1e-3


def batched_problems(count):
    """The seeded uneven-size problems, drawn in parallel in spawned processes."""
    from concurrent.futures import ProcessPoolExecutor
    import multiprocessing as mp

    from paper_1009_0881_gb300 import synth

    sizes = synth.batched_sizes(count)
    workers = max(1, min(16, os.cpu_count() or 1))
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(synth.make_problem, side, side, n, r, 0.04 * side if side > 19 else 2.0, i)
                for i, (side, n, r) in enumerate(sizes)]
        return [f.result() for f in futs]


def _request(p, Md, algo, V=None, W=None, iters=None):
    return dict(M=Md, grid_h=p.grid_h, grid_w=p.grid_w, V=p.V.copy() if V is None else V,
                W=p.W.copy() if W is None else W, algo=algo, levels=BATCH_LEVELS,
                iters=(iters or BATCH_ITERS)[algo], rel_tol=BATCH_TOL)


def _batch_flops(pool, res, L, K):
    """Algorithmic flops of a solved batch (Appendix A.1 per sweep, 4 m_l n r + 4 (m_l + n) r^2)
    from each problem's schedule, its finest-level post-smoothing cut to the sweeps it ran."""
    import numpy as np

    from paper_1009_0881_gb300 import native

    total = 0.0
    for p, (_, sweeps, _) in zip(pool, res):
        m, n = p.M.shape
        r = p.V.shape[1]
        per_level = native.schedule("vcycle", L, K)
        full = int(np.sum(per_level))
        gh, gw = p.grid_h, p.grid_w
        for lvl, cnt in enumerate(per_level):
            ml = gh * gw
            if lvl == 0:
                cnt = cnt - (full - sweeps)
            total += cnt * (4.0 * ml * n * r + 4.0 * (ml + n) * r * r)
            gh, gw = (gh + 1) // 2, (gw + 1) // 2
    return total


def batched_form(args, pool, reps=3):
    """All 64 problems in one nmf_solve_batch (one CUDA graph of concurrent branches), FP32 and
    BF16, and in one nmf_solve_grouped (every half-sweep one persistent launch over the tiles
    of all 64; FP32), next to the plain FP32 path solving them one request at a time."""
    import torch

    from paper_1009_0881_gb300 import native

    stream = torch.cuda.current_stream()
    Mds = [torch.from_numpy(p.M).cuda() for p in pool]
    V0s = [torch.from_numpy(p.V).cuda() for p in pool]
    W0s = [torch.from_numpy(p.W).cuda() for p in pool]
    Vs = [v.clone() for v in V0s]
    Ws = [w.clone() for w in W0s]
    reqs = [_request(p, Md, "hals", V, W) for p, Md, V, W in zip(pool, Mds, Vs, Ws)]

    def reset():
        for V, W, V0, W0 in zip(Vs, Ws, V0s, W0s):
            V.copy_(V0)
            W.copy_(W0)

    out = {"problems": len(pool), "levels": BATCH_LEVELS, "iters_cap": BATCH_ITERS["hals"], "rel_tol": BATCH_TOL,
           "algo": "hals", "flops_per_batch_note": "sum over problems of the Appendix A.1 sweep cost"}
    for label, prec, batched in (("batched_fp32", native.NMF_FP32, True), ("batched_bf16", native.NMF_BF16, True),
                                 ("batched_bf16_fp32_finish", native.NMF_BF16_FP32, True),
                                 ("grouped_fp32", native.NMF_FP32, "grouped"),
                                 ("sequential_plain_fp32", native.NMF_FP32, False)):
        with native.Handle(0, precision=prec) as hh:
            hh.set_stream(stream.cuda_stream)
            ms = []
            for it in range(1 + reps):
                reset()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if batched == "grouped":
                    res = hh.solve_batch(reqs, grouped=True)
                elif batched:
                    res = hh.solve_batch(reqs)
                else:
                    res = [hh.solve_batch([d])[0] for d in reqs]
                e1.record(stream)
                e1.synchronize()
                if it:
                    ms.append(e0.elapsed_time(e1))
            t = statistics.median(ms)
            sweeps = sum(x[1] for x in res)
            fl = _batch_flops(pool, res, BATCH_LEVELS, BATCH_ITERS["hals"])
            out[label] = {"ms_per_batch": t, "solves_per_s": len(pool) / (t / 1e3), "sweeps": sweeps,
                          "sweeps_per_s": sweeps / (t / 1e3), "all_ok": all(x[0] == 0 for x in res),
                          "objective_sum": sum(x[2] for x in res), "algorithmic_tflop": fl / 1e12,
                          "tflop_per_s": fl / (t / 1e3) / 1e12}
    out["speedup_batched_bf16_vs_sequential_fp32"] = (out["sequential_plain_fp32"]["ms_per_batch"]
                                                      / out["batched_bf16"]["ms_per_batch"])
    out["speedup_batched_fp32_vs_sequential_fp32"] = (out["sequential_plain_fp32"]["ms_per_batch"]
                                                      / out["batched_fp32"]["ms_per_batch"])
    out["speedup_grouped_fp32_vs_sequential_fp32"] = (out["sequential_plain_fp32"]["ms_per_batch"]
                                                      / out["grouped_fp32"]["ms_per_batch"])
    out["speedup_batched_bf16_fp32_finish_vs_sequential_fp32"] = (out["sequential_plain_fp32"]["ms_per_batch"]
                                                                  / out["batched_bf16_fp32_finish"]["ms_per_batch"])
    del Mds, V0s, W0s, Vs, Ws
    torch.cuda.empty_cache()
    return out


def _sample_pool():
    """The 64 requests of tests/golden/served_sample.json with their FP64 oracle objectives."""
    from concurrent.futures import ProcessPoolExecutor
    import multiprocessing as mp

    from paper_1009_0881_gb300 import synth

    G = json.load(open(os.path.join(ROOT, "tests", "golden", "served_sample.json")))
    rows = G["requests"]
    workers = max(1, min(16, os.cpu_count() or 1))
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(synth.make_problem, q["side"], q["side"], q["n"], q["r"], q["sigma"], q["index"])
                for q in rows]
        return [(q, f.result()) for q, f in zip(rows, futs)]


def oracle_sample_forms(sample, reps=3):
    """The 64 sampled requests (uneven sizes, HALS / MU / ANLS, three levels, short fixed
    budgets) solved as one batch and through the server, in each precision, every result
    against the FP64 oracle's objective for the same request: time per batch, solves/s and
    the relative errors (the precision forms' time to results within 1e-3 of the oracle)."""
    import numpy as np
    import torch

    from paper_1009_0881_gb300 import native

    stream = torch.cuda.current_stream()
    Mds = [torch.from_numpy(p.M).cuda() for _, p in sample]
    out = {"requests": len(sample), "source": "tests/golden/served_sample.json (FP64 oracle objectives)"}
    for label, prec in (("fp32", native.NMF_FP32), ("bf16", native.NMF_BF16), ("bf16_fp32_finish", native.NMF_BF16_FP32),
                        ("auto", native.NMF_AUTO)):
        def reqs():
            return [dict(M=Md, grid_h=q["side"], grid_w=q["side"], V=p.V.copy(), W=p.W.copy(), algo=q["algo"],
                         levels=q["levels"], iters=q["iters"]) for (q, p), Md in zip(sample, Mds)]
        res = {}
        with native.Handle(0, precision=prec) as hh:
            hh.set_stream(stream.cuda_stream)
            ms = []
            for it in range(1 + reps):
                batch = reqs()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                got = hh.solve_batch(batch)
                e1.record(stream)
                e1.synchronize()
                if it:
                    ms.append(e0.elapsed_time(e1))
            errs = [abs(g[2] - q["objective"]) / q["objective"] for g, (q, _) in zip(got, sample)]
            res["batch"] = {"ms_per_batch": statistics.median(ms), "solves_per_s": len(sample) / (statistics.median(ms) / 1e3),
                            "max_rel_error": max(errs), "median_rel_error": float(np.median(errs)),
                            "within_1e-3": int(sum(e <= 1e-3 for e in errs))}
        with native.Server(0, hbm_budget_bytes=40 * 10**9, slots=8, precision=prec) as srv:
            t0 = time.perf_counter()
            tickets = [srv.submit(d) for d in reqs()]
            got = [srv.poll(t, -1) for t in tickets]
            wall = time.perf_counter() - t0
            errs = [abs(g[2] - q["objective"]) / q["objective"] for g, (q, _) in zip(got, sample)]
            lat = np.array([g[3] for g in got])
            res["served"] = {"wall_s": wall, "max_rel_error": max(errs), "median_rel_error": float(np.median(errs)),
                             "within_1e-3": int(sum(e <= 1e-3 for e in errs)),
                             "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                             "note": "all 64 submitted at once, first-seen shapes (plans and graphs built inside)"}
        out[label] = res
    del Mds
    torch.cuda.empty_cache()
    return out


def serving_form(args, pool):
    """Poisson arrivals into nmf_server: sizes from the 64-problem pool, algorithm uniform over
    HALS/MU/ANLS, 40 GB workspace budget.  M stays on the device; each request brings its
    initial V, W from host memory and gets the result back there.  Run at the configured
    rate and again at a lower rate the server sustains (latency without a standing queue)."""
    import torch

    from paper_1009_0881_gb300 import native

    # each request brings M from pinned host memory: its upload is part of its latency
    Mhs = [torch.from_numpy(p.M).pin_memory() for p in pool]
    algos = ("hals", "mu", "anls")
    budget = 40 * 10**9
    out = {"rate_per_s": args.serve_rate, "low_rate_per_s": args.serve_rate_low, "seconds": args.serve_seconds,
           "slots": args.serve_slots, "hbm_budget_bytes": budget, "levels": BATCH_LEVELS, "iters_cap": SERVE_ITERS,
           "rel_tol": BATCH_TOL, "sizes": "uniform over the 64 seeded batched-form problems",
           "latency": "from nmf_server_submit to completion; M, V0, W0 uploaded from pinned host memory "
                      "and V, W returned to it inside that time",
           "max_batch": "requests a slot takes at once (NMF_SERVE_MAX_BATCH): 16 = one graph per combination "
                        "of shapes, 1 = the cached graph of each shape"}
    precs = {"fp32": native.NMF_FP32, "bf16": native.NMF_BF16, "bf16_fp32_finish": native.NMF_BF16_FP32,
             "auto": native.NMF_AUTO}
    for label in args.serve_precisions.split(","):
        prec = precs[label]
        for mb in (int(x) for x in args.serve_max_batches.split(",")):
            os.environ["NMF_SERVE_MAX_BATCH"] = str(mb)
            with native.Server(0, hbm_budget_bytes=budget, slots=args.serve_slots, precision=prec) as srv:
                # warm-up: every (problem, algorithm) once, so the slots' graphs and workspaces exist
                t0 = time.perf_counter()
                tickets = [srv.submit(_request(p, Mh, a, iters=SERVE_ITERS)) for p, Mh in zip(pool, Mhs) for a in algos]
                warm = [srv.poll(t, -1) for t in tickets]
                res = {"warmup_s": time.perf_counter() - t0, "warmup_ok": all(w[0] == 0 for w in warm)}
                res["offered"] = _poisson_run(srv, pool, Mhs, args.serve_rate, args.serve_seconds, seed=7)
                if mb == 16 or args.serve_max_batches == str(mb):
                    res["low_rate"] = _poisson_run(srv, pool, Mhs, args.serve_rate_low, args.serve_seconds, seed=8)
                out[f"{label}_max_batch{mb}"] = res
    os.environ.pop("NMF_SERVE_MAX_BATCH", None)
    del Mhs
    torch.cuda.empty_cache()
    return out


def _poisson_run(srv, pool, Mds, rate, seconds, seed):
    """Submit Poisson arrivals at `rate` for `seconds`, then drain; latency and throughput."""
    import numpy as np

    from paper_1009_0881_gb300 import synth

    algos = ("hals", "mu", "anls")
    n_req = int(rate * seconds * 1.5) + 16
    gaps = synth.exponential(seed, 11, n_req) / rate
    pick = synth.uniform(seed, 12, n_req)
    lat, outstanding, status, by_algo, held = [], {}, [], {a: 0 for a in algos}, 0
    t_start = time.perf_counter()
    t_next = t_start
    t_end = t_start + seconds
    i = 0

    def drain(wait):
        for t in list(outstanding):
            r = srv.poll(t, wait)
            if r is not None:
                status.append(r[0])
                lat.append(r[3])
                del outstanding[t]

    while True:
        now = time.perf_counter()
        if now >= t_end or i + 1 >= n_req:
            break
        if now >= t_next:
            k = min(int(pick[i] * 3 * len(pool)), 3 * len(pool) - 1)
            a = algos[k % 3]
            p, Md = pool[k // 3], Mds[k // 3]
            outstanding[srv.submit(_request(p, Md, a, iters=SERVE_ITERS))] = a
            by_algo[a] += 1
            i += 1
            t_next += gaps[i]
            continue
        drain(0)
        held = max(held, srv.stats()["bytes_held"])
        time.sleep(min(max(t_next - time.perf_counter(), 0.0), 0.001))
    submitted = i
    drain(-1)
    wall = time.perf_counter() - t_start
    lat_a = np.array(lat)
    return {"rate_per_s": rate, "submitted": submitted, "completed": len(lat), "all_ok": all(x == 0 for x in status),
            "solves_per_s": len(lat) / wall, "wall_s": wall,
            "latency_ms": {"p50": float(np.percentile(lat_a, 50)), "p99": float(np.percentile(lat_a, 99)),
                           "mean": float(lat_a.mean()), "max": float(lat_a.max())},
            "per_algo_requests": by_algo, "max_bytes_held": held}

if __name__ == "__main__":
    a = parse_args()
    if a._oracle_sample:
        oracle_sample_child(a)
    elif a.impl == "reference":
        reference_arm(a)
    else:
        main_ours(a)
