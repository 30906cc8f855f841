#!/usr/bin/env python3
"""Benchmark: implicit IB step time to a 1e-8 relative residual on GB300.

Workload (default): the 256^2 periodic MAC grid with the 512-point elastic
ellipse (semi-axes 0.28/0.22 at (0.5, 0.5), rest length 2*pi*0.25/512), rho =
mu = 1, swept over kappa in {1, 1e2, 1e4, 1e6} x dt in {1e-3, 1e-2}: one bench
step = one backward-Euler IB step (set-up + MG-preconditioned FGMRES to 1e-8
+ point update) for each of the 8 cases, inputs resident on the device.
value = mean wall time per implicit IB step (ms), CUDA events, L2 flushed
between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp32|fp64] [--box B]

Under torchrun each rank solves the whole sweep on its own GPU (independent
replicas, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import ib_workloads as W  # noqa: E402

METRIC = "implicit IB step time to 1e-8 residual; V-cycle DOF/s; mixed/learned vs FP64"
UNIT = "ms per implicit IB step"
CASES = [(k, dt) for dt in (1e-3, 1e-2) for k in (1.0, 1e2, 1e4, 1e6)]
N_GRID = 256
N_POINTS = 512


def workload_problems(box):
    probs = []
    for k, dt in CASES:
        p = W.single_ellipse(N=N_GRID, n_points=N_POINTS, kappa=k, dt=dt)
        p.box = box
        probs.append(p)
    return probs


def config_dict(args):
    return {"workload": "256^2 MAC grid, 512-point ellipse, kappa x dt sweep (8 cases)",
            "N": N_GRID, "n_points": N_POINTS, "cases": [[k, dt] for k, dt in CASES],
            "box": args.box, "precision": args.precision, "nu": [1, 1], "tol": 1e-8,
            "max_iters": args.max_iters, "escalate": args.precision == "fp32",
            "l2": "flushed (256 MiB write) before every timed step",
            "parallelism": "replicas" if args.world > 1 else "single GPU"}


# ----------------------------------------------------------------------------- clocks

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + CLOCK_QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# ----------------------------------------------------------------------------- distributed helpers

def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def reduce_max(value, world):
    """Max over ranks (a host scalar); identity at world size 1."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value, world):
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate(step_ms_local, n_ib_steps_local, world):
    """Whole-job ms per implicit IB step: the slowest rank's time over all ranks' steps."""
    t_max = reduce_max(sum(step_ms_local), world)
    n_tot = reduce_sum(n_ib_steps_local, world)
    return t_max / max(n_tot, 1.0), t_max


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ----------------------------------------------------------------------------- CPU oracle

def oracle_sample_ms(box, case_index=2):
    """Time the CPU oracle (as it stands) on one implicit step of one sweep case."""
    from oracle import ib_oracle as O

    p = workload_problems(box)[case_index]
    t = time.perf_counter()
    r = O.solve_step(p)
    dt = time.perf_counter() - t
    return 1e3 * dt, r.solve.iters


def run_reference(args):
    rank, world, _ = args.rank, args.world, args.local_rank
    if rank != 0:
        return 0
    times = []
    for s in range(args.warmup + args.steps):
        ms, its = oracle_sample_ms(args.box, case_index=s % len(CASES) if args.rotate else 2)
        if s >= args.warmup:
            times.append(ms)
    v = float(np.mean(times))
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_dict(args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "one implicit step of the kappa=1e4, dt=1e-3 case per bench step "
                                       "(scipy CSR oracle, single-threaded sparse kernels)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm

def run_ours(args):
    import torch

    import paper_1311_5614_gb300 as pkg

    rank, world, local_rank = args.rank, args.world, args.local_rank
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    probs = workload_problems(args.box)
    solvers = [pkg.IBSolver.from_problem(p, precision=args.precision, max_iters=args.max_iters) for p in probs]
    nn = 3 * N_GRID * N_GRID
    X0 = [torch.tensor(p.X, dtype=torch.float64, device=dev) for p in probs]
    Xw = [x.clone() for x in X0]
    up = [torch.zeros(nn, dtype=torch.float64, device=dev) for _ in probs]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream()
    stats = [None] * len(probs)

    def one_step():
        for i, s in enumerate(solvers):
            Xw[i].copy_(X0[i])
            stats[i] = s.solve_step(None, up[i], Xw[i])

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    # timed region
    clk = ClockSampler(local_rank)
    launches0 = sum(s.launch_count() for s in solvers)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    clk.start()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        one_step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    barrier(world)
    clocks = clk.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    gpu_launches = sum(s.launch_count() for s in solvers) - launches0
    per_ib_ms, t_max = aggregate(step_ms, args.steps * len(probs), world)
    iters = [st["iters"] for st in stats]
    status = [st["status"] for st in stats]
    escal = [st["escalated_at"] for st in stats]

    # end-to-end through the C ABI with host buffers: H2D of X^n, D2H of u, v, p and X^{n+1}
    Xh = [torch.tensor(p.X, dtype=torch.float64).pin_memory() for p in probs]
    uph = [torch.empty(nn, dtype=torch.float64).pin_memory() for _ in probs]
    Xoh = [torch.empty_like(x) .pin_memory() for x in Xh]
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i, s in enumerate(solvers):
            Xw[i].copy_(Xh[i], non_blocking=True)
            s.solve_step(None, up[i], Xw[i])
            uph[i].copy_(up[i], non_blocking=True)
            Xoh[i].copy_(Xw[i], non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    e2e_per, _ = aggregate(e2e_ms, args.steps * len(probs), world)
    h2d = sum(x.numel() * 8 for x in Xh)
    d2h = sum(u.numel() * 8 for u in uph) + sum(x.numel() * 8 for x in Xoh)

    # V-cycle throughput on the kappa = 1e4, dt = 1e-3 case (the preconditioner alone)
    vs = solvers[2]
    bv = torch.randn(nn, dtype=torch.float64, device=dev)
    wv = torch.zeros_like(bv)
    for _ in range(3):
        vs.vcycle(bv, wv)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nv = 20
    a.record(stream)
    for _ in range(nv):
        vs.vcycle(bv, wv)
    b.record(stream)
    torch.cuda.synchronize()
    vcycle_ms = a.elapsed_time(b) / nv
    vcycle_dofs = nn / (vcycle_ms * 1e-3)

    # profiled pass (separate from the timed region): per-class device time and bytes
    for s in solvers:
        s.profile(True)
    one_step()
    torch.cuda.synchronize()
    prof = {}
    for s in solvers:
        for name, (n_, ms_, by_) in s.profile_read().items():
            q = prof.setdefault(name, [0, 0.0, 0.0])
            q[0] += n_
            q[1] += ms_
            q[2] += by_
        s.profile(False)
    hot = [c for c in ("stokes", "box", "interp", "spread", "transfer")]
    dom = max(hot, key=lambda c: prof[c][1])
    n_, ms_, by_ = prof[dom]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    achieved = (by_ / n_) / (ms_ / n_ * 1e-3) / 1e9 if n_ and ms_ > 0 else 0.0
    roofline = {"bound": "hbm", "kernel_class": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src, "traffic": args.traffic,
                "launches": n_, "avg_launch_us": 1e3 * ms_ / max(n_, 1),
                "alg_bytes_per_launch": by_ / max(n_, 1),
                "share_of_step": ms_ / max(sum(v[1] for v in prof.values()), 1e-30)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ms_cpu, its_cpu = oracle_sample_ms(args.box, 2)
        cpu = {"value": ms_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "one implicit step of the kappa=1e4, dt=1e-3 case (%d FGMRES iterations)" % its_cpu}

    for s in solvers:
        s.close()
    if rank == 0:
        line = {"metric": METRIC, "value": per_ib_ms, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 V-cycle + f64 Krylov" if args.precision == "fp32" else "f64",
                "data": "synthetic", "config": config_dict(args),
                "e2e": {"value": e2e_per, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "roofline": roofline, "cpu_baseline": cpu, "gpu_launches": int(gpu_launches),
                "clocks": clocks, "iters": iters, "status": status, "escalated_at": escal,
                "vcycle": {"ms": vcycle_ms, "dof_per_s": vcycle_dofs, "dof": nn,
                           "case": "kappa=1e4, dt=1e-3"},
                "wall_s_timed": t_wall,
                "profile": {k: {"launches": v[0], "ms": v[1], "bytes": v[2]} for k, v in prof.items()}}
        print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--box", type=int, default=4)
    ap.add_argument("--max-iters", type=int, default=200)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--rotate", action="store_true", help="reference arm: rotate through the cases")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu DRAM bytes per launch of the dominant kernel (from a capture)")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)
    args.rank, args.world, args.local_rank = dist_env()
    if args.world > 1:
        import torch.distributed as dist

        if args.impl == "reference":
            dist.init_process_group("gloo")
        else:
            import torch

            torch.cuda.set_device(args.local_rank)
            dist.init_process_group("nccl")
    try:
        if args.impl == "reference":
            return run_reference(args)
        return run_ours(args)
    finally:
        if args.world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
