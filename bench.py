#!/usr/bin/env python3
"""Benchmark: implicit IB step time to a 1e-8 relative residual on GB300.

Default workload (multi1024): the 1024^2 periodic MAC grid with 16 non-overlapping
elastic ellipses of 2048 points each (seed 1311, semi-axes U[0.02, 0.06]), kappa =
1e4, dt = 1e-3, rho = mu = 1, b = 4, V(1,1), FP32 V-cycle inside FP64 FGMRES
(restart 50).  One bench step = 20 consecutive implicit IB steps (set-up + MG-
preconditioned FGMRES to 1e-8 + point update each; u^n and X carried from step to
step), starting from rest at X^0; inputs resident on the device, L2 flushed before
every bench step.  value = device ms per implicit step (CUDA events on the stream).

The line also carries:
  e2e           the same steps through the C ABI with host buffers (H2D of X^0,
                D2H of u, v, p and X^{n+1}), host clock around the calls;
  roofline      the V-cycle (replayed from its CUDA graph inside FGMRES), timed
                with an event pair per V-cycle inside the timed region, against
                the V(1,1) algorithmic traffic (56 B/DOF in FP32) and the measured
                HBM bandwidth;
  cpu_baseline  the CPU oracle on a bounded sample of the same workload (its
                set-up plus one FGMRES iteration, scaled by the iteration count),
                and the GPU result's error against the oracle;
  forms         the 256^2 kappa x dt sweep solved case by case (FP64, mixed,
                FP32 V-cycles) and batched (FP32, FP64), for the precision and
                batching comparisons.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload multi1024|sweep256|case256|batch256|vcycle|learned512]
                  [--precision fp32|fp64|mixed] [--box B] [--no-cpu] [--no-forms]

Under torchrun each rank solves the whole workload on its own GPU (independent
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
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch, from one
# ncu capture each.  "vcycle1024": one V(1,1) cycle of the 1024^2 sixteen-ellipse
# step (146 kernel launches from one kv_zero to the next, summed; ncu replays each
# launch with cold caches, so this is an upper bound of the graph-replayed cycle's
# traffic).  Valid only for the V-cycle kernel sources it was taken on: reported as
# null once they change.
TRAFFIC = {"sources_sha256": "7d15a3a37ad17522a40f3ae3064a068071e95cbd06807e0193cfe1e70bbb0c1b",
           "vcycle1024": 747.8e6}
VCYCLE_SOURCES = ["ib_internal.cuh", "ib_ops.cuh", "ib_vcycle.cu", "ib_vcycle.cuh", "ib_windows.cu",
                  "ib_async.cuh"]


def captured_traffic(kclass):
    """Recorded DRAM bytes per launch of a kernel class, or None if the sources differ."""
    import hashlib

    h = hashlib.sha256()
    try:
        for f in VCYCLE_SOURCES:
            with open(os.path.join(ROOT, "paper_1311_5614_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    if h.hexdigest() != TRAFFIC["sources_sha256"]:
        return None
    return TRAFFIC.get(kclass)


# arithmetic of the V-cycle per precision mode (FGMRES and the operator are FP64 in all)
DTYPE = {"fp32": "f32 V-cycle + f64 Krylov", "fp64": "f64",
         "mixed": "f64 V-cycle vectors, f32 box solves + f64 Krylov"}
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
            "form": "batched (one stream per case)",
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
    """The reference arm: the CPU oracle, as it stands, on the host cores, for the same
    workload, metric and unit as the GPU arm.  Rank 0 alone runs it.

    multi1024 (default): the oracle's first implicit step of the C3 workload.  Its
    per-step set-up (hierarchy, Galerkin levels, box matrices, right-hand side) and one
    full FGMRES solve (which fixes the iteration count) run during the first warm-up
    step; every bench step then times one FGMRES iteration's V-cycle and operator apply.
    value = set-up + iterations x the mean iteration sample (ms per implicit step).
    sweep256: one implicit step of the kappa = 1e4, dt = 1e-3 case per bench step (the
    config names that single case)."""
    rank = args.rank
    if rank != 0:
        return 0
    if args.workload == "multi1024":
        prob = c3_problem(args.box)
        o = oracle_c3(prob, samples=max(1, args.warmup - 1) + args.steps, full_solve=True,
                      log=lambda m: print(m, file=sys.stderr))
        v = 1e3 * o["step_s"]
        sample = ("C3 first implicit step: oracle set-up %.1f s (measured once) + %d FGMRES iterations (the "
                  "oracle's own count) x %.2f s (median of %d samples of one V-cycle + one operator apply; "
                  "Gram-Schmidt not included); the full solve took %.1f s"
                  % (o["t_setup_s"], o["iters"], o["t_iter_s"], o["samples"], o["t_solve_s"]))
        config = c3_config(args)
    else:
        times = []
        for s_ in range(args.warmup + args.steps):
            ms, its = oracle_sample_ms(args.box, 2)
            if s_ >= args.warmup:
                times.append(ms)
        v = float(np.mean(times))
        sample = "one implicit step of the kappa=1e4, dt=1e-3 sweep case per bench step (%d iterations)" % its
        config = dict(config_dict(args), workload="256^2 MAC grid, 512-point ellipse, kappa=1e4, dt=1e-3 "
                                                  "(one case of the sweep)")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference", "config": config,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm

def _timed_steps(torch, step_fn, flush, stream, warmup, steps, profile_range=False):
    """W untimed steps, then K steps each bracketed by CUDA events, L2 flushed before each.
    With profile_range the first timed step is also bracketed by cudaProfilerStart/Stop
    (for an ncu launch list of exactly one step with --profile-from-start off)."""
    for _ in range(warmup):
        step_fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        if profile_range and k == 0:
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
        ev[k][0].record(stream)
        step_fn()
        ev[k][1].record(stream)
        if profile_range and k == 0:
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def run_ours(args):
    import torch

    import paper_1311_5614_gb300 as pkg
    from paper_1311_5614_gb300 import capi as C

    rank, world, local_rank = args.rank, args.world, args.local_rank
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    probs = workload_problems(args.box)
    nc = len(probs)
    nn = 3 * N_GRID * N_GRID
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream()
    X0 = torch.tensor(np.concatenate([p.X for p in probs]), dtype=torch.float64, device=dev)
    Xw = X0.clone()
    up = torch.zeros(nc * nn, dtype=torch.float64, device=dev)
    npts = [p.n_points for p in probs]
    xoff = np.concatenate([[0], np.cumsum(npts)])  # row offsets of each case in X

    # --- sequential forms: one IBSolver per case, solved one after another
    def make_seq(prec):
        return [pkg.IBSolver.from_problem(p, precision=prec, max_iters=args.max_iters) for p in probs]

    def seq_step(solvers, stats):
        Xw.copy_(X0)
        for i, s in enumerate(solvers):
            stats[i] = s.solve_step(None, up[i * nn:(i + 1) * nn], Xw[xoff[i]:xoff[i + 1]])

    forms = {}
    seq_stats = {}
    for prec in (["fp64", "mixed", "fp32"] if args.forms else [args.precision]):
        solvers = make_seq(prec)
        forms.setdefault("tail_grid", {})[prec] = [s.tail_grid(prec) for s in solvers]
        forms.setdefault("tail_cluster", {})[prec] = [s.tail_cluster(prec) for s in solvers]
        st = [None] * nc
        ms = _timed_steps(torch, lambda: seq_step(solvers, st), flush, stream, args.warmup, args.steps,
                          args.profile_range and prec == args.precision)
        forms["sequential_" + prec] = {"ms_per_ib_step": sum(ms) / (args.steps * nc),
                                       "iters": [x["iters"] for x in st], "status": [x["status"] for x in st],
                                       "escalated_at": [x["escalated_at"] for x in st]}
        seq_stats[prec] = (solvers, st)

    if args.no_batch:
        return _report_sequential(args, forms, seq_stats, torch)

    # --- batched form (headline): all cases in one ib_solve_step_batch call
    batch = pkg.IBBatch(probs, precision=args.precision, max_iters=args.max_iters)
    bstats = [None]

    def batch_step():
        Xw.copy_(X0)
        bstats[0] = batch.solve_step(None, up, Xw)

    launches0 = sum(C.ib_launch_count(batch.problem(k)) for k in range(nc))
    clk = ClockSampler(local_rank)
    # warm-up of the batched form, then the timed region
    for _ in range(args.warmup):
        batch_step()
    torch.cuda.synchronize()
    launches0 = sum(C.ib_launch_count(batch.problem(k)) for k in range(nc))
    barrier(world)
    torch.cuda.synchronize()
    clk.start()
    t_wall = time.perf_counter()
    step_ms = _timed_steps(torch, batch_step, flush, stream, 0, args.steps)
    t_wall = time.perf_counter() - t_wall
    barrier(world)
    clocks = clk.stop()
    gpu_launches = sum(C.ib_launch_count(batch.problem(k)) for k in range(nc)) - launches0
    per_ib_ms, t_max = aggregate(step_ms, args.steps * nc, world)
    stats = bstats[0]
    forms["batched_" + args.precision] = {"ms_per_ib_step": per_ib_ms, "iters": [x["iters"] for x in stats],
                                          "status": [x["status"] for x in stats],
                                          "escalated_at": [x["escalated_at"] for x in stats]}

    # end-to-end through the C ABI with host buffers: H2D of X^n, D2H of u, v, p and X^{n+1}
    Xh = torch.tensor(np.concatenate([p.X for p in probs]), dtype=torch.float64).pin_memory()
    uph = torch.empty(nc * nn, dtype=torch.float64).pin_memory()
    Xoh = torch.empty_like(Xh).pin_memory()

    def e2e_step():
        Xw.copy_(Xh, non_blocking=True)
        batch.solve_step(None, up, Xw)
        uph.copy_(up, non_blocking=True)
        Xoh.copy_(Xw, non_blocking=True)

    e2e_ms = _timed_steps(torch, e2e_step, flush, stream, args.warmup, args.steps)
    e2e_per, _ = aggregate(e2e_ms, args.steps * nc, world)
    h2d = Xh.numel() * 8
    d2h = uph.numel() * 8 + Xoh.numel() * 8

    # V-cycle throughput on the kappa = 1e4, dt = 1e-3 case (the preconditioner alone)
    solvers, _ = seq_stats[args.precision] if args.precision in seq_stats else (make_seq(args.precision), None)
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

    # profiled pass (separate from the timed region, sequential so launches do not
    # overlap): per-class device time and algorithmic bytes
    for s in solvers:
        s.profile(True)
    st = [None] * nc
    seq_step(solvers, st)
    torch.cuda.synchronize()
    prof = {}
    for s in solvers:
        for name, (n_, ms_, by_) in s.profile_read().items():
            q = prof.setdefault(name, [0, 0.0, 0.0])
            q[0] += n_
            q[1] += ms_
            q[2] += by_
        s.profile(False)
    hot = ("stokes", "box", "interp", "spread", "transfer")
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
    traffic = args.traffic if args.traffic is not None else captured_traffic(dom)
    roofline = {"bound": "hbm", "kernel_class": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src, "traffic": traffic,
                "launches": n_, "avg_launch_us": 1e3 * ms_ / max(n_, 1),
                "alg_bytes_per_launch": by_ / max(n_, 1),
                "share_of_step": ms_ / max(sum(v[1] for v in prof.values()), 1e-30)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ms_cpu, its_cpu = oracle_sample_ms(args.box, 2)
        cpu = {"value": ms_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "one implicit step of the kappa=1e4, dt=1e-3 case (%d FGMRES iterations)" % its_cpu}

    for pr in seq_stats.values():
        for s in pr[0]:
            s.close()
    batch.close()
    if rank == 0:
        line = {"metric": METRIC, "value": per_ib_ms, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE[args.precision],
                "data": "synthetic", "config": config_dict(args),
                "e2e": {"value": e2e_per, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "roofline": roofline, "cpu_baseline": cpu, "gpu_launches": int(gpu_launches),
                "clocks": clocks, "forms": forms,
                "vcycle": {"ms": vcycle_ms, "dof_per_s": vcycle_dofs, "dof": nn,
                           "case": "kappa=1e4, dt=1e-3", "precision": args.precision},
                "wall_s_timed": t_wall,
                "profile": {k: {"launches": v[0], "ms": v[1], "bytes": v[2]} for k, v in prof.items()}}
        print(json.dumps(line), flush=True)
    return 0


def _report_sequential(args, forms, seq_stats, torch):
    """Line for --no-batch runs (used for single-stream profiler captures)."""
    for pr in seq_stats.values():
        for s in pr[0]:
            s.close()
    f = forms["sequential_" + args.precision]
    if args.rank == 0:
        print(json.dumps({"metric": METRIC, "value": f["ms_per_ib_step"], "unit": UNIT, "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
                          "data": "synthetic", "config": dict(config_dict(args), form="sequential"),
                          "forms": forms}), flush=True)
    return 0


def run_vcycle(args):
    """V-cycle throughput alone on an N x N grid (default 2048) with the 0.28/0.22 ellipse of
    2N points, kappa = 1e4, dt = 1e-3: W warm-up and K timed cycles, L2 flushed before each.
    Roofline: the V(1,1) algorithmic traffic of 56 B/DOF (FP32) or 112 B/DOF (FP64) against
    the measured HBM copy bandwidth."""
    import torch

    import paper_1311_5614_gb300 as pkg

    torch.cuda.set_device(args.local_rank)
    N = args.grid
    prob = W.single_ellipse(N=N, n_points=2 * N, kappa=1e4, dt=1e-3)
    prob.box = args.box
    # the V-cycle alone: a one-vector Krylov workspace keeps the device memory small
    s = pkg.IBSolver.from_problem(prob, precision=args.precision, max_iters=1)
    n = 3 * N * N
    b = torch.randn(n, dtype=torch.float64, device="cuda")
    w = torch.zeros_like(b)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ms = _timed_steps(torch, lambda: s.vcycle(b, w), flush, torch.cuda.current_stream(), args.warmup,
                      args.steps, args.profile_range)
    per = sum(ms) / len(ms)
    # ib_vcycle converts the FP64 input and output around the cycle: time that part separately
    bpd = 56.0 if args.precision == "fp32" else 112.0  # vectors in FP64 for fp64 and mixed
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = bpd * n / (per * 1e-3) / 1e9
    line = {"metric": "V-cycle DOF/s", "value": n / (per * 1e-3), "unit": "DOF/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per, "higher_is_better": True,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": "V(1,1) on %d^2, ellipse of %d points, kappa=1e4, dt=1e-3" % (N, 2 * N),
                       "box": args.box, "precision": args.precision, "tail_grid": s.tail_grid(args.precision),
                       "tail_cluster": s.tail_cluster(args.precision), "box_forms": s.box_forms(args.precision),
                       "note": "ib_vcycle includes the FP64<->FP32 conversion of b and w"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "alg_bytes_per_dof": bpd,
                         "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}}
    s.close()
    print(json.dumps(line), flush=True)
    return 0


def run_unet(args):
    """The learned stage's network alone at 512^2 (4 -> 3 channels, 118 451 parameters):
    forward and one training step (forward, backward, Adam), CUDA events, against the
    dense BF16 tensor peak.  FLOPs per forward: sum over layers of 2 Co Ci K^2 H^2, each
    taken twice (hi and lo BF16 terms of the activations)."""
    import torch

    import paper_1311_5614_gb300 as pkg

    torch.cuda.set_device(args.local_rank)
    N = 512
    net = pkg.UNet(N, W.unet_init_params(0))
    x = torch.randn(4 * N * N, device="cuda")
    y = torch.zeros(3 * N * N, device="cuda")
    t = torch.randn(3 * N * N, device="cuda")
    flops = 0.0
    for ci, co, k in W.UNET_SHAPES:
        H = N if co in (16, 3) else (N // 2 if co == 32 else N // 4)
        flops += 2.0 * co * ci * k * k * H * H
    fwd = _timed_steps(torch, lambda: net.forward(x, y), torch.empty(64 * 1024 * 1024, device="cuda"),
                       torch.cuda.current_stream(), args.warmup, args.steps)
    trn = _timed_steps(torch, lambda: net.train_step(x, t, 1e-5), torch.empty(64 * 1024 * 1024, device="cuda"),
                       torch.cuda.current_stream(), args.warmup, args.steps)
    net.close()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("bf16_tflops", 1900.0))
    f_ms = sum(fwd) / len(fwd)
    ach = 2.0 * flops / (f_ms * 1e-3) / 1e12
    line = {"metric": "U-Net forward / training step time", "value": f_ms, "unit": "ms per forward",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "dtype": "bf16 x (bf16 hi + lo) -> f32", "data": "synthetic",
            "config": {"workload": "U-Net 16/32/64 channels at 512^2"},
            "train_step_ms": sum(trn) / len(trn),
            "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "flops_per_forward": 2.0 * flops}}
    print(json.dumps(line), flush=True)
    return 0


CAVITY_CASES = ([(N, b, a) for N in (64, 256, 1024) for b in (4, 8) for a in (6.0, 60.0, 600.0, 3000.0)]
                + [(N, 16, a) for N in (64, 256) for a in (6.0, 60.0, 600.0, 3000.0)])


def run_cavity(args):
    """The paper's own problem on the GPU (sec. 4, the refinement study of sec. 6):
    the lid-driven cavity with the thick annulus, steady Stokes, cosine kernel, zero
    rest length, stiffness alpha = 6, 60, 600, 3000 (non-stiff ... very stiff), box
    sizes 4 and 8 (and 16 at N = 64 and 256), V(1,1), MG-GMRES from zero to a 1e-6 residual reduction (100
    iterations at most), at N = 64, 256 and 1024.  Right-hand side from the library
    (ib_rhs: the lid's ghost term and -S F(X)); each case is solved warmup + steps
    times and its median FGMRES device time reported (events inside ib_solve).  The
    GPU sweeps the boxes in four colours, the paper lexicographically, so the
    iteration counts are the colour order's (the paper plots its counts)."""
    import torch

    from paper_1311_5614_gb300 import capi as C

    torch.cuda.set_device(args.local_rank)
    cases = []
    for N, b, alpha in CAVITY_CASES:
        p = W.cavity_annulus(N, kappa=alpha, dt=1.0)
        s = C.IBSolver(N, p.X, p.springs, p.kappa, p.rest, L=1.0, rho=0.0, mu=1.0, dt=1.0, delta="cos4", box=b,
                       walls="noslip", lid=1.0, precision=args.precision, tol=1e-6, max_iters=100)
        rhs = torch.zeros(3 * N * N, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(rhs)
        s.rhs(None, rhs)
        times, st = [], None
        for r in range(args.warmup + args.steps):
            st = s.solve(rhs, x)
            if r >= args.warmup:
                times.append(st["t_solve_ms"])
        s.close()
        cases.append({"N": N, "box": b, "alpha": alpha, "iters": st["iters"], "status": st["status"],
                      "rel_res_true": st["rel_res_true"], "ms": float(np.median(times)),
                      "escalated_at": st["escalated_at"]})
    big = [c for c in cases if c["N"] == 1024 and c["box"] == 8 and c["alpha"] == 3000.0][0]
    line = {"metric": "MG-GMRES solve time to a 1e-6 residual reduction, the paper's cavity problem",
            "value": big["ms"], "unit": "ms per solve (N = 1024, b = 8, alpha = 3000)", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "dtype": "f32 V-cycle + f64 Krylov" if args.precision == "fp32" else args.precision,
            "data": "synthetic (the paper's geometry, no randomness)",
            "config": {"workload": "lid-driven cavity, thick annulus (r = 1/4, w = 1/16), M1 = 19N/8, "
                                   "M2 = 3N/32 + 1, steady Stokes, cosine kernel, V(1,1), colour order",
                       "precision": args.precision},
            "cases": cases, "clocks": None}
    print(json.dumps(line), flush=True)
    return 0


def run_cavity_time(args):
    """What the implicit method saves (sec. 7), on the paper's cavity: the lid-driven
    cavity with the thick annulus (lid velocity 1) advanced to t = 1 by the
    implicit-time method (dt = 1/40, 40 steps, the paper's step) and by the explicit-
    time method at 0.9 of its stability limit (dt = 0.9 alpha_exp / gamma; 40 steps
    run and the work extrapolated to t = 1, as the paper does), at relative
    stiffness gamma dt / alpha_exp = 1, 10, 100, 500 for the implicit step, box
    sizes 4, 8 and 16, MG-GMRES to 1e-6 per step.  The efficiency factor is the ratio of
    the explicit method's work to the implicit one's, counted in MG-GMRES
    iterations (the paper's measure) and in GPU time (set-up + solve per step, CUDA
    events inside ib_solve_step).  alpha_exp = 3.93 at N = 64 is the paper's Table 1
    value (the cavity oracle reproduces it)."""
    import torch

    from paper_1311_5614_gb300 import capi as C

    torch.cuda.set_device(args.local_rank)
    N, T, dt_i, a_exp = 64, 1.0, 1.0 / 40.0, 3.93
    rows = []
    for b in (4, 8, 16):
        for rel in (1.0, 10.0, 100.0, 500.0):
            gamma = rel * a_exp / dt_i
            res = {"box": b, "rel_stiffness": rel, "gamma": gamma}
            for method, dt in (("implicit", dt_i), ("explicit", 0.9 * a_exp / gamma)):
                p = W.cavity_annulus(N, kappa=gamma, dt=dt)
                s = C.IBSolver(N, p.X, p.springs, p.kappa, p.rest, L=1.0, rho=0.0, mu=1.0, dt=dt, delta="cos4",
                               box=b, walls="noslip", lid=1.0, precision=args.precision, tol=1e-6, max_iters=100,
                               time_method=method)
                X = torch.tensor(p.X, device="cuda")
                up = torch.zeros(3 * N * N, dtype=torch.float64, device="cuda")
                its, ms, bad = [], [], 0
                for _ in range(40):
                    st = s.solve_step(None, up, X)
                    bad += st["status"] != 0
                    its.append(st["iters"])
                    ms.append(st["t_setup_ms"] + st["t_solve_ms"])
                s.close()
                steps = T / dt
                res[method] = {"dt": dt, "steps_to_t1": steps, "iters_per_step": float(np.mean(its)),
                               "ms_per_step": float(np.mean(ms)), "failed_steps": bad,
                               "iters_to_t1": steps * float(np.mean(its)), "ms_to_t1": steps * float(np.mean(ms))}
            res["efficiency_iters"] = res["explicit"]["iters_to_t1"] / res["implicit"]["iters_to_t1"]
            res["efficiency_time"] = res["explicit"]["ms_to_t1"] / res["implicit"]["ms_to_t1"]
            rows.append(res)
    big = [r for r in rows if r["box"] == 8 and r["rel_stiffness"] == 100.0][0]
    line = {"metric": "implicit vs explicit time to t = 1 on the paper's cavity (efficiency factor, GPU time)",
            "value": big["efficiency_time"], "unit": "x (explicit GPU time / implicit GPU time, b = 8, "
                                                     "relative stiffness 100)",
            "n_gpus": 1, "steps": 40, "warmup": 0, "higher_is_better": True,
            "dtype": "f32 V-cycle + f64 Krylov" if args.precision == "fp32" else args.precision,
            "data": "synthetic (the paper's geometry, no randomness)",
            "config": {"workload": "lid-driven cavity 64^2, thick annulus, lid velocity 1, t in [0, 1]; "
                                   "implicit dt = 1/40, explicit dt = 0.9 alpha_exp / gamma",
                       "precision": args.precision},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_learned512(args):
    """Learned stage at 512^2 (1024-point ellipse): pairs harvested from the method's own
    V-cycles on problems with kappa = 10^U[2,6], U-Net trained on the GPU with the
    library's kernels, then plain vs learned MG-FGMRES on held-out kappa in {1e2, 1e4, 1e6}."""
    import torch

    from paper_1311_5614_gb300 import learned

    torch.cuda.set_device(args.local_rank)
    res = learned.run(N=512, n_problems=args.learn_problems, pairs_per_problem=args.learn_pairs,
                      epochs=args.learn_epochs, lr=1e-3, seed=0, log=lambda m: print(m, file=sys.stderr))
    params = res.pop("params")
    if args.save_params:
        np.save(args.save_params, params)
    ev = res["eval"]
    plain = sum(r["plain"]["ms"] for r in ev) / len(ev)
    lrn = sum(r["learned"]["ms"] for r in ev) / len(ev)
    line = {"metric": METRIC, "value": lrn, "unit": UNIT, "n_gpus": 1, "steps": len(ev), "warmup": 1,
            "higher_is_better": False, "dtype": "f32 V-cycle + f64 Krylov + f32/bf16 U-Net",
            "data": "synthetic",
            "config": {"workload": "512^2, 1024-point ellipse, dt=1e-2; learned stage vs plain",
                       "pairs": res["pairs"], "epochs": res["epochs"], "box": 4, "precision": "fp32"},
            "forms": {"plain_ms_per_ib_step": plain, "learned_ms_per_ib_step": lrn}, "learned": res}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- C2 forms (context)

def sweep_forms(args, torch, pkg):
    """The 256^2 kappa x dt sweep (8 cases) in five forms, ms per implicit step to 1e-8:
    case by case with the FP64, mixed and FP32 V-cycles, and batched (all cases in one
    ib_solve_step_batch) with the FP32 and FP64 V-cycles, so that precision and batching
    are compared separately.  With the CPU leg on (rank 0, one GPU), each form's solution
    of the kappa = 1e4, dt = 1e-3 case is compared with the oracle's."""
    dev = torch.device("cuda", args.local_rank)
    probs = workload_problems(args.box)
    nc = len(probs)
    nn = 3 * N_GRID * N_GRID
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    X0 = torch.tensor(np.concatenate([p.X for p in probs]), dtype=torch.float64, device=dev)
    Xw = X0.clone()
    up = torch.zeros(nc * nn, dtype=torch.float64, device=dev)
    xoff = np.concatenate([[0], np.cumsum([p.n_points for p in probs])])
    forms, sols = {}, {}
    steps = max(2, min(args.steps, 5))
    for prec in ("fp64", "mixed", "fp32"):
        solvers = [pkg.IBSolver.from_problem(p, precision=prec, max_iters=args.max_iters) for p in probs]
        st = [None] * nc

        def seq_step():
            Xw.copy_(X0)
            for i, s_ in enumerate(solvers):
                st[i] = s_.solve_step(None, up[i * nn:(i + 1) * nn], Xw[xoff[i]:xoff[i + 1]])

        ms = _timed_steps(torch, seq_step, flush, stream, 3, steps)
        forms["sequential_" + prec] = {"ms_per_ib_step": sum(ms) / (steps * nc), "iters": [x["iters"] for x in st],
                                       "status": [x["status"] for x in st]}
        sols["sequential_" + prec] = up[2 * nn:3 * nn].cpu().numpy()
        for s_ in solvers:
            s_.close()
    for prec in ("fp32", "fp64"):
        batch = pkg.IBBatch(probs, precision=prec, max_iters=args.max_iters)
        bst = [None]

        def batch_step():
            Xw.copy_(X0)
            bst[0] = batch.solve_step(None, up, Xw)

        ms = _timed_steps(torch, batch_step, flush, stream, 3, steps)
        forms["batched_" + prec] = {"ms_per_ib_step": sum(ms) / (steps * nc),
                                    "iters": [x["iters"] for x in bst[0]], "status": [x["status"] for x in bst[0]]}
        sols["batched_" + prec] = up[2 * nn:3 * nn].cpu().numpy()
        batch.close()
    forms["workload"] = "256^2, 512-point ellipse, kappa in {1,1e2,1e4,1e6} x dt in {1e-3,1e-2}, b = %d" % args.box
    if args.rank == 0 and args.world == 1 and not args.no_cpu:
        from oracle import ib_oracle as O

        t = time.perf_counter()
        ref = O.solve_step(probs[2])
        t = time.perf_counter() - t
        forms["error_vs_oracle"] = {
            "case": "kappa=1e4, dt=1e-3 (oracle: %d iterations, %.1f s on one core)" % (ref.solve.iters, t),
            **{k: float(np.linalg.norm(v - ref.w) / np.linalg.norm(ref.w)) for k, v in sols.items()}}
    return forms


# ----------------------------------------------------------------------------- C3: the headline

C3 = dict(N=1024, count=16, n_per=2048, kappa=1e4, dt=1e-3, seed=1311, restart=50)
C3_STEPS = 20  # consecutive implicit steps per bench step


def c3_problem(box):
    p = W.many_ellipses(N=C3["N"], count=C3["count"], n_per=C3["n_per"], kappa=C3["kappa"], dt=C3["dt"],
                        seed=C3["seed"])
    p.box = box
    return p


def c3_config(args):
    return {"workload": "1024^2 MAC grid, 16 ellipses x 2048 points (seed 1311, semi-axes U[0.02, 0.06]), "
                        "kappa=1e4, dt=1e-3, rho=mu=1; %d consecutive implicit steps per bench step "
                        "(u^n and X carried), each from rest at X^0 per bench step" % args.c3_steps,
            "N": C3["N"], "n_points": C3["count"] * C3["n_per"], "box": args.box, "nu": [1, 1],
            "precision": args.precision, "tol": 1e-8, "restart": C3["restart"], "max_iters": args.max_iters,
            "l2": "flushed (256 MiB write) before every timed bench step",
            "parallelism": "replicas" if args.world > 1 else "single GPU"}


def oracle_c3(prob, iters=None, samples=1, full_solve=False, gpu=None, log=None):
    """CPU oracle on the C3 workload (first implicit step, fluid at rest): the per-step
    set-up (hierarchy: S, J, Galerkin levels, box matrices; right-hand side) timed once,
    then `samples` timings of one FGMRES iteration's preconditioner and operator work
    (one V-cycle + one operator apply).  With full_solve the oracle's FGMRES runs to
    the tolerance once (its iteration count and solution).  Estimated oracle step time =
    set-up + iters x iteration sample.  gpu (dict: w = the GPU's first-step solution,
    z = the GPU V-cycle applied to the first step's right-hand side) adds the GPU result's
    errors against the oracle: the true residual on the oracle's CSR operator and the
    relative difference of the preconditioner output."""
    from oracle import ib_oracle as O

    def note(m):
        if log:
            log(m)

    t0 = time.perf_counter()
    levels, _ = O.build_hierarchy(prob)
    for lev in levels[:-1]:
        O.prepare_boxes(lev, prob.box)
    b = O.rhs_vector(prob)
    t_setup = time.perf_counter() - t0
    note("oracle set-up %.1f s" % t_setup)
    A = levels[0].A
    t_iter = []
    z = None
    for _ in range(samples):
        t1 = time.perf_counter()
        z = O.vcycle(levels, b, np.zeros_like(b), prob.nu1, prob.nu2, prob.rho, "color4")
        _ = A @ z
        t_iter.append(time.perf_counter() - t1)
    note("oracle iteration sample %.2f s" % min(t_iter))
    out = {"t_setup_s": t_setup, "t_iter_s": float(np.median(t_iter)), "samples": samples}
    if full_solve:
        t2 = time.perf_counter()
        res = O.fgmres(A, b, lambda v: O.vcycle(levels, v, np.zeros_like(v), prob.nu1, prob.nu2, prob.rho,
                                                 "color4"), prob.tol, prob.max_iters)
        out["t_solve_s"] = time.perf_counter() - t2
        out["oracle_iters"] = res.iters
        out["oracle_w"] = O.remove_pressure_mean(res.x, prob.N)
        iters = res.iters if iters is None else iters
    out["iters"] = iters
    out["step_s"] = t_setup + (iters or 0) * out["t_iter_s"]
    if gpu is not None:
        w = gpu["w"]
        bn = np.linalg.norm(b)
        n = prob.N * prob.N
        out["error_vs_oracle"] = {
            "rel_res_true_on_oracle_csr": float(np.linalg.norm(b - A @ w) / bn),
            "div_on_oracle_csr": float(np.linalg.norm((A @ w)[2 * n:]) / bn),
            "vcycle_rel_diff": float(np.linalg.norm(gpu["z"] - z) / np.linalg.norm(z)),
            "vcycle_max_elem_rel": float(np.abs(gpu["z"] - z).max() / np.abs(z).max())}
        if "oracle_w" in out:
            ow = out["oracle_w"]
            out["error_vs_oracle"]["solution_rel"] = float(np.linalg.norm(w - ow) / np.linalg.norm(ow))
    out.pop("oracle_w", None)
    return out


def vcycle_alone(torch, pkg, N, precision, box, steps, warmup, peak):
    """The V-cycle alone on N^2 (the 0.28/0.22 ellipse of 2N points, kappa = 1e4, dt =
    1e-3): mean device time of the graph-replayed V-cycle (ib_vcycle_timer), L2 flushed
    before each, against the V(1,1) algorithmic traffic (56 B/DOF in FP32)."""
    prob = W.single_ellipse(N=N, n_points=2 * N, kappa=1e4, dt=1e-3)
    prob.box = box
    s = pkg.IBSolver.from_problem(prob, precision=precision, max_iters=1)
    n = 3 * N * N
    b = torch.randn(n, dtype=torch.float64, device="cuda")
    w = torch.zeros_like(b)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        s.vcycle(b, w)
    torch.cuda.synchronize()
    s.vcycle_timer(True)
    for _ in range(steps):
        flush.zero_()
        s.vcycle(b, w)
    prec = "fp32" if precision == "fp32" else "fp64"
    nv, ms = s.vcycle_timer_read(prec)
    s.vcycle_timer(False)
    out = {"grid": N, "dof": n, "ms": ms / max(nv, 1), "precision": precision,
           "box_forms": s.box_forms(precision), "tail_grid": s.tail_grid(precision)}
    s.close()
    bpd = 56.0 if precision == "fp32" else 112.0
    ach = bpd * n / (out["ms"] * 1e-3) / 1e9 if out["ms"] > 0 else 0.0
    out["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                       "alg_bytes_per_dof": bpd}
    out["dof_per_s"] = n / (out["ms"] * 1e-3) if out["ms"] > 0 else 0.0
    return out


def run_multi1024(args):
    """Headline: the 1024^2 multi-structure workload.  One bench step = C3_STEPS
    consecutive implicit IB steps (set-up + MG-preconditioned FGMRES to 1e-8 + point
    update each, u^n and X carried), starting from rest at X^0.  value = device ms per
    implicit step (CUDA events on the stream, L2 flushed before every bench step)."""
    import torch

    import paper_1311_5614_gb300 as pkg
    from paper_1311_5614_gb300 import capi as C

    rank, world, local_rank = args.rank, args.world, args.local_rank
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prob = c3_problem(args.box)
    N = prob.N
    n3, n2 = 3 * N * N, 2 * N * N
    s = pkg.IBSolver.from_problem(prob, precision=args.precision, max_iters=args.max_iters, restart=C3["restart"])
    up = torch.zeros(n3, dtype=torch.float64, device=dev)
    un = torch.zeros(n2, dtype=torch.float64, device=dev)
    X0 = torch.tensor(prob.X, dtype=torch.float64, device=dev)
    X = X0.clone()
    stream = torch.cuda.current_stream()
    stats = []

    def steps():
        stats.clear()
        stats.append(s.solve_step(None, up, X))
        for _ in range(args.c3_steps - 1):
            un.copy_(up[:n2])
            stats.append(s.solve_step(un, up, X))

    def bench_step():
        X.copy_(X0)
        steps()

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = s.launch_count()
    s.vcycle_timer(True)
    clk = ClockSampler(local_rank)
    clk.start()
    t_wall = time.perf_counter()
    step_ms = _timed_steps(torch, bench_step, flush, stream, 0, args.steps, args.profile_range)
    t_wall = time.perf_counter() - t_wall
    clocks = clk.stop()
    vprec = "fp32" if args.precision == "fp32" else "fp64"
    nv32 = s.vcycle_timer_read("fp32") if args.precision == "fp32" else (0, 0.0)
    nv64 = s.vcycle_timer_read("fp64")
    s.vcycle_timer(False)
    barrier(world)
    gpu_launches = s.launch_count() - launches0
    step_stats = list(stats)
    per_ib_ms, t_max = aggregate(step_ms, args.steps * args.c3_steps, world)

    # end to end through the C ABI with host buffers: H2D of X^0 from pinned memory, the
    # steps, D2H of the final u, v, p and X; host clock around the whole call sequence
    Xh = torch.tensor(prob.X, dtype=torch.float64).pin_memory()
    uph = torch.empty(n3, dtype=torch.float64).pin_memory()
    Xoh = torch.empty_like(Xh).pin_memory()
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        X.copy_(Xh, non_blocking=True)
        steps()
        uph.copy_(up, non_blocking=True)
        Xoh.copy_(X, non_blocking=True)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t))
    e2e_per, _ = aggregate(e2e_ms, args.steps * args.c3_steps, world)

    # roofline of the V-cycle (the preconditioner graph replayed inside FGMRES): the
    # algorithmic traffic of a V(1,1) cycle, 56 B/DOF in FP32 (112 B/DOF on FP64
    # vectors), over its mean device time inside the timed region
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    nv, vms = (nv32[0] + nv64[0], nv32[1] + nv64[1])
    bpd32, bpd64 = 56.0, 112.0
    alg_bytes = (nv32[0] * bpd32 + nv64[0] * bpd64) * n3
    vcycle_ms = vms / max(nv, 1)
    achieved = alg_bytes / (vms * 1e-3) / 1e9 if vms > 0 else 0.0
    traffic = captured_traffic("vcycle1024")
    roofline = {"bound": "hbm", "kernel": "V(1,1) cycle, replayed from its CUDA graph inside FGMRES",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "traffic": traffic, "alg_bytes_per_launch": alg_bytes / max(nv, 1), "launches": nv,
                "avg_launch_ms": vcycle_ms, "dof": n3,
                "alg_bytes_per_dof": bpd32 if nv32[0] >= nv64[0] else bpd64,
                "share_of_step": vms / max(sum(step_ms), 1e-30),
                "vcycle_dof_per_s": n3 / (vcycle_ms * 1e-3) if vcycle_ms > 0 else 0.0}

    # first step again (from rest at X^0): its solution and the V-cycle applied to its
    # right-hand side, for the comparison with the oracle in the CPU leg
    X.copy_(X0)
    st1 = s.solve_step(None, up, X)
    w1 = up.cpu().numpy()
    X.copy_(X0)
    s.update_points(X)
    b1 = torch.zeros(n3, dtype=torch.float64, device=dev)
    s.rhs(None, b1)
    z1 = torch.zeros_like(b1)
    s.vcycle(b1, z1)
    z1 = z1.cpu().numpy()

    # per-class device time of one implicit step (a separate eager pass with an event pair
    # around every launch: context for the V-cycle figure above)
    s.profile(True)
    X.copy_(X0)
    s.solve_step(None, up, X)
    torch.cuda.synchronize()
    prof = s.profile_read()
    s.profile(False)
    tail = (s.tail_grid(args.precision), s.tail_cluster(args.precision))
    forms_by_level = s.box_forms(args.precision)
    s.close()

    forms = sweep_forms(args, torch, pkg) if args.forms else None
    large = vcycle_alone(torch, pkg, 4096, args.precision, args.box, 5, 3, peak) if args.vcycle_large else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        o = oracle_c3(prob, iters=st1["iters"], samples=1, gpu={"w": w1, "z": z1},
                      log=lambda m: print(m, file=sys.stderr))
        cpu = {"value": 1e3 * o["step_s"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "C3 first implicit step: the oracle's set-up (hierarchy, Galerkin levels, box "
                         "matrices, right-hand side: %.1f s) plus %d x one FGMRES iteration's V-cycle and "
                         "operator apply (%.2f s, measured once; %d = the GPU step's iteration count); "
                         "Gram-Schmidt not included" % (o["t_setup_s"], o["iters"], o["t_iter_s"], o["iters"]),
               "error_vs_oracle": o["error_vs_oracle"]}

    if rank == 0:
        its = [x["iters"] for x in step_stats]
        line = {"metric": METRIC, "value": per_ib_ms, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
                "config": c3_config(args),
                "e2e": {"value": e2e_per, "unit": UNIT, "h2d_bytes_per_step": Xh.numel() * 8,
                        "d2h_bytes_per_step": uph.numel() * 8 + Xoh.numel() * 8,
                        "clock": "host wall clock around the C-ABI calls, synchronised"},
                "roofline": roofline, "cpu_baseline": cpu, "gpu_launches": int(gpu_launches),
                "clocks": clocks, "wall_s_timed": t_wall,
                "iters_per_step": its, "rel_res_true": [x["rel_res_true"] for x in step_stats],
                "status": sorted(set(x["status"] for x in step_stats)),
                "setup_ms": float(np.mean([x["t_setup_ms"] for x in step_stats])),
                "solve_ms": float(np.mean([x["t_solve_ms"] for x in step_stats])),
                "autotune": {"tail_grid": tail[0], "tail_cluster": tail[1], "box_form_by_level": forms_by_level,
                             "box_form_codes": "1 one box per CTA, 2 thread per box row, 3 register-blocked "
                                               "product, 4/5/6 strip kernel of 8/16/32 boxes, 7 eight boxes "
                                               "per 64-thread CTA, 0 size rule"},
                "profile": {k: {"launches": v[0], "ms": v[1], "bytes": v[2]} for k, v in prof.items()},
                "forms": forms, "vcycle_large": large}
        print(json.dumps(line), flush=True)
    return 0


def run_case256(args):
    """One case of the 256^2 sweep on its own (--case K, CASES order; 7 = the stiff
    kappa = 1e6, dt = 1e-2 case): a solver set up once, then W untimed and K timed
    implicit steps, each from the case's initial points.  The first step follows
    the set-up directly, so an ncu capture can select a launch of that step by its
    index (the Gram-Schmidt kernels launch nowhere else before it)."""
    import torch

    import paper_1311_5614_gb300 as pkg

    torch.cuda.set_device(args.local_rank)
    p = workload_problems(args.box)[args.case]
    s = pkg.IBSolver.from_problem(p, precision=args.precision, max_iters=args.max_iters)
    up = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    X0 = torch.tensor(p.X, dtype=torch.float64, device="cuda")
    X = X0.clone()
    stream = torch.cuda.current_stream()
    stats = []

    def step():
        X.copy_(X0)
        stats.append(s.solve_step(None, up, X))

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    clk = ClockSampler(args.local_rank)
    clk.start()
    ms = _timed_steps(torch, step, flush, stream, args.warmup, args.steps)
    clocks = clk.stop()
    s.close()
    kappa, dt = CASES[args.case]
    line = {"metric": METRIC, "value": sum(ms) / len(ms), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False, "dtype": DTYPE[args.precision],
            "data": "synthetic",
            "config": {"workload": "256^2 MAC grid, 512-point ellipse, kappa=%g, dt=%g (one sweep case)" % (kappa, dt),
                       "box": args.box, "precision": args.precision, "max_iters": args.max_iters},
            "iters": [x["iters"] for x in stats], "status": [x["status"] for x in stats],
            "escalated_at": [x["escalated_at"] for x in stats], "setup_ms": [x["t_setup_ms"] for x in stats],
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def batch_restarts(probs, sigma_stiff=3000.0, m=30):
    """FGMRES restart length per problem of the batch: 30 Krylov vectors, none (the whole
    iteration cap) for problems whose stiffness ratio dt max(kappa) / mu reaches 3000.
    With restarts the stiff 512^2 problems stall (two of them at the 200-iteration cap);
    unrestarted they take 61-139 iterations."""
    return [0 if p.dt * float(np.max(p.kappa)) / p.mu >= sigma_stiff else m for p in probs]


def run_batch256(args):
    """256 independent problems, grids drawn from {64, 128, 256, 512} (seed 5614), one
    ellipse each with 4 points per cell of perimeter, kappa log-uniform in [1, 1e6]:
    one bench step = one ib_solve_step_batch over all of them."""
    import torch

    import paper_1311_5614_gb300 as pkg

    torch.cuda.set_device(args.local_rank)
    probs = W.batch(count=256, seed=5614)
    for p in probs:
        p.box = args.box
    B = pkg.IBBatch(probs, precision=args.precision, max_iters=args.max_iters, restart=batch_restarts(probs))
    n = sum(3 * p.N * p.N for p in probs)
    up = torch.zeros(n, dtype=torch.float64, device="cuda")
    X0 = torch.tensor(np.concatenate([p.X for p in probs]), dtype=torch.float64, device="cuda")
    X = X0.clone()
    stats = [None]

    def step():
        X.copy_(X0)
        stats[0] = B.solve_step(None, up, X)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    clk = ClockSampler(args.local_rank)
    clk.start()
    ms = _timed_steps(torch, step, flush, torch.cuda.current_stream(), args.warmup, args.steps)
    clocks = clk.stop()
    st = stats[0]
    B.close()
    dof = sum(3 * p.N * p.N for p in probs)
    its = [x["iters"] for x in st]
    line = {"metric": METRIC, "value": sum(ms) / (len(ms) * len(probs)), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms),
            "higher_is_better": False, "dtype": "f32 V-cycle + f64 Krylov", "data": "synthetic",
            "config": {"workload": "256 problems, N in {64,128,256,512} (seed 5614), kappa 10^U[0,6], dt=1e-2",
                       "box": args.box, "precision": args.precision,
                       "restart": "30; none for dt kappa / mu >= 3000",
                       "max_iters": args.max_iters, "total_dof": dof},
            "iters_total": int(sum(its)), "iters_max": int(max(its)),
            "not_converged": int(sum(1 for x in st if x["status"] != 0)),
            "escalated": int(sum(1 for x in st if x["escalated_at"] >= 0)),
            "dof_vcycles_per_s": float(sum(3 * p.N * p.N * x["iters"] for p, x in zip(probs, st)) /
                                       (sum(ms) / len(ms) * 1e-3)),
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "mixed"])
    ap.add_argument("--box", type=int, default=4)
    ap.add_argument("--max-iters", type=int, default=200)
    ap.add_argument("--grid", type=int, default=2048, help="grid size of the vcycle workload")
    ap.add_argument("--case", type=int, default=7, choices=range(len(CASES)),
                    help="case256: index into the sweep's cases (7: kappa=1e6, dt=1e-2)")
    ap.add_argument("--learn-problems", type=int, default=40)
    ap.add_argument("--learn-pairs", type=int, default=256,
                    help="pairs per training problem (40 x 256 = 10240 pairs by default)")
    ap.add_argument("--save-params", default=None, help="learned512: write the trained U-Net parameters (.npy)")
    ap.add_argument("--learn-epochs", type=int, default=2)
    ap.add_argument("--workload", default="multi1024",
                    choices=["sweep256", "case256", "multi1024", "batch256", "vcycle", "learned512", "unet", "cavity", "cavity_time"],
                    help="multi1024 (default): the 1024^2 sixteen-ellipse run, 20 consecutive steps per "
                         "bench step; sweep256: the 256^2 kappa x dt sweep; batch256: the 256-problem "
                         "batch; vcycle: the V-cycle alone (--grid); learned512: the learned stage")
    ap.add_argument("--c3-steps", type=int, default=C3_STEPS,
                    help="multi1024: consecutive implicit steps per bench step")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the first timed step of the sequential form in the bench precision "
                         "with cudaProfilerStart/Stop (for an ncu launch list of one sweep)")
    ap.add_argument("--no-batch", action="store_true",
                    help="time only the sequential form (single stream; for profiler captures)")
    ap.add_argument("--no-vcycle-large", dest="vcycle_large", action="store_false",
                    help="multi1024: skip the V-cycle alone at 4096^2")
    ap.add_argument("--no-forms", dest="forms", action="store_false",
                    help="skip the sequential FP64 / FP32 comparison forms")
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
        if args.workload == "multi1024":
            return run_multi1024(args)
        if args.workload == "batch256":
            return run_batch256(args)
        if args.workload == "case256":
            return run_case256(args)
        if args.workload == "vcycle":
            return run_vcycle(args)
        if args.workload == "learned512":
            return run_learned512(args)
        if args.workload == "cavity":
            return run_cavity(args)
        if args.workload == "cavity_time":
            return run_cavity_time(args)
        if args.workload == "unet":
            return run_unet(args)
        if args.workload == "sweep256":
            return run_ours(args)
        return run_multi1024(args)
    finally:
        if args.world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
