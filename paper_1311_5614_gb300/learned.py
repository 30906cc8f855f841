"""Training and evaluation of the learned FGMRES stage (orchestration only).

Every numerical step runs in libibmg.so: pairs come from ib_learned_pair (the
problem's own operator and V-cycle), training from ib_unet_train_step (the
library's forward, backward and Adam kernels).  This module only draws the
seeded inputs, orders the calls and keeps the pairs in device memory.

Pair recipe (not in the paper): the residual -> error pairs the method produces
while it solves.  For a training problem (random stiffness, jittered centre) and a
right-hand side b = -(rho/dt) u^n - S F (u^n a random smooth velocity of random
amplitude), x* is solved to 1e-10; multigrid as a stand-alone solver (sec. 5) from
x_0 = 0 then gives e_0 = x* and e_{k+1} = e_k - MG(A e_k), and every step yields the
pair (r_{k+1} = A e_{k+1}, e_{k+1}): the residual left by a V-cycle and the error
that remains (ib_learned_chain).  That residual is what the FGMRES stage receives
(r = v - A MG(v)).  The network learns r/|r| (+ the structure channel) -> e/|r|.
The earlier recipe (b = A x for random smooth fields x, one V-cycle) is kept as
mode "smooth".
"""
from __future__ import annotations

import time

import numpy as np

import ib_workloads as W

from . import capi as C


def harvest_chain(N=512, n_points=1024, n_problems=40, rhs_per_problem=4, chain=64, seed=0,
                  log_kappa=(2.0, 6.0), dt=1e-2, box=4, precision="fp32"):
    """Pairs along multigrid-solver chains of solved steps: device tensors X [P, 4 N^2],
    T [P, 3 N^2] (float32), P = n_problems x rhs_per_problem x chain, and the kappas."""
    import torch

    rng = np.random.default_rng(seed)
    P = n_problems * rhs_per_problem * chain
    X = torch.empty((P, 4 * N * N), dtype=torch.float32, device="cuda")
    T = torch.empty((P, 3 * N * N), dtype=torch.float32, device="cuda")
    kappas = []
    k = 0
    for _ in range(n_problems):
        kap = float(10.0 ** rng.uniform(*log_kappa))
        cx, cy = 0.5 + 0.02 * rng.standard_normal(2)
        prob = W.single_ellipse(N=N, n_points=n_points, kappa=kap, dt=dt, center=(cx, cy))
        prob.box = box
        s = C.IBSolver.from_problem(prob, precision=precision, tol=1e-10, max_iters=400)
        X0 = torch.tensor(prob.X, dtype=torch.float64, device="cuda")
        for _ in range(rhs_per_problem):
            amp = float(10.0 ** rng.uniform(-2.0, 0.0))
            un = torch.tensor(amp * W.random_smooth_field(N, int(rng.integers(1 << 31)), count=2).ravel(),
                              dtype=torch.float64, device="cuda")
            e = torch.zeros(3 * N * N, dtype=torch.float64, device="cuda")
            s.solve_step(un, e, X0.clone())  # e = x*, the error of x_0 = 0
            s.update_points(X0)              # the step moved the problem's points: restore X^n
            e0 = float(torch.linalg.vector_norm(e))
            for _ in range(chain):
                # a chain that has converged (or overflowed) yields no further pairs
                en = float(torch.linalg.vector_norm(e))
                if not (1e-12 * e0 < en < 1e30 * e0):
                    break
                s.learned_chain(e, X[k], T[k])
                k += 1
        s.close()
        kappas.append(kap)
    torch.cuda.synchronize()
    # drop pairs with a non-finite or vanishing target
    ok = torch.isfinite(X[:k]).all(dim=1) & torch.isfinite(T[:k]).all(dim=1) & (T[:k].abs().sum(dim=1) > 0)
    idx = torch.nonzero(ok).flatten()
    return X[idx], T[idx], kappas


def holdout_loss(net, X, T):
    """Mean relative squared error of the network over pairs (no update)."""
    tot = 0.0
    for i in range(X.shape[0]):
        L, _ = net.loss_grad(X[i], T[i])
        tot += L
    return tot / max(X.shape[0], 1)


def harvest(N=512, n_points=1024, n_problems=40, pairs_per_problem=256, seed=0, log_kappa=(2.0, 6.0),
            dt=1e-2, box=4, precision="fp32"):
    """Mode "smooth": b = A x for random smooth fields x.  Return device tensors X
    [P, 4 N^2], T [P, 3 N^2] (float32) and the problems' kappas."""
    import torch

    from concurrent.futures import ThreadPoolExecutor

    rng = np.random.default_rng(seed)
    P = n_problems * pairs_per_problem
    X = torch.empty((P, 4 * N * N), dtype=torch.float32, device="cuda")
    T = torch.empty((P, 3 * N * N), dtype=torch.float32, device="cuda")
    # draw every seed in the fixed order first, then generate the fields on host
    # threads ahead of the device work (the FFTs release the GIL)
    plan = []
    for i in range(n_problems):
        kap = float(10.0 ** rng.uniform(*log_kappa))
        cx, cy = 0.5 + 0.02 * rng.standard_normal(2)
        seeds = [int(rng.integers(1 << 31)) for _ in range(pairs_per_problem)]
        plan.append((kap, (cx, cy), seeds))
    kappas = []
    k = 0
    with ThreadPoolExecutor(max_workers=8) as pool:
        for kap, centre, seeds in plan:
            fields = pool.map(lambda sd: W.random_smooth_field(N, sd).ravel(), seeds)
            prob = W.single_ellipse(N=N, n_points=n_points, kappa=kap, dt=dt, center=centre)
            prob.box = box
            s = C.IBSolver.from_problem(prob, precision=precision)
            for f in fields:
                s.learned_pair(torch.tensor(f, device="cuda"), X[k], T[k])
                k += 1
            s.close()
            kappas.append(kap)
    torch.cuda.synchronize()
    return X, T, kappas


def train(net, X, T, epochs=2, lr=1e-3, seed=0, log=None):
    """Adam over the pairs in a seeded random order; returns the per-epoch mean losses."""
    import torch

    rng = np.random.default_rng(seed)
    P = X.shape[0]
    losses = []
    total = epochs * P
    step = 0
    for ep in range(epochs):
        order = rng.permutation(P)
        acc = 0.0
        for idx in order:
            # cosine decay of the learning rate over the whole run
            a = lr * 0.5 * (1.0 + np.cos(np.pi * step / max(total, 1)))
            L = net.train_step(X[int(idx)], T[int(idx)], float(max(a, 1e-5)))
            acc += L if np.isfinite(L) else 0.0
            step += 1
        losses.append(acc / P)
        if log:
            log("epoch %d loss %.4f" % (ep, losses[-1]))
    torch.cuda.synchronize()
    return losses


def evaluate(net, N=512, n_points=1024, kappas=(1e2, 1e4, 1e6), dt=1e-2, box=4, precision="fp32",
             seed=1000003, repeats=3):
    """Plain MG-FGMRES vs MG-FGMRES with the learned stage on held-out problems:
    iterations and device time of one implicit step each."""
    import torch

    rng = np.random.default_rng(seed)
    out = []
    for kap in kappas:
        cx, cy = 0.5 + 0.02 * rng.standard_normal(2)
        prob = W.single_ellipse(N=N, n_points=n_points, kappa=kap, dt=dt, center=(cx, cy))
        prob.box = box
        row = {"kappa": kap}
        for mode in ("plain", "learned"):
            s = C.IBSolver.from_problem(prob, precision=precision, max_iters=400)
            if mode == "learned":
                s.set_learned_stage(net)
            up = torch.zeros(3 * N * N, dtype=torch.float64, device="cuda")
            X0 = torch.tensor(prob.X, device="cuda")
            times, st = [], None
            for r in range(repeats + 1):
                X = X0.clone()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                st = s.solve_step(None, up, X)
                b.record()
                torch.cuda.synchronize()
                if r > 0:
                    times.append(a.elapsed_time(b))
            row[mode] = {"iters": st["iters"], "ms": float(np.median(times)), "status": st["status"],
                         "rel_res_true": st["rel_res_true"], "learned_used": st["learned_used"],
                         "escalated_at": st["escalated_at"]}
            if mode == "learned":
                s.set_learned_stage(None)
            s.close()
        out.append(row)
    return out


def run(N=512, n_problems=40, pairs_per_problem=256, epochs=2, lr=1e-3, seed=0, log=print, mode="chain",
        rhs_per_problem=4, chain=64, n_holdout=4, n_points=None):
    """Harvest, train from a seeded initialisation, evaluate; returns a summary dict.
    mode "chain": n_problems x rhs_per_problem x chain pairs from multigrid-solver
    chains (held-out loss on n_holdout further problems); mode "smooth": n_problems x
    pairs_per_problem pairs from random smooth fields."""
    n_points = n_points or 2 * N
    t0 = time.perf_counter()
    if mode == "chain":
        X, T, kap = harvest_chain(N=N, n_points=n_points, n_problems=n_problems, rhs_per_problem=rhs_per_problem,
                                  chain=chain, seed=seed)
        Xh, Th, _ = harvest_chain(N=N, n_points=n_points, n_problems=n_holdout, rhs_per_problem=1, chain=chain,
                                  seed=seed + 99991)
    else:
        X, T, kap = harvest(N=N, n_points=n_points, n_problems=n_problems, pairs_per_problem=pairs_per_problem,
                            seed=seed)
        Xh, Th = X[:0], T[:0]
    t1 = time.perf_counter()
    net = C.UNet(N, W.unet_init_params(seed + 7))
    h0 = holdout_loss(net, Xh, Th) if Xh.shape[0] else None
    losses = train(net, X, T, epochs=epochs, lr=lr, seed=seed, log=log)
    h1 = holdout_loss(net, Xh, Th) if Xh.shape[0] else None
    t2 = time.perf_counter()
    pairs = int(X.shape[0])
    del X, T, Xh, Th
    ev = evaluate(net, N=N, n_points=n_points)
    t3 = time.perf_counter()
    params = net.get_params()
    net.close()
    return {"mode": mode, "pairs": pairs, "train_kappas": kap, "epochs": epochs, "losses": losses,
            "holdout_loss_before": h0, "holdout_loss_after": h1,
            "harvest_s": t1 - t0, "train_s": t2 - t1, "eval_s": t3 - t2, "eval": ev, "params": params}
