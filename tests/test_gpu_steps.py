"""Consecutive implicit steps against the oracle: u^n and X carried from step to step.

The path of the 1024^2 multi-structure workload, at a size the oracle finishes in
seconds: each step starts from the previous step's velocity and points (the
-(rho/dt) u^n term of the right-hand side, Eq. 20's point update feeding the next
step's S, J and hierarchy).  Bars: every step reaches the FP64 relative residual
1e-8 on the oracle's own CSR operator; the fields agree with the oracle's to 1e-6
relative and the points to 1e-6 h after each step (solver tolerance times the
conditioning margin, compounded over three steps); FP64 iteration counts within
one of the oracle's.
"""
import numpy as np
import pytest

import ib_workloads as W
from oracle import ib_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_5614_gb300 as P

    P.lib()
    return P


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("prec,box", [("fp64", 4), ("fp32", 4), ("mixed", 2)])
def test_three_consecutive_steps_match_oracle(pkg, prec, box):
    p = W.many_ellipses(N=64, count=3, n_per=96, kappa=1e4, dt=1e-3, seed=1311, lo=0.08, hi=0.14)
    p.box = box
    n2 = 2 * p.N * p.N
    s = pkg.IBSolver.from_problem(p, precision=prec)
    up = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    un = torch.zeros(n2, dtype=torch.float64, device="cuda")
    X = dev(p.X)
    u_ref, X_ref = None, p.X.copy()
    moved = 0.0
    for step in range(3):
        ref = O.solve_step(p, u_n=u_ref, X=X_ref)
        st = s.solve_step(un if step else None, up, X)
        w = up.cpu().numpy()
        assert st["status"] == 0 and st["rel_res_true"] <= p.tol, (step, st)
        A = O.build_hierarchy(p, X_ref)[0][0].A
        assert np.linalg.norm(ref.b - A @ w) <= 1.01 * p.tol * np.linalg.norm(ref.b), step
        err = np.linalg.norm(w - ref.w) / np.linalg.norm(ref.w)
        assert err <= 1e-6, (step, err)
        xe = np.abs(X.cpu().numpy() - ref.X).max()
        assert xe <= 1e-6 * p.h, (step, xe)
        if prec == "fp64":
            assert abs(st["iters"] - ref.solve.iters) <= 1, (step, st["iters"], ref.solve.iters)
        moved = max(moved, np.abs(ref.X - X_ref).max())
        u_ref, X_ref = ref.w[:n2], ref.X
        un.copy_(up[:n2])
    assert moved > 1e-3 * p.h  # the points really move between steps
    s.close()


@pytest.mark.parametrize("prec,kappa,dt,N", [("fp64", 1e4, 1e-3, 64), ("fp32", 1e6, 1e-2, 128), ("mixed", 1e6, 1e-2, 128)])
def test_step_is_bitwise_reproducible(pkg, prec, kappa, dt, N):
    """The same step solved twice (each with its own set-up) gives bit-identical
    velocity, pressure and points and the same iteration count: the right-hand
    side's spread, the FP64 operator's spread and the level-0 row assembly gather
    through per-row point lists in a fixed order, and every reduction sums in a
    fixed order (no floating-point atomics on the path).  The stiff cases are the
    ones whose count varied with the summation order of atomic spreads."""
    p = W.single_ellipse(N=N, n_points=2 * N, kappa=kappa, dt=dt)
    p.box = 4
    s = pkg.IBSolver.from_problem(p, precision=prec, max_iters=200)
    outs = []
    for _ in range(2):
        up = torch.zeros(3 * N * N, dtype=torch.float64, device="cuda")
        X = dev(p.X)
        st = s.solve_step(None, up, X)
        assert st["status"] == 0
        outs.append((st["iters"], up.clone(), X.clone()))
    s.close()
    (i0, u0, x0), (i1, u1, x1) = outs
    assert i0 == i1
    assert torch.equal(u0, u1) and torch.equal(x0, x1)


def test_repeated_setups_give_identical_vcycles(pkg):
    """Six set-ups of the same points (ib_update_points) give bit-identical FP32
    and FP64 V-cycles on the 512^2 strip-kernel case: nothing in the set-up depends
    on the order in which threads run (slot numbers do, values do not).  A race in
    the shared-memory Gauss-Jordan inversion of the box blocks used to make about
    one set-up in ten wrong here."""
    import os

    os.environ["IB_BOX_STRIP_MIN"] = "1"
    os.environ["IB_BOX_STRIP_W"] = "32"
    try:
        p = W.single_ellipse(N=512, n_points=1024, kappa=1e4, dt=1e-3)
        p.box = 4
        rhs = dev(O.rhs_vector(p))
        for prec in ("fp32", "fp64"):
            s = pkg.IBSolver.from_problem(p, precision=prec)
            X = dev(p.X)
            first = None
            for k in range(6):
                if k:
                    s.update_points(X)
                w = torch.zeros(3 * 512 * 512, dtype=torch.float64, device="cuda")
                s.vcycle(rhs, w)
                if first is None:
                    first = w.clone()
                assert torch.equal(w, first), (prec, k)
            s.close()
    finally:
        del os.environ["IB_BOX_STRIP_MIN"]
        del os.environ["IB_BOX_STRIP_W"]


def test_no_read_of_unwritten_device_memory(pkg, tmp_path):
    """With IB_POISON=1 every device allocation of the library starts as all-ones
    bytes (NaN in floating point): a fresh process then solves one step in each
    precision and runs the FP32 V-cycle, and every result is finite and matches
    the oracle as in the other tests, so nothing reads memory the library has not
    written."""
    import os
    import subprocess
    import sys

    code = r'''
import sys, numpy as np, torch
sys.path.insert(0, "."); sys.path.insert(0, "tests")
import ib_workloads as W
from oracle import ib_oracle as O
import paper_1311_5614_gb300 as pkg
p = W.many_ellipses(N=64, count=3, n_per=96, kappa=1e4, dt=1e-3, seed=1311, lo=0.08, hi=0.14)
p.box = 4
ref = O.solve_step(p)
for prec in ("fp64", "fp32", "mixed"):
    s = pkg.IBSolver.from_problem(p, precision=prec)
    up = torch.zeros(3 * 64 * 64, dtype=torch.float64, device="cuda")
    st = s.solve_step(None, up, torch.tensor(p.X, device="cuda"))
    w = up.cpu().numpy()
    assert st["status"] == 0 and np.all(np.isfinite(w)), (prec, st)
    err = np.linalg.norm(w - ref.w) / np.linalg.norm(ref.w)
    assert err <= 1e-6, (prec, err)
    s.close()
print("ok")
'''
    env = dict(os.environ, IB_POISON="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600,
                         cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert out.returncode == 0 and "ok" in out.stdout, out.stdout + out.stderr

