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
