"""The paper's own problem on the GPU: the square with no-slip walls and the thick
annulus (sec. 4), through the C ABI (IB_WALLS_NOSLIP), against the cavity oracle
in the colour order.

* every level's operator A_l (re-discretised wall Stokes + the Galerkin
  elasticity with the wall prolongation) element by element at 1e-10;
* one V-cycle in FP64 at 1e-10 for b = 1, 2, 4, 8; FP32 and mixed within the
  element-wise bars of the periodic tests;
* MG-GMRES solves of the lid-driven right-hand side: iteration counts equal to
  the oracle's (colour order) within one, the true residual on the oracle's CSR
  operator within the tolerance;
* points closer than 2h to a wall are refused.
"""
import types

import numpy as np
import pytest

import ib_workloads as W
from oracle import cavity_oracle as C

pytestmark = pytest.mark.gpu


def _geom(p):
    """The workload's annulus as the oracle's geometry object."""
    m = p.meta
    return types.SimpleNamespace(N=p.N, M1=m["M1"], M2=m["M2"], ds1=m["ds1"], ds2=m["ds2"], points=lambda: p.X)


def _problem(N, rel, b):
    """Relative stiffness rel = alpha / alpha_exp; the springs carry kappa = alpha with dt = 1."""
    a_exp = C.explicit_limit(N, "ds1^2")[0]
    alpha = rel * a_exp
    p = W.cavity_annulus(N, kappa=alpha, dt=1.0)
    levels = C.cavity_hierarchy(N, alpha, b, ann=_geom(p), order="color4")
    return p, levels


def _solver(p, b, precision="fp64", tol=1e-8, max_iters=200, lid=0.0):
    from paper_1311_5614_gb300 import capi as CA

    return CA.IBSolver(p.N, p.X, p.springs, p.kappa, p.rest, L=1.0, rho=0.0, mu=1.0, dt=p.dt, delta="cos4",
                       box=b, walls="noslip", precision=precision, tol=tol, max_iters=max_iters, lid=lid)


def _random_unknowns(N, seed):
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(3 * N * N)
    w[C.wall_rows(N)] = 0.0
    return w


def _rel_per_component(got, want, N):
    n = N * N
    out = []
    for c in range(3):
        g, r = got[c * n:(c + 1) * n], want[c * n:(c + 1) * n]
        out.append(np.abs(g - r).max() / max(np.abs(r).max(), 1e-300))
    return max(out)


@pytest.mark.parametrize("N,rel,b", [(32, 10.0, 4), (64, 100.0, 4), (32, 100.0, 1), (64, 10.0, 8)])
def test_cavity_apply_every_level(N, rel, b):
    import torch

    p, levels = _problem(N, rel, b)
    s = _solver(p, b)
    try:
        assert s.n_levels == len(levels)
        for l, lev in enumerate(levels):
            n = lev.N
            w = _random_unknowns(n, 7 + l)
            y = torch.zeros(3 * n * n, dtype=torch.float64, device="cuda")
            s.apply(l, torch.tensor(w, device="cuda"), y)
            want = lev.A @ w
            assert _rel_per_component(y.cpu().numpy(), want, n) < 1e-10, l
    finally:
        s.close()


@pytest.mark.parametrize("b", [1, 2, 4, 8])
def test_cavity_vcycle_fp64(b):
    import torch

    N = 32 if b < 8 else 64
    p, levels = _problem(N, 30.0, b)
    s = _solver(p, b)
    try:
        rhs = C.cavity_rhs(N, levels, ann=_geom(p))
        w = torch.zeros(3 * N * N, dtype=torch.float64, device="cuda")
        s.vcycle(torch.tensor(rhs, device="cuda"), w)
        want = C.cavity_vcycle(levels, rhs, np.zeros_like(rhs))
        assert _rel_per_component(w.cpu().numpy(), want, N) < 1e-10
    finally:
        s.close()


@pytest.mark.parametrize("precision,bar", [("fp32", 2e-5), ("mixed", 5e-7)])
def test_cavity_vcycle_reduced_precision(precision, bar):
    import torch

    N, b = 64, 4
    p, levels = _problem(N, 30.0, b)
    s = _solver(p, b, precision=precision)
    try:
        rhs = C.cavity_rhs(N, levels, ann=_geom(p))
        w = torch.zeros(3 * N * N, dtype=torch.float64, device="cuda")
        s.vcycle(torch.tensor(rhs, device="cuda"), w)
        want = C.cavity_vcycle(levels, rhs, np.zeros_like(rhs))
        assert _rel_per_component(w.cpu().numpy(), want, N) < bar
    finally:
        s.close()


@pytest.mark.parametrize("N,rel,b", [(32, 0.0, 1), (32, 10.0, 1), (64, 100.0, 4), (64, 500.0, 8), (64, 10.0, 2)])
def test_cavity_solve_counts(N, rel, b):
    import torch

    p, levels = _problem(N, rel, b)
    rhs = C.cavity_rhs(N, levels, ann=_geom(p))
    ref = C.cavity_mg_gmres(levels, rhs, tol=1e-8, max_iters=200)
    s = _solver(p, b, tol=1e-8, max_iters=200)
    try:
        x = torch.zeros(3 * N * N, dtype=torch.float64, device="cuda")
        st = s.solve(torch.tensor(rhs, device="cuda"), x)
        assert st["status"] == 0
        assert abs(st["iters"] - ref.iters) <= 1, (st["iters"], ref.iters)
        xs = x.cpu().numpy()
        A = levels[0].A
        assert np.linalg.norm(rhs - A @ xs) / np.linalg.norm(rhs) <= 1.05e-8
        assert np.all(xs[C.wall_rows(N)] == 0.0)
    finally:
        s.close()


def test_cavity_rhs_with_lid_and_step():
    """ib_rhs with the moving lid: the lid's ghost term plus -S F(X) (F = kappa A_f X ds1^2,
    the oracle's force term times kappa); one implicit step through ib_solve_step solves
    that system (true residual on the oracle's operator) and moves the points by S^* u."""
    import torch

    N, b = 64, 4
    p, levels = _problem(N, 10.0, b)
    s = _solver(p, b, lid=1.0)
    try:
        rhs = torch.zeros(3 * N * N, dtype=torch.float64, device="cuda")
        s.rhs(None, rhs)
        want = C.cavity_rhs(N, levels, ann=_geom(p), force_scale=float(p.kappa[0]))
        got = rhs.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
        up = torch.zeros_like(rhs)
        X = torch.tensor(p.X, device="cuda")
        st = s.solve_step(None, up, X)
        assert st["status"] == 0
        x = up.cpu().numpy()
        assert np.linalg.norm(want - levels[0].A @ x) / np.linalg.norm(want) <= 1.05e-8
        # X^{n+1} = X^n + dt S^* u with the interpolation of the oracle
        Ss = C.interp_matrix_from_kernel(p.X, N)
        U = Ss @ x[: 2 * N * N]
        npt = p.X.shape[0]
        Xn = p.X + p.dt * np.stack([U[:npt], U[npt:]], axis=1)
        assert np.abs(X.cpu().numpy() - Xn).max() <= 1e-9 / N
    finally:
        s.close()


def test_cavity_point_near_wall_is_refused():
    from paper_1311_5614_gb300 import capi as CA

    p = W.cavity_annulus(32, kappa=1.0)
    X = p.X.copy()
    X[0] = (1.5 / 32, 0.5)  # 1.5 h from the wall x = 0
    with pytest.raises(CA.IBError):
        CA.IBSolver(32, X, p.springs, p.kappa, p.rest, rho=0.0, mu=1.0, dt=1.0, delta="cos4", box=4,
                    walls="noslip")


def _explicit_solver(p, b, dt, lid=0.0, tol=1e-8):
    from paper_1311_5614_gb300 import capi as CA

    return CA.IBSolver(p.N, p.X, p.springs, p.kappa, p.rest, L=1.0, rho=0.0, mu=1.0, dt=dt, delta="cos4",
                       box=b, walls="noslip", tol=tol, max_iters=200, lid=lid, time_method="explicit")


def test_cavity_explicit_step_matches_oracle():
    """One step of the explicit-time method (sec. 2.3.1): the Stokes system alone with
    the force F(X^n) on the right-hand side, then X^{n+1} = X^n + dt S^* u."""
    import torch

    N, b, gamma, dt = 64, 4, 50.0, 0.01
    p = W.cavity_annulus(N, kappa=gamma, dt=dt)
    lev0 = C.cavity_hierarchy(N, 0.0, b, ann=_geom(p))  # Stokes alone
    want_b = C.cavity_rhs(N, lev0, ann=_geom(p), force_scale=gamma)
    s = _explicit_solver(p, b, dt, lid=1.0)
    try:
        up = torch.zeros(3 * N * N, dtype=torch.float64, device="cuda")
        X = torch.tensor(p.X, device="cuda")
        st = s.solve_step(None, up, X)
        assert st["status"] == 0 and st["n_struct_boxes"] > 0
        x = up.cpu().numpy()
        A = lev0[0].A
        assert np.linalg.norm(want_b - A @ x) / np.linalg.norm(want_b) <= 1.05e-8
        Ss = C.interp_matrix_from_kernel(p.X, N)
        U = Ss @ x[: 2 * N * N]
        npt = p.X.shape[0]
        assert np.abs(X.cpu().numpy() - (p.X + dt * np.stack([U[:npt], U[npt:]], axis=1))).max() <= 1e-12
    finally:
        s.close()


@pytest.mark.parametrize("frac,stable", [(0.9, True), (1.3, False)])
def test_cavity_explicit_stability_limit(frac, stable):
    """The explicit-time method is stable for gamma dt below alpha_exp (sec. 4.1, Table
    1: 6.09 at h = 2^-5, the oracle's value) and unstable above: from a small
    high-frequency perturbation of the annulus, the step-to-step displacement decays
    at 0.9 alpha_exp and grows at 1.3 alpha_exp (amplification |1 - 2 frac| per step of
    the stiffest mode)."""
    import torch

    N, b, gamma = 32, 4, 1.0e4
    a_exp = C.explicit_limit(N, "ds1^2")[0]
    dt = frac * a_exp / gamma
    p = W.cavity_annulus(N, kappa=gamma, dt=dt)
    rng = np.random.default_rng(3)
    X0 = p.X + (1e-3 / N) * rng.standard_normal(p.X.shape)
    s = _explicit_solver(p, b, dt)
    try:
        up = torch.zeros(3 * N * N, dtype=torch.float64, device="cuda")
        X = torch.tensor(X0, device="cuda")
        s.update_points(X)
        disp = []
        for _ in range(12):
            Xp = X.clone()
            st = s.solve_step(None, up, X)
            assert st["status"] == 0
            disp.append(float(torch.linalg.vector_norm(X - Xp)))
        growth = disp[-1] / disp[1]
        if stable:
            assert growth < 1.0, disp
        else:
            assert growth > 10.0, disp
    finally:
        s.close()
