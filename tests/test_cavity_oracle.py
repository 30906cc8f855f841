"""Pins of the cavity oracle (the paper's own test problem, sec. 4) against the
numbers the paper prints and against the mathematics.

* the no-slip Stokes operator: a manufactured solution converges at second
  order, the velocity block is symmetric negative definite and D = -G^T;
* the transfers: pressure restriction after prolongation is the identity,
  restriction rows of interior faces sum to one, prolongation reproduces a smooth
  field that vanishes on the walls to second order;
* Table 1: alpha_exp at h = 2^-5 ... 2^-7 (2^-8 with IB_ORACLE_SLOW=1);
* sec. 5: stand-alone multigrid and MG-GMRES iteration counts with 1 x 1 boxes,
  the spectral radius of the multigrid iteration matrix and the share of its
  eigenvalues outside two discs, the stiffnesses where the solvers give up;
* Table 2: all 36 MG-GMRES counts at h = 2^-6 for b = 1, 4, 8 and four
  smoothing schedules.

Counts are compared under the stopping rule's rounding: the paper's count must
lie between the first iteration whose residual is below 1.01e-6 and the first
below 0.99e-6 (two entries of Table 2 sit 0.1-0.3 % above 1e-6 one iteration
before the oracle stops).
"""
import math
import os

import numpy as np
import pytest

from oracle import cavity_oracle as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            out.append(line.split())
    return out


_AEXP = {}


def _alpha_exp(N):
    if N not in _AEXP:
        _AEXP[N] = C.explicit_limit(N, "ds1^2")[0]
    return _AEXP[N]


def _count_window(history, tol=1e-6, slack=0.01):
    """(first k with residual <= tol (1 + slack), first k with residual <= tol (1 - slack))."""
    lo = next((k for k, r in enumerate(history) if r <= tol * (1 + slack)), None)
    hi = next((k for k, r in enumerate(history) if r <= tol * (1 - slack)), None)
    return lo, hi


# ---------------------------------------------------------------- Stokes with walls

def _manufactured(N):
    """u = pi sin^2(pi x) sin(2 pi y), v = -pi sin(2 pi x) sin^2(pi y) (zero on every
    wall, divergence-free), p = cos(pi x) cos(pi y); f = -(Lap u - grad p)."""
    h = 1.0 / N
    k = np.arange(N)
    pi = math.pi
    xu, yu = np.meshgrid(k * h, (k + 0.5) * h, indexing="xy")
    xv, yv = np.meshgrid((k + 0.5) * h, k * h, indexing="xy")
    u = pi * np.sin(pi * xu) ** 2 * np.sin(2 * pi * yu)
    v = -pi * np.sin(2 * pi * xv) * np.sin(pi * yv) ** 2
    lap_u = 2 * pi ** 3 * np.sin(2 * pi * yu) * (2 * np.cos(2 * pi * xu) - 1)
    lap_v = -2 * pi ** 3 * np.sin(2 * pi * xv) * (2 * np.cos(2 * pi * yv) - 1)
    px = -pi * np.sin(pi * xu) * np.cos(pi * yu)
    py = -pi * np.cos(pi * xv) * np.sin(pi * yv)
    f = np.concatenate([-(lap_u - px).ravel(), -(lap_v - py).ravel()])
    return np.concatenate([u.ravel(), v.ravel()]), f


def test_wall_stokes_manufactured_solution_second_order():
    errs = []
    for N in (16, 32, 64):
        u_ex, f = _manufactured(N)
        u = C.stokes_velocity_solver(N)(f)
        free = np.setdiff1d(np.arange(2 * N * N), C.wall_rows(N))
        assert np.all(u[C.wall_rows(N)] == 0.0)
        errs.append(np.abs(u[free] - u_ex[free]).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.8, (errs, orders)
    assert errs[-1] < 1e-3 * math.pi  # 0.1 % of max |u|


def test_wall_stokes_symmetry_and_definiteness():
    N = 8
    A = C.cavity_stokes_matrix(N).toarray()
    n = N * N
    free = np.setdiff1d(np.arange(2 * n), C.wall_rows(N))
    K = A[np.ix_(free, free)]
    assert np.allclose(K, K.T, atol=0.0)
    assert np.linalg.eigvalsh(K).max() < 0.0
    G = -A[np.ix_(free, np.arange(2 * n, 3 * n))]
    D = A[np.ix_(np.arange(2 * n, 3 * n), free)]
    assert np.allclose(D, -G.T, atol=0.0)
    # wall rows are the identity and nothing else reads a wall face
    W = C.wall_rows(N)
    assert np.allclose(A[np.ix_(W, W)], np.eye(W.size))
    others = np.setdiff1d(np.arange(3 * n), W)
    assert np.all(A[np.ix_(others, W)] == 0.0)


def test_wall_transfers():
    Nc = 8
    Nf = 2 * Nc
    R = C.cavity_restriction(Nf).toarray()
    P = C.cavity_prolongation(Nc).toarray()
    pc = slice(2 * Nc * Nc, 3 * Nc * Nc)
    pf = slice(2 * Nf * Nf, 3 * Nf * Nf)
    assert np.allclose(R[pc, pf] @ P[pf, pc], np.eye(Nc * Nc))
    # interior coarse faces: restriction weights sum to one; wall faces have no row
    wc = C.wall_rows(Nc)
    rows = np.setdiff1d(np.arange(2 * Nc * Nc), wc)
    assert np.allclose(R[rows].sum(axis=1), 1.0)
    assert np.all(R[wc] == 0.0)
    # prolongation of a smooth field vanishing on the walls: second order
    errs = []
    for nc in (8, 16, 32):
        u_c, _ = _manufactured(nc)
        u_f, _ = _manufactured(2 * nc)
        Pm = C.cavity_prolongation(nc).toarray()[: 8 * nc * nc, : 2 * nc * nc]
        errs.append(np.abs(Pm @ u_c - u_f).max())
    assert math.log2(errs[0] / errs[1]) > 1.8 and math.log2(errs[1] / errs[2]) > 1.8, errs


# ---------------------------------------------------------------- Table 1

def test_annulus_geometry():
    a = C.Annulus(64)
    assert (a.M1, a.M2) == (152, 7)
    r = np.hypot(a.X[..., 0] - 0.5, a.X[..., 1] - 0.5)
    assert np.allclose(r[0], 0.25) and np.allclose(r[-1], 0.25 + 1.0 / 16.0)
    # adjacent nodes about 2/3 h apart along the inner fibre (sec. 4)
    d = np.hypot(*(a.X[0, 1] - a.X[0, 0]))
    assert abs(d * 64 - 2.0 / 3.0) < 0.01
    # A_f on one fibre: the closed-form spectrum of the circulant second difference
    Af = C.force_operator(a)[: a.M1, : a.M1].toarray()
    m = np.arange(a.M1)
    want = np.sort(-4.0 * np.sin(np.pi * m / a.M1) ** 2 / a.ds1 ** 2)
    assert np.allclose(np.sort(np.linalg.eigvalsh(Af)), want, rtol=1e-10, atol=1e-6)


def test_spread_and_interp_are_adjoint():
    N = 32
    a = C.Annulus(N)
    X = a.points()
    w = a.ds1 ** 2
    S = C.spread_matrix(X, N, w)
    Ss = C.interp_matrix_from_kernel(X, N)
    rng = np.random.default_rng(5)
    F = rng.standard_normal(S.shape[1])
    u = rng.standard_normal(S.shape[0])
    h = 1.0 / N
    assert abs(h * h * u @ (S @ F) - w * F @ (Ss @ u)) < 1e-12 * abs(w * F @ (Ss @ u)) + 1e-14
    # total force is conserved: h^2 sum(S F) = w sum(F) per component
    n = N * N
    Np = X.shape[0]
    assert abs(h * h * (S @ F)[:n].sum() - w * F[:Np].sum()) < 1e-12


@pytest.mark.parametrize("N", [32, 64, 128])
def test_table1_alpha_exp(N):
    printed = {int(r[0]): float(r[1]) for r in _rows("table1_alpha_exp.txt")}
    a = _alpha_exp(N)
    assert abs(a - printed[N]) <= 3e-3 * printed[N], (N, a, printed[N])
    # the other reading of the spreading weight (ds1 ds2) is 0.8 % off
    if N == 32:
        b = C.explicit_limit(N, "ds1ds2")[0]
        assert abs(b - printed[N]) > 5e-3 * printed[N]


@pytest.mark.skipif(not os.environ.get("IB_ORACLE_SLOW"), reason="about two minutes; set IB_ORACLE_SLOW=1")
def test_table1_alpha_exp_finest():
    printed = {int(r[0]): float(r[1]) for r in _rows("table1_alpha_exp.txt")}
    a = _alpha_exp(256)
    assert abs(a - printed[256]) <= 3e-3 * printed[256], a


# ---------------------------------------------------------------- sec. 5

def _sec5():
    counts, rho, outside = [], [], []
    for r in _rows("sec5_multigrid.txt"):
        if r[0] == "counts":
            counts.append((float(r[1]), int(r[2]), int(r[3])))
        elif r[0] == "rho":
            rho.append((float(r[1]), float(r[2])))
        else:
            outside.append((float(r[1]), float(r[2]), float(r[3])))
    return counts, rho, outside


def _mg_history(levels, b, max_cycles=100):
    A = levels[0].A
    w = np.zeros_like(b)
    bn = np.linalg.norm(b)
    hist = [1.0]
    for _ in range(max_cycles):
        w = C.cavity_vcycle(levels, b, w)
        hist.append(np.linalg.norm(b - A @ w) / bn)
        if hist[-1] <= 0.99e-6:
            break
    return hist


def test_sec5_iteration_counts():
    N = 32
    counts, _, _ = _sec5()
    for rel, mg, gm in counts:
        lev = C.cavity_hierarchy(N, rel * _alpha_exp(N), 1)
        b = C.cavity_rhs(N, lev)
        lo, hi = _count_window(_mg_history(lev, b))
        assert lo is not None and lo <= mg <= hi, (rel, mg, lo, hi)
        g = C.cavity_mg_gmres(lev, b, tol=0.99e-6)
        lo, hi = _count_window(g.history)
        assert lo is not None and lo <= gm <= hi, (rel, gm, lo, hi)


def test_sec5_limits_of_the_solvers():
    """Stand-alone multigrid gives up (more than 100 cycles) between relative
    stiffness 160 and 200; MG-GMRES reaches 100 iterations near 800 (sec. 5)."""
    N = 32
    a = _alpha_exp(N)
    lev = C.cavity_hierarchy(N, 160 * a, 1)
    assert C.cavity_mg_solve(lev, C.cavity_rhs(N, lev), max_cycles=100) is not None
    lev = C.cavity_hierarchy(N, 200 * a, 1)
    assert C.cavity_mg_solve(lev, C.cavity_rhs(N, lev), max_cycles=100) is None
    lev = C.cavity_hierarchy(N, 800 * a, 1)
    g = C.cavity_mg_gmres(lev, C.cavity_rhs(N, lev), max_iters=120)
    assert 95 <= g.iters <= 105, g.iters


def test_sec5_spectrum():
    N = 32
    _, rho, outside = _sec5()
    frac = {}
    for rel, want in rho:
        lev = C.cavity_hierarchy(N, rel * _alpha_exp(N), 1)
        M, _ = C.cavity_iteration_matrix(lev)
        ev = np.abs(C.cavity_spectrum(M, N))
        assert abs(ev.max() - want) <= 0.005, (rel, ev.max(), want)
        frac[rel] = ev
    for rel, radius, pct in outside:
        got = 100.0 * (frac[rel] > radius).mean()
        assert abs(got - pct) <= 0.5 if pct >= 5.0 else abs(got - pct) <= 0.1, (radius, got, pct)


# ---------------------------------------------------------------- Table 2

def test_table2_iteration_counts():
    N = 64
    a = _alpha_exp(N)
    rows = _rows("table2_iterations.txt")
    by_b = {}
    for r in rows:
        by_b.setdefault(int(r[0]), []).append(r)
    for b, entries in by_b.items():
        for col, rel in ((3, 10), (4, 100), (5, 500)):
            lev = C.cavity_hierarchy(N, rel * a, b)
            rhs = C.cavity_rhs(N, lev)
            for r in entries:
                nu1, nu2 = int(r[1]), int(r[2])
                g = C.cavity_mg_gmres(lev, rhs, tol=0.99e-6, max_iters=100, nu1=nu1, nu2=nu2)
                lo, hi = _count_window(g.history)
                if r[col] == "ge100":
                    assert lo is None, (b, nu1, nu2, rel, lo)
                else:
                    want = int(r[col])
                    assert lo is not None and lo <= want <= hi, (b, nu1, nu2, rel, want, lo, hi)


def test_workload_annulus_matches_oracle():
    """The shared input generator builds the same annulus the oracle pins (both restate
    sec. 4's formula), its fibres closed chains of zero-rest-length springs."""
    import ib_workloads as W

    for N in (32, 64):
        p = W.cavity_annulus(N, kappa=3.0)
        a = C.Annulus(N)
        assert np.array_equal(p.X, a.points())
        assert (p.meta["M1"], p.meta["M2"]) == (a.M1, a.M2) and p.meta["ds1"] == a.ds1
        assert p.springs.shape == (a.M1 * a.M2, 2) and np.all(p.rest == 0.0) and np.all(p.kappa == 3.0)
        # every point has exactly two springs, to its neighbours on the same fibre
        deg = np.bincount(p.springs.ravel(), minlength=p.X.shape[0])
        assert np.all(deg == 2)
        assert np.all(p.springs[:, 0] // a.M1 == p.springs[:, 1] // a.M1)


@pytest.mark.parametrize("frac,stable", [(0.9, True), (1.3, False)])
def test_explicit_method_stability_matches_alpha_exp(frac, stable):
    """Sec. 4.1 by a second route: forward Euler X <- X + alpha S^* L^{-1} S A_f X (the
    explicit-time method with the structure held at X^0 in S) started from a random
    X decays for alpha = 0.9 alpha_exp and grows for alpha = 1.3 alpha_exp, alpha_exp
    from the Lanczos eigenvalue."""
    N = 32
    a_exp = _alpha_exp(N)
    ann = C.Annulus(N)
    X0 = ann.points()
    S = C.spread_matrix(X0, N, ann.ds1 ** 2)
    Ss = C.interp_matrix_from_kernel(X0, N)
    Af = C.force_operator(ann)
    solve = C.stokes_velocity_solver(N)
    alpha = frac * a_exp
    rng = np.random.default_rng(11)
    x = rng.standard_normal(Af.shape[0])
    norms = []
    for _ in range(25):
        x = x + alpha * (Ss @ solve(S @ (Af @ x)))
        norms.append(np.linalg.norm(Af @ x))
    if stable:
        assert norms[-1] < norms[4], norms
    else:
        assert norms[-1] > 100.0 * norms[4], norms
