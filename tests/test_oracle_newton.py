"""Pins of the oracle's Newton step (the backward-Euler step with the spring force at
the new positions, sec. 8): checked against the nonlinear equations themselves,
written out from the pinned Stokes matrix, spreading and spring force, not
against the linearisation the iteration uses.

* the first iterate is the linearised step (sec. 2.3), bit for bit;
* zero rest length: the force is linear (F = kappa A_f X), so the first iterate
  already solves the step and the second changes nothing;
* the converged step solves mu Lap u - (rho/dt) u - G p + S F(X^n + dt S^* u) = 0,
  D u = 0, to the linear solver's tolerance, where the linearised step leaves a
  residual hundreds of times larger;
* with the exact Jacobian the changes fall quadratically, with the clamped one
  linearly, to the same fixed point.
"""
import numpy as np
import pytest

import ib_workloads as W
from oracle import ib_oracle as O


def _case(clamped, rest=None, kappa=1e4):
    kw = dict(N=32, n_points=80, kappa=kappa, dt=1e-2)
    if rest is not None:
        kw["rest"] = rest
    p = W.single_ellipse(**kw)
    p.box = 4
    p.clamped = clamped
    return p


def _nonlinear_residual(p, w, X_new):
    """mu Lap u - (rho/dt) u - G p + S(X^n) F(X_new) (and D u), relative to |S F(X^n)|."""
    N, h = p.N, p.h
    A = O.stokes_matrix(N, h, p.mu, p.rho, p.dt)
    S = O.spread_matrix(p.X, N, p.L, p.delta)
    F = O.spring_force(X_new, p.springs, p.kappa, p.rest, p.L)
    F0 = O.spring_force(p.X, p.springs, p.kappa, p.rest, p.L)
    r = A @ w
    r[:2 * N * N] += S @ np.concatenate([F[:, 0], F[:, 1]])
    ref = np.linalg.norm(S @ np.concatenate([F0[:, 0], F0[:, 1]]))
    return np.linalg.norm(r) / ref


def test_first_newton_iterate_is_the_linearised_step():
    p = _case(clamped=True)
    r = O.solve_step_newton(p, max_newton=1)
    ref = O.solve_step(p)
    assert r.iters == 1
    assert np.array_equal(r.w, ref.w) and np.array_equal(r.X, ref.X)


def test_zero_rest_length_needs_no_correction():
    p = _case(clamped=True, rest=0.0, kappa=1e3)
    r = O.solve_step_newton(p, max_newton=5, tol=1e-9)
    assert r.iters == 2 and r.changes[1] <= 1e-10, r.changes


def test_converged_step_solves_the_nonlinear_equations():
    p = _case(clamped=False)
    r = O.solve_step_newton(p, max_newton=12, tol=1e-10)
    lin = O.solve_step(p)
    res_newton = _nonlinear_residual(p, r.w, r.X)
    res_lin = _nonlinear_residual(p, lin.w, lin.X)
    assert res_newton <= 1e-7, res_newton
    assert res_lin >= 300 * res_newton, (res_lin, res_newton)
    n = p.N * p.N
    D = O.stokes_matrix(p.N, p.h, p.mu, p.rho, p.dt)[2 * n:]
    assert np.linalg.norm(D @ r.w) <= 1e-7 * np.linalg.norm(r.w)


def test_exact_jacobian_converges_quadratically_clamped_linearly_same_point():
    pe = _case(clamped=False)
    re = O.solve_step_newton(pe, max_newton=12, tol=1e-10)
    c = re.changes
    for k in range(1, len(c) - 1):
        if c[k] > 1e-10:
            assert c[k + 1] <= 2.0 * c[k] ** 2, c
    pc = _case(clamped=True)
    rc = O.solve_step_newton(pc, max_newton=30, tol=1e-10)
    cc = rc.changes
    ratios = [cc[k + 1] / cc[k] for k in range(1, len(cc) - 1)]
    assert max(ratios) < 0.5 and min(ratios) > 1e-3, ratios  # linear, not quadratic
    assert rc.iters > re.iters
    assert np.abs(rc.X - re.X).max() <= 1e-8 * pe.h
    assert np.linalg.norm(rc.w - re.w) <= 1e-7 * np.linalg.norm(re.w)


@pytest.mark.parametrize("rho", [1.0])
def test_newton_with_u_n_term(rho):
    """The -(rho/dt) u^n term enters every iterate's right-hand side: the converged
    step with u^n solves the nonlinear equations with that term."""
    p = _case(clamped=False)
    p.rho = rho
    rng = np.random.default_rng(5)
    N = p.N
    u_n = 0.05 * rng.standard_normal(2 * N * N)
    r = O.solve_step_newton(p, u_n=u_n, max_newton=12, tol=1e-10)
    A = O.stokes_matrix(N, p.h, p.mu, p.rho, p.dt)
    S = O.spread_matrix(p.X, N, p.L, p.delta)
    F = O.spring_force(r.X, p.springs, p.kappa, p.rest, p.L)
    res = A @ r.w
    res[:2 * N * N] += S @ np.concatenate([F[:, 0], F[:, 1]]) + (p.rho / p.dt) * u_n
    b = np.concatenate([(p.rho / p.dt) * u_n, np.zeros(N * N)])
    assert np.linalg.norm(res) <= 1e-7 * np.linalg.norm(b)
