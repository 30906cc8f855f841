"""The Newton step on the GPU (ib_solve_step_newton: the spring force at the new
positions, sec. 8) against the oracle's Newton step.

* the exact Jacobian: the same number of Newton solves as the oracle, the fields
  within 1e-6 relative and the points within 1e-6 h of the oracle's converged step;
* the clamped Jacobian converges (linearly) to the same step;
* zero rest length: one correction that changes nothing (the force is linear);
* the first iterate alone is ib_solve_step's result, bit for bit.
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


def _case(clamped, rest=None, kappa=1e4, N=32, n_points=80):
    kw = dict(N=N, n_points=n_points, kappa=kappa, dt=1e-2)
    if rest is not None:
        kw["rest"] = rest
    p = W.single_ellipse(**kw)
    p.box = 4
    p.clamped = clamped
    return p


def _gpu_newton(pkg, p, prec="fp64", max_newton=30, tol=1e-10, u_n=None):
    s = pkg.IBSolver.from_problem(p, precision=prec)
    try:
        up = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
        X = dev(p.X)
        st = s.solve_step_newton(None if u_n is None else dev(u_n), up, X, max_newton=max_newton, tol_newton=tol)
        return st, up.cpu().numpy(), X.cpu().numpy()
    finally:
        s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_newton_exact_jacobian_matches_oracle(pkg, prec):
    p = _case(clamped=False)
    ref = O.solve_step_newton(p, max_newton=30, tol=1e-10)
    st, w, X = _gpu_newton(pkg, p, prec)
    assert st["status"] == 0, st
    assert abs(st["newton_iters"] - ref.iters) <= 1, (st["newton_iters"], ref.iters, ref.changes)
    assert st["newton_change"] <= 1e-10
    assert np.linalg.norm(w - ref.w) <= 1e-6 * np.linalg.norm(ref.w)
    assert np.abs(X - ref.X).max() <= 1e-6 * p.h


def test_newton_clamped_jacobian_reaches_the_same_step(pkg):
    pe = _case(clamped=False)
    ref = O.solve_step_newton(pe, max_newton=30, tol=1e-10)
    pc = _case(clamped=True)
    st, w, X = _gpu_newton(pkg, pc, "fp64", max_newton=40)
    assert st["status"] == 0 and st["newton_iters"] > ref.iters, st
    assert np.abs(X - ref.X).max() <= 1e-6 * pe.h
    assert np.linalg.norm(w - ref.w) <= 1e-6 * np.linalg.norm(ref.w)


def test_newton_zero_rest_length_one_correction(pkg):
    p = _case(clamped=True, rest=0.0, kappa=1e3, n_points=64)
    st, w, X = _gpu_newton(pkg, p, "fp64", max_newton=5, tol=1e-9)
    assert st["status"] == 0 and st["newton_iters"] == 2 and st["newton_change"] <= 1e-9, st


def test_newton_first_iterate_is_the_linearised_step(pkg):
    p = _case(clamped=True)
    st, w, X = _gpu_newton(pkg, p, "fp64", max_newton=1)
    s = pkg.IBSolver.from_problem(p)
    try:
        up = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
        Xl = dev(p.X)
        s.solve_step(None, up, Xl)
        assert st["newton_iters"] == 1
        assert np.array_equal(w, up.cpu().numpy()) and np.array_equal(X, Xl.cpu().numpy())
    finally:
        s.close()


def test_newton_with_u_n(pkg):
    p = _case(clamped=False)
    rng = np.random.default_rng(5)
    u_n = 0.05 * rng.standard_normal(2 * p.N * p.N)
    ref = O.solve_step_newton(p, u_n=u_n, max_newton=30, tol=1e-10)
    st, w, X = _gpu_newton(pkg, p, "fp64", u_n=u_n)
    assert st["status"] == 0
    assert np.linalg.norm(w - ref.w) <= 1e-6 * np.linalg.norm(ref.w)
    assert np.abs(X - ref.X).max() <= 1e-6 * p.h


def test_newton_rejects_bad_arguments(pkg):
    from paper_1311_5614_gb300 import capi as CA

    p = _case(clamped=True)
    s = pkg.IBSolver.from_problem(p)
    try:
        up = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
        with pytest.raises(CA.IBError):
            s.solve_step_newton(None, up, dev(p.X), max_newton=0)
        with pytest.raises(CA.IBError):
            s.solve_step_newton(None, up, dev(p.X), tol_newton=-1.0)
    finally:
        s.close()
