"""Failure paths of the C ABI, made on the host (no fault, trap or hang of the GPU).

Each case feeds the library an input or a setting that it must turn into a status
code, and then checks that the CUDA context is still usable by solving a normal
problem in the same process:

* a non-finite velocity u^n gives a non-finite right-hand side: IB_ERR_BREAKDOWN;
* two spring end points moved onto each other through ib_update_points: the
  spring kernel flags the zero length, IB_ERR_INVALID_ARG, and the problem
  accepts valid points again afterwards;
* an iteration cap of 1 on a stiff step: IB_ERR_NOT_CONVERGED with the iterate
  written and the points moved;
* a bounded device-side wait forced to run out: the environment variable
  IB_WAIT_LIMIT_NS = 0 at set-up (with IB_CGS_REG = 0, so that small bases also
  take the bulk-copy form) makes every wait of the Gram-Schmidt pass for
  its bulk copies give up at once (the copies still land: the block waits for
  them before it exits), which the solve reports as IB_ERR_TIMEOUT.
"""
import numpy as np
import pytest

import ib_workloads as W

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


def _healthy_solve(pkg):
    p = W.single_ellipse(N=32, n_points=64, kappa=1e2, dt=1e-2)
    s = pkg.IBSolver.from_problem(p)
    up = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    st = s.solve_step(None, up, dev(p.X))
    s.close()
    assert st["status"] == 0 and st["rel_res_true"] <= p.tol
    assert torch.isfinite(up).all()


def test_nonfinite_velocity_is_a_breakdown(pkg):
    p = W.single_ellipse(N=32, n_points=64, kappa=1e2, dt=1e-2)
    s = pkg.IBSolver.from_problem(p)
    n2 = 2 * p.N * p.N
    un = torch.zeros(n2, dtype=torch.float64, device="cuda")
    un[17] = float("nan")
    up = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.capi.IBError) as e:
        s.solve_step(un, up, dev(p.X))
    assert e.value.code == pkg.capi.IB_ERR_BREAKDOWN
    # the same problem solves a finite step afterwards
    st = s.solve_step(torch.zeros_like(un), up, dev(p.X))
    assert st["status"] == 0
    s.close()
    _healthy_solve(pkg)


def test_coincident_points_through_update_points(pkg):
    p = W.single_ellipse(N=32, n_points=64, kappa=1e2, dt=1e-2)
    s = pkg.IBSolver.from_problem(p)
    X = p.X.copy()
    X[5] = X[4]  # points 4 and 5 share a spring
    with pytest.raises(pkg.capi.IBError) as e:
        s.update_points(dev(X))
    assert e.value.code == pkg.capi.IB_ERR_INVALID_ARG
    assert "coincident" in str(e.value)
    s.update_points(dev(p.X))  # valid points are accepted again
    up = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    st = s.solve_step(None, up, dev(p.X))
    assert st["status"] == 0 and st["rel_res_true"] <= p.tol
    s.close()
    _healthy_solve(pkg)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_iteration_cap_reports_not_converged(pkg, prec):
    p = W.single_ellipse(N=32, n_points=80, kappa=1e6, dt=1e-2)
    p.box = 4
    s = pkg.IBSolver.from_problem(p, precision=prec, max_iters=1)
    up = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    X = dev(p.X)
    X0 = X.clone()
    st = s.solve_step(None, up, X)
    assert st["status"] == pkg.capi.IB_ERR_NOT_CONVERGED and st["iters"] == 1
    assert st["rel_res_true"] > p.tol and np.isfinite(st["rel_res_true"])
    assert float(up.abs().max()) > 0.0 and float((X - X0).abs().max()) > 0.0  # iterate written, points moved
    with pytest.raises(pkg.capi.IBError) as e:
        s.solve_step(None, up, X0.clone(), raise_on_not_converged=True)
    assert e.value.code == pkg.capi.IB_ERR_NOT_CONVERGED
    s.close()
    _healthy_solve(pkg)


def test_zero_wait_limit_reports_timeout(pkg, monkeypatch):
    monkeypatch.setenv("IB_WAIT_LIMIT_NS", "0")
    monkeypatch.setenv("IB_CGS_REG", "0")  # small bases on the bulk-copy form, whose waits are bounded
    p = W.single_ellipse(N=32, n_points=64, kappa=1e2, dt=1e-2)
    s = pkg.IBSolver.from_problem(p)
    monkeypatch.delenv("IB_WAIT_LIMIT_NS")
    monkeypatch.delenv("IB_CGS_REG")
    up = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.capi.IBError) as e:
        s.solve_step(None, up, dev(p.X))
    assert e.value.code == pkg.capi.IB_ERR_TIMEOUT
    s.close()
    torch.cuda.synchronize()
    _healthy_solve(pkg)
