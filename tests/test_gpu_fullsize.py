"""GPU checks at the full workload sizes.

Where the oracle cannot run the whole method in seconds, the operator is
compared element by element with the oracle's assembled one, and the solves are
checked through properties that hold at any size: the FP64 true residual
against the oracle's operator and right-hand side, the discrete divergence, and
the point update X^{n+1} = X^n + dt S*(X^n) u^{n+1} (Eq. 20) with the oracle's S*.
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


def rel_elementwise(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def fine_operator(p):
    E, S, Ss, _ = O.fine_elasticity(p)
    return O.with_elasticity(O.stokes_matrix(p.N, p.h, p.mu, p.rho, p.dt), E, p.dt, p.N), Ss


def check_solution(p, A, Ss, x, X_new):
    b = O.rhs_vector(p)
    bn = np.linalg.norm(b)
    Ax = A @ x
    assert np.linalg.norm(b - Ax) <= 1.01 * p.tol * bn
    n = p.N * p.N
    assert np.linalg.norm(Ax[2 * n:]) <= 1.01 * p.tol * bn  # discretely divergence-free
    U = Ss @ x[:2 * n]
    Xref = p.X + p.dt * np.stack([U[:p.n_points], U[p.n_points:]], axis=1)
    assert np.abs(X_new - Xref).max() <= 1e-9 * p.h


def test_sweep_stiff_case_full_size(pkg):
    """256^2 sweep, kappa = 1e6, dt = 1e-2 (the case that dominates the sweep): the
    FP32 preconditioner stalls, escalates to the mixed V-cycle, and the step still
    meets the FP64 tolerance."""
    p = W.single_ellipse(N=256, n_points=512, kappa=1e6, dt=1e-2)
    p.box = 4
    A, Ss = fine_operator(p)
    s = pkg.IBSolver.from_problem(p, precision="fp32", max_iters=200)
    up = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    X = dev(p.X)
    st = s.solve_step(None, up, X)
    s.close()
    assert st["status"] == 0 and st["escalated_at"] >= 0, st
    check_solution(p, A, Ss, up.cpu().numpy(), X.cpu().numpy())


def test_sweep_stiff_case_fp32_elimination_then_escalation(pkg, monkeypatch):
    """The same case held on the FP32 V-cycle (stiffness threshold raised): its
    structure boxes are eliminated in FP32; the FP32 iteration stalls and escalates
    mid-solve to the mixed V-cycle, which first re-forms and inverts the boxes in
    FP64; the step meets the FP64 tolerance on the oracle's operator."""
    monkeypatch.setenv("IB_STIFF_SIGMA", "1e12")
    p = W.single_ellipse(N=256, n_points=512, kappa=1e6, dt=1e-2)
    p.box = 4
    A, Ss = fine_operator(p)
    s = pkg.IBSolver.from_problem(p, precision="fp32", max_iters=200)
    up = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    X = dev(p.X)
    st = s.solve_step(None, up, X)
    s.close()
    assert st["status"] == 0 and st["escalated_at"] > 0, st
    check_solution(p, A, Ss, up.cpu().numpy(), X.cpu().numpy())


def test_multi_ellipse_1024_apply_and_step(pkg):
    """1024^2 grid, 16 ellipses x 2048 points (seed 1311): the fine operator element
    by element, then one FP32-preconditioned step to the FP64 tolerance."""
    p = W.many_ellipses()
    p.box = 4
    A, Ss = fine_operator(p)
    s = pkg.IBSolver.from_problem(p, precision="fp32", max_iters=200, restart=50)
    w = np.random.default_rng(11).standard_normal(3 * p.N * p.N)
    y = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    s.apply(0, dev(w), y)
    assert rel_elementwise(y.cpu().numpy(), A @ w) < 1e-10
    up = torch.zeros_like(y)
    X = dev(p.X)
    st = s.solve_step(None, up, X)
    s.close()
    assert st["status"] == 0, st
    check_solution(p, A, Ss, up.cpu().numpy(), X.cpu().numpy())


def test_full_batch_256(pkg):
    """All 256 problems of the batched workload (seed 5614; FGMRES restarted every 30
    iterations, unrestarted for stiffness ratios dt kappa / mu >= 3000): every problem
    meets the FP64 tolerance 1e-8, and a seeded sample matches the oracle."""
    import bench

    probs = W.batch(count=256, seed=5614)
    for p in probs:
        p.box = 4
    B = pkg.IBBatch(probs, precision="fp32", max_iters=200, restart=bench.batch_restarts(probs))
    sizes = [3 * p.N * p.N for p in probs]
    up = torch.zeros(sum(sizes), dtype=torch.float64, device="cuda")
    X = dev(np.concatenate([p.X for p in probs]))
    stats = B.solve_step(None, up, X)
    B.close()
    upc, Xc = up.cpu().numpy(), X.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(sizes)])
    xoff = np.concatenate([[0], np.cumsum([p.n_points for p in probs])])
    for st in stats:
        assert st["status"] == 0 and st["rel_res_true"] <= 1e-8, st
    rng = np.random.default_rng(3)
    stiff = [k for k, p in enumerate(probs) if p.dt * p.kappa.max() / p.mu >= 3000 and p.N <= 256]
    sample = [int(k) for k in rng.permutation(256)[:4]] + stiff[:1]
    for k in sample:
        p = probs[k]
        A, Ss = fine_operator(p)
        check_solution(p, A, Ss, upc[off[k]:off[k + 1]], Xc[xoff[k]:xoff[k + 1]])
