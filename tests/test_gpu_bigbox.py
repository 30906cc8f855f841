"""16 x 16 boxes on the GPU (the big boxes of sec. 6: 2 * 16 * 17 velocity faces and
256 cells, 800 unknowns per box) against the oracle, and the blocked Gauss-Jordan
inversion that their box matrices (and the 769-unknown coarsest level of N_c = 16)
need: they are too large for shared memory.

* FP64 V-cycle element by element at 1e-10 on the periodic ellipse (two smoothing
  levels at 64^2, one at 32^2 with the stiff kappa = 1e6) and on the paper's
  cavity with the thick annulus;
* FP32 and mixed V-cycles within the element-wise bars of the other box sizes;
* implicit steps: the FP64 tolerance on the oracle's CSR operator, iteration
  counts within one of the oracle's, fewer than with 8 x 8 boxes on the stiff case.
The 8 x 8 boxes (208 unknowns) take the same blocked inversion; their FP64
V-cycle parity tests are in the periodic and cavity test files.
"""
import types

import numpy as np
import pytest

import ib_workloads as W
from oracle import cavity_oracle as C
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


def rel_per_component(got, ref, N):
    n = N * N
    return [float(np.abs(got[c * n:(c + 1) * n] - ref[c * n:(c + 1) * n]).max()
                  / max(np.abs(ref[c * n:(c + 1) * n]).max(), 1e-300)) for c in range(3)]


CASES = {
    "ellipse_64": dict(N=64, n_points=128, kappa=1e2, dt=1e-2),
    "stiff_32": dict(N=32, n_points=80, kappa=1e6, dt=1e-2),
    "stiff_64": dict(N=64, n_points=160, kappa=1e6, dt=1e-2),
}


def make_case(name, box=16):
    p = W.single_ellipse(**CASES[name])
    p.box = box
    return p


def _oracle_vcycle(p, rhs):
    levels, _ = O.build_hierarchy(p)
    for lev in levels[:-1]:
        O.prepare_boxes(lev, p.box)
    return O.vcycle(levels, rhs, np.zeros_like(rhs), p.nu1, p.nu2, p.rho, "color4")


def _rhs(p, seed=11):
    rng = np.random.default_rng(seed)
    rhs = O.rhs_vector(p) + 0.1 * np.abs(O.rhs_vector(p)).max() * rng.standard_normal(3 * p.N * p.N)
    n = p.N * p.N
    rhs[2 * n:] -= rhs[2 * n:].mean()
    return rhs


@pytest.mark.parametrize("name", ["ellipse_64", "stiff_32"])
def test_vcycle_fp64_box16(pkg, name):
    p = make_case(name)
    rhs = _rhs(p)
    ref = _oracle_vcycle(p, rhs)
    s = pkg.IBSolver.from_problem(p)
    try:
        assert s.n_levels == len(O.level_sizes(p.N, 16))
        w = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
        s.vcycle(dev(rhs), w)
        err = rel_per_component(w.cpu().numpy(), ref, p.N)
        assert max(err) < 1e-10, err
    finally:
        s.close()


@pytest.mark.parametrize("prec,bar,box", [("fp32", 2e-5, 16), ("mixed", 5e-7, 16), ("fp32", 2e-5, 8)])
def test_vcycle_reduced_precision_box16(pkg, prec, bar, box):
    """FP32 (on this non-stiff case its big structure boxes are eliminated in FP32 by
    the blocked form) and mixed V-cycles within the element-wise bars."""
    p = make_case("ellipse_64", box)
    rhs = O.rhs_vector(p)
    ref = _oracle_vcycle(p, rhs)
    s = pkg.IBSolver.from_problem(p, precision=prec)
    try:
        w = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
        s.vcycle(dev(rhs), w)
        got = w.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 2e-4 * np.linalg.norm(ref)
        assert max(rel_per_component(got, ref, p.N)) <= bar, rel_per_component(got, ref, p.N)
    finally:
        s.close()


@pytest.mark.parametrize("name,prec", [("ellipse_64", "fp64"), ("stiff_64", "fp64"), ("stiff_64", "mixed")])
def test_solve_step_box16(pkg, name, prec):
    p = make_case(name)
    ref = O.solve_step(p)
    s = pkg.IBSolver.from_problem(p, precision=prec)
    try:
        up = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
        X = dev(p.X)
        st = s.solve_step(None, up, X)
        assert st["status"] == 0 and st["rel_res_true"] <= p.tol, st
        A = O.build_hierarchy(p)[0][0].A
        w = up.cpu().numpy()
        assert np.linalg.norm(ref.b - A @ w) <= p.tol * np.linalg.norm(ref.b) * 1.01
        if prec == "fp64":
            assert abs(st["iters"] - ref.solve.iters) <= 1, (st["iters"], ref.solve.iters)
        else:
            assert st["iters"] <= ref.solve.iters + 2
        assert np.abs(X.cpu().numpy() - ref.X).max() <= 1e-6 * p.h
    finally:
        s.close()


def test_big_boxes_take_fewer_iterations_on_the_stiff_case(pkg):
    """Sec. 6: bigger boxes lower the iteration count of stiff problems."""
    its = {}
    for box in (4, 8, 16):
        p = make_case("stiff_64", box)
        s = pkg.IBSolver.from_problem(p)
        try:
            up = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
            st = s.solve_step(None, up, dev(p.X))
            assert st["status"] == 0
            its[box] = st["iters"]
        finally:
            s.close()
    assert its[16] < its[8] < its[4], its


def _cavity(N, rel, b):
    a_exp = C.explicit_limit(N, "ds1^2")[0]
    p = W.cavity_annulus(N, kappa=rel * a_exp, dt=1.0)
    m = p.meta
    geom = types.SimpleNamespace(N=p.N, M1=m["M1"], M2=m["M2"], ds1=m["ds1"], ds2=m["ds2"], points=lambda: p.X)
    levels = C.cavity_hierarchy(N, rel * a_exp, b, ann=geom, order="color4")
    return p, levels, geom


def _cavity_solver(pkg, p, b, tol=1e-8):
    return pkg.IBSolver(p.N, p.X, p.springs, p.kappa, p.rest, L=1.0, rho=0.0, mu=1.0, dt=p.dt, delta="cos4",
                        box=b, walls="noslip", precision="fp64", tol=tol, max_iters=200)


def test_cavity_vcycle_and_solve_box16(pkg):
    """The paper's cavity at h = 2^-6 with 16 x 16 boxes, relative stiffness 100:
    one FP64 V-cycle at 1e-10 per component, MG-GMRES counts within one."""
    N, b = 64, 16
    p, levels, geom = _cavity(N, 100.0, b)
    rhs = C.cavity_rhs(N, levels, ann=geom)
    s = _cavity_solver(pkg, p, b)
    try:
        w = torch.zeros(3 * N * N, dtype=torch.float64, device="cuda")
        s.vcycle(dev(rhs), w)
        want = C.cavity_vcycle(levels, rhs, np.zeros_like(rhs))
        assert max(rel_per_component(w.cpu().numpy(), want, N)) < 1e-10
        ref = C.cavity_mg_gmres(levels, rhs, tol=1e-8, max_iters=200)
        x = torch.zeros(3 * N * N, dtype=torch.float64, device="cuda")
        st = s.solve(dev(rhs), x)
        assert st["status"] == 0
        assert abs(st["iters"] - ref.iters) <= 1, (st["iters"], ref.iters)
        xs = x.cpu().numpy()
        assert np.linalg.norm(rhs - levels[0].A @ xs) / np.linalg.norm(rhs) <= 1.05e-8
    finally:
        s.close()
