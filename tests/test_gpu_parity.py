"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bars (written here, derived in the design notes):
* FP64 operator apply, right-hand side, V-cycle: every element within 1e-10 of
  the oracle, relative to the largest oracle element (per-apply bar);
* FP32 V-cycle: every element within 2e-5 of the oracle, relative to the largest
  oracle element of its component (u, v or p), and 2e-4 in the 2-norm.  FP32
  rounding (unit roundoff 6e-8) through 2 x nu sweeps on every level, amplified by
  the structure rows, whose elastic terms (dt kappa / h^2 against mu / h^2) cancel
  in the FP32 residual; measured on GB300: at most 4.3e-6 (1 x 1 to 8 x 8 boxes,
  kappa up to 1e6), 2.8e-7 without the 8 x 8 stiff case;
* mixed V-cycle (FP64 vectors, FP32 free-box inverse): every element within 5e-7
  per component (the FP32 inverse's rounding enters once per box solve and is
  damped by the FP64 residual; measured at most 4.7e-8);
* solves: both sides reach the 1e-8 relative residual; the solutions agree to
  1e-6 relative (tolerance times the conditioning margin) and the iteration
  counts agree within one for FP64.
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


def rel_elementwise(gpu, ref):
    return float(np.abs(gpu - ref).max() / max(np.abs(ref).max(), 1e-300))


def rel_per_component(gpu, ref, N):
    """Largest elementwise error of each component (u, v, p) relative to that
    component's largest oracle element."""
    n = N * N
    return [rel_elementwise(gpu[c * n:(c + 1) * n], ref[c * n:(c + 1) * n]) for c in range(3)]


CASES = {
    "c1_64": dict(N=64, n_points=128, kappa=1e2, dt=1e-2),
    "stiff_32_exact": dict(N=32, n_points=80, kappa=1e6, dt=1e-2, jac="exact"),
    "stiff_32": dict(N=32, n_points=80, kappa=1e6, dt=1e-2),
    "steady_cos4_32": dict(N=32, n_points=64, kappa=1e3, dt=1e-1, rho=0.0, delta="cos4", rest=0.0),
    "offcentre_16": dict(N=16, n_points=24, kappa=50.0, dt=1e-2, center=(0.93, 0.07), a=0.2, b=0.15),
}


def make_case(name, box=1):
    c = dict(CASES[name])
    jac = c.pop("jac", "clamped")
    p = W.single_ellipse(**c)
    p.box = box
    p.clamped = jac == "clamped"
    return p


@pytest.mark.parametrize("name", list(CASES))
def test_apply_every_level_fp64(pkg, name):
    p = make_case(name)
    levels, _ = O.build_hierarchy(p)
    s = pkg.IBSolver.from_problem(p)
    assert s.n_levels == len(levels)
    rng = np.random.default_rng(7)
    for li, lev in enumerate(levels):
        n = 3 * lev.N * lev.N
        w = rng.standard_normal(n)
        y = torch.zeros(n, dtype=torch.float64, device="cuda")
        s.apply(li, dev(w), y)
        ref = lev.A @ w
        assert rel_elementwise(y.cpu().numpy(), ref) < 1e-10, (name, li)
    s.close()


@pytest.mark.parametrize("name", ["c1_64", "offcentre_16"])
def test_rhs_fp64(pkg, name):
    p = make_case(name)
    s = pkg.IBSolver.from_problem(p)
    n = 3 * p.N * p.N
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(3)
    un = rng.standard_normal(2 * p.N * p.N)
    s.rhs(dev(un), b)
    ref = O.rhs_vector(p, un)
    assert rel_elementwise(b.cpu().numpy(), ref) < 1e-10
    s.rhs(None, b)
    assert rel_elementwise(b.cpu().numpy(), O.rhs_vector(p)) < 1e-10
    s.close()


def _oracle_vcycle(p, rhs):
    levels, _ = O.build_hierarchy(p)
    for lev in levels[:-1]:
        O.prepare_boxes(lev, p.box)
    return O.vcycle(levels, rhs, np.zeros_like(rhs), p.nu1, p.nu2, p.rho, "color4")


@pytest.mark.parametrize("name,box", [("c1_64", 1), ("stiff_32_exact", 1), ("steady_cos4_32", 1),
                                      ("offcentre_16", 1), ("c1_64", 2), ("stiff_32_exact", 4),
                                      ("c1_64", 8)])
def test_vcycle_fp64(pkg, name, box):
    p = make_case(name, box)
    if p.N < 2 * max(4, box):
        pytest.skip("grid too small for the box")
    rng = np.random.default_rng(11)
    rhs = O.rhs_vector(p) + 0.1 * np.abs(O.rhs_vector(p)).max() * rng.standard_normal(3 * p.N * p.N)
    n = p.N * p.N
    rhs[2 * n:] -= rhs[2 * n:].mean()
    ref = _oracle_vcycle(p, rhs)
    s = pkg.IBSolver.from_problem(p)
    w = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    s.vcycle(dev(rhs), w)
    got = w.cpu().numpy()
    assert rel_elementwise(got, ref) < 1e-10, (name, box, rel_elementwise(got, ref))
    s.close()


@pytest.mark.parametrize("name,box", [("c1_64", 2), ("c1_64", 4), ("stiff_32_exact", 4)])
def test_vcycle_fp64_gemm_box_kernel(pkg, name, box, monkeypatch):
    """The register-blocked box kernel (used on large levels) forced on every level."""
    monkeypatch.setenv("IB_BOX_GEMM_MIN", "0")
    test_vcycle_fp64(pkg, name, box)


@pytest.mark.parametrize("name,box", [("c1_64", 2), ("c1_64", 4), ("stiff_32_exact", 4)])
def test_vcycle_fp64_multi_box_cta(pkg, name, box, monkeypatch):
    """The several-boxes-per-CTA kernel (used on mid-size levels) forced on every level."""
    monkeypatch.setenv("IB_BOX_ONE_MAX", "0")
    test_vcycle_fp64(pkg, name, box)


@pytest.mark.parametrize("name,box,nmax", [("c1_64", 1, 64), ("c1_64", 2, 32), ("c1_64", 4, 64),
                                           ("stiff_32_exact", 4, 32), ("c1_64", 8, 64), ("stiff_32", 2, 16)])
def test_vcycle_fp64_cluster_tail(pkg, name, box, nmax, monkeypatch):
    """The coarse levels from N = nmax down run on one thread-block cluster (arrays
    in global memory, phases separated by the cluster barrier); nmax = N puts the
    whole V-cycle there."""
    monkeypatch.setenv("IB_TAIL_NMAX", str(nmax))
    monkeypatch.setenv("IB_TAIL_CLUSTER", "1")
    p = make_case(name, box)
    rng = np.random.default_rng(11)
    rhs = O.rhs_vector(p) + 0.1 * np.abs(O.rhs_vector(p)).max() * rng.standard_normal(3 * p.N * p.N)
    n = p.N * p.N
    rhs[2 * n:] -= rhs[2 * n:].mean()
    ref = _oracle_vcycle(p, rhs)
    s = pkg.IBSolver.from_problem(p)
    w = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    s.vcycle(dev(rhs), w)
    assert s.tail_cluster("fp64") >= 8 and s.tail_grid("fp64") == nmax
    got = w.cpu().numpy()
    assert rel_elementwise(got, ref) < 1e-10, (name, box, rel_elementwise(got, ref))
    s.vcycle(dev(rhs), w)  # graph replay gives the same result
    assert rel_elementwise(w.cpu().numpy(), ref) < 1e-10
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_vcycle_cluster_tail_low_precision(pkg, prec, monkeypatch):
    monkeypatch.setenv("IB_TAIL_NMAX", "32")
    monkeypatch.setenv("IB_TAIL_CLUSTER", "1")
    p = make_case("stiff_32_exact", 4)
    rhs = O.rhs_vector(p)
    ref = _oracle_vcycle(p, rhs)
    s = pkg.IBSolver.from_problem(p, precision=prec)
    w = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    s.vcycle(dev(rhs), w)
    assert s.tail_cluster(prec) >= 8
    got = w.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 2e-4 * np.linalg.norm(ref)
    assert max(rel_per_component(got, ref, p.N)) <= (2e-5 if prec == "fp32" else 5e-7)
    s.close()


@pytest.mark.parametrize("name,box", [("c1_64", 1), ("c1_64", 4), ("stiff_32_exact", 4), ("stiff_32", 8),
                                      ("steady_cos4_32", 2), ("offcentre_16", 2)])
def test_vcycle_fp32(pkg, name, box):
    p = make_case(name, box)
    rhs = O.rhs_vector(p)
    ref = _oracle_vcycle(p, rhs)
    s = pkg.IBSolver.from_problem(p, precision="fp32")
    w = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    s.vcycle(dev(rhs), w)
    got = w.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 2e-4 * np.linalg.norm(ref)
    assert max(rel_per_component(got, ref, p.N)) <= 2e-5, rel_per_component(got, ref, p.N)
    s.close()


@pytest.mark.parametrize("name,box", [("c1_64", 1), ("c1_64", 4), ("stiff_32_exact", 4), ("stiff_32", 8),
                                      ("steady_cos4_32", 2), ("offcentre_16", 2)])
def test_vcycle_mixed(pkg, name, box):
    """FP64 vectors and residuals, FP32 box inverses: within FP32 rounding of the
    oracle's FP64 V-cycle."""
    p = make_case(name, box)
    rhs = O.rhs_vector(p)
    ref = _oracle_vcycle(p, rhs)
    s = pkg.IBSolver.from_problem(p, precision="mixed")
    w = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    s.vcycle(dev(rhs), w)
    got = w.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 2e-4 * np.linalg.norm(ref)
    assert max(rel_per_component(got, ref, p.N)) <= 5e-7, rel_per_component(got, ref, p.N)
    s.close()


@pytest.mark.parametrize("name,box,prec", [("c1_64", 1, "fp64"), ("c1_64", 1, "fp32"),
                                           ("stiff_32", 4, "fp64"), ("stiff_32", 8, "fp32"),
                                           ("stiff_32", 4, "mixed"), ("c1_64", 2, "mixed"),
                                           ("steady_cos4_32", 1, "fp64"),
                                           ("offcentre_16", 2, "fp32")])
def test_solve_step(pkg, name, box, prec):
    p = make_case(name, box)
    ref = O.solve_step(p)
    s = pkg.IBSolver.from_problem(p, precision=prec)
    n = 3 * p.N * p.N
    up = torch.zeros(n, dtype=torch.float64, device="cuda")
    X = dev(p.X)
    st = s.solve_step(None, up, X)
    w = up.cpu().numpy()
    assert st["status"] == 0 and st["rel_res_true"] <= p.tol, st
    A = O.build_hierarchy(p)[0][0].A
    assert np.linalg.norm(ref.b - A @ w) <= p.tol * np.linalg.norm(ref.b) * 1.01
    if p.rho == 0.0:
        nn = p.N * p.N
        for c in range(2):
            w[c * nn:(c + 1) * nn] -= w[c * nn:(c + 1) * nn].mean() - ref.w[c * nn:(c + 1) * nn].mean()
    assert np.linalg.norm(w - ref.w) <= 1e-6 * np.linalg.norm(ref.w), np.linalg.norm(w - ref.w) / np.linalg.norm(ref.w)
    if prec == "fp64":
        assert abs(st["iters"] - ref.solve.iters) <= 1, (st["iters"], ref.solve.iters)
    else:
        assert st["iters"] <= ref.solve.iters + 2
    Xn = X.cpu().numpy()
    assert np.abs(Xn - ref.X).max() <= 1e-6 * p.h
    s.close()


@pytest.mark.parametrize("name,box,prec", [("c1_64", 1, "fp64"), ("stiff_32", 4, "mixed")])
def test_solve_step_cluster_tail(pkg, name, box, prec, monkeypatch):
    """One implicit step with the coarse levels on a thread-block cluster."""
    monkeypatch.setenv("IB_TAIL_NMAX", "32")
    monkeypatch.setenv("IB_TAIL_CLUSTER", "1")
    test_solve_step(pkg, name, box, prec)


@pytest.mark.parametrize("name,box,prec", [("c1_64", 1, "fp64"), ("stiff_32", 4, "mixed")])
def test_solve_step_two_pass_gram_schmidt(pkg, name, box, prec, monkeypatch):
    """The middle Gram-Schmidt step as two passes (subtract, then project), the
    form taken when the basis slice does not fit in shared memory."""
    monkeypatch.setenv("IB_CGS_FUSED", "0")
    test_solve_step(pkg, name, box, prec)


@pytest.mark.parametrize("name,box,prec", [("c1_64", 1, "fp64"), ("stiff_32", 4, "mixed")])
def test_solve_step_bulk_copy_gram_schmidt(pkg, name, box, prec, monkeypatch):
    """Bases of up to 16 vectors on the bulk-copy form of the fused Gram-Schmidt
    step (by default they take the register form)."""
    monkeypatch.setenv("IB_CGS_REG", "0")
    test_solve_step(pkg, name, box, prec)


def test_no_structure_and_zero_rhs(pkg):
    """Edge cases: no Lagrangian points (pure Stokes, b = 0 -> zero solution)."""
    p = W.single_ellipse(N=16, n_points=8)
    s = pkg.IBSolver(16, np.zeros((0, 2)), np.zeros((0, 2), dtype=np.int32), np.zeros(0), np.zeros(0))
    up = torch.ones(3 * 256, dtype=torch.float64, device="cuda")
    st = s.solve_step(None, up, None)
    assert st["iters"] == 0 and float(up.abs().max()) == 0.0
    # the operator is still the Stokes operator
    levels, _ = O.build_hierarchy(W.single_ellipse(N=16, n_points=8, kappa=0.0))
    w = np.random.default_rng(0).standard_normal(768)
    y = torch.zeros(768, dtype=torch.float64, device="cuda")
    s.apply(0, dev(w), y)
    assert rel_elementwise(y.cpu().numpy(), levels[0].A @ w) < 1e-12
    s.close()


def test_struct_box_count_matches_oracle(pkg):
    """Boxes whose rows meet the elasticity operator are exactly the structure boxes."""
    p = make_case("c1_64")
    levels, _ = O.build_hierarchy(p)
    s = pkg.IBSolver.from_problem(p)
    for li, lev in enumerate(levels[:-1]):
        rows = set(np.nonzero(np.asarray(abs(lev.E).sum(axis=1)).ravel())[0].tolist())
        bx = O.prepare_boxes(lev, 1)
        touched = sum(1 for k in range(bx["lex"].shape[0]) if set(bx["lex"][k].tolist()) & rows)
        assert s.struct_boxes(li) >= touched
        assert s.struct_boxes(li) <= touched + 4 * lev.N  # conservative marking only at zero weights
    s.close()


def test_full_size_256_apply_and_fp32_solve(pkg):
    """The 256^2 workload (512-point ellipse): apply parity at full size and an FP32
    V-cycle solve that reaches the FP64 tolerance; the solution is compared with the
    oracle's at sampled entries via the true residual and divergence."""
    p = W.single_ellipse(N=256, n_points=512, kappa=1e4, dt=1e-2)
    levels, _ = O.build_hierarchy(p)
    s = pkg.IBSolver.from_problem(p, precision="fp32")
    rng = np.random.default_rng(2)
    w = rng.standard_normal(3 * 256 * 256)
    y = torch.zeros_like(dev(w))
    s.apply(0, dev(w), y)
    assert rel_elementwise(y.cpu().numpy(), levels[0].A @ w) < 1e-10
    up = torch.zeros(3 * 256 * 256, dtype=torch.float64, device="cuda")
    X = dev(p.X)
    st = s.solve_step(None, up, X)
    b = O.rhs_vector(p)
    x = up.cpu().numpy()
    assert np.linalg.norm(b - levels[0].A @ x) <= 1.01e-8 * np.linalg.norm(b)
    n = 256 * 256
    assert np.linalg.norm((levels[0].A @ x)[2 * n:]) <= 1.01e-8 * np.linalg.norm(b)
    assert st["iters"] <= 30
    s.close()


# ---------------------------------------------------------------- strip kernel for 4 x 4 boxes
# Levels whose N_l / 8 is a multiple of the strip width run the colour phases of
# 4 x 4 boxes with the strip kernel (a strip of W boxes of one colour per CTA
# iteration, staged tile, register-blocked free-box product).  IB_BOX_STRIP_MIN=1
# lets it run on every level it fits and IB_BOX_STRIP_W pins the width, so each
# width is compared with the oracle, with one strip per box row (N_l = 8 W) and with
# several (the staged rows then wrap only at the row ends); IB_BOX_STRIP=0 turns it off.

def _strip_case(N):
    if N == 64:
        return make_case("c1_64", 4)
    p = W.single_ellipse(N=N, n_points=2 * N, kappa=1e4, dt=1e-3)
    p.box = 4
    return p


@pytest.mark.parametrize("N,width,prec", [(64, 8, "fp64"), (64, 8, "fp32"), (64, 8, "mixed"),
                                          (128, 16, "fp64"), (128, 16, "mixed"),
                                          (256, 32, "fp64"), (256, 32, "fp32"), (256, 8, "fp32"),
                                          (256, 16, "mixed"), (512, 32, "fp64"), (512, 32, "fp32")])
def test_vcycle_strip_kernel(pkg, N, width, prec, monkeypatch):
    monkeypatch.setenv("IB_BOX_STRIP_MIN", "1")
    monkeypatch.setenv("IB_BOX_STRIP_W", str(width))
    p = _strip_case(N)
    rhs = O.rhs_vector(p)
    ref = _oracle_vcycle(p, rhs)
    s = pkg.IBSolver.from_problem(p, precision=prec)
    assert s.struct_boxes(0) > 0
    w = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    s.vcycle(dev(rhs), w)
    got = w.cpu().numpy()
    if prec == "fp64":
        assert rel_elementwise(got, ref) < 1e-10, rel_elementwise(got, ref)
    else:
        bar = 2e-5 if prec == "fp32" else 5e-7
        assert max(rel_per_component(got, ref, p.N)) <= bar, rel_per_component(got, ref, p.N)
    s.vcycle(dev(rhs), w)  # graph replay: same result
    got2 = w.cpu().numpy()
    assert np.abs(got2 - got).max() <= (1e-12 if prec == "fp64" else 1e-6) * np.abs(got).max()
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_solve_step_strip_kernel(pkg, prec, monkeypatch):
    monkeypatch.setenv("IB_BOX_STRIP_MIN", "1")
    test_solve_step(pkg, "c1_64", 4, prec)


# ---------------------------------------------------------------- assembled elasticity rows
# By default every level's elasticity block is kept as assembled rows (level 0 from
# the points, coarse levels by Galerkin products of them), which the operator apply
# and the V-cycle gather from.  IB_WINDOWS=0 keeps the point-based path (patches,
# atomics); a spring too long for a row's window makes a step fall back to it.

@pytest.mark.parametrize("name", ["c1_64", "stiff_32_exact", "offcentre_16"])
def test_point_path_apply_and_vcycle(pkg, name, monkeypatch):
    monkeypatch.setenv("IB_WINDOWS", "0")
    test_apply_every_level_fp64(pkg, name)
    test_vcycle_fp64(pkg, name, 4 if name != "offcentre_16" else 2)


def test_long_spring_falls_back_to_point_path(pkg):
    """A spring spanning about 2.5 cells: its coupling leaves the level-0 windows,
    so the step uses the point path; operator and V-cycle still match the oracle."""
    p = W.single_ellipse(N=32, n_points=24, kappa=1e3, dt=1e-2)
    p.box = 2
    assert np.abs(np.diff(p.X, axis=0)).max() > 1.6 * p.h
    levels, _ = O.build_hierarchy(p)
    s = pkg.IBSolver.from_problem(p)
    rng = np.random.default_rng(4)
    for li, lev in enumerate(levels):
        w = rng.standard_normal(3 * lev.N * lev.N)
        y = torch.zeros(3 * lev.N * lev.N, dtype=torch.float64, device="cuda")
        s.apply(li, dev(w), y)
        assert rel_elementwise(y.cpu().numpy(), lev.A @ w) < 1e-10, li
    rhs = O.rhs_vector(p)
    ref = _oracle_vcycle(p, rhs)
    z = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
    s.vcycle(dev(rhs), z)
    assert rel_elementwise(z.cpu().numpy(), ref) < 1e-10
    s.close()


@pytest.mark.parametrize("N", [64, 256])
def test_vcycle_fp32_eight_box_form(pkg, N, monkeypatch):
    """The eight-boxes-per-CTA FP32 form (IB_BOX_FORMS code 7) on every smoothing
    level: within the FP32 bars of the oracle, and bit for bit the V-cycle of the
    thread-per-row form (code 2), whose sums it forms in the same order."""
    p = _strip_case(N)
    rhs = O.rhs_vector(p)
    ref = _oracle_vcycle(p, rhs)
    out = {}
    for form in ("7", "2"):
        monkeypatch.setenv("IB_BOX_FORMS", ",".join([form] * 16))
        s = pkg.IBSolver.from_problem(p, precision="fp32")
        try:
            assert s.struct_boxes(0) > 0
            assert s.box_forms("fp32")[0] == int(form)
            w = torch.zeros(3 * p.N * p.N, dtype=torch.float64, device="cuda")
            s.vcycle(dev(rhs), w)
            out[form] = w.cpu().numpy()
        finally:
            s.close()
    assert max(rel_per_component(out["7"], ref, p.N)) <= 2e-5, rel_per_component(out["7"], ref, p.N)
    assert np.array_equal(out["7"], out["2"])
