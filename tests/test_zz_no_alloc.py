"""The allocation-free operator apply against the regular one.

ib_apply_noalloc serves callers that cannot allocate device memory (no
cudaMalloc stall inside a time step, or all device memory owned by the caller's
own pool).  It keeps its scratch in a static device array shared by every call,
so this test makes two calls in a row with different structures (the second
with fewer points, over the first call's leftover contents) and checks each
against ib_apply on a problem built from the same inputs, element by element
within the 1e-10 bar of the other operator-apply parity tests.  The file is
named to be collected last.
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


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _check_case(pkg, prob, jacobian, seed):
    from paper_1311_5614_gb300 import capi as C

    solver = pkg.IBSolver.from_problem(prob, jacobian=jacobian)
    n = 3 * prob.N * prob.N
    w = _dev(np.random.default_rng(seed).standard_normal(n))
    y_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
    solver.apply(0, w, y_ref)
    y = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    C.ib_apply_noalloc(solver.params, _dev(prob.X), _dev(prob.springs, torch.int32), _dev(prob.kappa),
                       _dev(prob.rest), w, y)
    torch.cuda.synchronize()
    a, b = y.cpu().numpy(), y_ref.cpu().numpy()
    solver.close()
    assert np.all(np.isfinite(a))
    assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()


def test_noalloc_apply_matches_ib_apply_twice(pkg):
    first = W.single_ellipse(N=64, n_points=128, kappa=1e2, dt=1e-2)
    second = W.single_ellipse(N=32, n_points=80, kappa=1e6, dt=1e-2, center=(0.9, 0.1), a=0.2, b=0.12)
    _check_case(pkg, first, "clamped", 1)
    _check_case(pkg, second, "exact", 2)


def test_noalloc_rejects_too_many_points(pkg):
    from paper_1311_5614_gb300 import capi as C

    p = C.make_params(16)
    n = 3 * 16 * 16
    big = C.IB_NOALLOC_MAX_POINTS + 1
    X = torch.rand(big, 2, dtype=torch.float64, device="cuda")
    sp = torch.stack([torch.arange(big), (torch.arange(big) + 1) % big], 1).to(torch.int32).cuda()
    k = torch.ones(big, dtype=torch.float64, device="cuda")
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(C.IBError) as e:
        C.ib_apply_noalloc(p, X, sp, k, k, w, y)
    assert e.value.code == C.IB_ERR_INVALID_ARG and "IB_NOALLOC_MAX_POINTS" in str(e.value)
