"""Batched independent problems: ib_solve_step_batch against one ib_solve_step per
problem (same kernels, own streams) and against the oracle."""
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


def _problems():
    a = W.single_ellipse(N=32, n_points=64, kappa=1e3, dt=1e-2)
    b = W.single_ellipse(N=64, n_points=128, kappa=1e2, dt=1e-3, center=(0.4, 0.6), a=0.2, b=0.15)
    c = W.single_ellipse(N=16, n_points=24, kappa=1e4, dt=1e-2, a=0.3, b=0.2)
    c.box = 2
    return [a, b, c]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_single_solves_and_oracle(pkg, prec):
    probs = _problems()
    B = pkg.IBBatch(probs, precision=prec)
    sizes = [3 * p.N * p.N for p in probs]
    up = torch.zeros(sum(sizes), dtype=torch.float64, device="cuda")
    X = torch.tensor(np.concatenate([p.X for p in probs]), dtype=torch.float64, device="cuda")
    stats = B.solve_step(None, up, X)
    torch.cuda.synchronize()
    upc = up.cpu().numpy()
    Xc = X.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(sizes)])
    xoff = np.concatenate([[0], np.cumsum([p.n_points for p in probs])])
    for k, p in enumerate(probs):
        s = pkg.IBSolver.from_problem(p, precision=prec)
        u1 = torch.zeros(sizes[k], dtype=torch.float64, device="cuda")
        X1 = torch.tensor(p.X, dtype=torch.float64, device="cuda")
        st1 = s.solve_step(None, u1, X1)
        s.close()
        wb = upc[off[k]:off[k + 1]]
        assert stats[k]["status"] == 0 and stats[k]["iters"] == st1["iters"]
        assert np.abs(wb - u1.cpu().numpy()).max() <= 1e-12 * np.abs(wb).max()
        ref = O.solve_step(p)
        assert np.linalg.norm(wb - ref.w) <= 1e-6 * np.linalg.norm(ref.w)
        assert np.abs(Xc[xoff[k]:xoff[k + 1]] - ref.X).max() <= 1e-6 * p.h
    B.close()


def test_batch_rejects_bad_offsets(pkg):
    from paper_1311_5614_gb300 import capi as C
    import ctypes

    p = C.make_params(16)
    P = (C.ib_params * 1)(p)
    pt = np.array([0, -1], dtype=np.int32)
    sp = np.array([0, 0], dtype=np.int32)
    out = ctypes.c_void_p()
    code = C.lib().ib_setup_batch(1, P, pt.ctypes.data_as(ctypes.c_void_p), None,
                                  sp.ctypes.data_as(ctypes.c_void_p), None, None, None, None, ctypes.byref(out))
    assert code == C.IB_ERR_INVALID_ARG
