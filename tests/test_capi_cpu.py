"""Host-side checks of the C ABI: the library loads, exports every entry point
declared in include/ib.h, and rejects invalid arguments before any GPU work."""
import ctypes
import os
import re

import numpy as np
import pytest

import ib_workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_1311_5614_gb300 import capi as C

    if not os.path.exists(C.LIB_PATH):
        from paper_1311_5614_gb300 import build as B

        B.build()
    C.lib()
    return C


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ib.h")).read()
    return sorted(set(re.findall(r"IB_API\s+[\w\s\*]+?\b(ib_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ib_setup", "ib_apply", "ib_vcycle", "ib_solve_step", "ib_destroy"):
        assert n in names
    assert len(names) >= 13


def test_library_exports_every_declared_symbol(capi):
    L = capi.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in capi._SIGS, "binding has no signature for " + name


def test_version_and_defaults(capi):
    assert "sm_103a" in capi.ib_version()
    p = capi.ib_default_params()
    assert (p.N, p.box, p.nu1, p.nu2, p.max_iters) == (64, 1, 1, 1, 100)
    assert p.tol == 1e-8 and p.rho == 1.0 and p.mu == 1.0 and p.dt == 1e-2
    assert ctypes.sizeof(capi.ib_params) == 104  # include/ib.h's ib_params, natural alignment
    assert p.escalate == 1 and p.restart == 0
    assert p.walls == 0 and p.lid == 0.0 and p.time_method == 0  # periodic, at rest, implicit


@pytest.mark.parametrize("field,value", [
    ("N", 48), ("N", 4), ("box", 3), ("box", 32), ("mu", 0.0), ("dt", -1.0), ("rho", -1.0), ("tol", 0.0),
    ("max_iters", 0), ("max_iters", 1000), ("nu1", 9), ("delta", 5), ("precision", 7), ("L", 0.0),
    ("restart", -1), ("escalate", 2)])
def test_setup_rejects_bad_params(capi, field, value):
    prob = W.single_ellipse(N=32, n_points=16)
    p = capi.make_params(32)
    setattr(p, field, value)
    with pytest.raises(capi.IBError) as e:
        capi.ib_setup(p, prob.X, prob.springs, prob.kappa, prob.rest, stream=0)
    assert e.value.code == capi.IB_ERR_INVALID_ARG


def test_setup_rejects_bad_structure(capi):
    prob = W.single_ellipse(N=32, n_points=16)
    p = capi.make_params(32)
    bad = prob.springs.copy()
    bad[3, 1] = 99
    with pytest.raises(capi.IBError):
        capi.ib_setup(p, prob.X, bad, prob.kappa, prob.rest, stream=0)
    bad = prob.springs.copy()
    bad[2, 1] = bad[2, 0]
    with pytest.raises(capi.IBError):
        capi.ib_setup(p, prob.X, bad, prob.kappa, prob.rest, stream=0)
    X = prob.X.copy()
    X[0, 0] = np.nan
    with pytest.raises(capi.IBError):
        capi.ib_setup(p, X, prob.springs, prob.kappa, prob.rest, stream=0)
    k = prob.kappa.copy()
    k[0] = -1.0
    with pytest.raises(capi.IBError):
        capi.ib_setup(p, prob.X, prob.springs, k, prob.rest, stream=0)
    # a point with more springs than the elasticity assembly supports
    sp = np.array([[0, j] for j in range(1, 10)], dtype=np.int32)
    with pytest.raises(capi.IBError) as e:
        capi.ib_setup(p, prob.X, sp, np.ones(9), np.zeros(9), stream=0)
    assert "7 springs" in str(e.value)


def test_null_handles_are_rejected(capi):
    L = capi.lib()
    assert L.ib_apply(None, 0, None, None) == capi.IB_ERR_INVALID_ARG
    assert L.ib_vcycle(None, None, None) == capi.IB_ERR_INVALID_ARG
    assert L.ib_solve_step(None, None, None, None, None) == capi.IB_ERR_INVALID_ARG
    assert L.ib_solve_step_newton(None, None, None, None, 5, 1e-9, None, None) == capi.IB_ERR_INVALID_ARG
    assert L.ib_num_levels(None) == 0
    L.ib_destroy(None)
