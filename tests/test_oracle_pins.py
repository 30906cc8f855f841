"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
values, exact discrete identities, convergence orders, symmetries, brute-force
dense solves.  A plausible slip (dropped term, wrong sign, wrong staggering
offset, transposed operand) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import ib_workloads as W
from oracle import ib_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- delta kernels (sec. 2.2)

def _golden_delta():
    rows = []
    with open(os.path.join(GOLDEN, "delta_kernels.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, r, v = line.split()[:3]
            rows.append((k, float(r), float(v)))
    return rows


def test_delta_golden_values():
    rows = _golden_delta()
    assert len(rows) == 13
    for k, r, v in rows:
        phi = O.KERNELS[k]
        assert abs(float(phi(np.array([r]))[0]) - v) < 1e-15, (k, r)
        assert abs(float(phi(np.array([-r]))[0]) - v) < 1e-15, (k, -r)


@pytest.mark.parametrize("kernel", ["peskin4", "cos4"])
def test_delta_moment_conditions(kernel):
    phi = O.KERNELS[kernel]
    j = np.arange(-4, 5)
    for r in np.linspace(0.0, 1.0, 41):
        w = phi(r - j)
        assert abs(w.sum() - 1.0) < 1e-14                      # partition of unity
        assert abs(w[j % 2 == 0].sum() - 0.5) < 1e-14          # even/odd split
        assert abs((w * w).sum() - 3.0 / 8.0) < 1e-14          # sum of squares
        assert np.count_nonzero(w) <= 4                        # 4-point support
        m1 = ((r - j) * w).sum()
        if kernel == "peskin4":
            assert abs(m1) < 1e-14                             # exact first moment
        else:
            assert abs(m1) < 0.022                             # cos4: bounded, not zero
    if kernel == "cos4":
        r = np.linspace(0, 1, 401)
        m1 = np.array([((x - j) * phi(x - j)).sum() for x in r])
        assert 0.02 < np.abs(m1).max() < 0.0215


# ---------------------------------------------------------------- spreading / interpolation

def _small_problem(N=32, n=40, kappa=10.0, rest=None, seed=0, **kw):
    p = W.single_ellipse(N=N, n_points=n, kappa=kappa, a=0.23, b=0.17,
                         center=(0.47, 0.53), rest=rest, **kw)
    return p


@pytest.mark.parametrize("kernel", ["peskin4", "cos4"])
def test_spread_conserves_force_and_interp_reproduces_constants(kernel):
    p = _small_problem()
    N, h = p.N, p.h
    S = O.spread_matrix(p.X, N, p.L, kernel)
    Ss = O.interp_matrix(S, h)
    F = W.random_points_field(p.n_points, 3)
    Fv = np.concatenate([F[:, 0], F[:, 1]])
    f = S @ Fv
    n2 = N * N
    # total force is conserved: h^2 sum_x f(x) = sum_k F_k (per component)
    assert abs(h * h * f[:n2].sum() - F[:, 0].sum()) < 1e-12
    assert abs(h * h * f[n2:].sum() - F[:, 1].sum()) < 1e-12
    # constants interpolate exactly
    u = np.concatenate([np.full(n2, 2.5), np.full(n2, -1.25)])
    U = Ss @ u
    assert np.allclose(U[: p.n_points], 2.5, atol=1e-13)
    assert np.allclose(U[p.n_points:], -1.25, atol=1e-13)


def test_interp_linear_exact_peskin4_pins_staggering():
    """Peskin4 has a zero first moment, so interpolating a linear field is exact,
    which fails if a face is placed at the wrong half-cell offset."""
    N, L = 32, 1.0
    h = L / N
    X = np.array([[0.431, 0.517], [0.55, 0.47], [0.5 + 0.25 * h, 0.5 - 0.375 * h]])
    S = O.spread_matrix(X, N, L, "peskin4")
    Ss = O.interp_matrix(S, h)
    i = np.arange(N)
    xu, yu = np.meshgrid(i * h, (i + 0.5) * h, indexing="xy")
    xv, yv = np.meshgrid((i + 0.5) * h, i * h, indexing="xy")
    u = 1.0 + 3.0 * xu - 2.0 * yu
    v = -0.5 + 0.7 * xv + 1.9 * yv
    U = Ss @ np.concatenate([u.ravel(), v.ravel()])
    n = X.shape[0]
    assert np.allclose(U[:n], 1.0 + 3.0 * X[:, 0] - 2.0 * X[:, 1], atol=1e-13)
    assert np.allclose(U[n:], -0.5 + 0.7 * X[:, 0] + 1.9 * X[:, 1], atol=1e-13)
    # and the spread force has its first moment at the point positions
    F = np.array([[1.0, 2.0], [-0.5, 0.3], [0.25, -1.0]])
    f = S @ np.concatenate([F[:, 0], F[:, 1]])
    n2 = N * N
    assert abs(h * h * (f[:n2] * xu.ravel()).sum() - (F[:, 0] * X[:, 0]).sum()) < 1e-13
    assert abs(h * h * (f[n2:] * yv.ravel()).sum() - (F[:, 1] * X[:, 1]).sum()) < 1e-13


def test_interp_of_smooth_field_second_order():
    """S* u approximates u(X) with O(h^2) error (pins offsets for both kernels)."""
    for kernel in ("peskin4", "cos4"):
        errs = []
        X = np.array([[0.3127, 0.6711], [0.7, 0.21]])
        for N in (32, 64, 128):
            h = 1.0 / N
            i = np.arange(N)
            xu, yu = np.meshgrid(i * h, (i + 0.5) * h, indexing="xy")
            xv, yv = np.meshgrid((i + 0.5) * h, i * h, indexing="xy")
            u = np.sin(2 * np.pi * xu) * np.cos(2 * np.pi * yu)
            v = np.cos(2 * np.pi * xv + 0.3) * np.sin(4 * np.pi * yv)
            S = O.spread_matrix(X, N, 1.0, kernel)
            U = O.interp_matrix(S, h) @ np.concatenate([u.ravel(), v.ravel()])
            ue = np.sin(2 * np.pi * X[:, 0]) * np.cos(2 * np.pi * X[:, 1])
            ve = np.cos(2 * np.pi * X[:, 0] + 0.3) * np.sin(4 * np.pi * X[:, 1])
            errs.append(max(np.abs(U[:2] - ue).max(), np.abs(U[2:] - ve).max()))
        assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, (kernel, errs)


def test_spread_interp_adjoint_and_sts_psd():
    p = _small_problem(N=16, n=24)
    h = p.h
    S = O.spread_matrix(p.X, p.N, p.L, "peskin4")
    Ss = O.interp_matrix(S, h)
    rng = np.random.default_rng(1)
    F = rng.standard_normal(2 * p.n_points)
    u = rng.standard_normal(2 * p.N * p.N)
    # <S F, u>_h = h^2 sum (S F) u  equals  <F, S* u>
    assert abs(h * h * (S @ F) @ u - F @ (Ss @ u)) < 1e-11 * np.abs(F).sum() * np.abs(u).max()
    M = (Ss @ S).toarray()
    assert np.allclose(M, M.T, atol=1e-12)
    assert np.linalg.eigvalsh(M).min() > -1e-12


# ---------------------------------------------------------------- springs

def test_spring_force_sums_to_zero_and_jacobian_matches_fd():
    p = _small_problem(n=20, kappa=7.0, rest=0.03)
    F = O.spring_force(p.X, p.springs, p.kappa, p.rest, p.L)
    assert np.abs(F.sum(axis=0)).max() < 1e-12
    Jx = O.spring_jacobian(p.X, p.springs, p.kappa, p.rest, p.L, clamped=False).toarray()
    n = p.n_points
    eps = 1e-6
    Jfd = np.zeros((2 * n, 2 * n))
    for c in range(2):
        for k in range(n):
            Xp = p.X.copy()
            Xm = p.X.copy()
            Xp[k, c] += eps
            Xm[k, c] -= eps
            dF = (O.spring_force(Xp, p.springs, p.kappa, p.rest, p.L)
                  - O.spring_force(Xm, p.springs, p.kappa, p.rest, p.L)) / (2 * eps)
            Jfd[:, c * n + k] = np.concatenate([dF[:, 0], dF[:, 1]])
    assert np.abs(Jx - Jfd).max() < 1e-6 * np.abs(Jx).max()
    assert np.allclose(Jx, Jx.T, atol=1e-12)


def test_clamped_jacobian_nsd_and_zero_rest_length_is_kappa_af():
    p = _small_problem(n=24, kappa=3.0, rest=0.06)   # compressed springs: exact J indefinite
    Jc = O.spring_jacobian(p.X, p.springs, p.kappa, p.rest, p.L, clamped=True).toarray()
    Je = O.spring_jacobian(p.X, p.springs, p.kappa, p.rest, p.L, clamped=False).toarray()
    assert np.linalg.eigvalsh(Jc).max() < 1e-12
    assert np.linalg.eigvalsh(Je).max() > 1e-3
    # zero rest length: J = kappa * A_f (x) I_2 with A_f the closed-curve second difference
    q = _small_problem(n=24, kappa=3.0, rest=0.0)
    J0 = O.spring_jacobian(q.X, q.springs, q.kappa, q.rest, q.L, clamped=True).toarray()
    n = q.n_points
    Af = -2.0 * np.eye(n) + np.roll(np.eye(n), 1, axis=1) + np.roll(np.eye(n), -1, axis=1)
    ref = np.kron(np.eye(2), 3.0 * Af)
    assert np.abs(J0 - ref).max() < 1e-12
    # and F = kappa A_f X for zero rest length
    F = O.spring_force(q.X, q.springs, q.kappa, q.rest, q.L)
    assert np.abs(F - 3.0 * Af @ q.X).max() < 1e-12


# ---------------------------------------------------------------- Stokes operator (sec. 2.2)

def _mms(N, mu=1.0):
    h = 1.0 / N
    i = np.arange(N)
    tp = 2 * np.pi
    xu, yu = np.meshgrid(i * h, (i + 0.5) * h, indexing="xy")
    xv, yv = np.meshgrid((i + 0.5) * h, i * h, indexing="xy")
    xp, yp = np.meshgrid((i + 0.5) * h, (i + 0.5) * h, indexing="xy")
    u = np.sin(tp * xu) * np.cos(tp * yu)
    v = -np.cos(tp * xv) * np.sin(tp * yv)
    p = np.sin(tp * xp) * np.sin(tp * yp)
    # continuous mu Lap u - grad p and div u at the same points
    fu = -2 * tp * tp * mu * u - tp * np.cos(tp * xu) * np.sin(tp * yu)
    fv = -2 * tp * tp * mu * v - tp * np.sin(tp * xv) * np.cos(tp * yv)
    w = np.concatenate([u.ravel(), v.ravel(), p.ravel()])
    exact = np.concatenate([fu.ravel(), fv.ravel(), np.zeros(N * N)])
    return w, exact


def test_stokes_manufactured_second_order():
    errs = []
    for N in (16, 32, 64, 128):
        A = O.stokes_matrix(N, 1.0 / N, 1.0, 0.0, 1.0)
        w, ex = _mms(N)
        errs.append(np.abs(A @ w - ex).max() / np.abs(ex).max())
    rates = [errs[k] / errs[k + 1] for k in range(3)]
    assert all(3.5 < r < 4.5 for r in rates), (errs, rates)


def test_stokes_unsteady_term_and_symmetry():
    N = 16
    h = 1.0 / N
    A0 = O.stokes_matrix(N, h, 1.3, 0.0, 0.1)
    A1 = O.stokes_matrix(N, h, 1.3, 2.0, 0.1)
    D = (A1 - A0).toarray()
    n = N * N
    assert np.allclose(np.diag(D)[: 2 * n], -20.0) and np.allclose(np.diag(D)[2 * n:], 0.0)
    assert np.abs(D - np.diag(np.diag(D))).max() == 0.0
    # [[K, -G], [D, 0]] with D = -G^T is symmetric
    assert abs(A1 - A1.T).max() < 1e-12


def test_stokes_divergence_free_solution_check():
    """A solve with a manufactured forcing gives an O(h^2)-accurate, exactly
    (discretely) divergence-free field."""
    errs = []
    for N in (16, 32, 64):
        A = O.stokes_matrix(N, 1.0 / N, 1.0, 0.0, 1.0)
        w, ex = _mms(N)
        sol = O.direct_solve(A, ex, N, 0.0) if N <= 32 else None
        if sol is None:
            import scipy.sparse.linalg as sla
            Z = O.nullspace_basis(N, 0.0)
            M = sp.bmat([[A, sp.csr_matrix(Z)], [sp.csr_matrix(Z.T), None]], format="csc")
            sol = sla.spsolve(M, np.concatenate([ex, np.zeros(3)]))[: 3 * N * N]
        n = N * N
        sol[2 * n:] -= sol[2 * n:].mean()
        div = (A @ sol)[2 * n:]
        assert np.abs(div).max() < 1e-9
        errs.append(np.abs(sol[: 2 * n] - w[: 2 * n]).max())
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


def _divfree_mode(N, kx, ky, phase=0.3):
    """A discretely divergence-free MAC velocity from a stream function psi on the
    cell corners: u = (psi[i, j+1] - psi[i, j]) / h, v = -(psi[i+1, j] - psi[i, j]) / h.
    psi is one real Fourier mode, so u and v are eigenvectors of the 5-point
    Laplacian with eigenvalue -lambda_k, lambda_k = (4/h^2)(sin^2(pi kx h) + sin^2(pi ky h))."""
    h = 1.0 / N
    i = np.arange(N)[None, :]
    j = np.arange(N)[:, None]

    def psi(ii, jj):
        return np.cos(2 * np.pi * (kx * ii + ky * jj) / N + phase)

    u = (psi(i, j + 1) - psi(i, j)) / h
    v = -(psi(i + 1, j) - psi(i, j)) / h
    lam = 4.0 / h ** 2 * (math.sin(math.pi * kx * h) ** 2 + math.sin(math.pi * ky * h) ** 2)
    return u, v, lam


@pytest.mark.parametrize("kx,ky", [(1, 0), (2, 3), (5, 1)])
def test_unsteady_step_decays_a_divergence_free_mode_exactly(kx, ky):
    """The u^n term of the right-hand side (backward Euler, sec. 2.3; the unsteady
    form named in sec. 8).  With no structure and u^n a discretely divergence-free
    Fourier mode, (mu Lap - (rho/dt) I) u - G p = -(rho/dt) u^n, D u = 0 is solved by
    u = c u^n, p = const, c = (rho/dt) / (rho/dt + mu lambda_k).  A sign slip in the
    u^n term gives -c, a dropped 1/dt gives rho / (rho + mu lambda_k dt)."""
    N, rho, mu, dt = 16, 2.0, 0.5, 0.1
    u, v, lam = _divfree_mode(N, kx, ky)
    n = N * N
    prob = W.Problem(N=N, L=1.0, rho=rho, mu=mu, dt=dt, X=np.zeros((0, 2)),
                     springs=np.zeros((0, 2), np.int32), kappa=np.zeros(0), rest=np.zeros(0))
    u_n = np.concatenate([u.ravel(), v.ravel()])
    A = O.stokes_matrix(N, 1.0 / N, mu, rho, dt)
    assert np.abs((A @ np.concatenate([u_n, np.zeros(n)]))[2 * n:]).max() < 1e-9  # D u^n = 0
    b = O.rhs_vector(prob, u_n=u_n)
    w = O.direct_solve(A, b, N, rho)
    c = (rho / dt) / (rho / dt + mu * lam)
    assert np.abs(w[: 2 * n] - c * u_n).max() <= 1e-10 * np.abs(u_n).max()
    assert np.abs(w[2 * n:] - w[2 * n:].mean()).max() <= 1e-10 * np.abs(u_n).max()
    # the multigrid-preconditioned step reaches the same field to its tolerance
    prob.box, prob.tol = 2, 1e-12
    st = O.solve_step(prob, u_n=u_n)
    assert np.abs(st.w[: 2 * n] - c * u_n).max() <= 1e-9 * np.abs(u_n).max()


def test_fluid_at_rest_without_structure_stays_at_rest():
    """u^n = None (and u^n = 0) with no structure: the right-hand side vanishes."""
    N = 16
    prob = W.Problem(N=N, L=1.0, rho=1.0, mu=1.0, dt=1e-2, X=np.zeros((0, 2)),
                     springs=np.zeros((0, 2), np.int32), kappa=np.zeros(0), rest=np.zeros(0))
    assert not O.rhs_vector(prob).any()
    assert not O.rhs_vector(prob, u_n=np.zeros(2 * N * N)).any()


# ---------------------------------------------------------------- transfers (sec. 3.1)

def test_transfer_constants_and_pressure_identity():
    Nf = 16
    R = O.restriction_matrix(Nf)
    P = O.prolongation_matrix(Nf // 2)
    assert np.allclose(np.asarray(R.sum(axis=1)).ravel(), 1.0)
    assert np.allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0)
    nc = (Nf // 2) ** 2
    Rp = R[2 * nc:, 2 * Nf * Nf:]
    Pp = P[2 * Nf * Nf:, 2 * nc:]
    assert abs(Rp @ Pp - sp.identity(nc)).max() < 1e-15
    # the u stencil is 1/8 [1 2 1; 1 2 1]: 6 fine faces, weights sum 1
    row = R[0].toarray().ravel()
    assert sorted(np.round(row[row != 0] * 8).tolist()) == [1, 1, 1, 1, 2, 2]


def _staggered_fields(N, f):
    h = 1.0 / N
    i = np.arange(N)
    xu, yu = np.meshgrid(i * h, (i + 0.5) * h, indexing="xy")
    xv, yv = np.meshgrid((i + 0.5) * h, i * h, indexing="xy")
    xp, yp = np.meshgrid((i + 0.5) * h, (i + 0.5) * h, indexing="xy")
    return np.concatenate([f(xu, yu, 0).ravel(), f(xv, yv, 1).ravel(), f(xp, yp, 2).ravel()])


def test_transfers_second_order_at_staggered_positions():
    """R and P of a smooth field match the field at the target points to O(h^2);
    a wrong staggering offset would leave an O(h) error."""
    def f(x, y, c):
        return np.sin(2 * np.pi * x + 0.4 * c) * np.cos(2 * np.pi * y - 0.3 * c)
    er, ep = [], []
    for N in (16, 32, 64, 128):
        R = O.restriction_matrix(N)
        P = O.prolongation_matrix(N // 2)
        fine = _staggered_fields(N, f)
        coarse = _staggered_fields(N // 2, f)
        n2 = 2 * N * N
        nc2 = 2 * (N // 2) ** 2
        er.append(np.abs((R @ fine)[:nc2] - coarse[:nc2]).max())
        ep.append(np.abs((P @ coarse)[:n2] - fine[:n2]).max())
    for e in (er, ep):
        assert all(e[k] / e[k + 1] > 3.5 for k in range(3)), e


# ---------------------------------------------------------------- elasticity operator, hierarchy

def test_elasticity_symmetric_nsd_and_kills_translations():
    p = _small_problem(N=16, n=24, kappa=50.0, rest=0.04)
    levels, ops = O.build_hierarchy(p)
    E0 = levels[0].E.toarray()
    assert np.allclose(E0, E0.T, atol=1e-9 * np.abs(E0).max())
    assert np.linalg.eigvalsh(0.5 * (E0 + E0.T)).max() < 1e-9 * np.abs(E0).max()
    for lev in levels:
        n2 = lev.N * lev.N
        c = np.concatenate([np.full(n2, 1.0), np.full(n2, -2.0)])
        assert np.abs(lev.E @ c).max() < 1e-9 * abs(lev.E).max()


def test_box_sizes_colours_and_free_boxes():
    p = _small_problem(N=32, n=30, kappa=100.0)
    levels, _ = O.build_hierarchy(p)
    for b in (1, 2, 4, 8):
        lev = levels[0]
        bx = O.prepare_boxes(lev, b)
        nb = 2 * b * (b + 1) + b * b
        assert bx["lex"].shape[1] == nb
        assert [5, 16, 56, 208][[1, 2, 4, 8].index(b)] == nb
        for c in range(4):
            idx = bx["color"][c][0]
            assert len(np.unique(idx)) == idx.size       # same-colour boxes share no unknowns
        # boxes away from the structure all carry the same matrix (sec. 8 remark)
        nbx = lev.N // b
        E = lev.E
        touched = set(np.nonzero(np.asarray(abs(E).sum(axis=1)).ravel())[0].tolist())
        free = [k for k in range(nbx * nbx) if not (set(bx["lex"][k].tolist()) & touched)]
        assert len(free) > 4
        A0 = bx["lexA"][free[0]]
        for k in free[1:]:
            assert np.array_equal(bx["lexA"][k], A0)
        # every unknown belongs to some box
        assert len(np.unique(bx["lex"])) == 3 * lev.N * lev.N


# ---------------------------------------------------------------- V-cycle and solves

def test_vcycle_stokes_contraction():
    """Without structure, one V(1,1) cycle contracts the error by well under 1/2."""
    p = _small_problem(N=64, n=8, kappa=0.0)
    levels, _ = O.build_hierarchy(p)
    for lev in levels[:-1]:
        O.prepare_boxes(lev, 1)
    rng = np.random.default_rng(5)
    b = levels[0].A @ rng.standard_normal(3 * 64 * 64)
    for order in ("color4", "lex"):
        w = np.zeros_like(b)
        r0 = np.linalg.norm(b)
        rs = []
        for _ in range(6):
            w = O.vcycle(levels, b, w, 1, 1, p.rho, order)
            rs.append(np.linalg.norm(b - levels[0].A @ w))
        rate = (rs[-1] / rs[1]) ** (1 / 4)
        assert rs[0] < r0 and rate < 0.35, (order, rate)


def _box_rows(N, b, color):
    """Unknowns of every b x b box of a colour, from the box definition (sec. 8):
    u faces x = I b .. I b + b on rows J b .. J b + b - 1, v faces y = J b .. J b + b
    on columns I b .. I b + b - 1, cells I b .. I b + b - 1 x J b .. J b + b - 1;
    layout [u | v | p], index j N + i, periodic wrap; colour (I mod 2) + 2 (J mod 2)."""
    n = N * N
    rows = set()
    for J in range(N // b):
        for I in range(N // b):
            if (I % 2) + 2 * (J % 2) != color:
                continue
            for j in range(J * b, J * b + b):
                for i in range(I * b, I * b + b + 1):
                    rows.add((j % N) * N + i % N)
            for j in range(J * b, J * b + b + 1):
                for i in range(I * b, I * b + b):
                    rows.add(n + (j % N) * N + i % N)
            for j in range(J * b, J * b + b):
                for i in range(I * b, I * b + b):
                    rows.add(2 * n + j * N + i)
    return np.array(sorted(rows))


@pytest.mark.parametrize("b,N", [(2, 16), (4, 16), (8, 16), (16, 32)])
@pytest.mark.parametrize("reverse", [False, True])
def test_colour_sweep_solves_last_colour_boxes_exactly(b, N, reverse):
    """Four-colour box smoother (sec. 6): n x n boxes (n >= 2) of one colour are
    farther apart than the 5-point stencil reaches, so without structure the last
    colour phase of a sweep solves its boxes' equations exactly: the residual
    vanishes on every unknown of that colour's boxes (colour 2 forward, colour 0
    reversed) and on no other colour's.  Up to the 16 x 16 boxes (800 unknowns)."""
    p = _small_problem(N=N, n=8, kappa=0.0)
    levels, _ = O.build_hierarchy(p)
    lev = levels[0]
    O.prepare_boxes(lev, b)
    rng = np.random.default_rng(21)
    rhs = rng.standard_normal(3 * N * N)
    w = O.smooth_color4(lev, rhs, rng.standard_normal(3 * N * N), reverse=reverse)
    r = rhs - lev.A @ w
    scale = np.abs(rhs).max()
    last = 0 if reverse else 2
    assert np.abs(r[_box_rows(N, b, last)]).max() <= 1e-10 * scale
    for c in range(4):
        if c != last:
            others = np.setdiff1d(_box_rows(N, b, c), _box_rows(N, b, last))
            assert np.abs(r[others]).max() > 1e-3 * scale, c


@pytest.mark.parametrize("b", [1, 2, 4])
def test_colour_phase_is_block_jacobi_with_structure(b):
    """Reading of sec. 5-6 for the GPU order: inside a colour every box is solved
    from the colour's starting state.  With a stiff structure (same-colour
    boxes coupled through the elasticity term) the sweep is then independent of
    the order of the boxes inside each colour, which an in-place (Gauss-Seidel)
    update inside a colour would not be; and a colour's boxes share no unknown."""
    N = 32
    p = _small_problem(N=N, n=48, kappa=1e4)
    levels, _ = O.build_hierarchy(p)
    lev = levels[0]
    O.prepare_boxes(lev, b)
    for c in range(4):
        idx = lev.boxes["color"][c][0]
        assert np.unique(idx.ravel()).size == idx.size, c
    rng = np.random.default_rng(8)
    rhs = rng.standard_normal(3 * N * N)
    w0 = rng.standard_normal(3 * N * N)
    ref = O.smooth_color4(lev, rhs, w0)
    perm = {}
    for c in range(4):
        idx, Abb = lev.boxes["color"][c]
        q = rng.permutation(idx.shape[0])
        perm[c] = (idx[q], Abb[q])
    lev.boxes = dict(lev.boxes, color=perm)
    got = O.smooth_color4(lev, rhs, w0)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    moved = np.abs(O.smooth_color4(lev, rhs, ref) - ref).max()
    assert moved > 1e-6 * np.abs(ref).max()  # the sweep is not a fixed point


def test_fgmres_matches_dense_direct_solve_16():
    for rho, kap, rest in ((1.0, 1e3, None), (0.0, 1e2, 0.0)):
        p = W.single_ellipse(N=16, n_points=24, kappa=kap, dt=1e-2, rho=rho, rest=rest,
                             a=0.28, b=0.22)
        res = O.solve_step(p)
        levels, _ = O.build_hierarchy(p)
        xd = O.remove_pressure_mean(O.direct_solve(levels[0].A, res.b, p.N, rho), p.N)
        if rho == 0.0:
            n = p.N * p.N
            xd[:n] -= xd[:n].mean()
            xd[n:2 * n] -= xd[n:2 * n].mean()
            w = res.w.copy()
            w[:n] -= w[:n].mean()
            w[n:2 * n] -= w[n:2 * n].mean()
        else:
            w = res.w
        assert res.solve.converged and res.solve.rel_res_true <= 1e-8
        assert np.linalg.norm(w - xd) <= 1e-6 * np.linalg.norm(xd)
        n = p.N * p.N
        div = (levels[0].A @ res.w)[2 * n:]
        assert np.linalg.norm(div) <= 1e-8 * np.linalg.norm(res.b)


def test_iterations_flat_under_refinement_and_rise_with_stiffness():
    its = []
    for N in (32, 64, 128):
        p = W.single_ellipse(N=N, n_points=2 * N, kappa=1e2, dt=1e-2)
        its.append(O.solve_step(p).solve.iters)
    assert max(its) - min(its) <= 2, its
    soft = O.solve_step(W.single_ellipse(N=32, n_points=64, kappa=1.0, dt=1e-2)).solve.iters
    stiff = O.solve_step(W.single_ellipse(N=32, n_points=64, kappa=1e6, dt=1e-2)).solve.iters
    assert stiff > soft, (soft, stiff)


def _iters(kappa, b=4, nu=(1, 1)):
    p = W.single_ellipse(N=32, n_points=64, kappa=kappa, dt=1e-2)
    p.box, (p.nu1, p.nu2), p.max_iters = b, nu, 200
    r = O.solve_step(p).solve
    return r.iters if r.converged else None


def test_bigger_boxes_fewer_iterations_most_when_stiff():
    """Sec. 6 (MG-GMRES for box sizes 1-8): the larger the box, the fewer the
    iterations, the more so the stiffer the structure, and for very stiff
    structures the single-box smoother does not converge within the cap while
    the big boxes do."""
    mild = [_iters(1e4, b) for b in (1, 2, 4, 8)]
    stiff = [_iters(1e6, b) for b in (1, 2, 4, 8)]
    assert all(x is not None for x in mild) and mild == sorted(mild, reverse=True), mild
    assert stiff[0] is None and None not in stiff[1:], stiff
    assert stiff[1] > stiff[2] > stiff[3], stiff
    assert stiff[1] - stiff[3] > mild[1] - mild[3], (mild, stiff)


def test_refinement_small_boxes_grow_big_boxes_flat_when_stiff():
    """Sec. 6 (grid refinement): for a stiff structure the MG-GMRES iteration
    count grows as the grid is refined with 1 x 1 boxes and stays about flat with
    8 x 8 boxes; for a milder one both stay flat."""
    def its(N, kappa, b):
        p = W.single_ellipse(N=N, n_points=2 * N, kappa=kappa, dt=1e-2)
        p.box, p.max_iters = b, 200
        r = O.solve_step(p).solve
        assert r.converged
        return r.iters

    s1 = [its(N, 1e5, 1) for N in (32, 64)]
    s8 = [its(N, 1e5, 8) for N in (32, 64)]
    m1 = [its(N, 1e4, 1) for N in (32, 64)]
    assert s1[1] >= 1.3 * s1[0], s1
    assert abs(s8[1] - s8[0]) <= 2 and abs(m1[1] - m1[0]) <= 2, (s8, m1)


def test_more_smoothing_sweeps_fewer_iterations():
    """Sec. 6 (table of nu1, nu2 for b = 4): the iteration count falls as the
    number of pre- and post-smoothing sweeps grows."""
    its = [_iters(1e5, 4, nu) for nu in ((1, 0), (1, 1), (2, 1), (2, 2))]
    assert None not in its and its == sorted(its, reverse=True) and its[0] > its[-1], its


# ---------------------------------------------------------------- MG as a solver, iteration matrix (sec. 5)

def _mg16(kappa, b):
    p = W.single_ellipse(N=16, n_points=32, kappa=kappa, dt=1e-2, a=0.23, b=0.17, center=(0.47, 0.53))
    p.box, p.max_iters = b, 200
    levels, _ = O.build_hierarchy(p)
    for lev in levels[:-1]:
        O.prepare_boxes(lev, b)
    M = O.iteration_matrix(levels, p.nu1, p.nu2, p.rho)
    return p, levels, O.spectrum_mean_zero_pressure(M, 16), M


@pytest.mark.parametrize("kappa,b", [(1e5, 4), (1e6, 4), (1e5, 1)])
def test_mg_solver_contraction_equals_iteration_matrix_spectral_radius(kappa, b):
    """Two independent routes to one number: stand-alone multigrid (repeated
    cycles on b = A x*) contracts the residual asymptotically by the spectral
    radius of the iteration matrix built column by column from unit errors
    (sec. 5), on the zero-mean-pressure space; with b = 1 and kappa = 1e5 both
    exceed 1 (the stand-alone solver diverges)."""
    p, levels, ev, _ = _mg16(kappa, b)
    rho = np.abs(ev).max()
    assert rho > 0.4
    rng = np.random.default_rng(2)
    xs = rng.standard_normal(3 * 256)
    xs[512:] -= xs[512:].mean()
    h = O.mg_solve(levels, levels[0].A @ xs, tol=0.0, max_iters=40, rho=p.rho).history
    rate = (h[-1] / h[-11]) ** 0.1
    assert abs(rate - rho) <= 0.02 * rho, (rate, rho)


def test_iteration_matrix_spectrum_and_solver_against_preconditioner():
    """Sec. 5 with the single-box (1 x 1) smoother: for Stokes the nontrivial
    eigenvalues lie in a small disc (the paper reports 0.24 for its cavity), a
    mild structure leaves the radius about unchanged, and a stiff one pushes a
    few eigenvalues out (radius above 1: the stand-alone solver fails) while
    nearly all stay near the origin, so MG-preconditioned GMRES still converges
    (multigrid a poor solver but an effective preconditioner).  With 4 x 4 boxes
    (sec. 6) the stiff radius stays below 1 and the solver converges, in far more
    iterations than MG-GMRES."""
    _, _, e0, M0 = _mg16(0.0, 1)
    c = np.zeros(3 * 256)
    c[512:] = 1.0  # constant pressure: the trivial eigenvector, eigenvalue 1 (sec. 5)
    assert np.abs(M0 @ c - c).max() <= 1e-10
    _, _, e2, _ = _mg16(1e2, 1)
    p5, lv5, e5, _ = _mg16(1e5, 1)
    r0, r2, r5 = (np.abs(e).max() for e in (e0, e2, e5))
    assert r0 < 0.3 and r2 < 1.1 * r0, (r0, r2)
    assert r5 > 1.0 and np.mean(np.abs(e5) > 0.25) < 0.1, (r5, np.mean(np.abs(e5) > 0.25))
    assert O.solve_step(p5).solve.converged
    p6, lv6, e6, _ = _mg16(1e6, 4)
    assert np.abs(e6).max() < 1.0
    mg = O.mg_solve(lv6, O.rhs_vector(p6), tol=p6.tol, max_iters=200, rho=p6.rho)
    gm = O.solve_step(p6).solve
    assert mg.converged and gm.converged and mg.iters > 2 * gm.iters, (mg.iters, gm.iters)


def test_explicit_stiffness_limit_spectrum_and_refinement():
    """Sec. 4.1: S* L^{-1} S A (Stokes solution operator, symmetric positive
    semidefinite, times the spring Jacobian per unit stiffness, symmetric
    negative semidefinite) has real, nonpositive eigenvalues; with zero rest
    length its kernel holds exactly the two rigid translations; and
    alpha_exp = 2 / rho falls as the grid is refined with the structure (the
    paper's table falls from 6.09 to 2.28 for its annulus, h = 2^-5 .. 2^-8)."""
    a = {}
    for N in (16, 32):
        p = W.single_ellipse(N=N, n_points=2 * N, kappa=1.0, dt=1e-2)
        a[N], ev = O.explicit_stiffness_limit(p)
        big = np.abs(ev).max()
        assert np.abs(ev.imag).max() <= 1e-10 * big and ev.real.max() <= 1e-10 * big
        assert a[N] == pytest.approx(2.0 / big)
    assert a[32] < a[16], a
    p0 = W.single_ellipse(N=16, n_points=32, kappa=1.0, dt=1e-2, rest=0.0)
    _, ev0 = O.explicit_stiffness_limit(p0)
    assert int(np.sum(np.abs(ev0) < 1e-9 * np.abs(ev0).max())) == 2


def test_translation_by_one_cell_shifts_solution():
    N = 32
    p = W.single_ellipse(N=N, n_points=48, kappa=1e3, center=(0.45, 0.52))
    q = W.single_ellipse(N=N, n_points=48, kappa=1e3, center=(0.45 + 1.0 / N, 0.52))
    a = O.solve_step(p)
    b = O.solve_step(q)
    for c in range(3):
        fa = a.w[c * N * N:(c + 1) * N * N].reshape(N, N)
        fb = b.w[c * N * N:(c + 1) * N * N].reshape(N, N)
        assert np.abs(np.roll(fa, 1, axis=1) - fb).max() < 1e-7 * np.abs(fa).max()
    assert np.abs(a.X + np.array([1.0 / N, 0.0]) - b.X).max() < 1e-10


def test_mirror_symmetry():
    """Reflecting the geometry x -> 1 - x mirrors u (with a sign) and v, p."""
    N = 32
    p = W.single_ellipse(N=N, n_points=48, kappa=1e3, center=(0.41, 0.52))
    X = p.X
    p.X = np.stack([0.5 + 0.09 * np.cos(np.arange(48) * 2 * np.pi / 48) + 0.02 * np.sin(
        3 * np.arange(48) * 2 * np.pi / 48), X[:, 1]], axis=1)
    q = W.single_ellipse(N=N, n_points=48, kappa=1e3)
    q.X = np.stack([1.0 - p.X[:, 0], p.X[:, 1]], axis=1)
    q.springs = p.springs[:, ::-1].copy()
    a = O.solve_step(p)
    b = O.solve_step(q)
    n = N * N
    ua = a.w[:n].reshape(N, N)
    ub = b.w[:n].reshape(N, N)
    # u face i at x = i h maps to x = 1 - i h = face (N - i) mod N
    ua_m = -ua[:, (-np.arange(N)) % N]
    assert np.abs(ua_m - ub).max() < 1e-7 * np.abs(ua).max()
    va = a.w[n:2 * n].reshape(N, N)
    vb = b.w[n:2 * n].reshape(N, N)
    assert np.abs(va[:, ::-1] - vb).max() < 1e-7 * np.abs(va).max()
    pa = a.w[2 * n:].reshape(N, N)
    pb = b.w[2 * n:].reshape(N, N)
    assert np.abs(pa[:, ::-1] - pb).max() < 1e-7 * np.abs(pa).max()


def test_backward_euler_energy_decreases_for_any_dt():
    """Zero rest length, steady Stokes (rho = 0): the lagged-S backward-Euler step is
    unconditionally stable, so the elastic energy never increases (sec. 2.3)."""
    for dt in (1e-3, 1e-1, 10.0):
        p = W.single_ellipse(N=32, n_points=48, kappa=50.0, dt=dt, rho=0.0, rest=0.0)
        e = [O.elastic_energy(p.X, p.springs, p.kappa, p.rest, p.L)]
        X = p.X
        for _ in range(3):
            r = O.solve_step(p, X=X)
            assert r.solve.converged
            X = r.X
            e.append(O.elastic_energy(X, p.springs, p.kappa, p.rest, p.L))
        assert all(e[k + 1] <= e[k] * (1 + 1e-12) for k in range(3)), (dt, e)
        assert e[-1] < e[0]
