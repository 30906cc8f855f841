"""Plain FP64 CPU oracle of the paper's own test problem: the lid-driven cavity
with the thick elastic annulus (sec. 4), and its explicit-time stability limit
alpha_exp (sec. 4.1, Table 1).

TEST INFRASTRUCTURE ONLY.  Like ``ib_oracle``, only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import it; the
library never does, and it shares no code with the CUDA path.

What it computes:

* the steady MAC Stokes operator of sec. 2.2 on the unit square with no-slip
  walls (the operator of the lid-driven cavity: the lid's tangential velocity
  only enters the right-hand side, so the linear operator is the homogeneous
  Dirichlet one);
* the thick annulus of sec. 4 (its initial positions, M1 = 19N/8 points along
  each closed fibre, M2 = 3N/32 + 1 fibres across the thickness w = 1/16);
* the force-generation operator A_f (three-point second difference along each
  fibre, sec. 2.2), the spreading of a Lagrangian force density with the
  cosine kernel, and its adjoint, the interpolation (sec. 2.2);
* alpha_exp = 2 / rho(S^* L^{-1} S A_f), sec. 4.1, the largest alpha = gamma dt
  for which the explicit-time method is stable;
* the multigrid of sec. 3 on the cavity: the staggered transfers with the wall
  rules, re-discretised Stokes plus the Galerkin elasticity on the coarse
  levels, the lexicographic box (Vanka) smoother of sec. 5 and the n x n big
  boxes of sec. 6, the exact coarsest solve on N_c = max(4, n), the V-cycle of
  Algorithm 1, multigrid as a stand-alone solver, GMRES right-preconditioned
  by one V-cycle, and the iteration matrix of the stand-alone solver.

Readings (each also listed in the design notes):

* walls: the normal velocity on a wall is zero (those faces are not unknowns);
  the tangential velocity in the first row of faces next to a wall sees the
  ghost value -u (the wall value, the mean of the two, is zero), so its
  Laplacian row reads (u_{j+1} - 3 u_j + ...) / h^2; the lid's velocity enters
  the right-hand side through the ghost 2 u_lid - u;
* Lagrangian spacings: the paper writes ds1 = ds2 = ds, but its M1 and M2
  give ds1 = 2 pi r / M1 = 4 pi / (19 N) and ds2 = w / (M2 - 1) = 2 / (3 N),
  which differ by 0.8 %.  A_f differentiates along s1 and divides by ds1^2.
  For the spreading weight ds^2 Table 1 decides: ds = ds1 reproduces all four
  printed alpha_exp, ds1 ds2 is 0.8 % low at every grid ("ds1^2" is the
  default; the others remain selectable);
* the cosine kernel is (1 + cos(pi r / (2h))) / (4h) for |r| < 2h, as in
  ``ib_oracle``;
* prolongation next to a wall interpolates linearly to the wall's zero (the
  same as using the ghost rule on the coarse grid); restriction needs no wall
  rule (the fine faces it reads are interior or hold zero);
* the right-hand side is the printed one of sec. 3 (-S A_f X^n) plus the lid;
  the iteration counts do not depend on the force term's scale (checked with
  and without it);
* the same lexicographic order before and after the coarse correction;
* box unknowns leave out the wall faces.

Pins (tests/test_cavity_oracle.py): a manufactured no-slip Stokes solution at
second order; symmetry of the velocity block and D = -G^T; the transfers'
identities and second-order prolongation at the walls; the annulus geometry and
the closed-form spectrum of A_f; the S / S^* adjoint; Table 1 (all four
alpha_exp to within 0.3 %); the counts of sec. 5 (9 / 8 cycles and iterations
at low stiffness, 62 / 30 at relative stiffness 100), the spectral radii under
the spectrum figure (0.24, 0.22, 0.30, 0.85) and the share of eigenvalues
outside radius 0.25 and 0.5, where the two solvers give up; and all 36
counts of Table 2.

Vector layout: [u | v | p], each an N x N array, row-major with x fastest (index
j*N + i), the same as ``ib_oracle``.  u[j, i] sits at (i h, (j + 1/2) h); the
faces i = 0 (and the absent i = N) are the walls x = 0 and x = 1, so u[j, 0] is
not an unknown: its row is the identity and no other row couples to it.  v is
the same with x and y exchanged.  p[j, i] sits at the cell centres.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .ib_oracle import phi_cos4

# ----------------------------------------------------------------------------
# Stokes operator with no-slip walls (sec. 2.2 discretisation, sec. 4 domain)
# ----------------------------------------------------------------------------


def u_index(N, i, j):
    return np.asarray(j) * N + np.asarray(i)


def v_index(N, i, j):
    return N * N + np.asarray(j) * N + np.asarray(i)


def p_index(N, i, j):
    return 2 * N * N + np.asarray(j) * N + np.asarray(i)


def wall_rows(N):
    """Indices of the pinned wall faces: u[j, 0] and v[0, i]."""
    k = np.arange(N)
    return np.concatenate([u_index(N, 0, k), v_index(N, k, 0)])


def cavity_stokes_matrix(N, mu=1.0, L=1.0):
    """[[mu Lap, -G], [D, 0]] on the N x N MAC grid of the square with no-slip walls, CSR.

    Free u faces i = 1..N-1 (all j): (Lap u) couples to u[j, i +- 1] (the wall
    faces i = 0 and i = N hold zero and are dropped) and to u[j +- 1, i]; in the
    rows j = 0 and j = N - 1 the missing neighbour is the ghost -u[j, i], which
    adds -1/h^2 to the diagonal.  (G p) on the u face (i, j) = (p_{i,j} -
    p_{i-1,j}) / h; (D w)_{i,j} = (u_{i+1,j} - u_{i,j} + v_{i,j+1} - v_{i,j}) / h
    with the wall faces zero.  v: x and y exchanged.  Wall faces: identity rows.
    """
    h = L / N
    n = N * N
    rows, cols, vals = [], [], []

    def add(r, c, v):
        rows.append(int(r))
        cols.append(int(c))
        vals.append(float(v))

    c = mu / (h * h)
    for j in range(N):
        for i in range(N):
            for comp in (0, 1):
                # (a, b): coordinates along the face normal and tangent
                a, b = (i, j) if comp == 0 else (j, i)
                idx = (lambda a_, b_: u_index(N, a_, b_)) if comp == 0 else (lambda a_, b_: v_index(N, b_, a_))
                r = idx(a, b)
                if a == 0:  # wall face
                    add(r, r, 1.0)
                    continue
                diag = -4.0 * c
                for da in (-1, 1):  # along the normal: faces a +- 1, walls at 0 and N
                    if 0 < a + da < N:
                        add(r, idx(a + da, b), c)
                for db in (-1, 1):  # along the tangent: ghost -u beyond the wall
                    if 0 <= b + db < N:
                        add(r, idx(a, b + db), c)
                    else:
                        diag -= c
                add(r, r, diag)
                # -G p: cells on either side of the face
                pc = p_index(N, i, j)
                pm = p_index(N, i - 1, j) if comp == 0 else p_index(N, i, j - 1)
                add(r, pc, -1.0 / h)
                add(r, pm, 1.0 / h)
            # D w at cell (i, j)
            rp = p_index(N, i, j)
            if i + 1 < N:
                add(rp, u_index(N, i + 1, j), 1.0 / h)
            if i > 0:
                add(rp, u_index(N, i, j), -1.0 / h)
            if j + 1 < N:
                add(rp, v_index(N, i, j + 1), 1.0 / h)
            if j > 0:
                add(rp, v_index(N, i, j), -1.0 / h)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(3 * n, 3 * n))
    A.sum_duplicates()
    return A


def stokes_velocity_solver(N, mu=1.0, L=1.0):
    """f -> u with mu Lap u - G p + f = 0, D u = 0 (the steady Stokes system of
    sec. 2.3.1, Eq. "explicit1"), as a callable on blocks of force columns
    [2N^2, k].  With no-slip walls the continuity rows sum to zero (no net flux
    through the walls), so one of them is redundant: the row of cell (0, 0) is
    replaced by p_00 = 0, which fixes the pressure's free constant and leaves the
    velocity unchanged."""
    n = N * N
    A = cavity_stokes_matrix(N, mu, L).tolil()
    r0 = p_index(N, 0, 0)
    A.rows[r0] = [r0]
    A.data[r0] = [1.0]
    lu = spla.splu(A.tocsc(), permc_spec="COLAMD")
    walls = wall_rows(N)

    def solve(f):
        f = np.asarray(f, dtype=np.float64)
        one = f.ndim == 1
        F = f[:, None] if one else f
        rhs = np.zeros((3 * n, F.shape[1]))
        rhs[: 2 * n] = -F
        rhs[walls] = 0.0  # the wall faces hold zero whatever force lands there
        u = lu.solve(rhs)[: 2 * n]
        return u[:, 0] if one else u

    return solve


# ----------------------------------------------------------------------------
# The thick annulus and its elasticity (sec. 4, sec. 2.2)
# ----------------------------------------------------------------------------


class Annulus:
    """Nodes X[l, k] = (xc + (r + s2_l) cos(s1_k / r), yc + (r + s2_l) sin(s1_k / r))
    with s1_k = k ds1 (k < M1, closed fibres) and s2_l = l ds2 (l < M2), sec. 4."""

    def __init__(self, N, r=0.25, w=1.0 / 16.0, center=(0.5, 0.5)):
        if N % 32 != 0:
            raise ValueError("M1 = 19N/8 and M2 = 3N/32 + 1 need N a multiple of 32")
        self.N = N
        self.M1 = 19 * N // 8
        self.M2 = 3 * N // 32 + 1
        self.r, self.w = r, w
        self.ds1 = 2.0 * math.pi * r / self.M1
        self.ds2 = w / (self.M2 - 1)
        s1 = np.arange(self.M1) * self.ds1
        s2 = np.arange(self.M2) * self.ds2
        R = r + s2[:, None]
        self.X = np.stack([center[0] + R * np.cos(s1[None, :] / r),
                           center[1] + R * np.sin(s1[None, :] / r)], axis=-1)  # [M2, M1, 2]

    @property
    def n_points(self):
        return self.M1 * self.M2

    def points(self):
        """[Np, 2], fibre-major (point l*M1 + k)."""
        return self.X.reshape(-1, 2)


def force_operator(ann):
    """A_f on [X components of all points | Y components], (A_f X)_{k,l} =
    (X_{k-1,l} - 2 X_{k,l} + X_{k+1,l}) / ds1^2 along each closed fibre (sec. 2.2)."""
    M1, M2 = ann.M1, ann.M2
    D = sp.diags([np.ones(M1 - 1), -2.0 * np.ones(M1), np.ones(M1 - 1)], [-1, 0, 1], format="lil")
    D[0, M1 - 1] = 1.0
    D[M1 - 1, 0] = 1.0
    D = D.tocsr() / (ann.ds1 ** 2)
    one = sp.kron(sp.identity(M2), D, format="csr")
    return sp.block_diag([one, one], format="csr")


def spread_matrix(X, N, weight, L=1.0):
    """S_h as a (2N^2) x (2Np) CSR matrix: (f1) at the u face = sum_k F1_k
    delta_h(x_face - X_k) * weight, delta_h(x) = phi(x/h) phi(y/h) / h^2 (the
    cosine kernel), weight the Lagrangian quadrature weight (sec. 2.2).  The
    kernel's support must stay inside the square (the annulus does)."""
    X = np.asarray(X, dtype=np.float64)
    Np = X.shape[0]
    h = L / N
    if np.any(X < 2.0 * h) or np.any(X > L - 2.0 * h):
        raise ValueError("kernel support reaches a wall")
    grid = np.arange(N, dtype=np.float64)
    rows, cols, vals = [], [], []
    for comp, (ox, oy) in enumerate(((0.0, 0.5), (0.5, 0.0))):
        for k in range(Np):
            wx = phi_cos4(grid + ox - X[k, 0] / h)
            wy = phi_cos4(grid + oy - X[k, 1] / h)
            ii = np.nonzero(wx)[0]
            jj = np.nonzero(wy)[0]
            W = np.outer(wy[jj], wx[ii]) * (weight / (h * h))
            J2, I2 = np.meshgrid(jj, ii, indexing="ij")
            rows.append((comp * N * N + J2 * N + I2).ravel())
            cols.append(np.full(W.size, comp * Np + k))
            vals.append(W.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(2 * N * N, 2 * Np))


def interp_matrix_from_kernel(X, N, L=1.0):
    """S_h^*: U_k = sum over faces of u delta_h(x_face - X_k) h^2 (sec. 2.2), the
    kernel sum written out on its own (not as a transpose of the spreading)."""
    return spread_matrix(X, N, 1.0, L).T.tocsr() * ((L / N) ** 2)


# ----------------------------------------------------------------------------
# Explicit-time stability limit (sec. 4.1, Table 1)
# ----------------------------------------------------------------------------


def fibre_sqrt(ann):
    """(-A_f)^{1/2} on one fibre as a dense M1 x M1 matrix (symmetric square root of
    the positive semidefinite circulant second difference)."""
    M1 = ann.M1
    B = (-force_operator(ann)[:M1, :M1]).toarray()
    lam, Q = np.linalg.eigh(B)
    return (Q * np.sqrt(np.maximum(lam, 0.0))) @ Q.T


def explicit_limit(N, weight="ds1ds2", tol=1e-10):
    """alpha_exp = 2 / rho, rho the spectral radius of S^* L^{-1} S A_f on the
    annulus in the cavity at h = 1/N (sec. 4.1).  L^{-1} maps a force density to
    the steady Stokes velocity; weight names the spreading quadrature weight
    ("ds1ds2", "ds1^2" or "ds2^2").

    S^* L^{-1} S is symmetric positive semidefinite and -A_f symmetric positive
    semidefinite, so the eigenvalues of the product are those of the symmetric
    B^{1/2} (S^* L^{-1} S) B^{1/2}, B = -A_f, all >= 0; the largest is found by
    Lanczos (ARPACK), one Stokes solve per product.  Returns (alpha_exp, rho)."""
    ann = Annulus(N)
    wts = {"ds1ds2": ann.ds1 * ann.ds2, "ds1^2": ann.ds1 ** 2, "ds2^2": ann.ds2 ** 2}
    X = ann.points()
    S = spread_matrix(X, N, wts[weight])
    Ss = interp_matrix_from_kernel(X, N)
    solve = stokes_velocity_solver(N)
    Bh = fibre_sqrt(ann)
    M1, M2 = ann.M1, ann.M2
    n = 2 * ann.n_points

    def half(x):
        # B^{1/2} acts along s1 on every fibre and both components
        return (x.reshape(2 * M2, M1) @ Bh.T).ravel()

    def mv(x):
        y = half(np.asarray(x).ravel())
        y = Ss @ solve(S @ y)
        return half(y)

    op = spla.LinearOperator((n, n), matvec=mv, dtype=np.float64)
    lam = spla.eigsh(op, k=1, which="LA", tol=tol, return_eigenvectors=False)
    rho = float(lam[0])
    return 2.0 / rho, rho


# ----------------------------------------------------------------------------
# Grid transfers with walls (sec. 3.1)
# ----------------------------------------------------------------------------


def cavity_restriction(Nf):
    """I_{2h<-h} for [u|v|p] from an Nf grid to Nc = Nf/2 in the square with walls.

    The stencils of sec. 3.1: p the mean of the four fine cells; u the 1/8
    [1 2 1; 1 2 1] stencil (fine faces 2I-1, 2I, 2I+1 across x, fine rows 2J and
    2J+1); v the same with x and y exchanged.  Coarse wall faces (I = 0) get no
    row (they hold zero); the fine faces a coarse interior face reads are all
    interior or wall faces, which hold zero."""
    Nc = Nf // 2
    rows, cols, vals = [], [], []
    for J in range(Nc):
        for I in range(Nc):
            for a, wa in ((-1, 0.25), (0, 0.5), (1, 0.25)):
                for bb in (0, 1):
                    if I > 0:
                        rows.append(u_index(Nc, I, J))
                        cols.append(u_index(Nf, 2 * I + a, 2 * J + bb))
                        vals.append(0.5 * wa)
                        rows.append(v_index(Nc, J, I))
                        cols.append(v_index(Nf, 2 * J + bb, 2 * I + a))
                        vals.append(0.5 * wa)
            for a in (0, 1):
                for bb in (0, 1):
                    rows.append(p_index(Nc, I, J))
                    cols.append(p_index(Nf, 2 * I + a, 2 * J + bb))
                    vals.append(0.25)
    R = sp.csr_matrix((vals, (rows, cols)), shape=(3 * Nc * Nc, 3 * Nf * Nf))
    R.sum_duplicates()
    return R


def cavity_prolongation(Nc):
    """I_{h<-2h} for [u|v|p] from an Nc grid to Nf = 2Nc in the square with walls.

    p: constant.  u: linear across x (fine face 2I copies coarse face I, fine face
    2I+1 averages coarse faces I and I+1; the wall faces 0 and Nc hold zero) and
    linear along y between cell-centred rows (fine row 2J: 3/4 coarse row J + 1/4
    row J-1; fine row 2J+1: 3/4 row J + 1/4 row J+1); beyond a wall the coarse
    row is its ghost, minus the first row, so the wall's zero is interpolated
    linearly (fine row 0 takes 1/2 of coarse row 0).  v: x and y exchanged."""
    Nf = 2 * Nc
    rows, cols, vals = [], [], []

    def normal(k):
        if k % 2 == 0:
            return [(k // 2, 1.0)]
        return [((k - 1) // 2, 0.5), ((k + 1) // 2, 0.5)]

    def centred(k):
        K = k // 2
        far = K - 1 if k % 2 == 0 else K + 1
        if 0 <= far < Nc:
            return [(K, 0.75), (far, 0.25)]
        return [(K, 0.75), (K, -0.25)]  # the ghost beyond the wall is -(row K)

    for fj in range(Nf):
        for fi in range(Nf):
            if fi > 0:  # u face (fi, fj); fine wall faces stay zero
                for ci, wi in normal(fi):
                    if 0 < ci < Nc:
                        for cj, wj in centred(fj):
                            rows.append(u_index(Nf, fi, fj))
                            cols.append(u_index(Nc, ci, cj))
                            vals.append(wi * wj)
            if fj > 0:  # v face (fi, fj)
                for cj, wj in normal(fj):
                    if 0 < cj < Nc:
                        for ci, wi in centred(fi):
                            rows.append(v_index(Nf, fi, fj))
                            cols.append(v_index(Nc, ci, cj))
                            vals.append(wi * wj)
            rows.append(p_index(Nf, fi, fj))
            cols.append(p_index(Nc, fi // 2, fj // 2))
            vals.append(1.0)
    P = sp.csr_matrix((vals, (rows, cols)), shape=(3 * Nf * Nf, 3 * Nc * Nc))
    P.sum_duplicates()
    return P


# ----------------------------------------------------------------------------
# Hierarchy, box smoother and V-cycle on the cavity (sec. 3, sec. 5, sec. 6)
# ----------------------------------------------------------------------------


class CavityLevel:
    def __init__(self, N, A, E):
        self.N = N
        self.A = A          # level operator, CSR (wall rows: identity)
        self.E = E          # elasticity S A_f S^* on the velocity faces (Galerkin below level 0)
        self.R = None       # restriction to the next level
        self.P = None       # prolongation from the next level
        self.boxes = None


def cavity_box_unknowns(N, b, I, J):
    """Unknowns of the b x b box (I, J): its u faces (i = Ib..Ib+b, rows Jb..Jb+b-1),
    v faces (the same with x and y exchanged) and cells, without the wall faces
    (i = 0, i = N), which are not unknowns."""
    x0, y0 = I * b, J * b
    out = []
    for j in range(y0, y0 + b):
        for i in range(x0, x0 + b + 1):
            if 0 < i < N:
                out.append(int(u_index(N, i, j)))
    for j in range(y0, y0 + b + 1):
        for i in range(x0, x0 + b):
            if 0 < j < N:
                out.append(int(v_index(N, i, j)))
    for j in range(y0, y0 + b):
        for i in range(x0, x0 + b):
            out.append(int(p_index(N, i, j)))
    return np.array(out, dtype=np.int64)


def cavity_hierarchy(N, alpha, b, ann=None, weight="ds1^2", order="lex"):
    """Levels N, N/2, ..., N_c = max(4, b) (sec. 6): the re-discretised wall Stokes
    operator plus alpha times the elasticity, level 0's S A_f S^* from the annulus
    and each coarser one the Galerkin product R E P of the velocity blocks
    (sec. 3.2).  Each non-coarsest level gets its boxes with their dense A_BB
    blocks, in lexicographic order (rows of boxes bottom to top, x fastest;
    order="lex", the paper's) or in the four colours of the parallel order
    (order="color4": box (I, J) has colour (I mod 2) + 2 (J mod 2), the colours
    visited as in ``ib_oracle.COLOR_SEQUENCE``).  ann: any object with N, M1,
    M2, ds1, ds2 and points() (default: ``Annulus(N)``)."""
    ann = Annulus(N) if ann is None else ann
    wts = {"ds1ds2": ann.ds1 * ann.ds2, "ds1^2": ann.ds1 ** 2, "ds2^2": ann.ds2 ** 2}
    X = ann.points()
    S = spread_matrix(X, N, wts[weight])
    Ss = interp_matrix_from_kernel(X, N)
    E = (S @ force_operator(ann) @ Ss).tocsr()
    Nc = max(4, b)
    levels = []
    n = N
    while True:
        A = cavity_stokes_matrix(n).tolil()
        m = 2 * n * n
        Av = A[:m, :m].tocsr() + alpha * E
        A = sp.bmat([[Av, A[:m, m:]], [A[m:, :m], A[m:, m:]]], format="csr")
        # wall rows stay identity (E has no entries there: the spread never reaches a wall)
        levels.append(CavityLevel(n, A, E))
        if n <= Nc:
            break
        R = cavity_restriction(n)
        P = cavity_prolongation(n // 2)
        levels[-1].R, levels[-1].P = R, P
        mc = 2 * (n // 2) ** 2
        E = (R[:mc, :m] @ E @ P[:m, :mc]).tocsr()
        n //= 2
    for lev in levels[:-1]:
        nb = lev.N // b
        boxes = []
        colors = {c: [] for c in range(4)}
        for J in range(nb):
            for I in range(nb):
                idx = cavity_box_unknowns(lev.N, b, I, J)
                rows = lev.A[idx, :].tocsr()
                box = (idx, rows, np.linalg.inv(rows[:, idx].toarray()))
                boxes.append(box)
                colors[(I % 2) + 2 * (J % 2)].append(box)
        lev.boxes = boxes
        lev.colors = colors
        lev.order = order
        lev.b = b
    return levels


def cavity_smooth_lex(level, rhs, w):
    """One block Gauss-Seidel sweep over the boxes in lexicographic order (sec. 5):
    each box's unknowns are replaced by the solution of its own equations with
    every other unknown at its current value.  w may carry several columns."""
    w = w.copy()
    for idx, rows, inv in level.boxes:
        r = rhs[idx] - rows @ w
        w[idx] += inv @ r
    return w


def cavity_smooth_color4(level, rhs, w, reverse=False):
    """One sweep in the parallel order: the colours in ``COLOR_SEQUENCE`` (reversed
    when ``reverse``); every box of a colour is solved from the colour's starting
    residual, then all are updated (block Jacobi inside a colour; a colour's boxes
    share no unknown)."""
    from .ib_oracle import COLOR_SEQUENCE

    w = w.copy()
    for c in (COLOR_SEQUENCE[::-1] if reverse else COLOR_SEQUENCE):
        r = rhs - level.A @ w
        for idx, rows, inv in level.colors[c]:
            w[idx] += inv @ r[idx]
    return w


def cavity_coarse_solve(level, rhs):
    """Exact coarsest solve, bordered with a zero-mean pressure (Algorithm 1)."""
    N = level.N
    A = level.A.toarray()
    z = np.zeros(A.shape[0])
    z[2 * N * N:] = 1.0
    M = np.block([[A, z[:, None]], [z[None, :], np.zeros((1, 1))]])
    rhs2 = rhs if rhs.ndim == 2 else rhs[:, None]
    sol = np.linalg.solve(M, np.vstack([rhs2, np.zeros((1, rhs2.shape[1]))]))[: A.shape[0]]
    return sol if rhs.ndim == 2 else sol[:, 0]


def cavity_vcycle(levels, rhs, w, nu1=1, nu2=1, li=0):
    """MGV(w, rhs) of Algorithm 1 with box smoothing before and after the
    coarse-grid correction: lexicographic (the same order both times), or the
    colour order (post-smoothing in reverse for 1 x 1 boxes, as
    ``ib_oracle.post_reversed``)."""
    from .ib_oracle import post_reversed

    lev = levels[li]
    if li == len(levels) - 1:
        return cavity_coarse_solve(lev, rhs)
    color = getattr(lev, "order", "lex") == "color4"
    for _ in range(nu1):
        w = cavity_smooth_color4(lev, rhs, w) if color else cavity_smooth_lex(lev, rhs, w)
    rc = lev.R @ (rhs - lev.A @ w)
    w = w + lev.P @ cavity_vcycle(levels, rc, np.zeros_like(rc), nu1, nu2, li + 1)
    for _ in range(nu2):
        w = (cavity_smooth_color4(lev, rhs, w, reverse=post_reversed(lev.b)) if color
             else cavity_smooth_lex(lev, rhs, w))
    return w


def lid_rhs(N, mu=1.0, L=1.0):
    """The lid-driven cavity's right-hand side: the top wall's tangential velocity
    u(x, 1) = (1 - cos 2 pi x) / 2 (sec. 4) enters the row of u faces next to it
    through the ghost value 2 u_lid - u (the wall value is the mean of the two)."""
    h = L / N
    b = np.zeros(3 * N * N)
    i = np.arange(1, N)
    b[u_index(N, i, N - 1)] = -2.0 * mu * 0.5 * (1.0 - np.cos(2.0 * np.pi * i * h)) / (h * h)
    return b


def cavity_rhs(N, levels, ann=None, weight="ds1^2", force_scale=1.0):
    """b = [-force_scale S A_f X^n + lid terms; 0] (the system of sec. 3,
    Eq. "matrixeq", with the cavity's lid)."""
    ann = Annulus(N) if ann is None else ann
    wts = {"ds1ds2": ann.ds1 * ann.ds2, "ds1^2": ann.ds1 ** 2, "ds2^2": ann.ds2 ** 2}
    X = ann.points()
    S = spread_matrix(X, N, wts[weight])
    Xv = np.concatenate([X[:, 0], X[:, 1]])
    b = lid_rhs(N)
    b[: 2 * N * N] -= force_scale * (S @ (force_operator(ann) @ Xv))
    b[wall_rows(N)] = 0.0
    return b


def cavity_mg_solve(levels, b, tol=1e-6, max_cycles=100, nu1=1, nu2=1):
    """Multigrid as a stand-alone solver from w = 0 (sec. 5): the number of V-cycles
    until ||b - A w|| <= tol ||b||, or None if max_cycles do not get there."""
    A = levels[0].A
    w = np.zeros_like(b)
    bn = np.linalg.norm(b)
    for k in range(1, max_cycles + 1):
        w = cavity_vcycle(levels, b, w, nu1, nu2)
        rn = np.linalg.norm(b - A @ w)
        if not np.isfinite(rn):
            return None
        if rn <= tol * bn:
            return k
    return None


def cavity_mg_gmres(levels, b, tol=1e-6, max_iters=100, nu1=1, nu2=1):
    """GMRES right-preconditioned by one V-cycle from zero (sec. 3.3, sec. 5),
    from w = 0; returns the oracle's SolveResult."""
    from .ib_oracle import fgmres

    def M(v):
        return cavity_vcycle(levels, v, np.zeros_like(v), nu1, nu2)

    return fgmres(levels[0].A, b, M, tol=tol, max_iters=max_iters, max_restarts=0)


def cavity_iteration_matrix(levels, nu1=1, nu2=1):
    """The stand-alone multigrid's iteration matrix (sec. 5, spectrum): column k is
    one V-cycle with a zero right-hand side applied to the k-th unit vector of the
    unknowns (the wall faces, which are not unknowns, left out).  All columns go
    through the cycle together.  Returns (M, indices of the unknowns)."""
    N = levels[0].N
    n = 3 * N * N
    free = np.setdiff1d(np.arange(n), wall_rows(N))
    W = np.zeros((n, free.size))
    W[free, np.arange(free.size)] = 1.0
    out = cavity_vcycle(levels, np.zeros_like(W), W, nu1, nu2)
    return out[free], free


def cavity_spectrum(M, N):
    """Eigenvalues of the iteration matrix on the unknowns with zero-mean pressure
    (sec. 5: the constant pressure is a trivial eigenvector with eigenvalue 1).
    The pressure unknowns are the last N^2 of M's rows and columns."""
    m = M.shape[0]
    n = N * N
    Q = np.eye(m)
    Q[m - n:, m - n:] -= 1.0 / n
    return np.linalg.eigvals(Q @ M @ Q)
