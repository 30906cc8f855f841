"""Plain FP64 CPU oracle of one implicit immersed-boundary step.

TEST INFRASTRUCTURE ONLY.  This module is the independent reference the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library never does.  It
shares no code, tables or helpers with the CUDA path; the only shared module is
``ib_workloads`` (seeded geometry, no method arithmetic).

What it computes (Guy, Philip & Griffith, "Geometric multigrid for an
implicit-time immersed boundary method"):

* the staggered (MAC) Stokes operator, sec. 2.2 (Delta_h, grad_h, div_h);
* the regularised delta function, spreading S_h and interpolation S_h^*,
  sec. 2.2 (delta and spreading/interpolation equations);
* the backward-Euler step with lagged S, and the elimination of the
  Lagrangian unknowns onto the grid, sec. 2.3.2 (Eqs. 17-22 and the block
  system "matrixeq");
* the staggered restriction / prolongation of sec. 3.1, the hybrid coarse
  operator of sec. 3.2 (re-discretised Stokes + Galerkin elasticity);
* the V-cycle of Algorithm 1 with the box (Vanka) smoother of sec. 5 and the
  n x n "big boxes" of sec. 6, exact coarsest solve on N_c = max(4, n);
* flexible GMRES with the V-cycle as right preconditioner, sec. 3.3;
* the position update X^{n+1} = X^n + dt S^* u^{n+1}, Eq. 20;
* the same step with the spring force taken at X^{n+1} (a nonlinear step),
  solved by Newton's method over linearised systems of the same form (sec. 8).

Everything is assembled as explicit sparse matrices (scipy CSR) and applied
with plain matrix-vector products; box matrices are principal submatrices of
the assembled level operator, solved with LAPACK (partial pivoting).

Readings where the paper is silent or differs from the workloads (each is
also listed in the design notes):

* periodic unit square instead of the lid-driven cavity;
* time-dependent momentum operator mu*Delta - (rho/dt) I (the paper's
  discussion names I - dt*Delta - dt^2*gamma*S A_f S^* as the unsteady form;
  rho = 0 gives the paper's steady system exactly);
* point springs with rest length, linearised once per step about X^n
  (sec. 8 allows semi-implicit linearisation of nonlinear laws); the default
  Jacobian is clamped to be negative semidefinite; with zero rest length both
  variants equal kappa * A_f exactly;
* the right-hand side is -S F(X^n) - (rho/dt) u^n (the paper's Eq. 21 omits the
  stiffness factor gamma in front of S A_f X^n; the force F = gamma A_f X is
  what the elimination produces);
* the 1-D cosine kernel is read as (1 + cos(pi r / (2h))) / (4h) for |r| < 2h;
* the Peskin 4-point kernel (Peskin, Acta Numerica 2002) is the default;
* boxes are visited either lexicographically with in-place updates (the
  paper's block Gauss-Seidel) or in four colours (2 x 2 box parity) with
  block-Jacobi semantics inside a colour ("color4", the parallel order);
  color4 pre-smooths in the colour sequence (even,even), (odd,odd),
  (odd,even), (even,odd) and post-smooths in the reverse sequence for 1 x 1
  boxes and in the same sequence for larger boxes (the choice that measured
  the best V-cycle contraction for each box size; see post_reversed).

Pins (tests/test_oracle_pins.py) fix each part against the paper or the
mathematics: delta-kernel moments and golden values, the S / S^* adjoint and
conservation, spring force sums and finite-difference Jacobians, manufactured
Stokes solutions (second order), transfer identities, E symmetric and
negative semidefinite, the box count and free-box identity, the colour
sweep solving its last colour's n x n boxes exactly (pure Stokes), the block-
Jacobi update inside a colour (with structure, the sweep does not depend on
the order of a colour's boxes; a colour's boxes share no unknown), V-cycle
contraction, FGMRES against a dense direct solve at 16 x 16, flat iteration
counts under refinement, the paper's trends (sec. 6: bigger boxes and more
smoothing sweeps take fewer iterations, the 1 x 1 box smoother fails on very
stiff structures, and under refinement a stiff problem's count grows with
1 x 1 boxes and stays flat with 8 x 8 ones), the stand-alone multigrid solver's contraction equal to the
spectral radius of its iteration matrix and that spectrum's behaviour with
stiffness (sec. 5), the explicit-time operator's real nonpositive spectrum and
translation kernel with alpha_exp falling under refinement (sec. 4.1),
translation and mirror symmetry, energy decay, and the backward-Euler decay
of a discretely divergence-free Fourier mode of u^n by (rho/dt) / (rho/dt +
mu lambda_k) with no structure (the u^n term of the right-hand side).
Parity unpinned: the exact iteration counts of the periodic workloads (the
paper prints counts only for its lid-driven-cavity problem, and sweeps its
boxes in lexicographic order where this oracle, like the GPU path, uses four
colours).

Vector layout: w = [u | v | p], each an N x N array, row-major with x fastest
(index j*N + i).  u[j, i] sits at (i h, (j + 1/2) h), v[j, i] at
((i + 1/2) h, j h), p[j, i] at ((i + 1/2) h, (j + 1/2) h).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# ----------------------------------------------------------------------------
# 1-D regularised delta kernels (sec. 2.2).  phi is dimensionless: delta_h^1(r)
# = phi(r / h) / h.
# ----------------------------------------------------------------------------


def phi_peskin4(r):
    """Peskin's 4-point kernel (Acta Numerica 2002), support |r| < 2."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(r)
    a = r < 1.0
    b = (r >= 1.0) & (r < 2.0)
    ra = r[a]
    rb = r[b]
    out[a] = (3.0 - 2.0 * ra + np.sqrt(1.0 + 4.0 * ra - 4.0 * ra * ra)) / 8.0
    out[b] = (5.0 - 2.0 * rb - np.sqrt(np.maximum(-7.0 + 12.0 * rb - 4.0 * rb * rb, 0.0))) / 8.0
    return out


def phi_cos4(r):
    """Cosine kernel of sec. 2.2: (1 + cos(pi r / 2)) / 4 for |r| < 2 (r in units of h)."""
    r = np.asarray(r, dtype=np.float64)
    out = np.where(np.abs(r) < 2.0, 0.25 * (1.0 + np.cos(0.5 * np.pi * r)), 0.0)
    return out


KERNELS = {"peskin4": phi_peskin4, "cos4": phi_cos4}

# ----------------------------------------------------------------------------
# Grid indexing
# ----------------------------------------------------------------------------


def uidx(N, i, j):
    return (np.asarray(j) % N) * N + (np.asarray(i) % N)


def vidx(N, i, j):
    return N * N + (np.asarray(j) % N) * N + (np.asarray(i) % N)


def pidx(N, i, j):
    return 2 * N * N + (np.asarray(j) % N) * N + (np.asarray(i) % N)


def _wrap(d, n):
    """Minimum-image representative of d on a periodic line of length n."""
    return d - n * np.round(d / n)


# ----------------------------------------------------------------------------
# Spreading and interpolation (sec. 2.2)
# ----------------------------------------------------------------------------


def spread_matrix(X, N, L, kernel="peskin4"):
    """S_h as a (2N^2) x (2Np) CSR matrix.

    Rows: u faces then v faces.  Columns: x-components of all points, then
    y-components.  Entry = delta_h(x_face - X_k) = phi(dx/h) phi(dy/h) / h^2, with
    periodic minimum-image displacement.  Point forces: the Lagrangian measure
    (ds^2 in the paper's force-density form) is already inside F.
    """
    phi = KERNELS[kernel]
    X = np.asarray(X, dtype=np.float64)
    Np = X.shape[0]
    h = L / N
    grid = np.arange(N, dtype=np.float64)
    rows, cols, vals = [], [], []
    for comp, (ox, oy) in enumerate(((0.0, 0.5), (0.5, 0.0))):
        for k in range(Np):
            # 1-D weights over all grid lines (tensor-product kernel)
            wx = phi(_wrap((grid + ox) - X[k, 0] / h, N))
            wy = phi(_wrap((grid + oy) - X[k, 1] / h, N))
            ii = np.nonzero(wx)[0]
            jj = np.nonzero(wy)[0]
            W = np.outer(wy[jj], wx[ii]) / (h * h)
            J2, I2 = np.meshgrid(jj, ii, indexing="ij")
            r = comp * N * N + J2 * N + I2
            rows.append(r.ravel())
            cols.append(np.full(r.size, comp * Np + k))
            vals.append(W.ravel())
    if Np == 0:  # no structure: an empty operator
        return sp.csr_matrix((2 * N * N, 0))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * N * N, 2 * Np))


def interp_matrix(S, h):
    """S_h^* = h^2 S_h^T: U_k = sum over faces of u * delta_h(x - X_k) * h^2 (sec. 2.2)."""
    return (S.T * (h * h)).tocsr()


# ----------------------------------------------------------------------------
# Springs: force F(X) and Jacobian J = dF/dX (sec. 2.2 force law, sec. 8
# linearisation of nonlinear laws)
# ----------------------------------------------------------------------------


def _min_image(d, L):
    return d - L * np.round(d / L)


def spring_force(X, springs, kappa, rest, L):
    """F_i = sum over springs (i, j) of kappa (1 - L0 / l) (X_j - X_i), and the opposite on j."""
    X = np.asarray(X, dtype=np.float64)
    F = np.zeros_like(X)
    for e in range(springs.shape[0]):
        i, j = int(springs[e, 0]), int(springs[e, 1])
        d = _min_image(X[j] - X[i], L)
        l = math.hypot(d[0], d[1])
        f = kappa[e] * (1.0 - rest[e] / l) * d
        F[i] += f
        F[j] -= f
    return F


def spring_block(d, kap, L0, clamped):
    """2x2 block K_e with dF_i/dX_j = K_e for the spring's displacement d = X_j - X_i.

    Exact derivative: kappa [ (1 - L0/l)(I - t t^T) + t t^T ], t = d / l.
    Clamped: the transverse factor (1 - L0/l) replaced by max(0, 1 - L0/l), which
    keeps K_e positive semidefinite (J negative semidefinite).
    """
    l = math.hypot(d[0], d[1])
    t = d / l
    tt = np.outer(t, t)
    s = 1.0 - L0 / l
    if clamped:
        s = max(0.0, s)
    return kap * (s * (np.eye(2) - tt) + tt)


def spring_jacobian(X, springs, kappa, rest, L, clamped=True):
    """J = dF/dX as a (2Np) x (2Np) CSR matrix in the [x-block; y-block] layout."""
    X = np.asarray(X, dtype=np.float64)
    Np = X.shape[0]
    rows, cols, vals = [], [], []
    for e in range(springs.shape[0]):
        i, j = int(springs[e, 0]), int(springs[e, 1])
        d = _min_image(X[j] - X[i], L)
        K = spring_block(d, kappa[e], rest[e], clamped)
        for a in range(2):
            for b in range(2):
                # dF_i/dX_j = K, dF_i/dX_i = -K, dF_j/dX_i = K, dF_j/dX_j = -K
                for (r, c, s) in ((i, j, 1.0), (i, i, -1.0), (j, i, 1.0), (j, j, -1.0)):
                    rows.append(a * Np + r)
                    cols.append(b * Np + c)
                    vals.append(s * K[a, b])
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * Np, 2 * Np))


def elastic_energy(X, springs, kappa, rest, L):
    """Sum over springs of kappa/2 (l - L0)^2."""
    e = 0.0
    for s in range(springs.shape[0]):
        i, j = int(springs[s, 0]), int(springs[s, 1])
        d = _min_image(X[j] - X[i], L)
        e += 0.5 * kappa[s] * (math.hypot(d[0], d[1]) - rest[s]) ** 2
    return e


# ----------------------------------------------------------------------------
# MAC Stokes operator (sec. 2.2), re-discretised on every level (sec. 3.2)
# ----------------------------------------------------------------------------


def stokes_matrix(N, h, mu, rho, dt):
    """[[mu Lap - (rho/dt) I, -G], [D, 0]] on the periodic N x N MAC grid, CSR.

    (Lap u)_{i,j} = (u_{i+1,j} + u_{i-1,j} + u_{i,j+1} + u_{i,j-1} - 4 u_{i,j}) / h^2
    (G p) on the u face (i, j) = (p_{i,j} - p_{i-1,j}) / h, on the v face (i, j) =
    (p_{i,j} - p_{i,j-1}) / h;  (D w)_{i,j} = (u_{i+1,j} - u_{i,j} + v_{i,j+1} - v_{i,j}) / h.
    """
    n = N * N
    I, J = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    I = I.ravel()
    J = J.ravel()
    rows, cols, vals = [], [], []

    def add(r, c, v):
        rows.append(np.asarray(r).ravel())
        cols.append(np.asarray(c).ravel())
        vals.append(np.broadcast_to(np.asarray(v, dtype=np.float64), np.asarray(r).shape).ravel())

    diag = -4.0 * mu / (h * h) - (rho / dt if rho != 0.0 else 0.0)
    off = mu / (h * h)
    for idx in (uidx, vidx):
        r = idx(N, I, J)
        add(r, r, diag)
        add(r, idx(N, I + 1, J), off)
        add(r, idx(N, I - 1, J), off)
        add(r, idx(N, I, J + 1), off)
        add(r, idx(N, I, J - 1), off)
    # -G p
    ru = uidx(N, I, J)
    add(ru, pidx(N, I, J), -1.0 / h)
    add(ru, pidx(N, I - 1, J), 1.0 / h)
    rv = vidx(N, I, J)
    add(rv, pidx(N, I, J), -1.0 / h)
    add(rv, pidx(N, I, J - 1), 1.0 / h)
    # D w
    rp = pidx(N, I, J)
    add(rp, uidx(N, I + 1, J), 1.0 / h)
    add(rp, uidx(N, I, J), -1.0 / h)
    add(rp, vidx(N, I, J + 1), 1.0 / h)
    add(rp, vidx(N, I, J), -1.0 / h)
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(3 * n, 3 * n))
    A.sum_duplicates()
    return A


# ----------------------------------------------------------------------------
# Grid transfers (sec. 3.1)
# ----------------------------------------------------------------------------


def restriction_matrix(Nf):
    """I_{2h<-h} for [u|v|p] from an Nf grid to Nf/2, CSR of shape (3Nc^2, 3Nf^2).

    p: average of the four fine cells.  u: full weighting (1,2,1)/4 across the
    faces normal to x (fine faces 2I-1, 2I, 2I+1) times two-point averaging of
    the fine rows 2J, 2J+1; together the 1/8 [1 2 1; 1 2 1] stencil.  v: the same
    with x and y exchanged.
    """
    Nc = Nf // 2
    I, J = np.meshgrid(np.arange(Nc), np.arange(Nc), indexing="xy")
    I = I.ravel()
    J = J.ravel()
    rows, cols, vals = [], [], []
    for a, wa in ((-1, 0.25), (0, 0.5), (1, 0.25)):
        for b in (0, 1):
            rows.append(uidx(Nc, I, J))
            cols.append(uidx(Nf, 2 * I + a, 2 * J + b))
            vals.append(np.full(I.size, wa * 0.5))
            rows.append(vidx(Nc, I, J))
            cols.append(vidx(Nf, 2 * I + b, 2 * J + a))
            vals.append(np.full(I.size, wa * 0.5))
    for a in (0, 1):
        for b in (0, 1):
            rows.append(pidx(Nc, I, J))
            cols.append(pidx(Nf, 2 * I + a, 2 * J + b))
            vals.append(np.full(I.size, 0.25))
    R = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(3 * Nc * Nc, 3 * Nf * Nf))
    R.sum_duplicates()
    return R


def prolongation_matrix(Nc):
    """I_{h<-2h} for [u|v|p] from an Nc grid to 2Nc, CSR of shape (3Nf^2, 3Nc^2).

    p: constant (each fine cell takes its coarse cell's value).  u: linear in x
    (fine face 2I copies coarse face I; fine face 2I+1 averages coarse faces I and
    I+1) times linear in y between the cell-centred rows (fine row 2J: 3/4 coarse
    row J + 1/4 row J-1; fine row 2J+1: 3/4 row J + 1/4 row J+1).  v: x and y
    exchanged.  This is the bilinear interpolation of sec. 3.1 on the staggered
    positions.
    """
    Nf = 2 * Nc
    i, j = np.meshgrid(np.arange(Nf), np.arange(Nf), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    rows, cols, vals = [], [], []

    def normal_weights(k):
        # (coarse index, weight) pairs along the face-normal direction
        if k % 2 == 0:
            return [(k // 2, 1.0)]
        return [((k - 1) // 2, 0.5), ((k + 1) // 2, 0.5)]

    def centred_weights(k):
        K = k // 2
        if k % 2 == 0:
            return [(K, 0.75), (K - 1, 0.25)]
        return [(K, 0.75), (K + 1, 0.25)]

    for f in range(i.size):
        fi, fj = int(i[f]), int(j[f])
        for (ci, wi) in normal_weights(fi):
            for (cj, wj) in centred_weights(fj):
                rows.append(int(uidx(Nf, fi, fj)))
                cols.append(int(uidx(Nc, ci, cj)))
                vals.append(wi * wj)
        for (cj, wj) in normal_weights(fj):
            for (ci, wi) in centred_weights(fi):
                rows.append(int(vidx(Nf, fi, fj)))
                cols.append(int(vidx(Nc, ci, cj)))
                vals.append(wi * wj)
        rows.append(int(pidx(Nf, fi, fj)))
        cols.append(int(pidx(Nc, fi // 2, fj // 2)))
        vals.append(1.0)
    P = sp.csr_matrix((vals, (rows, cols)), shape=(3 * Nf * Nf, 3 * Nc * Nc))
    P.sum_duplicates()
    return P


def velocity_block(M, Na, Nb):
    """The [u|v] x [u|v] block of a 3-component transfer matrix."""
    return M[: 2 * Na * Na, : 2 * Nb * Nb].tocsr()


# ----------------------------------------------------------------------------
# Level hierarchy (sec. 3.2): re-discretised Stokes + Galerkin elasticity
# ----------------------------------------------------------------------------


@dataclass
class Level:
    N: int
    h: float
    A: sp.csr_matrix                  # full level operator [K + dt E, -G; D, 0]
    E: sp.csr_matrix                  # elasticity block S J S^* (Galerkin coarsened), 2N^2 x 2N^2
    R: sp.csr_matrix | None = None    # restriction to the next coarser level
    P: sp.csr_matrix | None = None    # prolongation from the next coarser level
    boxes: dict = field(default_factory=dict)


def coarsest_size(b):
    """N_c = max(4, b) (sec. 6.1)."""
    return max(4, b)


def level_sizes(N, b):
    Nc = coarsest_size(b)
    out = [N]
    while out[-1] > Nc:
        out.append(out[-1] // 2)
    return out


def fine_elasticity(prob, X=None, Xj=None):
    """E_0 = S J S^* on the finest grid (the block alpha S A_f S^* of the paper's system).
    S at the points X; the springs' Jacobian J at Xj (default: X as well)."""
    X = prob.X if X is None else X
    Xj = X if Xj is None else Xj
    N, L = prob.N, prob.L
    h = L / N
    S = spread_matrix(X, N, L, prob.delta)
    Ss = interp_matrix(S, h)
    Jm = spring_jacobian(Xj, prob.springs, prob.kappa, prob.rest, L, prob.clamped)
    return (S @ Jm @ Ss).tocsr(), S, Ss, Jm


def with_elasticity(Astokes, E, dt, N):
    """Add dt * E to the velocity block of a level's Stokes operator."""
    n2 = 2 * N * N
    n3 = 3 * N * N
    Ebig = sp.bmat([[E, None], [None, sp.csr_matrix((N * N, N * N))]], format="csr")
    assert Ebig.shape == (n3, n3) and E.shape == (n2, n2)
    return (Astokes + dt * Ebig).tocsr()


def build_hierarchy(prob, X=None, Xj=None):
    """Levels N, N/2, ..., N_c with A_l = Stokes_l + dt E_l, E_{l+1} = R E_l P (S at X,
    the springs' Jacobian at Xj, default X)."""
    sizes = level_sizes(prob.N, prob.box)
    E, S, Ss, Jm = fine_elasticity(prob, X, Xj)
    levels = []
    for li, N in enumerate(sizes):
        h = prob.L / N
        As = stokes_matrix(N, h, prob.mu, prob.rho, prob.dt)
        lev = Level(N=N, h=h, A=with_elasticity(As, E, prob.dt, N), E=E)
        if li + 1 < len(sizes):
            lev.R = restriction_matrix(N)
            lev.P = prolongation_matrix(N // 2)
            Rv = velocity_block(lev.R, N // 2, N)
            Pv = velocity_block(lev.P, N, N // 2)
            E = (Rv @ E @ Pv).tocsr()
        levels.append(lev)
    return levels, dict(S=S, Ss=Ss, J=Jm)


# ----------------------------------------------------------------------------
# Box smoother (sec. 5, sec. 6)
# ----------------------------------------------------------------------------


def box_unknowns(N, b, I, J):
    """Indices of the unknowns of the b x b box (I, J): all its u faces, v faces and cells.

    u faces i = Ib..Ib+b, rows j = Jb..Jb+b-1; v faces i = Ib..Ib+b-1, j = Jb..Jb+b;
    cells Ib..Ib+b-1 x Jb..Jb+b-1.  2b(b+1) + b^2 unknowns (sec. 8).
    Order: u (row-major), v (row-major), p (row-major).
    """
    x0, y0 = I * b, J * b
    out = []
    for j in range(y0, y0 + b):
        for i in range(x0, x0 + b + 1):
            out.append(int(uidx(N, i, j)))
    for j in range(y0, y0 + b + 1):
        for i in range(x0, x0 + b):
            out.append(int(vidx(N, i, j)))
    for j in range(y0, y0 + b):
        for i in range(x0, x0 + b):
            out.append(int(pidx(N, i, j)))
    return np.array(out, dtype=np.int64)


def box_color(I, J):
    """Colour of box (I, J) in the 2x2 parity colouring: (I mod 2) + 2 (J mod 2)."""
    return (I % 2) + 2 * (J % 2)


# Colour sequence of one forward sweep: (even, even), (odd, odd), (odd, even),
# (even, odd) box parities.
COLOR_SEQUENCE = (0, 3, 1, 2)


def post_reversed(b):
    """Whether post-smoothing visits the colours in reverse.  1 x 1 boxes of one
    colour are coupled through the stencil (block Jacobi inside a colour) and
    contract best with the reversed (symmetric) sequence; n x n boxes (n >= 2) of
    one colour are uncoupled and contract best with the same sequence."""
    return b == 1


def submatrices(A, idx):
    """Dense principal submatrices A[idx_k, idx_k] for a batch of index sets idx [nb, m]."""
    nb, m = idx.shape
    r = np.repeat(idx, m, axis=1).ravel()
    c = np.tile(idx, (1, m)).ravel()
    vals = np.asarray(A[r, c]).ravel()
    return vals.reshape(nb, m, m)


def prepare_boxes(level, b):
    """Box index sets per colour and their dense A_BB blocks (setup, once per step)."""
    N = level.N
    nbx = N // b
    per_color = {}
    for c in range(4):
        idx = []
        for J in range(nbx):
            for I in range(nbx):
                if box_color(I, J) == c:
                    idx.append(box_unknowns(N, b, I, J))
        idx = np.array(idx)
        per_color[c] = (idx, submatrices(level.A, idx))
    lex = np.array([box_unknowns(N, b, I, J) for J in range(nbx) for I in range(nbx)])
    level.boxes = dict(color=per_color, lex=lex, lexA=submatrices(level.A, lex), b=b)
    return level.boxes


def smooth_color4(level, rhs, w, reverse=False):
    """One sweep over the colours in COLOR_SEQUENCE (reversed when ``reverse``);
    inside a colour every box is solved from the colour's starting state (block
    Jacobi), then all its corrections are added.  Boxes of one colour share no
    unknowns, so the updates do not overlap."""
    w = w.copy()
    for c in (COLOR_SEQUENCE[::-1] if reverse else COLOR_SEQUENCE):
        idx, Abb = level.boxes["color"][c]
        r = rhs - level.A @ w
        delta = np.linalg.solve(Abb, r[idx][..., None])[..., 0]
        w[idx] += delta
    return w


def smooth_lex(level, rhs, w, reverse=False):
    """One sweep of the paper's order: boxes row by row (x fastest), each solved from the
    current iterate and updated in place (block Gauss-Seidel, sec. 5).  The paper
    uses the same order before and after the coarse correction; ``reverse`` is
    accepted and ignored."""
    w = w.copy()
    A = level.A
    for k in range(level.boxes["lex"].shape[0]):
        idx = level.boxes["lex"][k]
        r = rhs[idx] - A[idx, :] @ w
        w[idx] += np.linalg.solve(level.boxes["lexA"][k], r)
    return w


# ----------------------------------------------------------------------------
# Coarsest solve (Algorithm 1, first branch)
# ----------------------------------------------------------------------------


def nullspace_basis(N, rho):
    """Columns spanning the constant pressure (and, with rho = 0, constant u and v)."""
    n = N * N
    cols = []
    comps = (2,) if rho != 0.0 else (0, 1, 2)
    for c in comps:
        e = np.zeros(3 * n)
        e[c * n:(c + 1) * n] = 1.0
        cols.append(e)
    return np.stack(cols, axis=1)


def coarse_solve(level, rhs, rho):
    """Exact solve of A w = rhs, bordered with zero mean of the null-space components."""
    A = level.A.toarray()
    Z = nullspace_basis(level.N, rho)
    k = Z.shape[1]
    M = np.block([[A, Z], [Z.T, np.zeros((k, k))]])
    sol = np.linalg.solve(M, np.concatenate([rhs, np.zeros(k)]))
    return sol[: A.shape[0]]


# ----------------------------------------------------------------------------
# V-cycle (Algorithm 1 of the paper; sec. 3)
# ----------------------------------------------------------------------------


def vcycle(levels, rhs, w, nu1=1, nu2=1, rho=1.0, order="color4", li=0):
    """MGV(w, rhs) on level li as a composition of three maps of the iterate:
    nu2 smoothing sweeps after the coarse-grid correction after nu1 smoothing sweeps.
    The coarse-grid correction adds P e, e the same cycle applied on the next level to
    the restricted residual from a zero start; on the coarsest level the cycle is the
    exact (bordered) solve."""
    lev = levels[li]
    if li == len(levels) - 1:
        return coarse_solve(lev, rhs, rho)
    smooth = smooth_color4 if order == "color4" else smooth_lex

    def sweeps(x, n, reverse=False):
        for _ in range(n):
            x = smooth(lev, rhs, x, reverse=reverse)
        return x

    def coarse_correction(x):
        rc = lev.R @ (rhs - lev.A @ x)
        return x + lev.P @ vcycle(levels, rc, np.zeros_like(rc), nu1, nu2, rho, order, li + 1)

    return sweeps(coarse_correction(sweeps(w, nu1)), nu2, reverse=post_reversed(lev.boxes["b"]))


# ----------------------------------------------------------------------------
# Flexible GMRES, right preconditioned (sec. 3.3)
# ----------------------------------------------------------------------------


@dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    rel_res_true: float
    history: list
    converged: bool


def fgmres(A, b, precond, tol=1e-8, max_iters=100, x0=None, max_restarts=3):
    """Flexible GMRES with classical Gram-Schmidt applied twice and Givens rotations.

    Stops when the Givens residual estimate falls below tol * ||b||, then
    confirms with the true residual ||b - A x|| / ||b||; restarts from x if the
    true residual is above tol.
    """
    n = b.size
    bnorm = np.linalg.norm(b)
    x = np.zeros(n) if x0 is None else x0.copy()
    if bnorm == 0.0:
        return SolveResult(x, 0, 0.0, [0.0], True)
    history = []
    total = 0
    for _restart in range(max_restarts + 1):
        r = b - A @ x
        beta = np.linalg.norm(r)
        history.append(beta / bnorm)
        if beta <= tol * bnorm:
            return SolveResult(x, total, beta / bnorm, history, True)
        m = max_iters - total
        if m <= 0:
            break
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_done = 0
        for j in range(m):
            Z[j] = precond(V[j])
            wv = A @ Z[j]
            h1 = V[: j + 1] @ wv
            wv = wv - V[: j + 1].T @ h1
            h2 = V[: j + 1] @ wv
            wv = wv - V[: j + 1].T @ h2
            H[: j + 1, j] = h1 + h2
            H[j + 1, j] = np.linalg.norm(wv)
            if H[j + 1, j] > 0.0:
                V[j + 1] = wv / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            k_done = j + 1
            history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm:
                break
        y = np.zeros(k_done)
        for i in range(k_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k_done] @ y[i + 1:]) / H[i, i]
        x = x + Z[:k_done].T @ y
        rt = np.linalg.norm(b - A @ x) / bnorm
        if rt <= tol:
            return SolveResult(x, total, rt, history, True)
        if total >= max_iters:
            break
    rt = np.linalg.norm(b - A @ x) / bnorm
    return SolveResult(x, total, rt, history, rt <= tol)


# ----------------------------------------------------------------------------
# The implicit step (sec. 2.3)
# ----------------------------------------------------------------------------


def rhs_vector(prob, u_n=None, X=None):
    """b = [-(rho/dt) u^n - S F(X^n); 0] (the right-hand side of the eliminated system)."""
    X = prob.X if X is None else X
    N = prob.N
    S = spread_matrix(X, N, prob.L, prob.delta)
    F = spring_force(X, prob.springs, prob.kappa, prob.rest, prob.L)
    Fv = np.concatenate([F[:, 0], F[:, 1]])
    b = np.zeros(3 * N * N)
    b[: 2 * N * N] = -(S @ Fv)
    if u_n is not None and prob.rho != 0.0:
        b[: 2 * N * N] -= (prob.rho / prob.dt) * np.asarray(u_n, dtype=np.float64).ravel()[: 2 * N * N]
    return b


def remove_pressure_mean(w, N):
    w = w.copy()
    n = N * N
    w[2 * n:] -= w[2 * n:].mean()
    return w


@dataclass
class StepResult:
    w: np.ndarray          # [u|v|p] at t^{n+1}, zero-mean pressure
    X: np.ndarray          # X^{n+1}
    solve: SolveResult
    b: np.ndarray


def solve_step(prob, u_n=None, order="color4", X=None):
    """One backward-Euler IB step: assemble, MG-preconditioned FGMRES, move the points."""
    X = prob.X if X is None else np.asarray(X, dtype=np.float64)
    levels, ops = build_hierarchy(prob, X)
    for lev in levels[:-1]:
        prepare_boxes(lev, prob.box)
    b = rhs_vector(prob, u_n, X)

    def M(v):
        return vcycle(levels, v, np.zeros_like(v), prob.nu1, prob.nu2, prob.rho, order)

    res = fgmres(levels[0].A, b, M, prob.tol, prob.max_iters)
    w = remove_pressure_mean(res.x, prob.N)
    N = prob.N
    U = ops["Ss"] @ w[: 2 * N * N]
    Np = X.shape[0]
    Xn = X + prob.dt * np.stack([U[:Np], U[Np:]], axis=1)
    return StepResult(w=w, X=Xn, solve=res, b=b)


@dataclass
class NewtonResult:
    w: np.ndarray          # [u|v|p] at t^{n+1}, zero-mean pressure
    X: np.ndarray          # X^{n+1}
    iters: int             # Newton iterations (linear solves)
    changes: list          # max |X^{k+1} - X^k| / h after each iteration (the first: the step)
    linear_iters: list     # FGMRES iterations of each linear solve


def solve_step_newton(prob, u_n=None, order="color4", X=None, max_newton=20, tol=1e-9):
    """The backward-Euler step with the spring force at the new positions, solved by
    Newton's method (sec. 8 names Newton's method for nonlinear force laws; it
    solves a sequence of linearised systems of the form of the linearised step).

    Unknowns u^{n+1}, p^{n+1}; S and S^* stay at X^n (lagged, sec. 2.3); with
    X(u) = X^n + dt S^* u the equations are
        mu Lap u - (rho/dt) u - G p + S F(X(u)) = -(rho/dt) u^n,   D u = 0.
    Iteration k linearises F about X^k = X(u^k):
        F(X) ~ F(X^k) + J(X^k) (X - X^k),  X - X^k = dt S^* (u - u^k),
    so u^{k+1} solves the linearised step's operator with J(X^k) in place of J(X^n)
    and the right-hand side -(rho/dt) u^n - S [F(X^k) - J(X^k)(X^k - X^n)]
    (X^k - X^n = dt S^* u^k).  u^0 = 0, X^0 = X^n: the first iterate is the
    linearised step.  Stops when max |X^{k+1} - X^k| <= tol h (k >= 1) or after
    max_newton solves.  The fixed point does not depend on J (its terms cancel), so
    the clamped Jacobian converges to the same step, only more slowly."""
    Xn = prob.X if X is None else np.asarray(X, dtype=np.float64)
    N, L = prob.N, prob.L
    h = L / N
    n2 = 2 * N * N
    Np = Xn.shape[0]
    S = spread_matrix(Xn, N, L, prob.delta)
    Ss = interp_matrix(S, h)
    Xk = Xn.copy()
    changes, lin = [], []
    w = None
    for k in range(max_newton):
        levels, _ = build_hierarchy(prob, Xn, Xj=Xk)
        for lev in levels[:-1]:
            prepare_boxes(lev, prob.box)
        Fk = spring_force(Xk, prob.springs, prob.kappa, prob.rest, L)
        Jk = spring_jacobian(Xk, prob.springs, prob.kappa, prob.rest, L, prob.clamped)
        d = np.array([_min_image(Xk[i] - Xn[i], L) for i in range(Np)]).reshape(Np, 2)
        Ft = np.concatenate([Fk[:, 0], Fk[:, 1]]) - Jk @ np.concatenate([d[:, 0], d[:, 1]])
        b = np.zeros(3 * N * N)
        b[:n2] = -(S @ Ft)
        if u_n is not None and prob.rho != 0.0:
            b[:n2] -= (prob.rho / prob.dt) * np.asarray(u_n, dtype=np.float64).ravel()[:n2]

        def M(v):
            return vcycle(levels, v, np.zeros_like(v), prob.nu1, prob.nu2, prob.rho, order)

        res = fgmres(levels[0].A, b, M, prob.tol, prob.max_iters)
        lin.append(res.iters)
        w = remove_pressure_mean(res.x, N)
        U = Ss @ w[:n2]
        Xnew = Xn + prob.dt * np.stack([U[:Np], U[Np:]], axis=1)
        changes.append(float(np.abs(Xnew - Xk).max() / h))
        Xk = Xnew
        if k >= 1 and changes[-1] <= tol:
            break
    return NewtonResult(w=w, X=Xk, iters=len(changes), changes=changes, linear_iters=lin)


def direct_solve(A, b, N, rho):
    """Plain definition: dense bordered solve of the full system (small N only)."""
    Ad = A.toarray()
    Z = nullspace_basis(N, rho)
    k = Z.shape[1]
    M = np.block([[Ad, Z], [Z.T, np.zeros((k, k))]])
    sol = np.linalg.solve(M, np.concatenate([b, np.zeros(k)]))
    return sol[: Ad.shape[0]]


# ----------------------------------------------------------------------------
# Multigrid as a stand-alone solver and its iteration matrix (sec. 5)
# ----------------------------------------------------------------------------


def mg_solve(levels, b, tol=1e-8, max_iters=100, nu1=1, nu2=1, rho=1.0, order="color4", x0=None):
    """Multigrid as a solver (sec. 5, solver performance): from x0 (zero by
    default) repeat x <- x + MGV(0, b - A x), one V-cycle per iteration, until
    ||b - A x|| <= tol ||b|| or max_iters cycles."""
    A = levels[0].A
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    history = []
    k = 0
    while True:
        r = b - A @ x
        rel = np.linalg.norm(r) / bnorm if bnorm > 0.0 else 0.0
        history.append(rel)
        if rel <= tol or k == max_iters:
            break
        x = x + vcycle(levels, r, np.zeros_like(r), nu1, nu2, rho, order)
        k += 1
    return SolveResult(x, k, history[-1], history, history[-1] <= tol)


def iteration_matrix(levels, nu1=1, nu2=1, rho=1.0, order="color4"):
    """Multigrid iteration matrix (sec. 5, spectrum): column k is one cycle
    applied to the error e_k (the k-th unit vector) with a zero right-hand
    side, e_k - MGV(0, A e_k).  Dense: small grids only."""
    A = levels[0].A
    n = A.shape[0]
    M = np.empty((n, n))
    e = np.zeros(n)
    for k in range(n):
        e[k] = 1.0
        M[:, k] = e - vcycle(levels, A @ e, np.zeros(n), nu1, nu2, rho, order)
        e[k] = 0.0
    return M


def spectrum_mean_zero_pressure(M, N):
    """Eigenvalues of the iteration matrix on the space of zero-mean pressure
    (sec. 5: a constant pressure is a trivial eigenvector with eigenvalue 1,
    which the paper excludes from the spectral radius).  Returns the eigenvalues
    of Q M Q, Q the orthogonal projector onto that space (the constant pressure
    maps to 0)."""
    n = N * N
    Q = np.eye(3 * n)
    Q[2 * n:, 2 * n:] -= 1.0 / n
    return np.linalg.eigvals(Q @ M @ Q)


# ----------------------------------------------------------------------------
# Explicit-time stability limit (sec. 4.1, characterizing the elastic stiffness)
# ----------------------------------------------------------------------------


def explicit_stiffness_limit(prob, X=None):
    """alpha_exp = 2 / rho(S* L^{-1} S A) (sec. 4.1): the largest alpha = kappa dt
    for which the explicit-time method (forward Euler on dX/dt = S* L^{-1} S F(X))
    is stable.  A is the spring-force Jacobian per unit stiffness (the paper's
    A_f when the rest length is zero); L^{-1} maps a force density to the
    velocity of the steady Stokes system (rho = 0; periodic, so the constant
    velocities and pressure are bordered out).  Returns (alpha_exp, eigenvalues
    of S* L^{-1} S A), which are real and nonpositive.  One sparse LU of the
    Stokes system and a dense eigenproblem in the points: small problems only."""
    X = prob.X if X is None else np.asarray(X, dtype=np.float64)
    N, L = prob.N, prob.L
    h = L / N
    S = spread_matrix(X, N, L, prob.delta)
    Ss = interp_matrix(S, h)
    A = spring_jacobian(X, prob.springs, np.ones(prob.springs.shape[0]), prob.rest, L, prob.clamped)
    Ast = stokes_matrix(N, h, prob.mu, 0.0, prob.dt)
    Z = sp.csr_matrix(nullspace_basis(N, 0.0))
    K = sp.bmat([[Ast, Z], [Z.T, None]], format="csc")
    n2 = 2 * N * N
    rhs = np.zeros((K.shape[0], A.shape[1]))
    rhs[:n2] = -(S @ A).toarray()  # momentum rows carry -f (the system's sign)
    u = spla.splu(K).solve(rhs)[:n2]
    ev = np.linalg.eigvals(Ss @ u)
    return 2.0 / np.abs(ev).max(), ev
