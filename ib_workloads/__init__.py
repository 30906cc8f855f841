"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws geometry and random vectors.  It holds none of the
method's arithmetic: no delta kernel, no operator, no spring law.  Both the CPU
oracle and the CUDA path consume what it produces, so that a parity test feeds
the two sides identical inputs.

Workload recipes (Lagrangian structures immersed in a 2-D periodic box):

* ``single_ellipse``: one closed elastic curve of ``n`` points equally spaced
  in parameter angle on an ellipse, nearest-neighbour springs with a common
  stiffness and rest length.  The standard case is semi-axes 0.28 / 0.22
  centred at (0.5, 0.5) with rest length 2*pi*0.25/n, i.e. the perimeter of
  a circle of radius 0.25 divided by ``n``.
* ``many_ellipses``: ``count`` ellipses with semi-axes drawn from U[lo, hi],
  random rotation, centres drawn uniformly and rejected until no two
  ellipses' bounding circles come within ``4h`` of each other.
* ``batch``: independent problems with grids drawn from a set of sizes, each
  with one ellipse sampled at 4 points per grid cell of perimeter and a
  log-uniform stiffness.
* ``cavity_annulus``: the paper's own test structure (sec. 4), no randomness:
  the thick annulus of inner radius 1/4 and width 1/16 centred at (0.5, 0.5),
  M1 = 19N/8 points on each of M2 = 3N/32 + 1 concentric closed fibres, every
  fibre a closed chain of zero-rest-length springs, in the unit square with
  no-slip walls.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem",
    "ellipse_points",
    "closed_chain",
    "ellipse_perimeter",
    "single_ellipse",
    "many_ellipses",
    "batch",
    "random_field",
    "random_points_field",
    "cavity_annulus",
]


@dataclass
class Problem:
    """One immersed-boundary problem instance (all host arrays, float64/int32)."""

    N: int                     # cells per side (power of two)
    L: float                   # domain side; h = L / N; periodic
    rho: float                 # fluid density (0 -> steady Stokes)
    mu: float                  # viscosity
    dt: float                  # backward-Euler time step
    X: np.ndarray              # [Np, 2] Lagrangian point positions
    springs: np.ndarray        # [Ns, 2] int32 point index pairs
    kappa: np.ndarray          # [Ns] spring stiffness
    rest: np.ndarray           # [Ns] rest lengths
    delta: str = "peskin4"     # "peskin4" or "cos4"
    box: int = 1               # smoother box size b
    nu1: int = 1
    nu2: int = 1
    tol: float = 1e-8
    max_iters: int = 100
    clamped: bool = True       # clamped (negative semidefinite) spring Jacobian
    meta: dict = field(default_factory=dict)

    @property
    def h(self) -> float:
        return self.L / self.N

    @property
    def n_points(self) -> int:
        return int(self.X.shape[0])


def ellipse_points(n, a, b, center=(0.5, 0.5), theta=0.0):
    """Points at parameter angles 2*pi*k/n on an ellipse rotated by ``theta``."""
    t = 2.0 * np.pi * np.arange(n) / n
    x = a * np.cos(t)
    y = b * np.sin(t)
    c, s = math.cos(theta), math.sin(theta)
    X = np.empty((n, 2), dtype=np.float64)
    X[:, 0] = center[0] + c * x - s * y
    X[:, 1] = center[1] + s * x + c * y
    return X


def closed_chain(n, offset=0):
    """Spring list (k, k+1 mod n) of a closed curve whose points start at ``offset``."""
    k = np.arange(n, dtype=np.int32)
    return np.stack([offset + k, offset + (k + 1) % n], axis=1).astype(np.int32)


def ellipse_perimeter(a, b):
    """Ramanujan's approximation of an ellipse perimeter (sizes the batch sampling)."""
    return math.pi * (3.0 * (a + b) - math.sqrt((3.0 * a + b) * (a + 3.0 * b)))


def single_ellipse(N=64, n_points=128, kappa=1e2, dt=1e-2, rho=1.0, mu=1.0, L=1.0,
                   a=0.28, b=0.22, center=(0.5, 0.5), rest=None, **kw):
    """One closed spring curve on an ellipse (the 64^2 / 256^2 workloads)."""
    X = ellipse_points(n_points, a, b, center)
    springs = closed_chain(n_points)
    if rest is None:
        rest = 2.0 * math.pi * 0.25 / n_points
    ns = springs.shape[0]
    return Problem(N=N, L=L, rho=rho, mu=mu, dt=dt, X=X, springs=springs,
                   kappa=np.full(ns, float(kappa)), rest=np.full(ns, float(rest)), **kw)


def cavity_annulus(N, kappa=1.0, dt=1.0, r=0.25, w=1.0 / 16.0, center=(0.5, 0.5), **kw):
    """The thick annulus of sec. 4 at h = 1/N: nodes (xc + (r + s2) cos(s1 / r),
    yc + (r + s2) sin(s1 / r)) for s1 = k ds1 (k < M1 = 19N/8, ds1 = 2 pi r / M1)
    and s2 = l ds2 (l < M2 = 3N/32 + 1, ds2 = w / (M2 - 1)), point l*M1 + k; each
    fibre (fixed l) a closed chain of springs with stiffness kappa and zero rest
    length.  Steady Stokes (rho = 0, mu = 1), the cosine kernel, no-slip walls
    (meta["walls"]).  meta carries M1, M2, ds1, ds2 and the nodes as [M2, M1, 2]."""
    if N % 32 != 0:
        raise ValueError("M1 = 19N/8 and M2 = 3N/32 + 1 need N a multiple of 32")
    M1, M2 = 19 * N // 8, 3 * N // 32 + 1
    ds1, ds2 = 2.0 * math.pi * r / M1, w / (M2 - 1)
    s1 = np.arange(M1) * ds1
    s2 = np.arange(M2) * ds2
    R = r + s2[:, None]
    nodes = np.stack([center[0] + R * np.cos(s1[None, :] / r), center[1] + R * np.sin(s1[None, :] / r)], axis=-1)
    springs = np.concatenate([closed_chain(M1, offset=l * M1) for l in range(M2)])
    ns = springs.shape[0]
    kw.setdefault("delta", "cos4")
    return Problem(N=N, L=1.0, rho=0.0, mu=1.0, dt=dt, X=nodes.reshape(-1, 2).copy(), springs=springs,
                   kappa=np.full(ns, float(kappa)), rest=np.zeros(ns),
                   meta=dict(M1=M1, M2=M2, ds1=ds1, ds2=ds2, nodes=nodes, walls="noslip"), **kw)


def _periodic_dist(p, q, L):
    d = np.abs(np.asarray(p) - np.asarray(q))
    d = np.minimum(d, L - d)
    return float(np.hypot(d[0], d[1]))


def many_ellipses(N=1024, count=16, n_per=2048, lo=0.02, hi=0.06, kappa=1e4, dt=1e-3,
                  seed=1311, rho=1.0, mu=1.0, L=1.0, **kw):
    """``count`` non-overlapping random ellipses (the 1024^2 multi-structure workload).

    Semi-axes a, b ~ U[lo, hi] independently, rotation ~ U[0, pi), centres ~ U[0, L)^2
    with rejection so that |c_i - c_j| >= max(a_i, b_i) + max(a_j, b_j) + 4h
    (periodic distance).  Rest length of each curve: the perimeter of the
    equal-area circle, 2*pi*sqrt(a*b), divided by ``n_per``.
    """
    rng = np.random.default_rng(seed)
    h = L / N
    shapes = []
    tries = 0
    while len(shapes) < count:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place non-overlapping ellipses")
        a, b = rng.uniform(lo, hi, size=2)
        th = rng.uniform(0.0, math.pi)
        c = rng.uniform(0.0, L, size=2)
        r = max(a, b)
        if all(_periodic_dist(c, s[3], L) >= r + max(s[0], s[1]) + 4 * h for s in shapes):
            shapes.append((a, b, th, c))
    Xs, sp, rl = [], [], []
    for i, (a, b, th, c) in enumerate(shapes):
        Xs.append(ellipse_points(n_per, a, b, tuple(c), th))
        sp.append(closed_chain(n_per, offset=i * n_per))
        rl.append(np.full(n_per, 2.0 * math.pi * math.sqrt(a * b) / n_per))
    X = np.concatenate(Xs)
    springs = np.concatenate(sp)
    rest = np.concatenate(rl)
    return Problem(N=N, L=L, rho=rho, mu=mu, dt=dt, X=X, springs=springs,
                   kappa=np.full(springs.shape[0], float(kappa)), rest=rest,
                   meta={"shapes": shapes, "seed": seed}, **kw)


def batch(count=256, sizes=(64, 128, 256, 512), seed=5614, dt=1e-2, rho=1.0, mu=1.0,
          L=1.0, a=0.28, b=0.22, log_kappa=(0.0, 6.0), **kw):
    """Independent problems of uneven size and stiffness (the batched workload).

    N_i uniform on ``sizes``; n_i = round(4 * perimeter / h_i) points on the
    standard ellipse; kappa_i = 10**U[log_kappa]; rest length 2*pi*0.25/n_i.
    """
    rng = np.random.default_rng(seed)
    per = ellipse_perimeter(a, b)
    out = []
    for _ in range(count):
        N = int(rng.choice(sizes))
        n = int(round(4.0 * per * N / L))
        kap = 10.0 ** rng.uniform(*log_kappa)
        out.append(single_ellipse(N=N, n_points=n, kappa=kap, dt=dt, rho=rho, mu=mu, L=L,
                                  a=a, b=b, **kw))
    return out


def random_field(N, seed, count=3):
    """Standard-normal grid vector [count, N, N] (u, v, p components), float64."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((count, N, N))


def random_points_field(n, seed):
    """Standard-normal Lagrangian vector [n, 2], float64."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 2))


# ----------------------------------------------------------------------------- learned stage inputs

# Parameter shapes of the learned stage's U-Net (c_in, c_out, kernel), in the
# parameter order [W_0 b_0 W_1 b_1 ...]; only used to draw initial values.
UNET_SHAPES = [(4, 16, 3), (16, 16, 3), (16, 32, 3), (32, 32, 3), (32, 64, 3), (64, 64, 3),
               (96, 32, 3), (32, 32, 3), (48, 16, 3), (16, 16, 3), (16, 3, 1)]


def unet_init_params(seed, scale=1.0):
    """Seeded He-normal weights (std scale*sqrt(2/fan_in)) and zero biases, float32."""
    rng = np.random.default_rng(seed)
    out = []
    for ci, co, k in UNET_SHAPES:
        out.append(rng.standard_normal(co * ci * k * k) * (scale * math.sqrt(2.0 / (ci * k * k))))
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)


def random_smooth_field(N, seed, count=3, kmax=12, noise=0.05):
    """[count, N, N] periodic field: random Fourier modes with |k| <= kmax and
    amplitudes falling off as 1/(1+|k|^2), plus white noise of relative size
    ``noise``; unit RMS per component."""
    rng = np.random.default_rng(seed)
    out = np.empty((count, N, N))
    ky = np.fft.fftfreq(N) * N
    kx = np.fft.rfftfreq(N) * N
    KY, KX = np.meshgrid(ky, kx, indexing="ij")
    kk = np.hypot(KX, KY)
    mask = kk <= kmax
    for c in range(count):
        coef = (rng.standard_normal(KX.shape) + 1j * rng.standard_normal(KX.shape)) * mask / (1.0 + kk ** 2)
        f = np.fft.irfft2(coef, s=(N, N))
        f /= max(np.sqrt((f ** 2).mean()), 1e-300)
        out[c] = f + noise * rng.standard_normal((N, N))
    return out
