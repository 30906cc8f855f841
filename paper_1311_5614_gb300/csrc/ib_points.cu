// Lagrangian-point kernels: regularised delta weights, spreading S and
// interpolation S^* (sec. 2.2), spring force and Jacobian (sec. 2.2 force law,
// sec. 8 linearisation), the elasticity term dt * S J S^* on every level with
// Galerkin-coarsened patches (sec. 3.2), and its contribution to the box and
// coarsest-level matrices.
#include <cmath>

#include "ib_internal.cuh"

namespace ib {

namespace {

constexpr int TPB = 128;

inline int nblk(long n, int t = TPB) { return (int)((n + t - 1) / t); }

// 1-D kernels in grid units (sec. 2.2).  Peskin's 4-point function and the
// paper's cosine function (1 + cos(pi r / 2)) / 4, both supported on |r| < 2.
__device__ inline double phi1(double r, int kind) {
  double a = fabs(r);
  if (a >= 2.0) return 0.0;
  if (kind == IB_DELTA_COS4) return 0.25 * (1.0 + cospi(0.5 * r));
  if (a < 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) * 0.125;
  return (5.0 - 2.0 * a - sqrt(fmax(-7.0 + 12.0 * a - 4.0 * a * a, 0.0))) * 0.125;
}

// Level-0 patches: for each component, the x and y 1-D weights over the 4 grid
// lines within 2h of the point.  A "normal" direction has nodes at integer
// multiples of h, a "centred" direction at half-integers.
// With no-slip walls a point must keep its kernel support off the walls (2h from
// every wall); otherwise DEV_ERR_WALL.
__global__ void k_fine_patches(Patches<double> pat, const double* __restrict__ X, int np, int N,
                               double h, int kind, int walls, int* err) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  double s[2] = {X[2 * k] / h, X[2 * k + 1] / h};
  if (walls && !(s[0] >= 2.0 && s[0] <= N - 2.0 && s[1] >= 2.0 && s[1] <= N - 2.0)) atomicOr(err, DEV_ERR_WALL);
  for (int comp = 0; comp < 2; ++comp) {
    for (int xy = 0; xy < 2; ++xy) {
      // u: x normal, y centred; v: x centred, y normal
      bool centred = (comp == 0) ? (xy == 1) : (xy == 0);
      double sc = centred ? s[xy] - 0.5 : s[xy];
      double fl = floor(sc);
      int x0 = (int)(fl - N * floor(fl / N)) - 1;  // in [-1, N - 2]
      double frac = sc - fl;                        // in [0, 1)
      for (int kd = 0; kd < 2; ++kd) {
        *pat.b_ptr(kd, comp, xy, k) = x0;
        for (int a = 0; a < PATCH; ++a)
          *pat.w_ptr(kd, comp, xy, a, k) = phi1((double)(a - 1) - frac, kind);
      }
    }
  }
}

// Galerkin coarsening of one 1-D weight window (length 4 at base x0) to the next
// coarser grid.  Spread weights take the restriction R (sec. 3.1): full
// weighting (1/4, 1/2, 1/4) across the normal direction, two-point averaging in
// the centred direction.  Interp weights take P^T: linear interpolation along
// the normal direction (even fine node = coarse node, odd = midpoint) and the
// 3/4-1/4 interpolation between cell-centred rows.  Every result fits a length
// 4 window again.
__device__ inline void coarsen_1d(int x0, const double w[4], bool spread, bool centred, int* X0,
                                  double W[4]) {
  for (int a = 0; a < 4; ++a) W[a] = 0.0;
  int base = x0 >> 1;
  if (!spread && centred) base -= 1;
  *X0 = base;
  for (int a = 0; a < 4; ++a) {
    int i = x0 + a;
    double v = w[a];
    int half = i >> 1;  // floor(i / 2)
    bool odd = (i & 1) != 0;
    if (spread && !centred) {
      if (!odd) {
        W[half - base] += 0.5 * v;
      } else {
        W[half - base] += 0.25 * v;
        W[half + 1 - base] += 0.25 * v;
      }
    } else if (spread && centred) {
      W[half - base] += 0.5 * v;
    } else if (!centred) {  // interp, normal
      if (!odd) {
        W[half - base] += v;
      } else {
        W[half - base] += 0.5 * v;
        W[half + 1 - base] += 0.5 * v;
      }
    } else {  // interp, centred
      W[half - base] += 0.75 * v;
      if (!odd) W[half - 1 - base] += 0.25 * v;
      else W[half + 1 - base] += 0.25 * v;
    }
  }
}

__global__ void k_coarse_patches(Patches<double> fine, Patches<double> coarse, int np) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= np * 8) return;
  int k = t % np;
  int combo = t / np;  // kind (2) x comp (2) x xy (2)
  int xy = combo & 1, comp = (combo >> 1) & 1, kd = combo >> 2;
  bool centred = (comp == 0) ? (xy == 1) : (xy == 0);
  double w[4], W[4];
  for (int a = 0; a < 4; ++a) w[a] = fine.w_at(kd, comp, xy, a, k);
  int X0;
  coarsen_1d(fine.b_at(kd, comp, xy, k), w, kd == 0, centred, &X0, W);
  *coarse.b_ptr(kd, comp, xy, k) = X0;
  for (int a = 0; a < 4; ++a) *coarse.w_ptr(kd, comp, xy, a, k) = W[a];
}

__global__ void k_cast_d2f(const double* __restrict__ x, float* __restrict__ y, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

// Spring force F_i += kappa (1 - L0 / l) d, F_j -= ..., d = X_j - X_i (minimum
// image), and the 2 x 2 block K = dF_i / dX_j = kappa [s (I - t t^T) + t t^T],
// s = 1 - L0 / l (clamped at 0 for the negative-semidefinite variant).
__global__ void k_springs(const double* __restrict__ X, const int* __restrict__ ij,
                          const double* __restrict__ kappa, const double* __restrict__ rest,
                          int ns, double L, int clamped, double* Fs, double* K64, float* K32,
                          int* err) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ns) return;
  int i = ij[2 * e], j = ij[2 * e + 1];
  double dx = X[2 * j] - X[2 * i], dy = X[2 * j + 1] - X[2 * i + 1];
  dx -= L * rint(dx / L);
  dy -= L * rint(dy / L);
  double l = sqrt(dx * dx + dy * dy);
  double kxx = 0, kxy = 0, kyy = 0, fx = 0, fy = 0;
  if (l > 0.0 && isfinite(l)) {
    double kap = kappa[e], s = 1.0 - rest[e] / l;
    fx = kap * s * dx;
    fy = kap * s * dy;
    double tx = dx / l, ty = dy / l;
    double st = clamped ? fmax(s, 0.0) : s;
    kxx = kap * (st * (1.0 - tx * tx) + tx * tx);
    kxy = kap * (1.0 - st) * tx * ty;
    kyy = kap * (st * (1.0 - ty * ty) + ty * ty);
  } else {
    atomicOr(err, DEV_ERR_NONFINITE);
  }
  Fs[2 * e] = fx;  // on end i; -f on end j (gathered per point by k_point_force)
  Fs[2 * e + 1] = fy;
  K64[e] = kxx;
  K64[ns + e] = kxy;
  K64[2 * ns + e] = kyy;
  if (K32) {
    K32[e] = (float)kxx;
    K32[ns + e] = (float)kxy;
    K32[2 * ns + e] = (float)kyy;
  }
}

// F at each point: the forces of its springs in adjacency order (+f on a spring's
// first end, -f on its second), one writer per point, so the sum's order is fixed.
__global__ void k_point_force(const int* __restrict__ adj_ptr, const int* __restrict__ adj_spring,
                              const int* __restrict__ ij, const double* __restrict__ Fs, int np,
                              double* __restrict__ F) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  double fx = 0.0, fy = 0.0;
  for (int q = adj_ptr[k]; q < adj_ptr[k + 1]; ++q) {
    const int e = adj_spring[q];
    const double sg = ij[2 * e] == k ? 1.0 : -1.0;
    fx += sg * Fs[2 * e];
    fy += sg * Fs[2 * e + 1];
  }
  F[2 * k] = fx;
  F[2 * k + 1] = fy;
}

// Newton iterate: D = X^k - X^n per point ([2][np], periodic minimum image).
__global__ void k_newton_disp(const double* __restrict__ Xk, const double* __restrict__ Xn, int np, double L,
                              double* __restrict__ D) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  double dx = Xk[2 * k] - Xn[2 * k], dy = Xk[2 * k + 1] - Xn[2 * k + 1];
  dx -= L * rint(dx / L);
  dy -= L * rint(dy / L);
  D[k] = dx;
  D[np + k] = dy;
}

// F <- F - G (G = J D in [2][np] layout, F interleaved).
__global__ void k_newton_force(const double* __restrict__ G, int np, double* __restrict__ F) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  F[2 * k] -= G[k];
  F[2 * k + 1] -= G[np + k];
}

// b_c -= (S F)_c on the fine grid: delta_h = phi phi / h^2 (point forces).
__global__ void k_spread_force(Patches<double> pat, const double* __restrict__ F, int np, int N,
                               double inv_h2, double* b) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  int n = N * N;
  for (int comp = 0; comp < 2; ++comp) {
    double f = -F[2 * k + comp] * inv_h2;
    int x0 = pat.b_at(0, comp, 0, k), y0 = pat.b_at(0, comp, 1, k);
    for (int bb = 0; bb < PATCH; ++bb) {
      double wy = pat.w_at(0, comp, 1, bb, k) * f;
      if (wy == 0.0) continue;
      int row = wrapi(y0 + bb, N) * N;
      for (int a = 0; a < PATCH; ++a) {
        double wx = pat.w_at(0, comp, 0, a, k);
        if (wx != 0.0) atomicAdd(&b[comp * n + row + wrapi(x0 + a, N)], wx * wy);
      }
    }
  }
}

// X += dt * S^* u with the level-0 interpolation weights (Eq. 20).
__global__ void k_move_points(Patches<double> pat, const double* __restrict__ up, int np, int N,
                              double dt, double* X) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  int n = N * N;
  for (int comp = 0; comp < 2; ++comp) {
    int x0 = pat.b_at(1, comp, 0, k), y0 = pat.b_at(1, comp, 1, k);
    double s = 0.0;
    for (int bb = 0; bb < PATCH; ++bb) {
      double wy = pat.w_at(1, comp, 1, bb, k);
      int row = wrapi(y0 + bb, N) * N;
      double sx = 0.0;
      for (int a = 0; a < PATCH; ++a) sx += pat.w_at(1, comp, 0, a, k) * up[comp * n + row + wrapi(x0 + a, N)];
      s += wy * sx;
    }
    X[2 * k + comp] += dt * s;
  }
}

// U_c[k] = sum over the level's interp patch of w_c * wx * wy  (S^*_l w)
template <typename T>
__global__ void k_interp(Patches<T> pat, const T* __restrict__ w, int np, int N, T* __restrict__ U) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * np) return;
  int comp = t / np, k = t - comp * np;
  const T* wc = w + (size_t)comp * N * N;
  int x0 = pat.b_at(1, comp, 0, k), y0 = pat.b_at(1, comp, 1, k);
  T wx[PATCH];
  int ix[PATCH];
  for (int a = 0; a < PATCH; ++a) {
    wx[a] = pat.w_at(1, comp, 0, a, k);
    ix[a] = wrapi(x0 + a, N);
  }
  T s = 0;
  for (int bb = 0; bb < PATCH; ++bb) {
    T wy = pat.w_at(1, comp, 1, bb, k);
    const T* row = wc + wrapi(y0 + bb, N) * N;
    T sx = 0;
    for (int a = 0; a < PATCH; ++a) sx += wx[a] * row[ix[a]];
    s += wy * sx;
  }
  U[comp * np + k] = s;
}

// y_c += coef * S_l (J U)_c:  (J U)_k = sum over springs s at k of K_s (U_o - U_k).
template <typename T>
__global__ void k_spread_JU(Patches<T> pat, Springs<T> sp, const T* __restrict__ U, int N, T coef,
                            T* y) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= sp.np) return;
  int np = sp.np, ns = sp.ns;
  T ux = U[k], uy = U[np + k];
  T gx = 0, gy = 0;
  for (int q = sp.adj_ptr[k]; q < sp.adj_ptr[k + 1]; ++q) {
    int s = sp.adj_spring[q], o = sp.adj_other[q];
    T dx = U[o] - ux, dy = U[np + o] - uy;
    T kxx = sp.K[s], kxy = sp.K[ns + s], kyy = sp.K[2 * ns + s];
    gx += kxx * dx + kxy * dy;
    gy += kxy * dx + kyy * dy;
  }
  int n = N * N;
  for (int comp = 0; comp < 2; ++comp) {
    T g = coef * (comp == 0 ? gx : gy);
    if (g == (T)0) continue;
    int x0 = pat.b_at(0, comp, 0, k), y0 = pat.b_at(0, comp, 1, k);
    for (int bb = 0; bb < PATCH; ++bb) {
      T wy = pat.w_at(0, comp, 1, bb, k) * g;
      if (wy == (T)0) continue;
      T* row = y + comp * n + wrapi(y0 + bb, N) * N;
      for (int a = 0; a < PATCH; ++a) {
        T wx = pat.w_at(0, comp, 0, a, k);
        if (wx != (T)0) atomicAdd(&row[wrapi(x0 + a, N)], wx * wy);
      }
    }
  }
}

// (J U)_k per point into G [2][np] (the spread then gathers it by rows).
__global__ void k_point_JU(Springs<double> sp, const double* __restrict__ U, double* __restrict__ G) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= sp.np) return;
  int np = sp.np, ns = sp.ns;
  double ux = U[k], uy = U[np + k];
  double gx = 0, gy = 0;
  for (int q = sp.adj_ptr[k]; q < sp.adj_ptr[k + 1]; ++q) {
    int s = sp.adj_spring[q], o = sp.adj_other[q];
    double dx = U[o] - ux, dy = U[np + o] - uy;
    double kxx = sp.K[s], kxy = sp.K[ns + s], kyy = sp.K[2 * ns + s];
    gx += kxx * dx + kxy * dy;
    gy += kxy * dx + kyy * dy;
  }
  G[k] = gx;
  G[np + k] = gy;
}

// Mark every box whose velocity rows meet a spread patch: those are the boxes
// whose block A_BB can contain elasticity (structure boxes).
__global__ void k_mark(Patches<double> pat, int np, int N, int b, int nb, int* flag) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * np) return;
  int comp = t / np, k = t - comp * np;
  int x0 = pat.b_at(0, comp, 0, k), y0 = pat.b_at(0, comp, 1, k);
  for (int bb = 0; bb < PATCH; ++bb) {
    if (pat.w_at(0, comp, 1, bb, k) == 0.0) continue;
    int j = wrapi(y0 + bb, N);
    for (int a = 0; a < PATCH; ++a) {
      if (pat.w_at(0, comp, 0, a, k) == 0.0) continue;
      int i = wrapi(x0 + a, N);
      int I = i / b, J = j / b;
      flag[J * nb + I] = 1;
      // a face on a box edge belongs to the two boxes on either side
      if (comp == 0 && i % b == 0) flag[J * nb + ((I - 1 + nb) % nb)] = 1;
      if (comp == 1 && j % b == 0) flag[((J - 1 + nb) % nb) * nb + I] = 1;
    }
  }
}

// No-slip walls: the boxes along the walls (first and last row and column of boxes)
// hold wall faces and ghost rows, so their blocks differ from the free box's: they
// get structure slots (their own inverses).  Those no structure row reaches are
// marked -2: their blocks do not change from step to step, so their slots come
// after the others' and take inverses computed once (k_assign_ring).
__global__ void k_mark_ring(int nb, int* flag) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb * nb) return;
  const int I = t % nb, J = t / nb;
  if ((I == 0 || J == 0 || I == nb - 1 || J == nb - 1) && flag[t] == 0) flag[t] = -2;
}

__global__ void k_assign_slots(int* flag, int nbox, int* count, int* box_of_slot) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nbox) return;
  if (flag[t] > 0) {
    const int s = atomicAdd(count, 1);
    flag[t] = s;
    box_of_slot[s] = t;
  } else if (flag[t] == 0) {
    flag[t] = -1;
  }
}

// Slots after the formed ones (count_form of them) for the wall boxes marked -2.
__global__ void k_assign_ring(int* flag, int nbox, const int* count_form, int* count_ring, int* box_of_slot) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nbox || flag[t] != -2) return;
  const int s = *count_form + atomicAdd(count_ring, 1);
  flag[t] = s;
  box_of_slot[s] = t;
}

// Add coef * (S_l J S^*_l) restricted to box rows/cols to the dense box blocks.
// Thread = (point k, coupling q, row component c, row node of k's spread patch):
// q = 0 is the diagonal block J_kk = -sum K_s, q >= 1 the off-diagonal block
// J_kl = K_s of the q-th spring at k (at most 7 springs per point).
// mode 0: structure boxes (column-major n_B x n_B blocks indexed by slot);
// mode 1: the whole coarsest grid (one dense matrix, leading dimension ldm).
template <int MODE>
__global__ void k_assemble_E(Patches<double> pat, Springs<double> sp, int N, int b, int nb,
                             const int* __restrict__ slot, double coef, double* M, int nB, int ldm,
                             int* err) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const int np = sp.np, ns = sp.ns;
  const int k = (int)(t >> 8), rem = (int)(t & 255);
  const int q = rem >> 5, c = (rem >> 4) & 1, node = rem & 15;
  if (k >= np) return;
  const int deg = sp.adj_ptr[k + 1] - sp.adj_ptr[k];
  if (q > deg) return;
  if (deg > 7 && rem == 0) atomicOr(err, DEV_ERR_INDEX);
  const int ra = node & 3, rb = node >> 2;
  const double ws = pat.w_at(0, c, 0, ra, k) * pat.w_at(0, c, 1, rb, k);
  if (ws == 0.0) return;
  int l;
  double J[2][2];
  if (q == 0) {
    l = k;
    J[0][0] = J[0][1] = J[1][1] = 0.0;
    for (int a = sp.adj_ptr[k]; a < sp.adj_ptr[k + 1]; ++a) {
      int s = sp.adj_spring[a];
      J[0][0] -= sp.K[s];
      J[0][1] -= sp.K[ns + s];
      J[1][1] -= sp.K[2 * ns + s];
    }
  } else {
    int a = sp.adj_ptr[k] + q - 1;
    int s = sp.adj_spring[a];
    l = sp.adj_other[a];
    J[0][0] = sp.K[s];
    J[0][1] = sp.K[ns + s];
    J[1][1] = sp.K[2 * ns + s];
  }
  J[1][0] = J[0][1];
  const int n = N * N;
  const int ri = wrapi(pat.b_at(0, c, 0, k) + ra, N), rj = wrapi(pat.b_at(0, c, 1, k) + rb, N);
  const int nbx = (MODE == 0) ? 2 : 1;
  for (int bx = 0; bx < nbx; ++bx) {
    int x0 = 0, y0 = 0, sl = 0;
    if (MODE == 0) {
      int I = ri / b, Jb = rj / b;
      if (bx == 1) {
        // a face on a box edge belongs to the two boxes on either side
        if (c == 0 && ri % b == 0) I = (I - 1 + nb) % nb;
        else if (c == 1 && rj % b == 0) Jb = (Jb - 1 + nb) % nb;
        else continue;
      }
      sl = slot[Jb * nb + I];
      if (sl < 0) { atomicOr(err, DEV_ERR_INDEX); continue; }
      x0 = I * b;
      y0 = Jb * b;
    }
    const int rq = (MODE == 0) ? box_local(c, ri, rj, x0, y0, b, N) : c * n + rj * N + ri;
    if (rq < 0) { atomicOr(err, DEV_ERR_INDEX); continue; }
    double* Mb = (MODE == 0) ? M + (size_t)sl * nB * nB : M;
    const int ld = (MODE == 0) ? nB : ldm;
    for (int cc = 0; cc < 2; ++cc) {  // column component (interp patch of l)
      const double jv = coef * ws * J[c][cc];
      if (jv == 0.0) continue;
      const int ix0 = pat.b_at(1, cc, 0, l), iy0 = pat.b_at(1, cc, 1, l);
      for (int cb = 0; cb < PATCH; ++cb) {
        const double wiy = pat.w_at(1, cc, 1, cb, l);
        if (wiy == 0.0) continue;
        const int cj = wrapi(iy0 + cb, N);
        for (int ca = 0; ca < PATCH; ++ca) {
          const double wi = pat.w_at(1, cc, 0, ca, l) * wiy;
          if (wi == 0.0) continue;
          const int ci = wrapi(ix0 + ca, N);
          const int cq = (MODE == 0) ? box_local(cc, ci, cj, x0, y0, b, N) : cc * n + cj * N + ci;
          if (cq < 0) continue;
          atomicAdd(&Mb[(size_t)cq * ld + rq], jv * wi);
        }
      }
    }
  }
}

}  // namespace

// ---------------------------------------------------------------- launchers

int launch_fine_patches(Problem& P) {
  if (P.np == 0) return IB_OK;
  LevelInfo& L0 = P.lev[0];
  KScope ks(P, IB_KC_SETUP, P.np * (16.0 + 8 * 36.0));
  k_fine_patches<<<nblk(P.np), TPB, 0, P.stream>>>(L0.pat64, P.X, P.np, L0.N, L0.h, P.prm.delta, P.prm.walls,
                                                    P.dev_err);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_coarse_patches(Problem& P, int level) {
  if (P.np == 0) return IB_OK;
  KScope ks(P, IB_KC_SETUP, P.np * 16 * 36.0);
  k_coarse_patches<<<nblk(8L * P.np), TPB, 0, P.stream>>>(P.lev[level - 1].pat64, P.lev[level].pat64,
                                                           P.np);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_cast_patches(Problem& P, int level) {
  if (P.np == 0) return IB_OK;
  LevelInfo& L = P.lev[level];
  long nw = 32L * P.np;
  KScope ks(P, IB_KC_SETUP, nw * 12.0);
  k_cast_d2f<<<nblk(nw, 256), 256, 0, P.stream>>>(L.pat64.w, L.pat32.w, nw);
  IB_LAUNCH_CHECK();
  IB_CUDA_TRY(cudaMemcpyAsync(L.pat32.base, L.pat64.base, sizeof(int) * 8 * P.np,
                              cudaMemcpyDeviceToDevice, P.stream));
  return IB_OK;
}

int launch_spring_force_jacobian(Problem& P) {
  if (P.np == 0) return IB_OK;
  if (P.ns == 0) {
    IB_CUDA_TRY(cudaMemsetAsync(P.F, 0, sizeof(double) * 2 * P.np, P.stream));
    return IB_OK;
  }
  KScope ks(P, IB_KC_SETUP, P.ns * 100.0);
  k_springs<<<nblk(P.ns), TPB, 0, P.stream>>>(P.Xs ? P.Xs : P.X, P.springs, P.kappa, P.rest, P.ns, P.prm.L,
                                              P.prm.jacobian == IB_JAC_CLAMPED, P.Fs, P.K64, P.K32,
                                              P.dev_err);
  IB_LAUNCH_CHECK();
  k_point_force<<<nblk(P.np), TPB, 0, P.stream>>>(P.adj_ptr, P.adj_spring, P.springs, P.Fs, P.np, P.F);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_spread_force(Problem& P, double* b) {
  if (P.np == 0) return IB_OK;
  LevelInfo& L0 = P.lev[0];
  if (P.rows_ready) return launch_spread_rows(P, P.F, 2, 1, -1.0 / (L0.h * L0.h), b);
  KScope ks(P, IB_KC_OTHER, P.np * (16.0 + 2 * (8 * 8 + 8) + 32 * 16.0));
  k_spread_force<<<nblk(P.np), TPB, 0, P.stream>>>(L0.pat64, P.F, P.np, L0.N, 1.0 / (L0.h * L0.h), b);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_move_points(Problem& P, const double* up) {
  if (P.np == 0) return IB_OK;
  LevelInfo& L0 = P.lev[0];
  KScope ks(P, IB_KC_OTHER, P.np * (32.0 + 2 * (8 * 8 + 8) + 32 * 8.0));
  k_move_points<<<nblk(P.np), TPB, 0, P.stream>>>(L0.pat64, up, P.np, L0.N, P.prm.dt, P.X);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

template <typename T>
static Springs<T> springs_view(Problem& P);
template <>
Springs<double> springs_view<double>(Problem& P) {
  Springs<double> s;
  s.np = P.np; s.ns = P.ns; s.adj_ptr = P.adj_ptr; s.adj_spring = P.adj_spring;
  s.adj_other = P.adj_other; s.K = P.K64;
  return s;
}
template <>
Springs<float> springs_view<float>(Problem& P) {
  Springs<float> s;
  s.np = P.np; s.ns = P.ns; s.adj_ptr = P.adj_ptr; s.adj_spring = P.adj_spring;
  s.adj_other = P.adj_other; s.K = P.K32;
  return s;
}
int launch_newton_force(Problem& P) {
  if (P.np == 0 || P.ns == 0 || !P.Xs) return IB_OK;
  KScope ks(P, IB_KC_OTHER, P.np * 80.0);
  k_newton_disp<<<nblk(P.np), TPB, 0, P.stream>>>(P.Xs, P.Xn, P.np, P.prm.L, P.Dk);
  IB_LAUNCH_CHECK();
  k_point_JU<<<nblk(P.np), TPB, 0, P.stream>>>(springs_view<double>(P), P.Dk, P.Gk);
  IB_LAUNCH_CHECK();
  k_newton_force<<<nblk(P.np), TPB, 0, P.stream>>>(P.Gk, P.np, P.F);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

template <typename T>
static Patches<T> patches_of(LevelInfo& L);
template <>
Patches<double> patches_of<double>(LevelInfo& L) { return L.pat64; }
template <>
Patches<float> patches_of<float>(LevelInfo& L) { return L.pat32; }

template <typename T>
int launch_elastic(Problem& P, int level, const T* w, T* y, double coef, T* U) {
  if (!op_elastic(P)) return IB_OK;
  // The operator FGMRES is judged by stays in the factored form S J (S^* w): its
  // cancellation happens on small velocity differences.  An assembled row's entries
  // are sums of large per-point terms that nearly cancel (a second difference along
  // the curve), and applying them carries that error; measured on the stiff 256^2
  // step (kappa = 1e6, dt = 1e-2) the assembled operator cost 8-10 more iterations,
  // while the V-cycle (a preconditioner) on the assembled rows costs none.
  LevelInfo& L = P.lev[level];
  Patches<T> pat = patches_of<T>(L);
  const double sT = sizeof(T);
  {
    // per point and component: 16 gathered grid values, 8 weights, 2 bases, 1 result
    KScope ks(P, IB_KC_INTERP, 2.0 * P.np * (25 * sT + 8));
    k_interp<T><<<nblk(2L * P.np), TPB, 0, P.stream>>>(pat, w, P.np, L.N, U);
    IB_LAUNCH_CHECK();
  }
  if constexpr (sizeof(T) == 8) {
    if (level == 0 && P.rows_ready) {  // J U per point, then the spread as a gather by rows
      {
        KScope ks(P, IB_KC_SPREAD, P.np * (2 * sT + 8 + 2.0 * P.ns / P.np * (5 * sT + 8)));
        k_point_JU<<<nblk(P.np), TPB, 0, P.stream>>>(springs_view<double>(P), U, P.G64);
        IB_LAUNCH_CHECK();
      }
      return launch_spread_rows(P, P.G64, 1, P.np, coef, y);
    }
  }
  {
    // per point: own U, per spring U_other + K + adjacency, 16 weights + 4 bases,
    // 32 read-modify-write grid updates
    double deg = P.np ? 2.0 * P.ns / P.np : 0.0;
    KScope ks(P, IB_KC_SPREAD, P.np * (2 * sT + 8 + deg * (5 * sT + 8) + 16 * sT + 16 + 64 * sT));
    k_spread_JU<T><<<nblk(P.np), TPB, 0, P.stream>>>(pat, springs_view<T>(P), U, L.N, (T)coef, y);
    IB_LAUNCH_CHECK();
  }
  return IB_OK;
}
template int launch_elastic<double>(Problem&, int, const double*, double*, double, double*);
template int launch_elastic<float>(Problem&, int, const float*, float*, double, float*);

int launch_mark_struct(Problem& P, int level) {
  LevelInfo& L = P.lev[level];
  int nbox = L.nb * L.nb;
  IB_CUDA_TRY(cudaMemsetAsync(L.flag, 0, sizeof(int) * nbox, P.stream));
  IB_CUDA_TRY(cudaMemsetAsync(P.count, 0, sizeof(int), P.stream));
  if (op_elastic(P)) {
    KScope ks(P, IB_KC_SETUP, 2.0 * P.np * (8 * 8 + 8 + 32 * 4));
    k_mark<<<nblk(2L * P.np), TPB, 0, P.stream>>>(L.pat64, P.np, L.N, P.prm.box, L.nb, L.flag);
    IB_LAUNCH_CHECK();
  }
  if (P.prm.walls) {
    KScope ksr(P, IB_KC_SETUP, nbox * 4.0);
    k_mark_ring<<<nblk(nbox), TPB, 0, P.stream>>>(L.nb, L.flag);
    IB_LAUNCH_CHECK();
  }
  KScope ks(P, IB_KC_SETUP, nbox * 8.0);
  k_assign_slots<<<nblk(nbox), TPB, 0, P.stream>>>(L.flag, nbox, P.count, L.box_of_slot);
  IB_LAUNCH_CHECK();
  if (P.prm.walls) {
    int* cring = P.count + 1 + MAX_LEVELS_ALLOC + level;
    IB_CUDA_TRY(cudaMemsetAsync(cring, 0, sizeof(int), P.stream));
    k_assign_ring<<<nblk(nbox), TPB, 0, P.stream>>>(L.flag, nbox, P.count, cring, L.box_of_slot);
    IB_LAUNCH_CHECK();
  }
  return IB_OK;
}

int launch_assemble_struct(Problem& P, int level) {
  LevelInfo& L = P.lev[level];
  if (!op_elastic(P) || L.n_struct == 0) return IB_OK;
  double coef = P.prm.dt / (P.lev[0].h * P.lev[0].h);
  KScope ks(P, IB_KC_SETUP, 0.0);
  k_assemble_E<0><<<nblk(256L * P.np), TPB, 0, P.stream>>>(L.pat64, springs_view<double>(P), L.N,
                                                          P.prm.box, L.nb, L.flag, coef, L.Mstruct,
                                                          P.nB, 0, P.dev_err);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_assemble_coarse(Problem& P) {
  if (!op_elastic(P)) return IB_OK;
  LevelInfo& L = P.lev[P.nlev - 1];
  double coef = P.prm.dt / (P.lev[0].h * P.lev[0].h);
  KScope ks(P, IB_KC_SETUP, 0.0);
  k_assemble_E<1><<<nblk(256L * P.np), TPB, 0, P.stream>>>(L.pat64, springs_view<double>(P), L.N,
                                                          P.prm.box, 1, nullptr, coef, P.Mcoarse, 0,
                                                          P.nc + P.nborder, P.dev_err);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

}  // namespace ib
