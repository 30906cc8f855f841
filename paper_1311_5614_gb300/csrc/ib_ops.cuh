// Element-level device functions of the V-cycle, shared by the grid-wide
// kernels of the fine levels and the tail kernel of the coarse levels (one CTA
// or one thread-block cluster).  Pointers may address global or shared memory.
#pragma once

#include "ib_internal.cuh"

namespace ib {

// (A_S w) at the unknown (comp, i, j) of an N x N level (sec. 2.2 stencils: mu Lap -
// rho/dt on velocities, -G p on faces, D w on cells), periodic or with no-slip walls
// (c.walls: a wall face's row is the identity; w holds zero on the wall faces, so
// the rows that read them need no change except the tangential ghost -u).
template <typename T>
__device__ __forceinline__ T stokes_row(const T* __restrict__ w, int N, const StokesCoef<T>& c, int comp,
                                        int i, int j) {
  const int n = N * N, m = N - 1;
  const int ip = (i + 1) & m, im = (i - 1) & m, jp = (j + 1) & m, jm = (j - 1) & m;
  const T* u = w;
  const T* v = w + n;
  const T* p = w + 2 * n;
  if (comp == 0) {
    const T uc = u[j * N + i];
    if (c.walls) {
      if (i == 0) return uc;
      const T un = (j == m) ? -uc : u[jp * N + i], us = (j == 0) ? -uc : u[jm * N + i];
      return c.diag * uc + c.off * (u[j * N + ip] + u[j * N + im] + un + us) - c.g * (p[j * N + i] - p[j * N + im]);
    }
    return c.diag * uc + c.off * (u[j * N + ip] + u[j * N + im] + u[jp * N + i] + u[jm * N + i]) -
           c.g * (p[j * N + i] - p[j * N + im]);
  }
  if (comp == 1) {
    const T vc = v[j * N + i];
    if (c.walls) {
      if (j == 0) return vc;
      const T ve = (i == m) ? -vc : v[j * N + ip], vw = (i == 0) ? -vc : v[j * N + im];
      return c.diag * vc + c.off * (ve + vw + v[jp * N + i] + v[jm * N + i]) - c.g * (p[j * N + i] - p[jm * N + i]);
    }
    return c.diag * vc + c.off * (v[j * N + ip] + v[j * N + im] + v[jp * N + i] + v[jm * N + i]) -
           c.g * (p[j * N + i] - p[jm * N + i]);
  }
  return c.g * (u[j * N + ip] - u[j * N + i] + v[jp * N + i] - v[j * N + i]);
}

// Residual r = b - A_S w + rE at (comp, i, j); rE (-dt E w, velocity rows only)
// may be NULL.  A wall face's residual is b - w (no elasticity row there).
template <typename T>
__device__ __forceinline__ T resid_at(const T* w, const T* b, const T* rE, int N, const StokesCoef<T>& c,
                                      int comp, int i, int j) {
  const int g = comp * N * N + j * N + i;
  T r = b[g] - stokes_row(w, N, c, comp, i, j);
  if (rE && comp < 2 && !(c.walls && wall_face(comp, i, j))) r += rE[g];
  return r;
}

// Restriction of the full residual to coarse cell (I, J) of an Nc grid (sec. 3.1,
// Eqs. 25-26): u by (1/8)[1 2 1; 1 2 1], v transposed, p by the four-cell average.
template <typename T>
__device__ __forceinline__ void restrict_resid_cell(const T* w, const T* b, const T* E, int N,
                                                    const StokesCoef<T>& c, int I, int J, T* ru, T* rv, T* rp) {
  const int m = N - 1;
  const int xm = (2 * I - 1) & m, x0 = 2 * I, x1 = 2 * I + 1;
  const int ym = (2 * J - 1) & m, y0 = 2 * J, y1 = 2 * J + 1;
  *ru = (T)0.125 * (resid_at(w, b, E, N, c, 0, xm, y0) + resid_at(w, b, E, N, c, 0, xm, y1) +
                    resid_at(w, b, E, N, c, 0, x1, y0) + resid_at(w, b, E, N, c, 0, x1, y1)) +
        (T)0.25 * (resid_at(w, b, E, N, c, 0, x0, y0) + resid_at(w, b, E, N, c, 0, x0, y1));
  *rv = (T)0.125 * (resid_at(w, b, E, N, c, 1, x0, ym) + resid_at(w, b, E, N, c, 1, x1, ym) +
                    resid_at(w, b, E, N, c, 1, x0, y1) + resid_at(w, b, E, N, c, 1, x1, y1)) +
        (T)0.25 * (resid_at(w, b, E, N, c, 1, x0, y0) + resid_at(w, b, E, N, c, 1, x1, y0));
  *rp = (T)0.25 * (resid_at(w, b, E, N, c, 2, x0, y0) + resid_at(w, b, E, N, c, 2, x1, y0) +
                   resid_at(w, b, E, N, c, 2, x0, y1) + resid_at(w, b, E, N, c, 2, x1, y1));
  if (c.walls) {  // coarse wall faces hold zero
    if (I == 0) *ru = (T)0;
    if (J == 0) *rv = (T)0;
  }
}

// Same restriction applied to a stored residual vector r (walls: the coarse wall
// faces get zero).
template <typename T>
__device__ __forceinline__ void restrict_cell(const T* r, int N, int I, int J, T* ru, T* rv, T* rp, int walls) {
  const int n = N * N, m = N - 1;
  const T* u = r;
  const T* v = r + n;
  const T* p = r + 2 * n;
  const int xm = (2 * I - 1) & m, x0 = 2 * I, x1 = 2 * I + 1;
  const int ym = (2 * J - 1) & m, y0 = 2 * J, y1 = 2 * J + 1;
  *ru = (T)0.125 * (u[y0 * N + xm] + u[y1 * N + xm] + u[y0 * N + x1] + u[y1 * N + x1]) +
        (T)0.25 * (u[y0 * N + x0] + u[y1 * N + x0]);
  *rv = (T)0.125 * (v[ym * N + x0] + v[ym * N + x1] + v[y1 * N + x0] + v[y1 * N + x1]) +
        (T)0.25 * (v[y0 * N + x0] + v[y0 * N + x1]);
  *rp = (T)0.25 * (p[y0 * N + x0] + p[y0 * N + x1] + p[y1 * N + x0] + p[y1 * N + x1]);
  if (walls) {
    if (I == 0) *ru = (T)0;
    if (J == 0) *rv = (T)0;
  }
}

// Prolongation (sec. 3.1) of the coarse correction e (Nc = N/2) to fine cell
// (i, j): returns the three fine corrections.  With no-slip walls the coarse row
// beyond a wall is its ghost, minus the row itself (so the fine row next to the
// wall takes half the coarse one); the coarse wall faces hold zero.
template <typename T>
__device__ __forceinline__ void prolong_cell(const T* e, int N, int i, int j, T* cu, T* cv, T* cp, int walls) {
  const int Nc = N / 2, nc = Nc * Nc, mc = Nc - 1;
  const int I = i >> 1, J = j >> 1;
  const T* u = e;
  const T* v = e + nc;
  const T* p = e + 2 * nc;
  const int Ju = (j & 1) ? J + 1 : J - 1, Iu = (i & 1) ? I + 1 : I - 1;
  const int Jn = Ju & mc, In = Iu & mc;
  const int I1 = (I + 1) & mc, J1 = (J + 1) & mc;
  // weights of the far row / column; at a wall the ghost folds onto the near one
  const bool gy = walls && (Ju < 0 || Ju > mc), gx = walls && (Iu < 0 || Iu > mc);
  const int Jf = gy ? J : Jn, If = gx ? I : In;
  const T fy = gy ? (T)-0.25 : (T)0.25, hy = gy ? (T)-0.125 : (T)0.125;
  const T fx = gx ? (T)-0.25 : (T)0.25, hx = gx ? (T)-0.125 : (T)0.125;
  if ((i & 1) == 0) *cu = (T)0.75 * u[J * Nc + I] + fy * u[Jf * Nc + I];
  else *cu = (T)0.375 * (u[J * Nc + I] + u[J * Nc + I1]) + hy * (u[Jf * Nc + I] + u[Jf * Nc + I1]);
  if ((j & 1) == 0) *cv = (T)0.75 * v[J * Nc + I] + fx * v[J * Nc + If];
  else *cv = (T)0.375 * (v[J * Nc + I] + v[J1 * Nc + I]) + hx * (v[J * Nc + If] + v[J1 * Nc + If]);
  *cp = p[J * Nc + I];
}

// Interpolated velocity component of point k on level grid N: sum over its
// interp patch of w_c * wx * wy.
template <typename T>
__device__ __forceinline__ T interp_point(const Patches<T>& pat, const T* w, int N, int comp, int k) {
  const T* wc = w + (size_t)comp * N * N;
  const int x0 = pat.b_at(1, comp, 0, k), y0 = pat.b_at(1, comp, 1, k), m = N - 1;
  T wx[PATCH];
  int ix[PATCH];
#pragma unroll
  for (int a = 0; a < PATCH; ++a) {
    wx[a] = pat.w_at(1, comp, 0, a, k);
    ix[a] = (x0 + a) & m;
  }
  T s = 0;
#pragma unroll
  for (int bb = 0; bb < PATCH; ++bb) {
    const T* row = wc + ((y0 + bb) & m) * N;
    T sx = 0;
#pragma unroll
    for (int a = 0; a < PATCH; ++a) sx += wx[a] * row[ix[a]];
    s += pat.w_at(1, comp, 1, bb, k) * sx;
  }
  return s;
}

// Whether velocity row (comp, i, j) of a level with b x b boxes is an unknown of
// a box of colour `color` (-1: any).  A face on the low edge of its box is also
// the far-edge unknown of the neighbouring box, whose colour parity differs.
__device__ __forceinline__ bool row_in_color(int comp, int i, int j, int b, int color) {
  if (color < 0) return true;
  const int cx = (i / b) & 1, cy = ((j / b) & 1) << 1;
  if ((cx | cy) == color) return true;
  if (comp == 0 && i % b == 0) return ((cx ^ 1) | cy) == color;
  if (comp == 1 && j % b == 0) return (cx | (cy ^ 2)) == color;
  return false;
}

// Programmatic dependent launch entry: wait until the grids this kernel depends
// on have completed (their results visible), then let the next kernel of the
// stream begin launching.  Only set-up data may be read before it.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Interpolation patch (kind 1) of one component of one point: bases and weights.
template <typename T>
struct IPatch {
  int x0, y0;
  T wx[PATCH], wy[PATCH];
};

template <typename T>
__device__ __forceinline__ IPatch<T> load_ipatch(const Patches<T>& pat, int comp, int k) {
  IPatch<T> p;
  p.x0 = pat.b_at(1, comp, 0, k);
  p.y0 = pat.b_at(1, comp, 1, k);
#pragma unroll
  for (int a = 0; a < PATCH; ++a) {
    p.wx[a] = pat.w_at(1, comp, 0, a, k);
    p.wy[a] = pat.w_at(1, comp, 1, a, k);
  }
  return p;
}

// sum over the patch of wc * wx * wy (wc: one component of a level vector)
template <typename T>
__device__ __forceinline__ T interp_ip(const IPatch<T>& p, const T* wc, int N) {
  const int m = N - 1;
  T s = 0;
#pragma unroll
  for (int bb = 0; bb < PATCH; ++bb) {
    const T* row = wc + ((p.y0 + bb) & m) * N;
    T sx = 0;
#pragma unroll
    for (int a = 0; a < PATCH; ++a) sx += p.wx[a] * row[(p.x0 + a) & m];
    s += p.wy[bb] * sx;
  }
  return s;
}

// rE += coef * S_l J S*_l w restricted to the rows of boxes of one colour (-1:
// all rows), for point k by an aligned quad of lanes (j = lane & 3, qmask the
// quad's lanes, qlane0 its first lane).  Lane 0 interpolates the point's own
// velocity, lanes 1..3 those of its first three spring neighbours (further ones
// round robin), all at the same time; the spring terms K_s (U_other - U_k) are
// summed over the quad; then lane j spreads component j & 1 over patch rows
// 2 (j >> 1) and 2 (j >> 1) + 1 with atomic additions.  Adjacency, spring
// blocks and both patches are loaded first; with WAIT the kernel's
// programmatic-launch wait comes after them, so that only the loads of w depend
// on the previous kernel.  Every lane of the quad must call this.
template <typename T, bool WAIT>
__device__ __forceinline__ void force_spread_quad(const Patches<T>& pat, const Springs<T>& sp, const T* w, int N,
                                                  T coef, int k, int j, unsigned qmask, int qlane0, int b, int color,
                                                  T* rE) {
  const int p0 = sp.adj_ptr[k], deg = sp.adj_ptr[k + 1] - p0, ns = sp.ns;
  int pid = -1, s = -1;
  if (j == 0) {
    pid = k;
  } else if (j - 1 < deg) {
    pid = sp.adj_other[p0 + j - 1];
    s = sp.adj_spring[p0 + j - 1];
  }
  IPatch<T> pu, pv;
  if (pid >= 0) {
    pu = load_ipatch(pat, 0, pid);
    pv = load_ipatch(pat, 1, pid);
  }
  T kxx = 0, kxy = 0, kyy = 0;
  if (s >= 0) {
    kxx = sp.K[s];
    kxy = sp.K[ns + s];
    kyy = sp.K[2 * ns + s];
  }
  const int comp = j & 1, r0 = 2 * (j >> 1);
  const int sx0 = pat.b_at(0, comp, 0, k), sy0 = pat.b_at(0, comp, 1, k);
  T swx[PATCH], swy[2];
#pragma unroll
  for (int a = 0; a < PATCH; ++a) swx[a] = pat.w_at(0, comp, 0, a, k);
  swy[0] = pat.w_at(0, comp, 1, r0, k);
  swy[1] = pat.w_at(0, comp, 1, r0 + 1, k);
  if (WAIT) pdl_enter();
  T ux = 0, uy = 0;
  if (pid >= 0) {
    ux = interp_ip(pu, w, N);
    uy = interp_ip(pv, w + (size_t)N * N, N);
  }
  const T ux0 = __shfl_sync(qmask, ux, qlane0);
  const T uy0 = __shfl_sync(qmask, uy, qlane0);
  T ax = 0, ay = 0;
  if (s >= 0) {
    const T dx = ux - ux0, dy = uy - uy0;
    ax = kxx * dx + kxy * dy;
    ay = kxy * dx + kyy * dy;
    for (int m = j + 2; m < deg; m += 3) {
      const int o2 = sp.adj_other[p0 + m], s2 = sp.adj_spring[p0 + m];
      const T ex = interp_point(pat, w, N, 0, o2) - ux0, ey = interp_point(pat, w, N, 1, o2) - uy0;
      const T k2xx = sp.K[s2], k2xy = sp.K[ns + s2], k2yy = sp.K[2 * ns + s2];
      ax += k2xx * ex + k2xy * ey;
      ay += k2xy * ex + k2yy * ey;
    }
  }
  ax += __shfl_xor_sync(qmask, ax, 1);
  ay += __shfl_xor_sync(qmask, ay, 1);
  ax += __shfl_xor_sync(qmask, ax, 2);
  ay += __shfl_xor_sync(qmask, ay, 2);
  const T g = coef * (comp ? ay : ax);  // the quad sum is in every lane
  if (g == (T)0) return;
  const int m = N - 1;
  T* yc = rE + (size_t)comp * N * N;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const T wy = swy[r] * g;
    if (wy == (T)0) continue;
    const int jj = (sy0 + r0 + r) & m;
#pragma unroll
    for (int a = 0; a < PATCH; ++a) {
      const int ii = (sx0 + a) & m;
      if (swx[a] != (T)0 && row_in_color(comp, ii, jj, b, color)) atomicAdd(&yc[jj * N + ii], swx[a] * wy);
    }
  }
}

// delta = M r for a box of nB unknowns, M column-major (M[s * nB + q]); rows q
// from q0 in steps of dq.
template <typename TM, typename TR, typename TW>
__device__ __forceinline__ void box_apply_rows(const TM* __restrict__ M, int nB, const TR* rs, int q0, int dq,
                                               TW* w, const int* gs) {
  for (int q = q0; q < nB; q += dq) {
    TM d = 0;
    for (int s = 0; s < nB; ++s) d += M[(size_t)s * nB + q] * (TM)rs[s];
    w[gs[q]] += (TW)d;
  }
}

}  // namespace ib
