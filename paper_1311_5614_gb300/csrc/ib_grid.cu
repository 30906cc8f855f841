// Grid kernels: the MAC Stokes operator (sec. 2.2) re-discretised per level
// (sec. 3.2), staggered restriction / prolongation (sec. 3.1), the box and
// big-box smoother solves (secs. 5-6), dense box / coarsest-level matrices and
// their Gauss-Jordan inverses, and the exact coarsest solve (Algorithm 1).
#include <cmath>

#include "ib_internal.cuh"

namespace ib {

namespace {

constexpr int TPB = 256;
inline int nblk(long n, int t = TPB) { return (int)((n + t - 1) / t); }

// y = A_S w  (apply) or  y = b - A_S w  (residual), one thread per cell (i, j)
// computing the u row of face (i, j), the v row of face (i, j) and the p row of
// cell (i, j).
template <typename T, bool RES>
__global__ void k_stokes(const T* __restrict__ w, const T* __restrict__ b, T* __restrict__ out,
                         int N, int shift, StokesCoef<T> c) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int n = N * N;
  if (idx >= n) return;
  int i = idx & (N - 1), j = idx >> shift;
  int ip = (i + 1) & (N - 1), im = (i - 1) & (N - 1);
  int jp = (j + 1) & (N - 1), jm = (j - 1) & (N - 1);
  const T* u = w;
  const T* v = w + n;
  const T* p = w + 2 * n;
  int e = j * N + ip, wq = j * N + im, nq = jp * N + i, sq = jm * N + i;
  T pc = p[idx];
  T au = c.diag * u[idx] + c.off * (u[e] + u[wq] + u[nq] + u[sq]) - c.g * (pc - p[wq]);
  T av = c.diag * v[idx] + c.off * (v[e] + v[wq] + v[nq] + v[sq]) - c.g * (pc - p[sq]);
  T ap = c.g * (u[e] - u[idx] + v[nq] - v[idx]);
  if (RES) {
    out[idx] = b[idx] - au;
    out[n + idx] = b[n + idx] - av;
    out[2 * n + idx] = b[2 * n + idx] - ap;
  } else {
    out[idx] = au;
    out[n + idx] = av;
    out[2 * n + idx] = ap;
  }
}

// Restriction (sec. 3.1) from an N grid to N/2, one thread per coarse cell.
template <typename T>
__global__ void k_restrict(const T* __restrict__ rf, T* __restrict__ bc, int Nc) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int nc = Nc * Nc;
  if (idx >= nc) return;
  int N = 2 * Nc, n = N * N;
  int I = idx % Nc, J = idx / Nc;
  const T* u = rf;
  const T* v = rf + n;
  const T* p = rf + 2 * n;
  int xm = (2 * I - 1) & (N - 1), x0 = 2 * I, x1 = 2 * I + 1;
  int ym = (2 * J - 1) & (N - 1), y0 = 2 * J, y1 = 2 * J + 1;
  // u: (1/8)[1 2 1; 1 2 1] -- faces 2I-1, 2I, 2I+1 in x, rows 2J, 2J+1 in y
  T su = (T)0.125 * (u[y0 * N + xm] + u[y1 * N + xm] + u[y0 * N + x1] + u[y1 * N + x1]) +
         (T)0.25 * (u[y0 * N + x0] + u[y1 * N + x0]);
  // v: transposed stencil
  T sv = (T)0.125 * (v[ym * N + x0] + v[ym * N + x1] + v[y1 * N + x0] + v[y1 * N + x1]) +
         (T)0.25 * (v[y0 * N + x0] + v[y0 * N + x1]);
  T sp = (T)0.25 * (p[y0 * N + x0] + p[y0 * N + x1] + p[y1 * N + x0] + p[y1 * N + x1]);
  bc[idx] = su;
  bc[nc + idx] = sv;
  bc[2 * nc + idx] = sp;
}

// w_f += P e_c (sec. 3.1): velocity linear along its normal direction and
// 3/4-1/4 between cell-centred rows, pressure constant.  One thread per fine cell.
template <typename T>
__global__ void k_prolong_add(const T* __restrict__ ec, T* __restrict__ wf, int N) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int n = N * N;
  if (idx >= n) return;
  int Nc = N / 2, nc = Nc * Nc;
  int i = idx & (N - 1), j = idx / N;
  int I = i >> 1, J = j >> 1;
  const T* u = ec;
  const T* v = ec + nc;
  const T* p = ec + 2 * nc;
  // centred-direction neighbour row/column: J-1 for even fine index, J+1 for odd
  int Jn = ((j & 1) ? J + 1 : J - 1) & (Nc - 1);
  int In = ((i & 1) ? I + 1 : I - 1) & (Nc - 1);
  int I1 = (I + 1) & (Nc - 1), J1 = (J + 1) & (Nc - 1);
  T cu, cv;
  if ((i & 1) == 0) {
    cu = (T)0.75 * u[J * Nc + I] + (T)0.25 * u[Jn * Nc + I];
  } else {
    cu = (T)0.375 * (u[J * Nc + I] + u[J * Nc + I1]) + (T)0.125 * (u[Jn * Nc + I] + u[Jn * Nc + I1]);
  }
  if ((j & 1) == 0) {
    cv = (T)0.75 * v[J * Nc + I] + (T)0.25 * v[J * Nc + In];
  } else {
    cv = (T)0.375 * (v[J * Nc + I] + v[J1 * Nc + I]) + (T)0.125 * (v[J * Nc + In] + v[J1 * Nc + In]);
  }
  wf[idx] += cu;
  wf[n + idx] += cv;
  wf[2 * n + idx] += p[J * Nc + I];
}

// Box solve for one colour, 1 x 1 boxes: one thread per box.  delta = A_BB^{-1} r_B,
// w_B += delta.  Structure boxes use their own FP64 inverse, the others the
// shared inverse of the structure-free box.
template <typename T>
__global__ void k_box1(const T* __restrict__ r, T* __restrict__ w, int N, int color,
                       const int* __restrict__ slot, const double* __restrict__ Ms,
                       const T* __restrict__ Mf) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int half = N >> 1;
  if (t >= half * half) return;
  int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
  int n = N * N;
  int I1 = (I + 1) & (N - 1), J1 = (J + 1) & (N - 1);
  int g[5] = {J * N + I, J * N + I1, n + J * N + I, n + J1 * N + I, 2 * n + J * N + I};
  int sl = slot[J * N + I];
  if (sl >= 0) {
    const double* M = Ms + (size_t)sl * 25;
    double rb[5];
    for (int q = 0; q < 5; ++q) rb[q] = (double)r[g[q]];
    for (int q = 0; q < 5; ++q) {
      double d = 0.0;
      for (int s = 0; s < 5; ++s) d += M[s * 5 + q] * rb[s];
      w[g[q]] += (T)d;
    }
  } else {
    T rb[5];
    for (int q = 0; q < 5; ++q) rb[q] = r[g[q]];
    for (int q = 0; q < 5; ++q) {
      T d = 0;
      for (int s = 0; s < 5; ++s) d += Mf[s * 5 + q] * rb[s];
      w[g[q]] += d;
    }
  }
}

// Box solve for one colour, b x b boxes (b >= 2): one warp per box; the box
// residual is staged in shared memory, lanes own rows of delta.
constexpr int BOX_WARPS = 4;
constexpr int MAX_NB = 208;  // 2 b (b + 1) + b^2 for b = 8
template <typename T>
__global__ void k_boxb(const T* __restrict__ r, T* __restrict__ w, int N, int b, int color,
                       const int* __restrict__ slot, const double* __restrict__ Ms,
                       const T* __restrict__ Mf) {
  __shared__ double rs[BOX_WARPS][MAX_NB];
  __shared__ int gs[BOX_WARPS][MAX_NB];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int nb = N / b, half = nb >> 1;
  int t = blockIdx.x * BOX_WARPS + warp;
  if (t >= half * half) return;
  int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
  int x0 = I * b, y0 = J * b, n = N * N;
  int nB = box_nunk(b);
  for (int q = lane; q < nB; q += 32) {
    int c, i, j;
    box_unknown(q, b, x0, y0, N, &c, &i, &j);
    int gq = c * n + j * N + i;
    gs[warp][q] = gq;
    rs[warp][q] = (double)r[gq];
  }
  __syncwarp();
  int sl = slot[J * nb + I];
  if (sl >= 0) {
    const double* M = Ms + (size_t)sl * nB * nB;
    for (int q = lane; q < nB; q += 32) {
      double d = 0.0;
      for (int s = 0; s < nB; ++s) d += M[(size_t)s * nB + q] * rs[warp][s];
      w[gs[warp][q]] += (T)d;
    }
  } else {
    for (int q = lane; q < nB; q += 32) {
      T d = 0;
      for (int s = 0; s < nB; ++s) d += Mf[(size_t)s * nB + q] * (T)rs[warp][s];
      w[gs[warp][q]] += d;
    }
  }
}

// Stokes block of a box at the origin of a level (identical for every box by
// translation invariance), column-major n_B x n_B.
__global__ void k_box_stokes(double* M, int N, int b, StokesCoef<double> c) {
  int nB = box_nunk(b);
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nB * nB) return;
  int q = e % nB, s = e / nB;
  int cq, iq, jq, cs, is, js;
  box_unknown(q, b, 0, 0, N, &cq, &iq, &jq);
  box_unknown(s, b, 0, 0, N, &cs, &is, &js);
  M[e] = stokes_entry(c, N, cq, iq, jq, cs, is, js);
}

__global__ void k_replicate(const double* __restrict__ src, double* dst, int m, long count) {
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= (long)m * count) return;
  dst[e] = src[e % m];
}

// Dense bordered coarsest matrix [[A_S, Z], [Z^T, 0]] (column-major, leading
// dimension ld = nc + nz); Z spans the constant pressure (and with rho = 0 the
// constant u and v).  The elasticity part is added by the point kernels.
__global__ void k_coarse_fill(double* M, int N, StokesCoef<double> c, int nz, int zfirst) {
  int nc = 3 * N * N, ld = nc + nz, n = N * N;
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= (long)ld * ld) return;
  int r = (int)(e % ld), col = (int)(e / ld);
  double v = 0.0;
  if (r < nc && col < nc) {
    int cr = r / n, rr = r % n, cc = col / n, rc = col % n;
    v = stokes_entry(c, N, cr, rr % N, rr / N, cc, rc % N, rc / N);
  } else if (r < nc && col >= nc) {
    v = (r / n == zfirst + (col - nc)) ? 1.0 : 0.0;
  } else if (r >= nc && col < nc) {
    v = (col / n == zfirst + (r - nc)) ? 1.0 : 0.0;
  }
  M[e] = v;
}

// In-place Gauss-Jordan inversion with partial pivoting, one CTA per matrix
// (row-major n x n storage; applied to a column-major A it returns A^{-1} in
// column-major order).  Row interchanges are undone by the reverse sequence of
// column interchanges at the end.
constexpr int INV_MAXN = 256;
__global__ void k_invert(double* Ms, int n, int* err) {
  __shared__ double f[INV_MAXN];
  __shared__ int perm[INV_MAXN];
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ int prow;
  double* M = Ms + (size_t)blockIdx.x * n * n;
  int tid = threadIdx.x, bd = blockDim.x;
  int lane = tid & 31, wid = tid >> 5, nw = (bd + 31) >> 5;
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = n;
    for (int i = k + tid; i < n; i += bd) {
      double a = fabs(M[(size_t)i * n + k]);
      if (a > best) { best = a; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_down_sync(0xffffffffu, best, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { rv[wid] = best; ri[wid] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b0 = rv[0];
      int i0 = ri[0];
      for (int q = 1; q < nw; ++q)
        if (rv[q] > b0 || (rv[q] == b0 && ri[q] < i0)) { b0 = rv[q]; i0 = ri[q]; }
      if (i0 >= n) i0 = k;
      prow = i0;
      perm[k] = i0;
    }
    __syncthreads();
    int p = prow;
    if (p != k) {
      for (int j = tid; j < n; j += bd) {
        double t = M[(size_t)k * n + j];
        M[(size_t)k * n + j] = M[(size_t)p * n + j];
        M[(size_t)p * n + j] = t;
      }
    }
    __syncthreads();
    double piv = M[(size_t)k * n + k];
    if (!(fabs(piv) > 0.0) || !isfinite(piv)) {
      if (tid == 0) atomicOr(err, DEV_ERR_SINGULAR);
      piv = 1.0;
    }
    __syncthreads();
    for (int j = tid; j < n; j += bd) {
      double v = (j == k) ? 1.0 : M[(size_t)k * n + j];
      M[(size_t)k * n + j] = v / piv;
    }
    for (int i = tid; i < n; i += bd) f[i] = (i == k) ? 0.0 : M[(size_t)i * n + k];
    __syncthreads();
    for (int i = tid; i < n; i += bd)
      if (i != k) M[(size_t)i * n + k] = 0.0;
    __syncthreads();
    for (long e = tid; e < (long)n * n; e += bd) {
      int i = (int)(e / n), j = (int)(e % n);
      if (i != k) M[e] -= f[i] * M[(size_t)k * n + j];
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    int p = perm[k];
    if (p != k) {
      for (int i = tid; i < n; i += bd) {
        double t = M[(size_t)i * n + k];
        M[(size_t)i * n + k] = M[(size_t)i * n + p];
        M[(size_t)i * n + p] = t;
      }
    }
    __syncthreads();
  }
}

// w = (M^{-1})[0:nc, 0:nc] b for the bordered coarsest system, one CTA.
template <typename T>
__global__ void k_coarse_solve(const double* __restrict__ M, int nc, int ld, const T* __restrict__ b,
                               T* __restrict__ w) {
  __shared__ double bs[3 * 64 + 8];
  for (int s = threadIdx.x; s < nc; s += blockDim.x) bs[s] = (double)b[s];
  __syncthreads();
  for (int r = threadIdx.x; r < nc; r += blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < nc; ++s) acc += M[(size_t)s * ld + r] * bs[s];
    w[r] = (T)acc;
  }
}

template <typename T>
__global__ void k_fill(T* x, long n, T v) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

template <typename A, typename B>
__global__ void k_cast(const A* __restrict__ x, B* __restrict__ y, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (B)x[i];
}

inline int log2i(int N) {
  int s = 0;
  while ((1 << s) < N) ++s;
  return s;
}

template <typename T>
StokesCoef<T> coef_of(const Problem& P, int level) {
  double h = P.lev[level].h;
  StokesCoef<T> c;
  double reac = (P.prm.rho != 0.0) ? P.prm.rho / P.prm.dt : 0.0;
  c.diag = (T)(-4.0 * P.prm.mu / (h * h) - reac);
  c.off = (T)(P.prm.mu / (h * h));
  c.g = (T)(1.0 / h);
  return c;
}

template <typename T>
const T* free_inverse(const LevelInfo& L);
template <>
const double* free_inverse<double>(const LevelInfo& L) { return L.Mfree; }
template <>
const float* free_inverse<float>(const LevelInfo& L) { return L.Mfree32; }

}  // namespace

template <typename T>
int launch_stokes(Problem& P, int level, const T* w, const T* b, T* out, bool residual) {
  int N = P.lev[level].N;
  StokesCoef<T> c = coef_of<T>(P, level);
  KScope ks(P, IB_KC_STOKES, (residual ? 9.0 : 6.0) * N * N * sizeof(T));
  if (residual)
    k_stokes<T, true><<<nblk((long)N * N), TPB, 0, P.stream>>>(w, b, out, N, log2i(N), c);
  else
    k_stokes<T, false><<<nblk((long)N * N), TPB, 0, P.stream>>>(w, b, out, N, log2i(N), c);
  IB_LAUNCH_CHECK();
  return IB_OK;
}
template int launch_stokes<double>(Problem&, int, const double*, const double*, double*, bool);
template int launch_stokes<float>(Problem&, int, const float*, const float*, float*, bool);

template <typename T>
int launch_restrict(Problem& P, int level, const T* rf, T* bc) {
  int Nc = P.lev[level + 1].N;
  KScope ks(P, IB_KC_TRANSFER, 15.0 * Nc * Nc * sizeof(T));
  k_restrict<T><<<nblk((long)Nc * Nc), TPB, 0, P.stream>>>(rf, bc, Nc);
  IB_LAUNCH_CHECK();
  return IB_OK;
}
template int launch_restrict<double>(Problem&, int, const double*, double*);
template int launch_restrict<float>(Problem&, int, const float*, float*);

template <typename T>
int launch_prolong_add(Problem& P, int level, const T* ec, T* wf) {
  int N = P.lev[level].N;
  KScope ks(P, IB_KC_TRANSFER, (6.0 * N * N + 0.75 * N * N) * sizeof(T));
  k_prolong_add<T><<<nblk((long)N * N), TPB, 0, P.stream>>>(ec, wf, N);
  IB_LAUNCH_CHECK();
  return IB_OK;
}
template int launch_prolong_add<double>(Problem&, int, const double*, double*);
template int launch_prolong_add<float>(Problem&, int, const float*, float*);

template <typename T>
int launch_box_solve(Problem& P, int level, int color, const T* r, T* w) {
  LevelInfo& L = P.lev[level];
  int b = P.prm.box;
  int half = L.nb / 2;
  long nbox = (long)half * half;
  // per box: n_B residual reads, n_B read-modify-writes of w, the slot; structure
  // boxes (about a quarter of them per colour) read their FP64 inverse; the shared
  // free-box inverse is read once
  int nB = P.nB;
  KScope ks(P, IB_KC_BOX, nbox * (3.0 * nB * sizeof(T) + 4) + 0.25 * L.n_struct * nB * nB * 8.0 +
                              (double)nB * nB * sizeof(T));
  if (b == 1) {
    k_box1<T><<<nblk(nbox, 128), 128, 0, P.stream>>>(r, w, L.N, color, L.flag, L.Mstruct,
                                                      free_inverse<T>(L));
  } else {
    k_boxb<T><<<nblk(nbox, BOX_WARPS), 32 * BOX_WARPS, 0, P.stream>>>(r, w, L.N, b, color, L.flag,
                                                                       L.Mstruct, free_inverse<T>(L));
  }
  IB_LAUNCH_CHECK();
  return IB_OK;
}
template int launch_box_solve<double>(Problem&, int, int, const double*, double*);
template int launch_box_solve<float>(Problem&, int, int, const float*, float*);

// Free-box Stokes block into L.Mfree, copied into every structure slot.
int launch_box_stokes_fill(Problem& P, int level, bool /*unused*/) {
  LevelInfo& L = P.lev[level];
  int nB = P.nB;
  StokesCoef<double> c = coef_of<double>(P, level);
  KScope ks(P, IB_KC_SETUP, nB * nB * 8.0);
  k_box_stokes<<<nblk((long)nB * nB), TPB, 0, P.stream>>>(L.Mfree, L.N, P.prm.box, c);
  IB_LAUNCH_CHECK();
  if (L.n_struct > 0) {
    long tot = (long)nB * nB * L.n_struct;
    KScope ks2(P, IB_KC_SETUP, tot * 8.0);
    k_replicate<<<nblk(tot), TPB, 0, P.stream>>>(L.Mfree, L.Mstruct, nB * nB, L.n_struct);
    IB_LAUNCH_CHECK();
  }
  return IB_OK;
}

int launch_invert(Problem& P, double* M, int n, int count) {
  if (count <= 0) return IB_OK;
  if (n > INV_MAXN) return fail(IB_ERR_INVALID_ARG, "matrix too large for the device inverse");
  int threads = n <= 32 ? 32 : (n <= 64 ? 64 : 256);
  KScope ks(P, IB_KC_SETUP, 2.0 * count * n * n * 8.0);
  k_invert<<<count, threads, 0, P.stream>>>(M, n, P.dev_err);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_coarse_fill(Problem& P) {
  LevelInfo& L = P.lev[P.nlev - 1];
  StokesCoef<double> c = coef_of<double>(P, P.nlev - 1);
  int ld = P.nc + P.nborder;
  int zfirst = (P.nborder == 1) ? 2 : 0;
  KScope ks(P, IB_KC_SETUP, (double)ld * ld * 8.0);
  k_coarse_fill<<<nblk((long)ld * ld), TPB, 0, P.stream>>>(P.Mcoarse, L.N, c, P.nborder, zfirst);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

template <typename T>
int launch_coarse_solve(Problem& P, const T* b, T* w) {
  KScope ks(P, IB_KC_COARSE, (double)P.nc * P.nc * 8.0 + 2.0 * P.nc * sizeof(T));
  k_coarse_solve<T><<<1, 256, 0, P.stream>>>(P.Mcoarse, P.nc, P.nc + P.nborder, b, w);
  IB_LAUNCH_CHECK();
  return IB_OK;
}
template int launch_coarse_solve<double>(Problem&, const double*, double*);
template int launch_coarse_solve<float>(Problem&, const float*, float*);

template <typename T>
int launch_fill(Problem& P, T* x, size_t n, T v) {
  if (n == 0) return IB_OK;
  KScope ks(P, IB_KC_OTHER, (double)n * sizeof(T));
  k_fill<T><<<nblk((long)n), TPB, 0, P.stream>>>(x, (long)n, v);
  IB_LAUNCH_CHECK();
  return IB_OK;
}
template int launch_fill<double>(Problem&, double*, size_t, double);
template int launch_fill<float>(Problem&, float*, size_t, float);

template <typename A, typename B>
int launch_cast(Problem& P, const A* x, B* y, size_t n) {
  if (n == 0) return IB_OK;
  KScope ks(P, IB_KC_OTHER, (double)n * (sizeof(A) + sizeof(B)));
  k_cast<A, B><<<nblk((long)n), TPB, 0, P.stream>>>(x, y, (long)n);
  IB_LAUNCH_CHECK();
  return IB_OK;
}
template int launch_cast<double, float>(Problem&, const double*, float*, size_t);
template int launch_cast<float, double>(Problem&, const float*, double*, size_t);
template int launch_cast<double, double>(Problem&, const double*, double*, size_t);

}  // namespace ib
