// Grid kernels: the MAC Stokes operator (sec. 2.2) re-discretised per level
// (sec. 3.2), staggered restriction / prolongation (sec. 3.1), the box and
// big-box smoother solves (secs. 5-6), dense box / coarsest-level matrices and
// their Gauss-Jordan inverses, and the exact coarsest solve (Algorithm 1).
#include <cmath>
#include <cstring>
#include <mutex>

#include "ib_internal.cuh"
#include "ib_ops.cuh"

namespace ib {

namespace {

constexpr int TPB = 256;
inline int nblk(long n, int t = TPB) { return (int)((n + t - 1) / t); }

// y = A_S w  (apply) or  y = b - A_S w  (residual), one thread per cell (i, j)
// computing the u row of face (i, j), the v row of face (i, j) and the p row of
// cell (i, j).  With no-slip walls (c.walls) the rows are those of stokes_row.
template <typename T, bool RES>
__global__ void k_stokes(const T* __restrict__ w, const T* __restrict__ b, T* __restrict__ out,
                         int N, int shift, StokesCoef<T> c) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int n = N * N;
  if (idx >= n) return;
  int i = idx & (N - 1), j = idx >> shift;
  T au, av, ap;
  if (c.walls) {
    au = stokes_row(w, N, c, 0, i, j);
    av = stokes_row(w, N, c, 1, i, j);
    ap = stokes_row(w, N, c, 2, i, j);
  } else {
    int ip = (i + 1) & (N - 1), im = (i - 1) & (N - 1);
    int jp = (j + 1) & (N - 1), jm = (j - 1) & (N - 1);
    const T* u = w;
    const T* v = w + n;
    const T* p = w + 2 * n;
    int e = j * N + ip, wq = j * N + im, nq = jp * N + i, sq = jm * N + i;
    T pc = p[idx];
    au = c.diag * u[idx] + c.off * (u[e] + u[wq] + u[nq] + u[sq]) - c.g * (pc - p[wq]);
    av = c.diag * v[idx] + c.off * (v[e] + v[wq] + v[nq] + v[sq]) - c.g * (pc - p[sq]);
    ap = c.g * (u[e] - u[idx] + v[nq] - v[idx]);
  }
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

// Stokes block of each structure slot's box at its own position (no-slip walls:
// the boxes along a wall differ from the free box), column-major n_B x n_B.
__global__ void k_struct_stokes(double* M, const int* __restrict__ box_of_slot, int nslot, int N, int b,
                                StokesCoef<double> c) {
  const int nB = box_nunk(b);
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= (long)nslot * nB * nB) return;
  const int s = (int)(e / ((long)nB * nB)), rem = (int)(e - (long)s * nB * nB);
  const int q = rem % nB, t = rem / nB;
  const int nb = N / b, box = box_of_slot[s], x0 = (box % nb) * b, y0 = (box / nb) * b;
  int cq, iq, jq, ct, it, jt;
  box_unknown(q, b, x0, y0, N, &cq, &iq, &jq);
  box_unknown(t, b, x0, y0, N, &ct, &it, &jt);
  M[e] = stokes_entry(c, N, cq, iq, jq, ct, it, jt);
}

// The wall faces of a no-slip level (u at x = 0, v at y = 0) set to zero.
__global__ void k_zero_walls(double* w, int N) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  w[(size_t)t * N] = 0.0;              // u(0, t)
  w[(size_t)N * N + t] = 0.0;          // v(t, 0)
}

// The moving lid of the cavity (sec. 4): u(x, L) = lid (1 - cos(2 pi x / L)) / 2.  The
// face row next to the lid, j = N - 1, reads the ghost 2 u_lid - u; its known part
// moves to the right-hand side: b -= 2 mu u_lid / h^2 (walls zeroed as well).
__global__ void k_wall_rhs(double* b, int N, double h, double mu, double lid) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  b[(size_t)i * N] = 0.0;
  b[(size_t)N * N + i] = 0.0;
  if (i > 0 && lid != 0.0) {
    const double x = i * h, L = N * h;
    const double ul = lid * 0.5 * (1.0 - cos(2.0 * M_PI * x / L));
    b[(size_t)(N - 1) * N + i] -= 2.0 * mu * ul / (h * h);
  }
}

// Position of box (I, J) in the ring of wall boxes of an nb x nb box grid: the first
// row, the last row, then the first and last column between them.
__host__ __device__ inline int ring_index(int I, int J, int nb) {
  if (nb == 1) return 0;
  if (J == 0) return I;
  if (J == nb - 1) return nb + I;
  return 2 * nb + 2 * (J - 1) + (I == 0 ? 0 : 1);
}
__host__ __device__ inline int ring_count(int nb) { return nb == 1 ? 1 : 4 * nb - 4; }

// Stokes blocks of all wall boxes of a level, in ring order (for their inverses).
__global__ void k_ring_stokes(double* M, int nring, int N, int b, StokesCoef<double> c) {
  const int nB = box_nunk(b), nb = N / b;
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= (long)nring * nB * nB) return;
  const int r = (int)(e / ((long)nB * nB)), rem = (int)(e - (long)r * nB * nB);
  int I = 0, J = 0;
  if (nb > 1) {
    if (r < nb) { I = r; J = 0; }
    else if (r < 2 * nb) { I = r - nb; J = nb - 1; }
    else { const int q = r - 2 * nb; J = 1 + q / 2; I = (q & 1) ? nb - 1 : 0; }
  }
  const int q = rem % nB, t = rem / nB;
  int cq, iq, jq, ct, it, jt;
  box_unknown(q, b, I * b, J * b, N, &cq, &iq, &jq);
  box_unknown(t, b, I * b, J * b, N, &ct, &it, &jt);
  M[e] = stokes_entry(c, N, cq, iq, jq, ct, it, jt);
}

// Slots [first, first + count) take their wall box's cached inverse.
__global__ void k_ring_copy(double* __restrict__ Ms, const int* __restrict__ box_of_slot, int first, int count,
                            const double* __restrict__ Mring, int nb, int nB2) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= (long)count * nB2) return;
  const int k = (int)(e / nB2), rem = (int)(e - (long)k * nB2);
  const int s = first + k, box = box_of_slot[s];
  Ms[(size_t)s * nB2 + rem] = Mring[(size_t)ring_index(box % nb, box / nb, nb) * nB2 + rem];
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

// Largest order inverted in shared memory (one CTA per matrix, n^2 doubles of
// dynamic shared memory up to 160 KB, so n <= 143 in practice); larger matrices
// take the blocked form below, up to INV_MAXN_BLOCKED.
constexpr int INV_MAXN = 256;
constexpr int INV_MAXN_BLOCKED = 1024;

// Magnitude of x as an integer key: a non-negative float or double orders like its
// bit pattern.
__device__ __forceinline__ unsigned long long mag_key(double x) {
  return (unsigned long long)__double_as_longlong(fabs(x));
}
__device__ __forceinline__ unsigned long long mag_key(float x) { return (unsigned long long)__float_as_uint(fabsf(x)); }

// Pivot row of column `col` among rows first..n-1 of the row-major matrix A (row
// stride ld): the largest magnitude, the lowest row on ties; found by one warp, the
// magnitudes compared as integer keys (so the floating-point pipe is left to the
// elimination; a NaN compares above every finite value and is then caught as a
// non-finite pivot).  Lane 0 holds the result.
template <typename TE>
__device__ __forceinline__ int warp_pivot_row(const TE* A, int ld, int col, int first, int n, int lane) {
  unsigned long long best = 0ull;
  int bi = n;
  for (int i = first + lane; i < n; i += 32) {
    const unsigned long long a = mag_key(A[(size_t)i * ld + col]);
    if (bi == n || a > best) { best = a; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_down_sync(0xffffffffu, best, o);
    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
    if (oi < n && (bi == n || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
  }
  return bi < n ? bi : first;
}

// Gauss-Jordan with partial pivoting on a matrix in shared memory, organised for
// the rank-1 update: thread t owns column t % n for the rows congruent to t / n
// modulo R = blockDim / n (blockDim >= n), so the update needs no index division and
// the pivot column is written in the same pass (M[i][k] = -f_i / pivot).  The row
// interchange of step k is folded into that pass: f_i and the scaled pivot row are
// read from the rows before the interchange (rows k and p trade places), so a step
// is one pivot search by warp 0 (which also forms the one reciprocal), one read
// pass and one update pass, three barriers.
template <typename TE>
__device__ void gj_invert_cols(TE* M, int n, int* err) {
  __shared__ TE f[INV_MAXN];
  __shared__ int perm[INV_MAXN];
  __shared__ TE sinv;
  __shared__ int prow;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int R = bd / n > 0 ? bd / n : 1;
  const int jc = tid % n, r0 = tid / n;
  for (int k = 0; k < n; ++k) {
    if (tid < 32) {
      const int p = warp_pivot_row(M, n, k, k, n, tid);
      if (tid == 0) {
        TE piv = M[p * n + k];
        if (!(fabs(piv) > 0.0) || !isfinite(piv)) {
          atomicOr(err, DEV_ERR_SINGULAR);
          piv = TE(1);
        }
        prow = p;
        perm[k] = p;
        sinv = TE(1) / piv;
      }
    }
    __syncthreads();
    const int p = prow;
    const TE inv = sinv;
    // after the interchange row k is the old row p and row p the old row k
    for (int i = tid; i < n; i += bd) f[i] = (i == k) ? TE(0) : M[(i == p ? k : i) * n + k];
    TE mkj = TE(0), okj = TE(0);
    if (r0 < R) {
      mkj = (jc == k ? TE(1) : M[p * n + jc]) * inv;
      okj = M[k * n + jc];
    }
    __syncthreads();
    // row k scaled (its pivot entry becomes 1/pivot); other rows updated, the
    // pivot column's entries as 0 - f_i / pivot so that a warp runs one FMA per row
    if (r0 < R) {
      for (int i = r0; i < n; i += R) {
        if (i == k) {
          M[k * n + jc] = mkj;
          continue;
        }
        const TE old = (jc == k) ? TE(0) : (i == p ? okj : M[i * n + jc]);
        M[i * n + jc] = fma(-f[i], mkj, old);
      }
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k)
      for (int i = tid; i < n; i += bd) {
        const TE t = M[i * n + k];
        M[i * n + k] = M[i * n + p];
        M[i * n + p] = t;
      }
    __syncthreads();
  }
}

// Blocked Gauss-Jordan for matrices too large for shared memory (the 8 x 8 and
// 16 x 16 boxes, the coarsest level of 16 x 16 boxes): the columns go in panels of
// GJ_PW.  k_bgj_panel runs the panel's Gauss-Jordan steps, with partial pivoting,
// on the panel's columns staged in shared memory, interchanging whole rows in
// global memory as it goes, and saves the pivot rows of every other column (after
// the interchanges, before any elimination) in U.  The steps change another column
// x only through its pivot-row entries: with Q the panel's final columns,
//   x_i <- [i not a pivot row of the panel] x_i + sum_s Q[i][s] x_{k0+s},
// which k_bgj_update applies to all other columns at once, a rank-GJ_PW product
// tiled 64 x 64 over the matrix.  These are the row operations of the unblocked
// elimination, grouped by panel; the pivots are the same.  k_bgj_unperm finally
// undoes the row interchanges as column interchanges.
constexpr int GJ_PW = 16;
constexpr int GJ_PANEL_THREADS = 512;

template <typename TE>
__global__ void __launch_bounds__(GJ_PANEL_THREADS) k_bgj_panel(TE* Ms, int n, int k0, int pw, TE* U, int* perms,
                                                                int* err) {
  extern __shared__ __align__(16) unsigned char bgj_raw[];
  TE* sP = reinterpret_cast<TE*>(bgj_raw);  // [n][GJ_PW] the panel, then f[n]
  TE* f = sP + (size_t)n * GJ_PW;
  __shared__ TE sinv;
  __shared__ int prow;
  TE* M = Ms + (size_t)blockIdx.x * n * n;
  int* perm = perms + (size_t)blockIdx.x * n;
  TE* Um = U + (size_t)blockIdx.x * GJ_PW * n;
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int e = tid; e < n * GJ_PW; e += bd) {
    const int i = e / GJ_PW, c = e - i * GJ_PW;
    sP[e] = c < pw ? M[(size_t)i * n + k0 + c] : TE(0);
  }
  __syncthreads();
  const int R = bd / GJ_PW, c = tid % GJ_PW, r0 = tid / GJ_PW;
  for (int s = 0; s < pw; ++s) {
    const int k = k0 + s;
    if (tid < 32) {
      const int p = warp_pivot_row(sP, GJ_PW, s, k, n, tid);
      if (tid == 0) {
        TE piv = sP[(size_t)p * GJ_PW + s];
        if (!(fabs(piv) > TE(0)) || !isfinite(piv)) {
          atomicOr(err, DEV_ERR_SINGULAR);
          piv = TE(1);
        }
        prow = p;
        perm[k] = p;
        sinv = TE(1) / piv;
      }
    }
    __syncthreads();
    const int p = prow;
    if (p != k) {  // whole rows: the panel here, the other columns in global memory
      for (int j = tid; j < n; j += bd) {
        if (j >= k0 && j < k0 + pw) continue;  // stale copy of the panel, rewritten below
        const TE t = M[(size_t)k * n + j];
        M[(size_t)k * n + j] = M[(size_t)p * n + j];
        M[(size_t)p * n + j] = t;
      }
      if (tid < GJ_PW) {
        const TE t = sP[(size_t)k * GJ_PW + tid];
        sP[(size_t)k * GJ_PW + tid] = sP[(size_t)p * GJ_PW + tid];
        sP[(size_t)p * GJ_PW + tid] = t;
      }
    }
    __syncthreads();
    const TE inv = sinv;
    for (int i = tid; i < n; i += bd) f[i] = (i == k) ? TE(0) : sP[(size_t)i * GJ_PW + s];
    const TE mkc = (c < pw) ? (c == s ? TE(1) : sP[(size_t)k * GJ_PW + c]) * inv : TE(0);
    __syncthreads();
    if (c < pw) {
      for (int i = r0; i < n; i += R) {
        TE* e = sP + (size_t)i * GJ_PW + c;
        if (i == k) *e = mkc;
        else if (c == s) *e = -f[i] * mkc;
        else *e -= f[i] * mkc;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < n * pw; e += bd) {
    const int i = e / pw, cc = e - i * pw;
    M[(size_t)i * n + k0 + cc] = sP[(size_t)i * GJ_PW + cc];
  }
  for (int e = tid; e < pw * n; e += bd) {
    const int s = e / n, j = e - s * n;
    Um[(size_t)s * n + j] = (j >= k0 && j < k0 + pw) ? TE(0) : M[(size_t)(k0 + s) * n + j];
  }
}

// grid (column tiles, row tiles, matrices): a 64 x 64 tile per CTA, 4 x 4 entries
// per thread, the panel's rows of the tile and the saved pivot rows staged in shared memory.
template <typename TE>
__global__ void __launch_bounds__(256) k_bgj_update(TE* Ms, int n, int k0, int pw, const TE* U, int z0) {
  __shared__ TE sQ[64][GJ_PW + 1];
  __shared__ TE sU[GJ_PW][64];
  const int z = z0 + blockIdx.z;
  TE* M = Ms + (size_t)z * n * n;
  const TE* Um = U + (size_t)z * GJ_PW * n;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64, tid = threadIdx.x;
  for (int e = tid; e < 64 * GJ_PW; e += 256) {
    const int r = e / GJ_PW, s = e - r * GJ_PW, i = i0 + r;
    sQ[r][s] = (i < n && s < pw) ? M[(size_t)i * n + k0 + s] : TE(0);
  }
  for (int e = tid; e < GJ_PW * 64; e += 256) {
    const int s = e >> 6, cc = e & 63, j = j0 + cc;
    sU[s][cc] = (j < n && s < pw) ? Um[(size_t)s * n + j] : TE(0);
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  TE acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q] = TE(0);
#pragma unroll
  for (int s = 0; s < GJ_PW; ++s) {
    TE qa[4], ub[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) qa[a] = sQ[ty + 16 * a][s];
#pragma unroll
    for (int q = 0; q < 4; ++q) ub[q] = sU[s][tx + 16 * q];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[a][q] = fma(qa[a], ub[q], acc[a][q]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty + 16 * a;
    if (i >= n) continue;
    const bool pivot_row = i >= k0 && i < k0 + pw;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + tx + 16 * q;
      if (j >= n || (j >= k0 && j < k0 + pw)) continue;
      TE* e = M + (size_t)i * n + j;
      *e = (pivot_row ? TE(0) : *e) + acc[a][q];
    }
  }
}

// Column j of the result is column idx[j] of the eliminated matrix, idx being
// 0..n-1 put through the column interchanges k <-> perm[k], k = n-1 down to 0.
// grid (groups of 8 rows, matrices z0 + y).
template <typename TE>
__global__ void k_bgj_unperm(TE* Ms, int n, const int* perms, int z0) {
  extern __shared__ __align__(16) unsigned char bgj_row[];
  TE* sRow = reinterpret_cast<TE*>(bgj_row);  // one row [n], then perm [n] and idx [n] as ints
  int* sp = reinterpret_cast<int*>(sRow + n);
  int* idx = sp + n;
  const int z = z0 + blockIdx.y;
  TE* M = Ms + (size_t)z * n * n;
  const int* perm = perms + (size_t)z * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    sp[j] = perm[j];
    idx[j] = j;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = n - 1; k >= 0; --k) {
      const int p = sp[k];
      if (p != k) {
        const int t = idx[k];
        idx[k] = idx[p];
        idx[p] = t;
      }
    }
  __syncthreads();
  const int r_end = min(n, (int)(blockIdx.x + 1) * 8);
  for (int i = blockIdx.x * 8; i < r_end; ++i) {
    TE* row = M + (size_t)i * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) sRow[j] = row[j];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) row[j] = sRow[idx[j]];
    __syncthreads();
  }
}

// The matrices of several arrays (one per level) in one launch: CTA b inverts
// matrix b - start[l] of array l, start[l] <= b < start[l + 1].
struct InvBatch {
  double* M[16];
  int start[17];
  int narr;
};

// TE: the type of the elimination (the matrices are stored in FP64 either way).
template <typename TE>
__global__ void k_invert_batch(InvBatch B, int n, int* err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TE* sm = reinterpret_cast<TE*>(smraw);
  int l = 0;
  while (l + 1 < B.narr && (int)blockIdx.x >= B.start[l + 1]) ++l;
  double* M = B.M[l] + (size_t)(blockIdx.x - B.start[l]) * n * n;
  const int nn = n * n;
  for (int e = threadIdx.x; e < nn; e += blockDim.x) sm[e] = (TE)M[e];
  __syncthreads();
  gj_invert_cols<TE>(sm, n, err);
  for (int e = threadIdx.x; e < nn; e += blockDim.x) M[e] = (double)sm[e];
}

// FP32 elimination of NB x NB box matrices (NB = 16 or 56: 2 x 2 and 4 x 4 boxes),
// one warp per matrix with the matrix in registers: lane t holds columns t and
// t + 32.  A step broadcasts column k through shared memory, finds the pivot
// (integer keys, a butterfly so that every lane has it), reads the pivot row and
// row k of its columns by selecting over the unrolled rows, and updates every row
// of its columns with the interchange of rows k and p folded in, as in
// gj_invert_cols; no block barriers.  The column interchanges that undo the row
// interchanges are applied as the columns are written back.
template <int NB>
__global__ void __launch_bounds__(128) k_invert_warp_f32(InvBatch B, int total, int* err) {
  constexpr int NC = (NB + 31) / 32;
  __shared__ float fcol[4][NB];
  __shared__ int sidx[4][NB];
  __shared__ int spos[4][NB];
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int mat = blockIdx.x * 4 + wq;
  if (mat >= total) return;  // whole warps: no barrier below involves other warps
  int l = 0;
  while (l + 1 < B.narr && mat >= B.start[l + 1]) ++l;
  double* M = B.M[l] + (size_t)(mat - B.start[l]) * NB * NB;
  float a[NC][NB];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int j = lane + 32 * c;
#pragma unroll
    for (int i = 0; i < NB; ++i) a[c][i] = j < NB ? (float)M[i * NB + j] : 0.f;
  }
  for (int k = 0; k < NB; ++k) {
    const int lk = k & 31, ck = k >> 5;
    if (lane == lk) {
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        float v = a[0][i];
#pragma unroll
        for (int c = 1; c < NC; ++c) v = ck == c ? a[c][i] : v;
        fcol[wq][i] = v;
      }
    }
    __syncwarp();
    unsigned key = 0u;
    int bi = NB;
    for (int i = k + lane; i < NB; i += 32) {
      const unsigned v = __float_as_uint(fabsf(fcol[wq][i]));
      if (bi == NB || v > key) { key = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned ok = __shfl_xor_sync(0xffffffffu, key, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (oi < NB && (bi == NB || ok > key || (ok == key && oi < bi))) { key = ok; bi = oi; }
    }
    const int p = bi < NB ? bi : k;
    float piv = fcol[wq][p];
    if (!(fabsf(piv) > 0.f) || !isfinite(piv)) {
      if (lane == 0) atomicOr(err, DEV_ERR_SINGULAR);
      piv = 1.f;
    }
    const float inv = 1.f / piv;
    if (lane == 0) sidx[wq][k] = p;
    float mk[NC], okv[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float ap = 0.f, akv = 0.f;
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        ap = i == p ? a[c][i] : ap;
        akv = i == k ? a[c][i] : akv;
      }
      mk[c] = (lane + 32 * c == k ? 1.f : ap) * inv;
      okv[c] = akv;
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const float fi = i == k ? 0.f : fcol[wq][i == p ? k : i];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float old = lane + 32 * c == k ? 0.f : (i == p ? okv[c] : a[c][i]);
        a[c][i] = i == k ? mk[c] : fmaf(-fi, mk[c], old);
      }
    }
    __syncwarp();
  }
  // column j of the result is eliminated column idx[j] (idx: 0..NB-1 through the
  // interchanges k <-> p_k, k = NB-1 down to 0); eliminated column t goes to pos[t]
  if (lane == 0) {
    for (int j = 0; j < NB; ++j) spos[wq][j] = j;
    for (int k = NB - 1; k >= 0; --k) {
      const int p = sidx[wq][k];
      if (p != k) {
        const int t = spos[wq][k];
        spos[wq][k] = spos[wq][p];
        spos[wq][p] = t;
      }
    }
  }
  __syncwarp();
  for (int j = lane; j < NB; j += 32) sidx[wq][spos[wq][j]] = j;
  __syncwarp();
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int j = lane + 32 * c;
    if (j >= NB) continue;
    const int jo = sidx[wq][j];
#pragma unroll
    for (int i = 0; i < NB; ++i) M[i * NB + jo] = (double)a[c][i];
  }
}

// One matrix per CTA, staged in shared memory (n^2 doubles of dynamic shared memory).
__global__ void k_invert_sm(double* Ms, int n, int* err) {
  extern __shared__ double sm[];
  double* M = Ms + (size_t)blockIdx.x * n * n;
  const int nn = n * n;
  for (int e = threadIdx.x; e < nn; e += blockDim.x) sm[e] = M[e];
  __syncthreads();
  gj_invert_cols<double>(sm, n, err);
  for (int e = threadIdx.x; e < nn; e += blockDim.x) M[e] = sm[e];
}

// 5 x 5 matrices (1 x 1 boxes), one per thread in registers: the same
// Gauss-Jordan steps with partial pivoting.
__global__ void k_invert5(double* Ms, int count, int* err) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  double* Mg = Ms + (size_t)t * 25;
  double M[25];
  int perm[5];
#pragma unroll
  for (int e = 0; e < 25; ++e) M[e] = Mg[e];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    int p = k;
    double best = fabs(M[k * 5 + k]);
#pragma unroll
    for (int i = k + 1; i < 5; ++i) {
      double a = fabs(M[i * 5 + k]);
      if (a > best) { best = a; p = i; }
    }
    perm[k] = p;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      double a = M[k * 5 + j], b = M[p * 5 + j];
      M[k * 5 + j] = (p == k) ? a : b;
      M[p * 5 + j] = (p == k) ? b : a;
    }
    double piv = M[k * 5 + k];
    if (!(fabs(piv) > 0.0) || !isfinite(piv)) {
      atomicOr(err, DEV_ERR_SINGULAR);
      piv = 1.0;
    }
    double inv = 1.0 / piv;
    M[k * 5 + k] = 1.0;
#pragma unroll
    for (int j = 0; j < 5; ++j) M[k * 5 + j] *= inv;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      if (i == k) continue;
      double fi = M[i * 5 + k];
      M[i * 5 + k] = 0.0;
#pragma unroll
      for (int j = 0; j < 5; ++j) M[i * 5 + j] -= fi * M[k * 5 + j];
    }
  }
#pragma unroll
  for (int k = 4; k >= 0; --k) {
    int p = perm[k];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      double a = M[i * 5 + k], b = M[i * 5 + p];
      M[i * 5 + k] = (p == k) ? a : b;
      M[i * 5 + p] = (p == k) ? b : a;
    }
  }
#pragma unroll
  for (int e = 0; e < 25; ++e) Mg[e] = M[e];
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
  c.walls = P.prm.walls;
  return c;
}

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

// Stokes block of the structure-free box of a level into L.Sfree and its inverse
// into L.Mfree (and L.Mfree32): it depends only on the grid and fluid
// parameters, so it is computed once per problem.
int launch_free_box(Problem& P, int level) {
  LevelInfo& L = P.lev[level];
  int nB = P.nB;
  StokesCoef<double> c = coef_of<double>(P, level);
  c.walls = 0;  // the free box is an interior box: no wall rows (the boxes along walls are structure slots)
  {
    KScope ks(P, IB_KC_SETUP, nB * nB * 8.0);
    k_box_stokes<<<nblk((long)nB * nB), TPB, 0, P.stream>>>(L.Sfree, L.N, P.prm.box, c);
    IB_LAUNCH_CHECK();
  }
  IB_CUDA_TRY(cudaMemcpyAsync(L.Mfree, L.Sfree, sizeof(double) * nB * nB, cudaMemcpyDeviceToDevice, P.stream));
  IB_TRY(launch_invert(P, L.Mfree, nB, 1));
  if (L.Mfree32) IB_TRY((launch_cast<double, float>(P, L.Mfree, L.Mfree32, (size_t)nB * nB)));
  return IB_OK;
}

int launch_zero_walls(Problem& P, double* w) {
  const int N = P.prm.N;
  KScope ks(P, IB_KC_OTHER, 16.0 * N);
  k_zero_walls<<<nblk(N), TPB, 0, P.stream>>>(w, N);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_wall_rhs(Problem& P, double* b) {
  const int N = P.prm.N;
  KScope ks(P, IB_KC_OTHER, 32.0 * N);
  k_wall_rhs<<<nblk(N), TPB, 0, P.stream>>>(b, N, P.prm.L / N, P.prm.mu, P.prm.lid);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

// The inverses of every wall box of a level (no-slip walls), computed once.
int launch_ring_prepare(Problem& P, int level) {
  LevelInfo& L = P.lev[level];
  const int nB = P.nB, nring = ring_count(L.nb);
  if (!L.Mring) IB_TRY(dalloc(&L.Mring, (size_t)nring * nB * nB));
  L.nring = nring;
  const long tot = (long)nring * nB * nB;
  {
    KScope ks(P, IB_KC_SETUP, tot * 8.0);
    k_ring_stokes<<<nblk(tot), TPB, 0, P.stream>>>(L.Mring, nring, L.N, P.prm.box, coef_of<double>(P, level));
    IB_LAUNCH_CHECK();
  }
  return launch_invert(P, L.Mring, nB, nring);
}

int launch_ring_copy(Problem& P, int level) {
  LevelInfo& L = P.lev[level];
  const int count = L.n_struct - L.n_form, nB2 = P.nB * P.nB;
  if (count <= 0) return IB_OK;
  const long tot = (long)count * nB2;
  KScope ks(P, IB_KC_SETUP, tot * 16.0);
  k_ring_copy<<<nblk(tot), TPB, 0, P.stream>>>(L.Mstruct, L.box_of_slot, L.n_form, count, L.Mring, L.nb, nB2);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

// Every structure slot starts from the Stokes block of its box: the free box's
// (periodic), or with no-slip walls the block at the box's own position.
int launch_struct_fill(Problem& P, int level) {
  LevelInfo& L = P.lev[level];
  int nB = P.nB;
  if (L.n_form > 0) {
    long tot = (long)nB * nB * L.n_form;
    KScope ks(P, IB_KC_SETUP, tot * (P.prm.walls ? 8.0 : 16.0));
    if (P.prm.walls)
      k_struct_stokes<<<nblk(tot), TPB, 0, P.stream>>>(L.Mstruct, L.box_of_slot, L.n_form, L.N, P.prm.box,
                                                      coef_of<double>(P, level));
    else
      k_replicate<<<nblk(tot), TPB, 0, P.stream>>>(L.Sfree, L.Mstruct, nB * nB, L.n_form);
    IB_LAUNCH_CHECK();
  }
  return IB_OK;
}

// The blocked Gauss-Jordan over count matrices: per panel of GJ_PW columns one
// panel launch (a CTA per matrix) and one update launch (64 x 64 tiles of every
// matrix), then the column interchanges.  Its workspace (saved pivot rows and
// pivot indices) grows on demand and is kept with the problem.
template <typename TE>
int run_bgj(Problem& P, TE* M, int n, int count) {
  const size_t smem_panel = (size_t)n * (GJ_PW + 1) * sizeof(TE);
  const size_t smem_unperm = (size_t)n * (sizeof(TE) + 2 * sizeof(int));
  static std::once_flag once;
  cudaError_t ae = cudaSuccess;
  std::call_once(once, [&] {
    const int mx = (int)((size_t)INV_MAXN_BLOCKED * (GJ_PW + 1) * sizeof(TE));
    ae = cudaFuncSetAttribute(k_bgj_panel<TE>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  });
  IB_CUDA_TRY(ae);
  TE* U = reinterpret_cast<TE*>(P.inv_ws);
  const int tiles = (n + 63) / 64;
  for (int k0 = 0; k0 < n; k0 += GJ_PW) {
    const int pw = n - k0 < GJ_PW ? n - k0 : GJ_PW;
    k_bgj_panel<TE><<<count, GJ_PANEL_THREADS, smem_panel, P.stream>>>(M, n, k0, pw, U, P.inv_perm, P.dev_err);
    IB_LAUNCH_CHECK();
    for (int z0 = 0; z0 < count; z0 += 65535) {
      const int nz = count - z0 < 65535 ? count - z0 : 65535;
      k_bgj_update<TE><<<dim3(tiles, tiles, nz), 256, 0, P.stream>>>(M, n, k0, pw, U, z0);
      IB_LAUNCH_CHECK();
    }
  }
  for (int z0 = 0; z0 < count; z0 += 65535) {
    const int nz = count - z0 < 65535 ? count - z0 : 65535;
    k_bgj_unperm<TE><<<dim3((n + 7) / 8, nz), 256, smem_unperm, P.stream>>>(M, n, P.inv_perm, z0);
    IB_LAUNCH_CHECK();
  }
  return IB_OK;
}

// fp32: the elimination in FP32 on a rounded copy of the matrices (a stream-ordered
// temporary), the inverses written back in FP64.
int launch_invert_blocked(Problem& P, double* M, int n, int count, bool fp32) {
  const size_t ws = (size_t)count * GJ_PW * n, wp = (size_t)count * n;
  if (ws > P.inv_ws_cap) {
    dfree(P.inv_ws);
    P.inv_ws_cap = 0;
    IB_TRY(dalloc(&P.inv_ws, ws));
    P.inv_ws_cap = ws;
  }
  if (wp > P.inv_perm_cap) {
    dfree(P.inv_perm);
    P.inv_perm_cap = 0;
    IB_TRY(dalloc(&P.inv_perm, wp));
    P.inv_perm_cap = wp;
  }
  if (!fp32) return run_bgj<double>(P, M, n, count);
  const size_t nn = (size_t)count * n * n;
  float* M32 = nullptr;
  IB_CUDA_TRY(cudaMallocAsync((void**)&M32, nn * sizeof(float), P.stream));
  int rc = launch_cast<double, float>(P, M, M32, nn);
  if (rc == IB_OK) rc = run_bgj<float>(P, M32, n, count);
  if (rc == IB_OK) rc = launch_cast<float, double>(P, M32, M, nn);
  cudaFreeAsync(M32, P.stream);
  return rc;
}

// Invert count n x n matrices stored back to back: 5 x 5 in registers (one per
// thread), n^2 doubles that fit in shared memory staged there (one CTA each),
// larger ones by the blocked form in global memory.
int launch_invert(Problem& P, double* M, int n, int count, bool fp32) {
  if (count <= 0) return IB_OK;
  size_t smem = (size_t)n * n * sizeof(double);
  if (smem > 160u * 1024u ? n > INV_MAXN_BLOCKED : n > INV_MAXN)
    return fail(IB_ERR_INVALID_ARG, "matrix too large for the device inverse");
  KScope ks(P, IB_KC_SETUP, 2.0 * count * n * n * 8.0);
  if (n == 5) {
    k_invert5<<<nblk(count, 128), 128, 0, P.stream>>>(M, count, P.dev_err);
  } else if (smem <= 160u * 1024u) {
    static std::once_flag once;
    cudaError_t ae = cudaSuccess;
    std::call_once(once, [&] {
      ae = cudaFuncSetAttribute(k_invert_sm, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    });
    IB_CUDA_TRY(ae);
    const int threads = 256;
    k_invert_sm<<<count, threads, smem, P.stream>>>(M, n, P.dev_err);
  } else {
    IB_TRY(launch_invert_blocked(P, M, n, count, fp32));
  }
  IB_LAUNCH_CHECK();
  return IB_OK;
}

// All structure-box inverses of the smoothing levels in one launch (n_B^2 doubles
// of shared memory per CTA); returns false if they do not fit in shared memory,
// in which case the caller inverts level by level.  fp32: the elimination in FP32
// (the inverses stored in FP64 as before).
int launch_invert_struct_all(Problem& P, bool* done, bool fp32) {
  *done = false;
  const int n = P.nB;
  const size_t smem = (size_t)n * n * (fp32 ? sizeof(float) : sizeof(double));
  if (n == 5 || smem > 160u * 1024u || P.nlev - 1 > 16) return IB_OK;
  InvBatch B;
  std::memset(&B, 0, sizeof(B));
  int tot = 0;
  for (int l = 0; l < P.nlev - 1; ++l) {
    B.M[B.narr] = P.lev[l].Mstruct;
    B.start[B.narr] = tot;
    tot += P.lev[l].n_form;
    ++B.narr;
  }
  B.start[B.narr] = tot;
  *done = true;
  if (tot == 0) return IB_OK;
  static std::once_flag once;
  cudaError_t ae = cudaSuccess;
  std::call_once(once, [&] {
    ae = cudaFuncSetAttribute(k_invert_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (ae == cudaSuccess)
      ae = cudaFuncSetAttribute(k_invert_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  });
  IB_CUDA_TRY(ae);
  const int threads = 256;
  KScope ks(P, IB_KC_SETUP, 2.0 * tot * n * n * sizeof(double));
  if (fp32 && n == 56)
    k_invert_warp_f32<56><<<(tot + 3) / 4, 128, 0, P.stream>>>(B, tot, P.dev_err);
  else if (fp32 && n == 16)
    k_invert_warp_f32<16><<<(tot + 3) / 4, 128, 0, P.stream>>>(B, tot, P.dev_err);
  else if (fp32)
    k_invert_batch<float><<<tot, threads, smem, P.stream>>>(B, n, P.dev_err);
  else
    k_invert_batch<double><<<tot, threads, smem, P.stream>>>(B, n, P.dev_err);
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
