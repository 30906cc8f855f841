// Flexible GMRES building blocks (sec. 3.3: GMRES right-preconditioned by the
// V-cycle; flexible form so that an FP32 preconditioner is admissible).  All
// vectors are FP64; reductions are two-stage and deterministic.  The Krylov
// bases (V, Z) are read with the streaming cache hint (evict first): at a few
// hundred MB they would otherwise push the V-cycle's working set out of L2
// between preconditioner applications.
#include <cmath>

#include "ib_internal.cuh"

namespace ib {

namespace {

constexpr int TPB = 256;
inline int nblk(long n, int t = TPB) { return (int)((n + t - 1) / t); }

__device__ inline double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sh[q];
  }
  return s;  // valid in thread 0
}

// partial[blk * stride + i] = sum over the block's range of V_i . w.  The basis
// vectors are taken MDG at a time: per element w is read once and MDG independent
// loads are in flight, and one block reduction serves the whole group.
constexpr int MDG = 8;
__global__ void k_multidot_partial(const double* __restrict__ V, int nvec, long n,
                                   const double* __restrict__ w, double* partial, int stride) {
  __shared__ double sh[32][MDG];  // [warp][vector of the group]
  const long per = (n + gridDim.x - 1) / gridDim.x;
  const long lo = blockIdx.x * per, hi = lo + per < n ? lo + per : n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i0 = 0; i0 < nvec; i0 += MDG) {
    const int nv = nvec - i0 < MDG ? nvec - i0 : MDG;
    const double* v0 = V + (size_t)i0 * n;
    double acc[MDG];
#pragma unroll
    for (int q = 0; q < MDG; ++q) acc[q] = 0.0;
    for (long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      const double we = w[e];
#pragma unroll
      for (int q = 0; q < MDG; ++q)
        if (q < nv) acc[q] += __ldcs(v0 + (size_t)q * n + e) * we;
    }
#pragma unroll
    for (int q = 0; q < MDG; ++q)
      for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], o);
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < MDG; ++q) sh[wid][q] = acc[q];
    __syncthreads();
    if (threadIdx.x < nv) {
      double s = 0.0;
      for (int q = 0; q < nw; ++q) s += sh[q][threadIdx.x];
      partial[(size_t)blockIdx.x * stride + i0 + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

__global__ void k_multidot_final(const double* __restrict__ partial, int nblocks, int stride,
                                 double* out) {
  __shared__ double sh[32];
  int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(size_t)b * stride + i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[i] = s;
}

// w -= sum_i coef[i] V_i
__global__ void k_multiaxpy(const double* __restrict__ V, int nvec, long n,
                            const double* __restrict__ coef, double* w) {
  __shared__ double c[520];
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) c[i] = coef[i];
  __syncthreads();
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  double s = w[e];
#pragma unroll 8
  for (int i = 0; i < nvec; ++i) s -= c[i] * __ldcs(V + (size_t)i * n + e);
  w[e] = s;
}

// y = x * s or y = x / s with the scalar s on the device
__global__ void k_scale_copy(const double* __restrict__ x, const double* __restrict__ s, double* y,
                             long n, int invert) {
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  double a = *s;
  y[e] = invert ? x[e] / a : x[e] * a;
}

// Givens step of FGMRES iteration j.  H (column-major, ld m + 1) column j is
// h1 + h2 from the two Gram-Schmidt passes and ||w|| below the diagonal; the
// previous rotations are applied, a new one is formed, and g is updated.
// scal layout: [0] |g_{j+1}|, [1] H_{j+1,j} (= ||w||), [2] non-finite flag.
__global__ void k_givens(double* H, int ld, int j, const double* h1, const double* h2,
                         const double* wnorm2, double* cs, double* sn, double* g, double* scal) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* col = H + (size_t)j * ld;
  for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
  double hn = sqrt(fmax(*wnorm2, 0.0));
  col[j + 1] = hn;
  scal[1] = hn;
  for (int i = 0; i < j; ++i) {
    double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  double a = col[j], b = col[j + 1];
  double den = hypot(a, b);
  double c = den > 0.0 ? a / den : 1.0, s = den > 0.0 ? b / den : 0.0;
  cs[j] = c;
  sn[j] = s;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  scal[0] = fabs(g[j + 1]);
  scal[2] = (isfinite(den) && isfinite(g[j + 1])) ? 0.0 : 1.0;
}

// y = R^{-1} g for the leading k x k triangle of H.
__global__ void k_backsolve(const double* H, int ld, int k, const double* g, double* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int q = i + 1; q < k; ++q) s -= H[(size_t)q * ld + i] * y[q];
    y[i] = s / H[(size_t)i * ld + i];
  }
}

template <typename T>
__global__ void k_update_x(const T* __restrict__ Z, int k, long n, const double* __restrict__ y,
                           double* x) {
  __shared__ double c[520];
  for (int i = threadIdx.x; i < k; i += blockDim.x) c[i] = y[i];
  __syncthreads();
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  double s = x[e];
#pragma unroll 8
  for (int i = 0; i < k; ++i) s += c[i] * (double)__ldcs(Z + (size_t)i * n + e);
  x[e] = s;
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* z, long n) {
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e < n) z[e] = a * x[e] + (y ? b * y[e] : 0.0);
}

__global__ void k_sub_scalar(double* x, long n, const double* s, double scale) {
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e < n) x[e] -= (*s) * scale;
}

}  // namespace

static inline long nvec_len(const Problem& P) { return 3L * P.lev[0].N * P.lev[0].N; }

int launch_multidot(Problem& P, const double* V, int nvec, const double* w, double* out) {
  long n = nvec_len(P);
  int stride = P.max_m + 2;
  {
    KScope ks(P, IB_KC_KRYLOV, (nvec + 1.0) * n * 8.0);
    k_multidot_partial<<<P.dot_blocks, TPB, 0, P.stream>>>(V, nvec, n, w, P.dots, stride);
    IB_LAUNCH_CHECK();
  }
  {
    KScope ks(P, IB_KC_KRYLOV, (double)nvec * P.dot_blocks * 8.0);
    k_multidot_final<<<nvec, TPB, 0, P.stream>>>(P.dots, P.dot_blocks, stride, out);
    IB_LAUNCH_CHECK();
  }
  return IB_OK;
}

int launch_multiaxpy(Problem& P, const double* V, int nvec, const double* coef, double* w) {
  long n = nvec_len(P);
  KScope ks(P, IB_KC_KRYLOV, (nvec + 2.0) * n * 8.0);
  k_multiaxpy<<<nblk(n), TPB, 0, P.stream>>>(V, nvec, n, coef, w);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_dot(Problem& P, const double* a, const double* b, double* out) {
  long n = nvec_len(P);
  int stride = P.max_m + 2;
  {
    KScope ks(P, IB_KC_KRYLOV, 2.0 * n * 8.0);
    k_multidot_partial<<<P.dot_blocks, TPB, 0, P.stream>>>(a, 1, n, b, P.dots, stride);
    IB_LAUNCH_CHECK();
  }
  {
    KScope ks(P, IB_KC_KRYLOV, (double)P.dot_blocks * 8.0);
    k_multidot_final<<<1, TPB, 0, P.stream>>>(P.dots, P.dot_blocks, stride, out);
    IB_LAUNCH_CHECK();
  }
  return IB_OK;
}

int launch_scale_copy(Problem& P, const double* x, const double* s, double* y, bool invert) {
  long n = nvec_len(P);
  KScope ks(P, IB_KC_KRYLOV, 2.0 * n * 8.0);
  k_scale_copy<<<nblk(n), TPB, 0, P.stream>>>(x, s, y, n, invert ? 1 : 0);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

// givens layout: cs[m] | sn[m] | g[m + 1] | y[m];  scal: [0..2] Givens outputs,
// [8 .. 8 + m + 1] h1, [8 + m + 2 ..] h2, then ||w||^2.
int launch_givens(Problem& P, int j, double /*unused*/, double* /*unused*/) {
  int m = P.max_m;
  double* cs = P.givens;
  double* sn = cs + m;
  double* g = sn + m;
  double* h1 = P.scal + 8;
  double* h2 = h1 + m + 2;
  double* wn = h2 + m + 2;
  KScope ks(P, IB_KC_KRYLOV, 8.0 * (4.0 * j + 8));
  k_givens<<<1, 32, 0, P.stream>>>(P.H, m + 1, j, h1, h2, wn, cs, sn, g, P.scal);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_backsolve(Problem& P, int k) {
  int m = P.max_m;
  double* g = P.givens + 2 * m;
  double* y = g + m + 1;
  KScope ks(P, IB_KC_KRYLOV, 8.0 * k * (k + 2.0));
  k_backsolve<<<1, 32, 0, P.stream>>>(P.H, m + 1, k, g, y);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

template <typename T>
int launch_update_x(Problem& P, const T* Z, int k, double* x, int first) {
  if (k <= 0) return IB_OK;
  int m = P.max_m;
  const double* y = P.givens + 3 * m + 1 + first;
  Z += (size_t)first * 3 * P.lev[0].N * P.lev[0].N;
  long n = nvec_len(P);
  KScope ks(P, IB_KC_KRYLOV, (double)k * n * sizeof(T) + 2.0 * n * 8.0);
  k_update_x<T><<<nblk(n), TPB, 0, P.stream>>>(Z, k, n, y, x);
  IB_LAUNCH_CHECK();
  return IB_OK;
}
template int launch_update_x<double>(Problem&, const double*, int, double*, int);
template int launch_update_x<float>(Problem&, const float*, int, double*, int);

int launch_axpby(Problem& P, double a, const double* x, double b, const double* y, double* z) {
  long n = nvec_len(P);
  KScope ks(P, IB_KC_KRYLOV, 3.0 * n * 8.0);
  k_axpby<<<nblk(n), TPB, 0, P.stream>>>(a, x, b, y, z, n);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

// Subtract the mean of the pressure block (the constant-pressure null space).
int launch_pressure_mean_remove(Problem& P, double* w) {
  int N = P.lev[0].N;
  long n = (long)N * N;
  double* ones = P.t64b;  // [0 | 0 | 1]
  IB_TRY(launch_fill<double>(P, ones, (size_t)(2 * n), 0.0));
  IB_TRY(launch_fill<double>(P, ones + 2 * n, (size_t)n, 1.0));
  int stride = P.max_m + 2;
  {
    KScope ks(P, IB_KC_OTHER, 6.0 * n * 8.0);
    k_multidot_partial<<<P.dot_blocks, TPB, 0, P.stream>>>(ones, 1, 3 * n, w, P.dots, stride);
    IB_LAUNCH_CHECK();
  }
  {
    KScope ks(P, IB_KC_OTHER, (double)P.dot_blocks * 8.0);
    k_multidot_final<<<1, TPB, 0, P.stream>>>(P.dots, P.dot_blocks, stride, P.scal + 3);
    IB_LAUNCH_CHECK();
  }
  {
    KScope ks(P, IB_KC_OTHER, 2.0 * n * 8.0);
    k_sub_scalar<<<nblk(n), TPB, 0, P.stream>>>(w + 2 * n, n, P.scal + 3, 1.0 / (double)n);
    IB_LAUNCH_CHECK();
  }
  return IB_OK;
}

}  // namespace ib
