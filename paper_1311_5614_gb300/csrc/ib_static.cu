// Allocation-free fine-level operator apply.
//
// ib_apply_noalloc computes the same y = A_0 w as ib_apply on level 0, but
// without a problem handle and without allocating any device memory: the
// caller passes the structure and the vectors as device pointers, and the one
// piece of scratch the elasticity term needs (the velocity interpolated to the
// points, S^* w) lives in a fixed-size array in this file's static device
// memory.  It exists for callers that cannot allocate device memory: code that
// must not stall on cudaMalloc's implicit device synchronisation in the middle
// of a time step, or a host framework that owns all device memory through its
// own pool and does not let libraries allocate.
//
// Rules of the shared static scratch (see include/ib.h):
//  * its size bounds n_points (IB_NOALLOC_MAX_POINTS); larger calls are rejected;
//  * every call on a device uses the same array, so calls that overlap on the
//    GPU (other streams, other host threads) race and must be serialised by the
//    caller;
//  * the array keeps the previous call's contents; each call writes every entry
//    it later reads (the interpolated velocities of its own points) and clears
//    the error word before its kernels run;
//  * the first call on each device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make that
//    first call before any stream capture.
#include <mutex>

#include "ib_internal.cuh"

namespace ib {
namespace {

constexpr int kMaxPoints = IB_NOALLOC_MAX_POINTS;
constexpr int kMaxDevices = 64;

// U[0 .. n) = x-velocity at the points, U[kMaxPoints .. kMaxPoints + n) = y-velocity.
static __device__ __align__(256) double g_scratch_U[2 * kMaxPoints];
static __device__ __align__(256) int g_scratch_err[4];

std::mutex g_mu;
double* g_U_addr[kMaxDevices] = {};
int* g_err_addr[kMaxDevices] = {};

// 1-D delta kernels in grid units: Peskin's 4-point function or the cosine function.
__device__ inline double na_phi(double r, int kind) {
  double a = fabs(r);
  if (a >= 2.0) return 0.0;
  if (kind == IB_DELTA_COS4) return 0.25 * (1.0 + cospi(0.5 * r));
  if (a < 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) * 0.125;
  return (5.0 - 2.0 * a - sqrt(fmax(-7.0 + 12.0 * a - 4.0 * a * a, 0.0))) * 0.125;
}

// Base node and the four 1-D weights along one direction of one component grid.
__device__ inline int na_weights(double xh, bool centred, int N, int kind, double w[4]) {
  double sc = centred ? xh - 0.5 : xh;
  double fl = floor(sc);
  double frac = sc - fl;
  for (int a = 0; a < 4; ++a) w[a] = na_phi((double)(a - 1) - frac, kind);
  return (int)(fl - N * floor(fl / N)) - 1;
}

__global__ void na_stokes(const double* __restrict__ w, double* __restrict__ y, int N, double diag,
                          double off, double g) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int n = N * N;
  if (idx >= n) return;
  int i = idx & (N - 1), j = idx / N;
  int ip = (i + 1) & (N - 1), im = (i - 1) & (N - 1);
  int jp = (j + 1) & (N - 1), jm = (j - 1) & (N - 1);
  const double* u = w;
  const double* v = w + n;
  const double* p = w + 2 * n;
  int e = j * N + ip, wq = j * N + im, nq = jp * N + i, sq = jm * N + i;
  y[idx] = diag * u[idx] + off * (u[e] + u[wq] + u[nq] + u[sq]) - g * (p[idx] - p[wq]);
  y[n + idx] = diag * v[idx] + off * (v[e] + v[wq] + v[nq] + v[sq]) - g * (p[idx] - p[sq]);
  y[2 * n + idx] = g * (u[e] - u[idx] + v[nq] - v[idx]);
}

// U = S^* w at every point (thread per point and component), into the scratch.
__global__ void na_interp(const double* __restrict__ X, int np, const double* __restrict__ w, int N,
                          double inv_h, int kind, double* U) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * np) return;
  int comp = t / np, k = t - comp * np;
  double wx[4], wy[4];
  int x0 = na_weights(X[2 * k] * inv_h, comp == 1, N, kind, wx);
  int y0 = na_weights(X[2 * k + 1] * inv_h, comp == 0, N, kind, wy);
  const double* wc = w + (size_t)comp * N * N;
  double s = 0.0;
  for (int b = 0; b < 4; ++b) {
    const double* row = wc + ((y0 + b) & (N - 1)) * N;
    double sx = 0.0;
    for (int a = 0; a < 4; ++a) sx += wx[a] * row[(x0 + a) & (N - 1)];
    s += wy[b] * sx;
  }
  U[comp * kMaxPoints + k] = s;
}

__device__ inline void na_spread_point(const double* X, int k, double gx, double gy, int N, double inv_h,
                                       int kind, double* y) {
  int n = N * N;
  for (int comp = 0; comp < 2; ++comp) {
    double g = comp == 0 ? gx : gy;
    if (g == 0.0) continue;
    double wx[4], wy[4];
    int x0 = na_weights(X[2 * k] * inv_h, comp == 1, N, kind, wx);
    int y0 = na_weights(X[2 * k + 1] * inv_h, comp == 0, N, kind, wy);
    for (int b = 0; b < 4; ++b) {
      double gy_ = g * wy[b];
      if (gy_ == 0.0) continue;
      double* row = y + comp * n + ((y0 + b) & (N - 1)) * N;
      for (int a = 0; a < 4; ++a)
        if (wx[a] != 0.0) atomicAdd(&row[(x0 + a) & (N - 1)], wx[a] * gy_);
    }
  }
}

// Per spring (i, j): g = K (U_j - U_i) with K = dF_i/dX_j at X; spread coef * g at
// point i and -coef * g at point j.  Bad indices or coincident end points set the
// error word and skip the spring.
__global__ void na_springs(const double* __restrict__ X, int np, const int* __restrict__ ij,
                           const double* __restrict__ kappa, const double* __restrict__ rest, int ns,
                           double L, int clamped, const double* __restrict__ U, int N, double inv_h,
                           int kind, double coef, double* y, int* err) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ns) return;
  int i = ij[2 * e], j = ij[2 * e + 1];
  if (i < 0 || j < 0 || i >= np || j >= np || i == j) {
    atomicOr(err, 1);
    return;
  }
  double dx = X[2 * j] - X[2 * i], dy = X[2 * j + 1] - X[2 * i + 1];
  dx -= L * rint(dx / L);
  dy -= L * rint(dy / L);
  double l = sqrt(dx * dx + dy * dy);
  if (!(l > 0.0) || !isfinite(l)) {
    atomicOr(err, 2);
    return;
  }
  double kap = kappa[e], s = 1.0 - rest[e] / l;
  double tx = dx / l, ty = dy / l;
  double st = clamped ? fmax(s, 0.0) : s;
  double kxx = kap * (st * (1.0 - tx * tx) + tx * tx);
  double kxy = kap * (1.0 - st) * tx * ty;
  double kyy = kap * (st * (1.0 - ty * ty) + ty * ty);
  double ux = U[j] - U[i], uy = U[kMaxPoints + j] - U[kMaxPoints + i];
  double gx = coef * (kxx * ux + kxy * uy), gy = coef * (kxy * ux + kyy * uy);
  na_spread_point(X, i, gx, gy, N, inv_h, kind, y);
  na_spread_point(X, j, -gx, -gy, N, inv_h, kind, y);
}

__global__ void na_clear_err(int* err) {
  if (threadIdx.x < 4) err[threadIdx.x] = 0;
}

// Device address of the static scratch for the current device (looked up once).
int scratch_for_current_device(double** U, int** err) {
  int dev = -1;
  IB_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(IB_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_U_addr[dev]) {
    double* u = nullptr;
    int* e = nullptr;
    IB_CUDA_TRY(cudaGetSymbolAddress((void**)&u, g_scratch_U));
    IB_CUDA_TRY(cudaGetSymbolAddress((void**)&e, g_scratch_err));
    g_U_addr[dev] = u;
    g_err_addr[dev] = e;
  }
  *U = g_U_addr[dev];
  *err = g_err_addr[dev];
  return IB_OK;
}

}  // namespace
}  // namespace ib

using namespace ib;

extern "C" int ib_apply_noalloc(const ib_params* prm, int32_t n_points, const double* X,
                                int32_t n_springs, const int32_t* springs, const double* kappa,
                                const double* rest, const double* w, double* y, void* stream) {
  set_error("");
  if (!prm || !w || !y) return fail(IB_ERR_INVALID_ARG, "NULL argument");
  int N = prm->N;
  if (N < 8 || N > (1 << 14) || (N & (N - 1)) != 0)
    return fail(IB_ERR_INVALID_ARG, "N must be a power of two in 8..16384");
  if (!(prm->L > 0) || !(prm->mu > 0) || !(prm->dt > 0) || !(prm->rho >= 0))
    return fail(IB_ERR_INVALID_ARG, "L, mu, dt must be > 0 and rho >= 0");
  if (prm->delta != IB_DELTA_PESKIN4 && prm->delta != IB_DELTA_COS4)
    return fail(IB_ERR_INVALID_ARG, "unknown delta kernel");
  if (prm->walls != IB_WALLS_PERIODIC)
    return fail(IB_ERR_INVALID_ARG, "ib_apply_noalloc is for the periodic square only");
  if (n_points < 0 || n_springs < 0) return fail(IB_ERR_INVALID_ARG, "negative counts");
  if (n_points > IB_NOALLOC_MAX_POINTS)
    return fail(IB_ERR_INVALID_ARG, "n_points exceeds IB_NOALLOC_MAX_POINTS (65536), the size of the "
                                    "static scratch of ib_apply_noalloc");
  if (n_springs > 0 && (n_points == 0 || !X || !springs || !kappa || !rest))
    return fail(IB_ERR_INVALID_ARG, "spring arrays need points and non-NULL pointers");
  if (w == y) return fail(IB_ERR_INVALID_ARG, "w and y must not alias");
  cudaStream_t s = (cudaStream_t)stream;
  double* U = nullptr;
  int* err = nullptr;
  IB_TRY(scratch_for_current_device(&U, &err));
  double h = prm->L / N;
  double reac = prm->rho != 0.0 ? prm->rho / prm->dt : 0.0;
  na_clear_err<<<1, 32, 0, s>>>(err);
  IB_LAUNCH_CHECK();
  int n = N * N;
  na_stokes<<<(n + 255) / 256, 256, 0, s>>>(w, y, N, -4.0 * prm->mu / (h * h) - reac, prm->mu / (h * h),
                                             1.0 / h);
  IB_LAUNCH_CHECK();
  if (n_springs > 0) {
    na_interp<<<(2 * n_points + 127) / 128, 128, 0, s>>>(X, n_points, w, N, 1.0 / h, prm->delta, U);
    IB_LAUNCH_CHECK();
    na_springs<<<(n_springs + 127) / 128, 128, 0, s>>>(X, n_points, springs, kappa, rest, n_springs,
                                                       prm->L, prm->jacobian == IB_JAC_CLAMPED, U, N,
                                                       1.0 / h, prm->delta, prm->dt / (h * h), y, err);
    IB_LAUNCH_CHECK();
  }
  int herr[4] = {0, 0, 0, 0};
  IB_CUDA_TRY(cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
  IB_CUDA_TRY(cudaStreamSynchronize(s));
  if (herr[0] & 1) return fail(IB_ERR_INVALID_ARG, "spring end points out of range or equal");
  if (herr[0] & 2) return fail(IB_ERR_INVALID_ARG, "a spring has coincident or non-finite end points");
  return IB_OK;
}
