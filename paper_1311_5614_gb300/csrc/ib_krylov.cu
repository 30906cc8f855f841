// Flexible GMRES building blocks (sec. 3.3: GMRES right-preconditioned by the
// V-cycle; flexible form so that an FP32 preconditioner is admissible).  All
// vectors are FP64; reductions are two-stage and deterministic.  The Krylov
// bases (V, Z) are read with the streaming cache hint (evict first): at a few
// hundred MB they would otherwise push the V-cycle's working set out of L2
// between preconditioner applications.
//
// Classical Gram-Schmidt applied twice takes three passes over the basis per
// iteration: h1 = V^T w; w -= V h1 and h2 = V^T w in one pass (basis slices
// brought into shared memory by bulk copies); w -= V h2 with ||w||^2, whose
// final reduction also runs the Givens step.  With one FP64 FMA per 8 bytes of
// basis, these passes are bound by GB300's FP64 rate rather than by HBM.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "ib_async.cuh"
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

// partial[bx * stride + i] = sum over the elements [bx * per, (bx + 1) * per) of
// V_i . w, for the MDG vectors of block row blockIdx.y.  Per step every thread has
// MDE x MDG independent loads in flight, and each block reduces once, at the end.
constexpr int MDG = 8;
constexpr int MDE = 4;
__global__ void __launch_bounds__(TPB) k_multidot_partial(const double* __restrict__ V, int nvec, long n,
                                                          const double* __restrict__ w, double* partial,
                                                          int stride, long per) {
  __shared__ double sh[TPB / 32][MDG];
  const int i0 = blockIdx.y * MDG;
  const int nv = nvec - i0 < MDG ? nvec - i0 : MDG;
  const double* v0 = V + (size_t)i0 * n;
  double acc[MDG];
#pragma unroll
  for (int q = 0; q < MDG; ++q) acc[q] = 0.0;
  const long lo = (long)blockIdx.x * per, hi = lo + per < n ? lo + per : n;
  for (long e0 = lo + threadIdx.x; e0 < hi; e0 += (long)TPB * MDE) {
    double we[MDE];
#pragma unroll
    for (int k = 0; k < MDE; ++k) we[k] = e0 + (long)k * TPB < hi ? w[e0 + (long)k * TPB] : 0.0;
    if (nv == MDG && e0 + (long)(MDE - 1) * TPB < hi) {
#pragma unroll
      for (int q = 0; q < MDG; ++q)
#pragma unroll
        for (int k = 0; k < MDE; ++k) acc[q] += __ldcs(v0 + (size_t)q * n + e0 + (long)k * TPB) * we[k];
    } else {
#pragma unroll
      for (int q = 0; q < MDG; ++q)
        if (q < nv)
#pragma unroll
          for (int k = 0; k < MDE; ++k)
            if (e0 + (long)k * TPB < hi) acc[q] += __ldcs(v0 + (size_t)q * n + e0 + (long)k * TPB) * we[k];
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < MDG; ++q) {
    double a = acc[q];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) sh[wid][q] = a;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double t = 0.0;
    for (int q = 0; q < TPB / 32; ++q) t += sh[q][threadIdx.x];
    partial[(size_t)blockIdx.x * stride + i0 + threadIdx.x] = t;
  }
}

// Fused Gram-Schmidt pass: w <- w - sum_i coef_i V_i, then partial[bx * stride + i]
// = the block's part of V_i . w (the updated w), so the basis is read from HBM
// once for the first subtraction and the second projection of CGS2.  A block
// takes chunks of CGS_CH elements: the lanes of warp 0 issue one bulk copy per
// basis vector (its 512-byte slice) into shared memory, the block subtracts (one
// thread per element), then thread t forms the dot products of vectors t, t + 64,
// ... with the chunk (rows read at a per-row rotation of the column, so a warp's
// 32 rows hit distinct banks) and keeps them in registers across chunks.  A bulk
// copy that has not landed after limit_ns (1 s unless set at ib_setup) sets
// DEV_ERR_TIMEOUT and ends the block once the copies in flight have landed (or
// after DRAIN_LIMIT_NS more).  Before the copies of the next chunk are issued, the
// issuing warp orders the block's earlier generic-proxy reads of sV and sw (made
// visible to it by the barrier ending the chunk) before its async-proxy writes
// with fence.proxy.async.
constexpr int CGS_CH = 64;
constexpr int CGS_KMAX = (513 + CGS_CH - 1) / CGS_CH;  // vectors per thread (nvec <= 513)
__global__ void __launch_bounds__(CGS_CH) k_cgs_sub_dot(const double* __restrict__ V, int nvec, long n,
                                                        const double* __restrict__ coef, double* __restrict__ w,
                                                        double* __restrict__ partial, int stride, int* err,
                                                        unsigned long long limit_ns) {
  extern __shared__ __align__(128) double sm[];
  double* sV = sm;                          // [nvec][CGS_CH]
  double* sw = sV + (size_t)nvec * CGS_CH;  // [CGS_CH] updated w of the chunk
  double* sc = sw + CGS_CH;                 // [nvec] coefficients
  __shared__ __align__(8) unsigned long long bar;
  const int t = threadIdx.x;
  for (int i = t; i < nvec; i += CGS_CH) sc[i] = coef[i];
  if (t == 0) mbar_init(&bar, 1);
  __syncthreads();
  double acc[CGS_KMAX];
#pragma unroll
  for (int k = 0; k < CGS_KMAX; ++k) acc[k] = 0.0;
  const long nch = (n + CGS_CH - 1) / CGS_CH;
  unsigned parity = 0;
  for (long ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const long c0 = ch * CGS_CH;
    const int len = (int)(n - c0 < CGS_CH ? n - c0 : CGS_CH);
    if (t < 32) {
      const unsigned bytes = (unsigned)len * 8u;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (t == 0) mbar_arrive_expect_tx(&bar, bytes * (unsigned)nvec);
      __syncwarp();
      for (int i = t; i < nvec; i += 32) bulk_g2s(sV + (size_t)i * CGS_CH, V + (size_t)i * n + c0, bytes, &bar);
    }
    const bool ok = mbar_wait_bounded(&bar, parity, limit_ns);
    if (__syncthreads_or(!ok)) {
      // thread 0 stays until this chunk's copies have landed, so the block's shared
      // memory outlives every write into it
      if (t == 0) {
        atomicOr(err, DEV_ERR_TIMEOUT);
        mbar_wait_bounded(&bar, parity, DRAIN_LIMIT_NS);
      }
      return;
    }
    parity ^= 1u;
    double s = 0.0;
    if (t < len) {
      double s0 = w[c0 + t], s1 = 0.0;
      int i = 0;
#pragma unroll 4
      for (; i + 1 < nvec; i += 2) {
        s0 -= sc[i] * sV[(size_t)i * CGS_CH + t];
        s1 -= sc[i + 1] * sV[(size_t)(i + 1) * CGS_CH + t];
      }
      if (i < nvec) s0 -= sc[i] * sV[(size_t)i * CGS_CH + t];
      s = s0 + s1;
      w[c0 + t] = s;
    }
    sw[t] = s;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < CGS_KMAX; ++k) {
      const int i = t + k * CGS_CH;
      if (i < nvec) {
        const double* r = sV + (size_t)i * CGS_CH;
        double d = 0.0;
        if (len == CGS_CH) {
#pragma unroll 16
          for (int e = 0; e < CGS_CH; ++e) {
            const int c = (e + i) & (CGS_CH - 1);
            d += r[c] * sw[c];
          }
        } else {
          for (int e = 0; e < len; ++e) d += r[e] * sw[e];
        }
        acc[k] += d;
      }
    }
    __syncthreads();  // sV and sw are refilled by the next chunk
  }
#pragma unroll
  for (int k = 0; k < CGS_KMAX; ++k) {
    const int i = t + k * CGS_CH;
    if (i < nvec) partial[(size_t)blockIdx.x * stride + i] = acc[k];
  }
}

// Last Gram-Schmidt subtraction with the norm: w <- w - sum_i coef_i V_i over
// the elements [bx * per, (bx + 1) * per), and partial[bx] = their part of ||w||^2.
__global__ void __launch_bounds__(TPB) k_sub_norm(const double* __restrict__ V, int nvec, long n,
                                                  const double* __restrict__ coef, double* __restrict__ w,
                                                  double* __restrict__ partial, long per) {
  __shared__ double c[520];
  __shared__ double sh[32];
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) c[i] = coef[i];
  __syncthreads();
  double s2 = 0.0;
  const long lo = (long)blockIdx.x * per, hi = lo + per < n ? lo + per : n;
  for (long e = lo + threadIdx.x; e < hi; e += TPB) {
    double s = w[e];
#pragma unroll 16
    for (int i = 0; i < nvec; ++i) s -= c[i] * __ldcs(V + (size_t)i * n + e);
    w[e] = s;
    s2 += s * s;
  }
  s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s2;
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

// y = x * s or y = x * (1 / s) with the scalar s on the device; the reciprocal is
// formed once per block (an FP64 division per element would cost more than the copy)
__global__ void k_scale_copy(const double* __restrict__ x, const double* __restrict__ s, double* y,
                             long n, int invert) {
  __shared__ double sa;
  if (threadIdx.x == 0) sa = invert ? 1.0 / *s : *s;
  __syncthreads();
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  y[e] = x[e] * sa;
}

// The fused middle step of classical Gram-Schmidt applied twice for a small basis
// (nvec <= K): w <- w - sum_i coef_i V_i and partial[block][i] = V_i . w (the
// updated w) over the block's contiguous range of elements.  Each thread keeps its
// element's nvec basis values in registers between the subtraction and the dots,
// so V is read once; the partial sums go through warp shuffles and shared memory
// in a fixed order.
template <int K>
__global__ void __launch_bounds__(TPB) k_cgs_sub_dot_reg(const double* __restrict__ V, int nvec, long n,
                                                         const double* __restrict__ coef, double* __restrict__ w,
                                                         double* __restrict__ partial, int stride, long per) {
  __shared__ double c[K];
  __shared__ double red[TPB / 32][K];
  if (threadIdx.x < K) c[threadIdx.x] = threadIdx.x < nvec ? coef[threadIdx.x] : 0.0;
  __syncthreads();
  double acc[K];
#pragma unroll
  for (int i = 0; i < K; ++i) acc[i] = 0.0;
  const long e0 = (long)blockIdx.x * per, e1 = e0 + per < n ? e0 + per : n;
  for (long e = e0 + threadIdx.x; e < e1; e += TPB) {
    double v[K];
    double s = w[e];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      v[i] = i < nvec ? V[(size_t)i * n + e] : 0.0;
      s -= c[i] * v[i];
    }
    w[e] = s;
#pragma unroll
    for (int i = 0; i < K; ++i) acc[i] += v[i] * s;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    double a = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) red[wid][i] = a;
  }
  __syncthreads();
  if (threadIdx.x < nvec) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < TPB / 32; ++q) t += red[q][threadIdx.x];
    partial[(size_t)blockIdx.x * stride + threadIdx.x] = t;
  }
}

// Givens step of FGMRES iteration j, one block.  H (column-major, ld m + 1)
// column j is h1 + h2 from the two Gram-Schmidt passes and ||w|| below the
// diagonal (||w||^2 summed here from the partials of k_sub_norm, in a fixed
// order); the previous rotations are applied, a new one is formed, and g is
// updated.  The column and the rotations are staged in shared memory so that the
// sequential rotation loop carries only two FMAs per step.
// scal layout: [0] |g_{j+1}|, [1] H_{j+1,j} (= ||w||), [2] non-finite flag.
constexpr int GIV_MAX = 514;
__global__ void k_norm_givens(const double* __restrict__ partial, int nb, double* wn2, double* H, int ld, int j,
                              const double* h1, const double* h2, double* cs, double* sn, double* g,
                              double* scal) {
  __shared__ double sh[32];
  __shared__ double col[GIV_MAX], scs[GIV_MAX], ssn[GIV_MAX];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[b];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = h1[i] + h2[i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    scs[i] = cs[i];
    ssn[i] = sn[i];
  }
  s = block_sum(s, sh);  // synchronises the block
  if (threadIdx.x == 0) {
    *wn2 = s;
    const double hn = sqrt(fmax(s, 0.0));
    scal[1] = hn;
    double a = col[0];
    for (int i = 0; i < j; ++i) {
      const double b = col[i + 1];
      col[i] = scs[i] * a + ssn[i] * b;
      a = -ssn[i] * a + scs[i] * b;
    }
    const double den = hypot(a, hn);
    const double c = den > 0.0 ? a / den : 1.0, sr = den > 0.0 ? hn / den : 0.0;
    cs[j] = c;
    sn[j] = sr;
    col[j] = den;
    col[j + 1] = 0.0;
    g[j + 1] = -sr * g[j];
    g[j] = c * g[j];
    scal[0] = fabs(g[j + 1]);
    scal[2] = (isfinite(den) && isfinite(g[j + 1])) ? 0.0 : 1.0;
  }
  __syncthreads();
  double* hc = H + (size_t)j * ld;
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) hc[i] = col[i];
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

// Block columns of k_multidot_partial: all block rows x columns resident at
// once (one wave), each column an equal contiguous range of at least one warp
// width per thread row.
static inline int dot_cols(const Problem& P, long n, int rows) {
  const long resident = (long)P.n_sm * std::max(1, P.occ_multidot);
  const long want = std::max(1L, resident / rows);
  const long most = std::max(1L, n / TPB);
  return (int)std::max(1L, std::min({want, most, (long)P.dot_blocks}));
}
static inline long range_per(long n, int cols) { return ((n + cols - 1) / cols + 31) / 32 * 32; }

int krylov_init(Problem& P) {
  int dev = 0;
  IB_CUDA_TRY(cudaGetDevice(&dev));
  IB_CUDA_TRY(cudaDeviceGetAttribute(&P.n_sm, cudaDevAttrMultiProcessorCount, dev));
  int optin = 0;
  IB_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  P.cgs_smem_max = std::max(0, optin - 256);  // leaves room for the static shared memory (one mbarrier)
  IB_CUDA_TRY(cudaFuncSetAttribute(k_cgs_sub_dot, cudaFuncAttributeMaxDynamicSharedMemorySize, P.cgs_smem_max));
  P.dot_blocks = 8 * std::max(1, P.n_sm);
  // IB_CGS_FUSED=0 takes the two-pass form of the middle Gram-Schmidt step always
  // (to test it: it is otherwise reached only above ~450 basis vectors)
  const char* e = std::getenv("IB_CGS_FUSED");
  P.cgs_fused = !(e && e[0] == '0');
  // IB_CGS_REG=0 keeps bases of up to 16 vectors on the bulk-copy form too (its
  // bounded waits are what the wait-limit test exercises)
  const char* er = std::getenv("IB_CGS_REG");
  P.cgs_reg = !(er && er[0] == '0');
  IB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&P.occ_multidot, k_multidot_partial, TPB, 0));
  IB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&P.occ_subnorm, k_sub_norm, TPB, 0));
  return IB_OK;
}

static int multidot_final(Problem& P, int nvec, int cols, double* out) {
  KScope ks(P, IB_KC_KRYLOV, (double)nvec * cols * 8.0);
  k_multidot_final<<<nvec, TPB, 0, P.stream>>>(P.dots, cols, P.max_m + 2, out);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_multidot(Problem& P, const double* V, int nvec, const double* w, double* out) {
  long n = nvec_len(P);
  const int rows = (nvec + MDG - 1) / MDG;
  const int cols = dot_cols(P, n, rows);
  {
    KScope ks(P, IB_KC_KRYLOV, (nvec + 1.0) * n * 8.0);
    k_multidot_partial<<<dim3(cols, rows), TPB, 0, P.stream>>>(V, nvec, n, w, P.dots, P.max_m + 2,
                                                               range_per(n, cols));
    IB_LAUNCH_CHECK();
  }
  return multidot_final(P, nvec, cols, out);
}

int launch_multiaxpy(Problem& P, const double* V, int nvec, const double* coef, double* w) {
  long n = nvec_len(P);
  KScope ks(P, IB_KC_KRYLOV, (nvec + 2.0) * n * 8.0);
  k_multiaxpy<<<nblk(n), TPB, 0, P.stream>>>(V, nvec, n, coef, w);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_dot(Problem& P, const double* a, const double* b, double* out) { return launch_multidot(P, a, 1, b, out); }

// w <- w - V coef, out = V^T w (the updated w): the first subtraction and the
// second projection of classical Gram-Schmidt applied twice, in one pass over V.
// Falls back to two passes when the chunk of V does not fit in shared memory.
int launch_cgs_sub_dot(Problem& P, const double* V, int nvec, const double* coef, double* w, double* out) {
  const long n = nvec_len(P);
  if (nvec <= 16 && P.cgs_fused && P.cgs_reg) {  // small basis: the register form, one wave of blocks
    if (P.occ_cgs_reg[0] == 0) {
      IB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&P.occ_cgs_reg[0], k_cgs_sub_dot_reg<8>, TPB, 0));
      IB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&P.occ_cgs_reg[1], k_cgs_sub_dot_reg<16>, TPB, 0));
      P.occ_cgs_reg[0] = std::max(1, P.occ_cgs_reg[0]);
      P.occ_cgs_reg[1] = std::max(1, P.occ_cgs_reg[1]);
    }
    const int occ = nvec <= 8 ? P.occ_cgs_reg[0] : P.occ_cgs_reg[1];
    const int cols = (int)std::min<long>({(long)P.n_sm * occ, (long)nblk(n), (long)P.dot_blocks});
    {
      KScope ks(P, IB_KC_KRYLOV, (nvec + 2.0) * n * 8.0);
      if (nvec <= 8)
        k_cgs_sub_dot_reg<8><<<cols, TPB, 0, P.stream>>>(V, nvec, n, coef, w, P.dots, P.max_m + 2, range_per(n, cols));
      else
        k_cgs_sub_dot_reg<16><<<cols, TPB, 0, P.stream>>>(V, nvec, n, coef, w, P.dots, P.max_m + 2,
                                                          range_per(n, cols));
      IB_LAUNCH_CHECK();
    }
    return multidot_final(P, nvec, cols, out);
  }
  const size_t smem = ((size_t)nvec * CGS_CH + CGS_CH + 2ul * nvec) * sizeof(double);
  if (!P.cgs_fused || smem > (size_t)P.cgs_smem_max || (n & 1)) {
    IB_TRY(launch_multiaxpy(P, V, nvec, coef, w));
    return launch_multidot(P, V, nvec, w, out);
  }
  if ((int)P.occ_cgs.size() <= nvec) P.occ_cgs.resize((size_t)nvec + 1, 0);
  int& per_sm = P.occ_cgs[nvec];
  if (per_sm == 0) {
    IB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cgs_sub_dot, CGS_CH, smem));
    per_sm = std::max(1, std::min(per_sm, 8));
  }
  const long chunks = (n + CGS_CH - 1) / CGS_CH;
  const int cols = (int)std::min<long>({chunks, (long)P.n_sm * per_sm, (long)P.dot_blocks});
  {
    KScope ks(P, IB_KC_KRYLOV, (nvec + 2.0) * n * 8.0);
    k_cgs_sub_dot<<<cols, CGS_CH, smem, P.stream>>>(V, nvec, n, coef, w, P.dots, P.max_m + 2, P.dev_err,
                                                     P.wait_limit_ns);
    IB_LAUNCH_CHECK();
  }
  return multidot_final(P, nvec, cols, out);
}

// givens layout: cs[m] | sn[m] | g[m + 1] | y[m];  scal: [0..2] Givens outputs,
// [8 .. 8 + m + 1] h1, [8 + m + 2 ..] h2, then ||w||^2.
// Last Gram-Schmidt subtraction w <- w - V h2, ||w||^2 and the Givens step of
// iteration j (nvec = j + 1).
int launch_cgs_finish(Problem& P, const double* V, int nvec, double* w, int j) {
  int m = P.max_m;
  double* cs = P.givens;
  double* sn = cs + m;
  double* g = sn + m;
  double* h1 = P.scal + 8;
  double* h2 = h1 + m + 2;
  double* wn = h2 + m + 2;
  const long n = nvec_len(P);
  const int cols = (int)std::min<long>({(long)P.n_sm * std::max(1, P.occ_subnorm), (long)nblk(n),
                                         (long)P.dot_blocks});
  {
    KScope ks(P, IB_KC_KRYLOV, (nvec + 2.0) * n * 8.0);
    k_sub_norm<<<cols, TPB, 0, P.stream>>>(V, nvec, n, h2, w, P.dots, range_per(n, cols));
    IB_LAUNCH_CHECK();
  }
  KScope ks(P, IB_KC_KRYLOV, 8.0 * (4.0 * j + 8 + cols));
  k_norm_givens<<<1, TPB, 0, P.stream>>>(P.dots, cols, wn, P.H, m + 1, j, h1, h2, cs, sn, g, P.scal);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_scale_copy(Problem& P, const double* x, const double* s, double* y, bool invert) {
  long n = nvec_len(P);
  KScope ks(P, IB_KC_KRYLOV, 2.0 * n * 8.0);
  k_scale_copy<<<nblk(n), TPB, 0, P.stream>>>(x, s, y, n, invert ? 1 : 0);
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
  const int cols = dot_cols(P, 3 * n, 1);
  {
    KScope ks(P, IB_KC_OTHER, 6.0 * n * 8.0);
    k_multidot_partial<<<dim3(cols, 1), TPB, 0, P.stream>>>(ones, 1, 3 * n, w, P.dots, P.max_m + 2,
                                                            range_per(3 * n, cols));
    IB_LAUNCH_CHECK();
  }
  {
    KScope ks(P, IB_KC_OTHER, (double)cols * 8.0);
    k_multidot_final<<<1, TPB, 0, P.stream>>>(P.dots, cols, P.max_m + 2, P.scal + 3);
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
