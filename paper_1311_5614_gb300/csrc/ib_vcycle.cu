// The V-cycle of Algorithm 1 as GB300 kernels.
//
// Fine levels (N_l above the tail size) run grid-wide kernels, one phase per
// launch: per colour the elasticity residual term rE = -dt E_l w (interp, then
// J U spread with atomics into the patch rows), then the box solves of that
// colour.  For n x n boxes (n >= 2) the Stokes residual of a box is evaluated
// inside the box kernel: boxes of one colour are at least n >= 2 cells apart,
// farther than the 5-point stencil reaches, so no box reads an unknown another
// box of its colour writes.  1 x 1 boxes of one colour are one cell apart, so
// their residual is formed by a separate kernel first (block-Jacobi semantics).
// Residual and restriction are fused.
//
// The coarse levels (N_l <= 64 in FP32, <= 32 in FP64, all fitting in shared
// memory) run in one kernel on a single CTA of 1024 threads: every sweep,
// transfer and the bordered coarsest solve, separated by __syncthreads.
//
// The whole sequence is captured once into a CUDA graph and replayed for every
// V-cycle; the graph is re-captured when a kernel argument changes.
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "ib_ops.cuh"
#include "ib_vcycle.cuh"

namespace ib {
namespace {

constexpr int TPB = 256;
inline int nblk(long n, int t = TPB) { return (int)((n + t - 1) / t); }
constexpr int kSeq[4] = {0, 3, 1, 2};  // forward colour sequence (host)
__device__ __forceinline__ int seq_color(int cc) { return cc == 0 ? 0 : (cc == 1 ? 3 : (cc == 2 ? 1 : 2)); }
constexpr int TAIL_THREADS = 1024;

template <typename T>
StokesCoef<T> coefs(const Problem& P, int l) {
  double h = P.lev[l].h;
  double reac = P.prm.rho != 0.0 ? P.prm.rho / P.prm.dt : 0.0;
  StokesCoef<T> c;
  c.diag = (T)(-4.0 * P.prm.mu / (h * h) - reac);
  c.off = (T)(P.prm.mu / (h * h));
  c.g = (T)(1.0 / h);
  return c;
}

template <typename T>
Patches<T> pats(LevelInfo& L);
template <>
Patches<double> pats<double>(LevelInfo& L) { return L.pat64; }
template <>
Patches<float> pats<float>(LevelInfo& L) { return L.pat32; }

template <typename T>
LevelBuf<T>& lbuf(LevelInfo& L);
template <>
LevelBuf<double>& lbuf<double>(LevelInfo& L) { return L.v64; }
template <>
LevelBuf<float>& lbuf<float>(LevelInfo& L) { return L.v32; }

template <typename T>
T* rEbuf(LevelInfo& L);
template <>
double* rEbuf<double>(LevelInfo& L) { return L.rE64; }
template <>
float* rEbuf<float>(LevelInfo& L) { return L.rE32; }

template <typename T>
const T* Mfree_of(const LevelInfo& L);
template <>
const double* Mfree_of<double>(const LevelInfo& L) { return L.Mfree; }
template <>
const float* Mfree_of<float>(const LevelInfo& L) { return L.Mfree32; }

template <typename T>
Springs<T> sview(Problem& P) {
  Springs<T> s;
  s.np = P.np;
  s.ns = P.ns;
  s.adj_ptr = P.adj_ptr;
  s.adj_spring = P.adj_spring;
  s.adj_other = P.adj_other;
  if constexpr (sizeof(T) == 8) s.K = (const T*)P.K64;
  else s.K = (const T*)P.K32;
  return s;
}

template <typename T>
T* Ubuf(Problem& P) {
  if constexpr (sizeof(T) == 8) return (T*)P.U64;
  else return (T*)P.U32;
}

// ------------------------------------------------------------------ fine-level kernels

// U = S^*_l w at every point, and zero the spread-patch rows of rE.
// Thread (row bb, component, point): bb == 0 also computes U.
template <typename T>
__global__ void kv_interp_zero(Patches<T> pat, const T* __restrict__ w, int np, int N, T* __restrict__ U,
                               T* __restrict__ rE) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 8 * np) return;
  int bb = t / (2 * np), rem = t - bb * 2 * np;
  int comp = rem / np, k = rem - comp * np;
  if (bb == 0) U[comp * np + k] = interp_point(pat, w, N, comp, k);
  zero_row(pat, N, comp, k, bb, rE);
}

// rE += coef * S_l (J U), thread (row bb, component, point).
template <typename T>
__global__ void kv_spread(Patches<T> pat, Springs<T> sp, const T* __restrict__ U, int N, T coef, T* rE) {
  int np = sp.np;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 8 * np) return;
  int bb = t / (2 * np), rem = t - bb * 2 * np;
  int comp = rem / np, k = rem - comp * np;
  T gx, gy;
  JU_point(sp, U, k, &gx, &gy);
  T g = coef * (comp == 0 ? gx : gy);
  if (g != (T)0) spread_row(pat, N, comp, k, bb, g, rE);
}

// n x n boxes (n >= 2) of one colour, Stokes residual inline.  One thread per
// box unknown (row of the box inverse), several boxes per CTA; the shared
// inverse of the structure-free box is staged in shared memory (n <= 4), the
// FP64 inverses of structure boxes are read column by column (coalesced over
// the box's threads).
template <int BS>
struct BoxShape {
  static constexpr int NB = 2 * BS * (BS + 1) + BS * BS;
  static constexpr int TPBOX = (NB + 31) / 32 * 32;
  static constexpr int BPC = BS == 2 ? 8 : (BS == 4 ? 4 : 1);
  static constexpr int THREADS = TPBOX * BPC;
  static constexpr bool SMEM_MF = BS <= 4;
};

template <typename T, int BS>
__global__ void __launch_bounds__(BoxShape<BS>::THREADS) kv_boxn(T* w, const T* __restrict__ b,
                                                                 const T* __restrict__ rE, int N, StokesCoef<T> c,
                                                                 int color, const int* __restrict__ slot,
                                                                 const double* __restrict__ Ms,
                                                                 const T* __restrict__ Mf) {
  using S = BoxShape<BS>;
  constexpr int NB = S::NB;
  __shared__ T sMf[S::SMEM_MF ? NB * NB : 1];
  __shared__ double rs[S::BPC][NB];
  const int tid = threadIdx.x;
  if (S::SMEM_MF)
    for (int e = tid; e < NB * NB; e += S::THREADS) sMf[e] = Mf[e];
  const int lb = tid / S::TPBOX, q = tid - lb * S::TPBOX;
  const int nb = N / BS, half = nb >> 1;
  const int t = blockIdx.x * S::BPC + lb;
  const bool valid = t < half * half && q < NB;
  int I = 0, J = 0, gq = 0;
  if (valid) {
    I = 2 * (t % half) + (color & 1);
    J = 2 * (t / half) + (color >> 1);
    int cc, i, j;
    box_unknown(q, BS, I * BS, J * BS, N, &cc, &i, &j);
    gq = cc * N * N + j * N + i;
    rs[lb][q] = (double)resid_at(w, b, rE, N, c, cc, i, j);
  }
  __syncthreads();
  if (!valid) return;
  const int sl = slot[J * nb + I];
  if (sl >= 0) {
    const double* M = Ms + (size_t)sl * NB * NB + q;
    double d = 0.0;
#pragma unroll 8
    for (int s = 0; s < NB; ++s) d += M[(size_t)s * NB] * rs[lb][s];
    w[gq] += (T)d;
  } else {
    const T* M = S::SMEM_MF ? sMf + q : Mf + q;
    T d = 0;
#pragma unroll 8
    for (int s = 0; s < NB; ++s) d += M[s * NB] * (T)rs[lb][s];
    w[gq] += d;
  }
}

// Register-blocked variant for n = 2, 4: the free-box solves of the CTA's boxes are
// one small GEMM (shared inverse x the block of box residuals), each thread owning
// an RB x CB tile (rows x boxes) and reading RB inverse entries with one vector
// load; structure boxes are then solved with their own FP64 inverse.
template <typename T, int BS>
struct BoxGemm {
  static constexpr int NB = 2 * BS * (BS + 1) + BS * BS;
  static constexpr int THREADS = 128;
  static constexpr int BPC = BS == 2 ? 32 : 16;   // boxes per CTA
  static constexpr int RB = sizeof(T) == 4 ? 4 : 2;  // rows per thread (one vector load)
  static constexpr int RG = NB / RB;                 // row groups
  // box groups: the largest power-of-two divisor of BPC with RG * BG <= THREADS
  static constexpr int bg_of(int g) { return RG * g <= THREADS ? g : bg_of(g / 2); }
  static constexpr int BG = bg_of(BPC);
  static constexpr int CB = BPC / BG;                // boxes per thread
  static_assert(NB % RB == 0, "rows");
  static_assert(BG * CB == BPC && RG * BG <= THREADS, "tiling");
};

template <typename T, int RB>
struct VecOf;
template <>
struct VecOf<float, 4> {
  using type = float4;
};
template <>
struct VecOf<double, 2> {
  using type = double2;
};

template <typename T, int BS>
__global__ void __launch_bounds__(128) kv_boxg(T* w, const T* __restrict__ b, const T* __restrict__ rE, int N,
                                               StokesCoef<T> c, int color, const int* __restrict__ slot,
                                               const double* __restrict__ Ms, const T* __restrict__ Mf) {
  using G = BoxGemm<T, BS>;
  using V = typename VecOf<T, G::RB>::type;
  constexpr int NB = G::NB;
  __shared__ __align__(16) T sMf[NB * NB];
  __shared__ T rs[G::BPC][NB];
  __shared__ int sslot[G::BPC];
  const int tid = threadIdx.x;
  const int nb = N / BS, half = nb >> 1, nbox = half * half;
  const int box0 = blockIdx.x * G::BPC;
  for (int e = tid; e < NB * NB; e += G::THREADS) sMf[e] = Mf[e];
  if (tid < G::BPC) {
    const int t = box0 + tid;
    int sl = -2;  // -2: no box
    if (t < nbox) {
      const int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
      sl = slot[J * nb + I];
    }
    sslot[tid] = sl;
  }
  for (int e = tid; e < G::BPC * NB; e += G::THREADS) {
    const int lb = e / NB, q = e - lb * NB, t = box0 + lb;
    T r = 0;
    if (t < nbox) {
      const int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
      int cc, i, j;
      box_unknown(q, BS, I * BS, J * BS, N, &cc, &i, &j);
      r = resid_at(w, b, rE, N, c, cc, i, j);
    }
    rs[lb][q] = r;
  }
  __syncthreads();
  // free boxes: delta[q][box] = sum_s Mf[s][q] r[box][s]
  const int rg = tid % G::RG, bg = tid / G::RG;
  if (bg < G::BG) {
    T acc[G::RB][G::CB];
#pragma unroll
    for (int a = 0; a < G::RB; ++a)
#pragma unroll
      for (int k = 0; k < G::CB; ++k) acc[a][k] = 0;
#pragma unroll 4
    for (int s2 = 0; s2 < NB; ++s2) {
      const V m = *reinterpret_cast<const V*>(&sMf[s2 * NB + rg * G::RB]);
      const T* mv = reinterpret_cast<const T*>(&m);
#pragma unroll
      for (int k = 0; k < G::CB; ++k) {
        const T rv = rs[bg * G::CB + k][s2];
#pragma unroll
        for (int a = 0; a < G::RB; ++a) acc[a][k] += mv[a] * rv;
      }
    }
#pragma unroll
    for (int k = 0; k < G::CB; ++k) {
      const int lb = bg * G::CB + k;
      if (sslot[lb] != -1) continue;  // structure box or no box
      const int t = box0 + lb;
      const int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
#pragma unroll
      for (int a = 0; a < G::RB; ++a) {
        int cc, i, j;
        box_unknown(rg * G::RB + a, BS, I * BS, J * BS, N, &cc, &i, &j);
        w[cc * N * N + j * N + i] += acc[a][k];
      }
    }
  }
  // structure boxes: their own FP64 inverse; all threads share the (box, row) pairs
  __shared__ int slist[G::BPC];
  __shared__ int ns;
  if (tid == 0) {
    int k = 0;
    for (int lb = 0; lb < G::BPC; ++lb)
      if (sslot[lb] >= 0) slist[k++] = lb;
    ns = k;
  }
  __syncthreads();
  for (int e = tid; e < ns * NB; e += G::THREADS) {
    const int lb = slist[e / NB], q = e % NB;
    const int t = box0 + lb;
    const int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
    const double* M = Ms + (size_t)sslot[lb] * NB * NB + q;
    double d0 = 0.0, d1 = 0.0;
#pragma unroll 4
    for (int s2 = 0; s2 < NB; s2 += 2) {
      d0 += M[(size_t)s2 * NB] * (double)rs[lb][s2];
      d1 += M[(size_t)(s2 + 1) * NB] * (double)rs[lb][s2 + 1];
    }
    int cc, i, j;
    box_unknown(q, BS, I * BS, J * BS, N, &cc, &i, &j);
    w[cc * N * N + j * N + i] += (T)(d0 + d1);
  }
}

template <typename T>
int launch_boxn(Problem& P, int l, T* w, const T* b, const T* rE, int color) {
  LevelInfo& L = P.lev[l];
  const StokesCoef<T> c = coefs<T>(P, l);
  const int half = L.nb / 2;
  const long nbox = (long)half * half;
  // the GEMM form pays off on large levels; small levels keep one box per CTA slot
  const bool gemm = nbox >= P.box_gemm_min;
  switch (P.prm.box) {
    case 2:
      if (!gemm) {
        kv_boxn<T, 2><<<nblk(nbox, BoxShape<2>::BPC), BoxShape<2>::THREADS, 0, P.stream>>>(
            w, b, rE, L.N, c, color, L.flag, L.Mstruct, Mfree_of<T>(L));
        break;
      }
      kv_boxg<T, 2><<<nblk(nbox, BoxGemm<T, 2>::BPC), 128, 0, P.stream>>>(w, b, rE, L.N, c, color, L.flag,
                                                                       L.Mstruct, Mfree_of<T>(L));
      break;
    case 4:
      if (!gemm) {
        kv_boxn<T, 4><<<nblk(nbox, BoxShape<4>::BPC), BoxShape<4>::THREADS, 0, P.stream>>>(
            w, b, rE, L.N, c, color, L.flag, L.Mstruct, Mfree_of<T>(L));
        break;
      }
      kv_boxg<T, 4><<<nblk(nbox, BoxGemm<T, 4>::BPC), 128, 0, P.stream>>>(w, b, rE, L.N, c, color, L.flag,
                                                                       L.Mstruct, Mfree_of<T>(L));
      break;
    default:
      kv_boxn<T, 8><<<nblk(nbox, BoxShape<8>::BPC), BoxShape<8>::THREADS, 0, P.stream>>>(
          w, b, rE, L.N, c, color, L.flag, L.Mstruct, Mfree_of<T>(L));
      break;
  }
  IB_LAUNCH_CHECK();
  return IB_OK;
}

// 1 x 1 boxes: residual of the colour's boxes first, then the solves.
template <typename T>
__global__ void kv_colres1(const T* __restrict__ w, const T* __restrict__ b, const T* __restrict__ rE,
                           T* __restrict__ r, int N, StokesCoef<T> c, int color) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int half = N >> 1;
  if (t >= half * half) return;
  int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
  int n = N * N, m = N - 1;
  int I1 = (I + 1) & m, J1 = (J + 1) & m;
  r[J * N + I] = resid_at(w, b, rE, N, c, 0, I, J);
  r[J * N + I1] = resid_at(w, b, rE, N, c, 0, I1, J);
  r[n + J * N + I] = resid_at(w, b, rE, N, c, 1, I, J);
  r[n + J1 * N + I] = resid_at(w, b, rE, N, c, 1, I, J1);
  r[2 * n + J * N + I] = resid_at(w, b, rE, N, c, 2, I, J);
}

template <typename T>
__global__ void kv_box1(const T* __restrict__ r, T* __restrict__ w, int N, int color,
                        const int* __restrict__ slot, const double* __restrict__ Ms, const T* __restrict__ Mf) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int half = N >> 1;
  if (t >= half * half) return;
  int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
  int n = N * N, m = N - 1;
  int g[5] = {J * N + I, J * N + ((I + 1) & m), n + J * N + I, n + ((J + 1) & m) * N + I, 2 * n + J * N + I};
  T rb[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) rb[q] = r[g[q]];
  int sl = slot[J * N + I];
  if (sl >= 0) box_apply_rows(Ms + (size_t)sl * 25, 5, rb, 0, 1, w, g);
  else box_apply_rows(Mf, 5, rb, 0, 1, w, g);
}

// b_{l+1} = R (b - A_l w) with the elasticity part from rE (may be NULL).
template <typename T>
__global__ void kv_resres(const T* __restrict__ w, const T* __restrict__ b, const T* __restrict__ rE,
                          T* __restrict__ bc, int Nc, StokesCoef<T> c) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int nc = Nc * Nc;
  if (idx >= nc) return;
  T ru, rv, rp;
  restrict_resid_cell(w, b, rE, 2 * Nc, c, idx % Nc, idx / Nc, &ru, &rv, &rp);
  bc[idx] = ru;
  bc[nc + idx] = rv;
  bc[2 * nc + idx] = rp;
}

template <typename T>
__global__ void kv_prolong(const T* __restrict__ ec, T* __restrict__ wf, int N) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int n = N * N;
  if (idx >= n) return;
  T cu, cv, cp;
  prolong_cell(ec, N, idx & (N - 1), idx / N, &cu, &cv, &cp);
  wf[idx] += cu;
  wf[n + idx] += cv;
  wf[2 * n + idx] += cp;
}

template <typename T>
__global__ void kv_zero(T* x, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) x[i] = (T)0;
}

// ------------------------------------------------------------------ single-CTA tail kernel

template <typename T>
__device__ void tail_residual(const TailLevel<T>& L, const TailArgs<T>& A, const T* w, const T* b, T* r) {
  const int N = L.N, n = N * N;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int i = e & (N - 1), j = e / N;
    r[e] = b[e] - stokes_row(w, N, L.c, 0, i, j);
    r[n + e] = b[n + e] - stokes_row(w, N, L.c, 1, i, j);
    r[2 * n + e] = b[2 * n + e] - stokes_row(w, N, L.c, 2, i, j);
  }
  if (A.sp.ns == 0) {
    __syncthreads();
    return;
  }
  const int np = A.sp.np;
  for (int t = threadIdx.x; t < 2 * np; t += blockDim.x) {
    const int comp = t / np, k = t - comp * np;
    A.U[comp * np + k] = interp_point(L.pat, w, N, comp, k);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 8 * np; t += blockDim.x) {
    const int bb = t / (2 * np), rem = t - bb * 2 * np;
    const int comp = rem / np, k = rem - comp * np;
    T gx, gy;
    JU_point(A.sp, A.U, k, &gx, &gy);
    const T g = A.coefE * (comp == 0 ? gx : gy);
    if (g != (T)0) spread_row(L.pat, N, comp, k, bb, g, r);
  }
  __syncthreads();
}

template <typename T>
__device__ void tail_boxes(const TailLevel<T>& L, const TailArgs<T>& A, const T* r, T* w, int color,
                           double* stage_r, int* stage_g) {
  const int N = L.N, n = N * N, bs = A.box;
  const int nb = N / bs, half = nb >> 1, nbox = half * half;
  if (bs == 1) {
    const int m = N - 1;
    for (int t = threadIdx.x; t < nbox; t += blockDim.x) {
      const int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
      int g[5] = {J * N + I, J * N + ((I + 1) & m), n + J * N + I, n + ((J + 1) & m) * N + I, 2 * n + J * N + I};
      T rb[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) rb[q] = r[g[q]];
      const int sl = L.slot[J * nb + I];
      if (sl >= 0) box_apply_rows(L.Ms + (size_t)sl * 25, 5, rb, 0, 1, w, g);
      else box_apply_rows(L.Mf, 5, rb, 0, 1, w, g);
    }
  } else {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nB = A.nB;
    if (warp < A.stage_warps) {
      double* rs = stage_r + warp * nB;
      int* gs = stage_g + warp * nB;
      for (int t = warp; t < nbox; t += A.stage_warps) {
        const int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
        for (int q = lane; q < nB; q += 32) {
          int cc, i, j;
          box_unknown(q, bs, I * bs, J * bs, N, &cc, &i, &j);
          const int gq = cc * n + j * N + i;
          gs[q] = gq;
          rs[q] = (double)r[gq];
        }
        __syncwarp();
        const int sl = L.slot[J * nb + I];
        if (sl >= 0) box_apply_rows(L.Ms + (size_t)sl * nB * nB, nB, rs, lane, 32, w, gs);
        else box_apply_rows(L.Mf, nB, rs, lane, 32, w, gs);
        __syncwarp();
      }
    }
  }
  __syncthreads();
}

template <typename T>
__device__ void tail_sweep(const TailLevel<T>& L, const TailArgs<T>& A, T* w, const T* b, T* r, bool rev,
                           double* sr, int* sg) {
  for (int cc = 0; cc < 4; ++cc) {
    const int color = rev ? seq_color(3 - cc) : seq_color(cc);
    tail_residual(L, A, w, b, r);
    tail_boxes(L, A, r, w, color, sr, sg);
  }
}

template <typename T>
__global__ void __launch_bounds__(TAIL_THREADS) kv_tail(TailArgs<T> A) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* W[MAX_LEVELS];
  T* B[MAX_LEVELS];
  const int nl = A.nlev;
  for (int l = 0; l < nl; ++l) {
    W[l] = (T*)(smem + A.off_w[l]);
    B[l] = (T*)(smem + A.off_b[l]);
  }
  T* r = (T*)(smem + A.off_r);
  double* sr = (double*)(smem + A.off_sr);
  int* sg = (int*)(smem + A.off_sg);
  {
    const int n0 = 3 * A.lev[0].N * A.lev[0].N;
    for (int e = threadIdx.x; e < n0; e += blockDim.x) B[0][e] = A.b_in[e];
  }
  __syncthreads();
  for (int l = 0; l < nl - 1; ++l) {
    const TailLevel<T>& L = A.lev[l];
    const int n3 = 3 * L.N * L.N;
    for (int e = threadIdx.x; e < n3; e += blockDim.x) W[l][e] = (T)0;
    __syncthreads();
    for (int s = 0; s < A.nu1; ++s) tail_sweep(L, A, W[l], B[l], r, false, sr, sg);
    tail_residual(L, A, W[l], B[l], r);
    const int Nc = L.N / 2, ncell = Nc * Nc;
    for (int e = threadIdx.x; e < ncell; e += blockDim.x) {
      T ru, rv, rp;
      restrict_cell(r, L.N, e % Nc, e / Nc, &ru, &rv, &rp);
      B[l + 1][e] = ru;
      B[l + 1][ncell + e] = rv;
      B[l + 1][2 * ncell + e] = rp;
    }
    __syncthreads();
  }
  {
    // exact bordered solve on the coarsest grid: w = (M^{-1})[0:nc, 0:nc] b
    const T* bc = B[nl - 1];
    T* wc = W[nl - 1];
    for (int q = threadIdx.x; q < A.nc; q += blockDim.x) {
      double acc = 0.0;
      for (int s = 0; s < A.nc; ++s) acc += A.Mc[(size_t)s * A.ldc + q] * (double)bc[s];
      wc[q] = (T)acc;
    }
    __syncthreads();
  }
  for (int l = nl - 2; l >= 0; --l) {
    const TailLevel<T>& L = A.lev[l];
    const int N = L.N, n = N * N;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      T cu, cv, cp;
      prolong_cell(W[l + 1], N, e & (N - 1), e / N, &cu, &cv, &cp);
      W[l][e] += cu;
      W[l][n + e] += cv;
      W[l][2 * n + e] += cp;
    }
    __syncthreads();
    for (int s = 0; s < A.nu2; ++s) tail_sweep(L, A, W[l], B[l], r, A.post_rev != 0, sr, sg);
  }
  {
    const int n0 = 3 * A.lev[0].N * A.lev[0].N;
    for (int e = threadIdx.x; e < n0; e += blockDim.x) A.w_out[e] = W[0][e];
  }
}

// ------------------------------------------------------------------ host side

template <typename T>
int build_tail_args(Problem& P, int lt, TailArgs<T>* A, size_t* smem_bytes) {
  std::memset((void*)A, 0, sizeof(*A));
  A->nlev = P.nlev - lt;
  if (A->nlev > MAX_LEVELS) return fail(IB_ERR_INVALID_ARG, "too many tail levels");
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 15) & ~size_t(15);
    return o;
  };
  int max_boxes = 1;
  for (int q = 0; q < A->nlev; ++q) {
    int l = lt + q;
    LevelInfo& L = P.lev[l];
    TailLevel<T>& t = A->lev[q];
    t.N = L.N;
    t.c = coefs<T>(P, l);
    t.pat = pats<T>(L);
    t.slot = L.flag;
    t.Ms = L.Mstruct;
    t.Mf = Mfree_of<T>(L);
    size_t n3 = 3ul * L.N * L.N * sizeof(T);
    A->off_w[q] = (int)take(n3);
    A->off_b[q] = (int)take(n3);
    if (l < P.nlev - 1) {
      int nb = L.N / P.prm.box;
      int bpc = (nb / 2) * (nb / 2);
      if (bpc > max_boxes) max_boxes = bpc;
    }
  }
  A->off_r = (int)take(3ul * P.lev[lt].N * P.lev[lt].N * sizeof(T));
  A->stage_warps = P.prm.box == 1 ? 0 : (max_boxes < 32 ? max_boxes : 32);
  A->off_sr = (int)take((size_t)A->stage_warps * P.nB * sizeof(double));
  A->off_sg = (int)take((size_t)A->stage_warps * P.nB * sizeof(int));
  A->U = Ubuf<T>(P);
  A->sp = sview<T>(P);
  A->coefE = (T)(-P.prm.dt / (P.lev[0].h * P.lev[0].h));
  A->Mc = P.Mcoarse;
  A->nc = P.nc;
  A->ldc = P.nc + P.nborder;
  A->nu1 = P.prm.nu1;
  A->nu2 = P.prm.nu2;
  A->box = P.prm.box;
  A->nB = P.nB;
  A->post_rev = P.prm.box == 1 ? 1 : 0;
  A->b_in = lbuf<T>(P.lev[lt]).b;
  A->w_out = lbuf<T>(P.lev[lt]).w;
  *smem_bytes = off;
  return IB_OK;
}

// Elasticity residual part rE = -dt E_l w on a fine level (two launches).
template <typename T>
int fine_elastic(Problem& P, int l, const T* w) {
  LevelInfo& L = P.lev[l];
  const double sT = sizeof(T);
  {
    KScope ks(P, IB_KC_INTERP, 2.0 * P.np * (25 * sT + 8) + 8.0 * P.np * 4 * sT);
    kv_interp_zero<T><<<nblk(8L * P.np), TPB, 0, P.stream>>>(pats<T>(L), w, P.np, L.N, Ubuf<T>(P), rEbuf<T>(L));
    IB_LAUNCH_CHECK();
  }
  {
    double deg = P.np ? 2.0 * P.ns / P.np : 0.0;
    KScope ks(P, IB_KC_SPREAD, P.np * (2 * sT + 8 + deg * (5 * sT + 8) + 16 * sT + 16 + 64 * sT));
    kv_spread<T><<<nblk(8L * P.np), TPB, 0, P.stream>>>(pats<T>(L), sview<T>(P), Ubuf<T>(P), L.N,
                                                        (T)(-P.prm.dt / (P.lev[0].h * P.lev[0].h)), rEbuf<T>(L));
    IB_LAUNCH_CHECK();
  }
  return IB_OK;
}

template <typename T>
int fine_sweep(Problem& P, int l, bool rev, bool w_is_zero) {
  LevelInfo& L = P.lev[l];
  LevelBuf<T>& B = lbuf<T>(L);
  const int N = L.N, bs = P.prm.box;
  const bool has_E = P.np > 0 && P.ns > 0;
  const StokesCoef<T> c = coefs<T>(P, l);
  const int half = L.nb / 2;
  const long nbox = (long)half * half;
  const int nB = P.nB;
  const double sT = sizeof(T);
  for (int cc = 0; cc < 4; ++cc) {
    const int color = rev ? kSeq[3 - cc] : kSeq[cc];
    const bool zero = w_is_zero && cc == 0;
    const T* rE = nullptr;
    if (has_E && !zero) {
      IB_TRY(fine_elastic<T>(P, l, B.w));
      rE = rEbuf<T>(L);
    }
    if (bs == 1) {
      {
        KScope ks(P, IB_KC_STOKES, nbox * 5.0 * (6 * sT + 2 * sT));
        kv_colres1<T><<<nblk(nbox), TPB, 0, P.stream>>>(B.w, B.b, rE, B.r, N, c, color);
        IB_LAUNCH_CHECK();
      }
      KScope ks(P, IB_KC_BOX, nbox * (15.0 * sT + 4) + 0.25 * L.n_struct * 25 * 8.0 + 25 * sT);
      kv_box1<T><<<nblk(nbox), TPB, 0, P.stream>>>(B.r, B.w, N, color, L.flag, L.Mstruct, Mfree_of<T>(L));
      IB_LAUNCH_CHECK();
    } else {
      // per box: its unknowns' rows read w (5-point stencils, counted once per
      // unknown plus the one-cell halo), b, rE on structure rows, write w
      const double box_bytes = sT * (3.0 * nB + (4.0 * bs + 4)) + 4;
      KScope ks(P, IB_KC_BOX, nbox * box_bytes + 0.25 * L.n_struct * nB * nB * 8.0 + (double)nB * nB * sT);
      IB_TRY(launch_boxn<T>(P, l, B.w, B.b, rE, color));
    }
  }
  return IB_OK;
}

template <typename T>
constexpr int pix() { return sizeof(T) == 8 ? 1 : 0; }

template <typename T>
int vcycle_eager(Problem& P) {
  const int lt = P.tail_level[pix<T>()];
  const bool has_E = P.np > 0 && P.ns > 0;
  for (int l = 0; l < lt; ++l) {
    LevelInfo& L = P.lev[l];
    LevelBuf<T>& B = lbuf<T>(L);
    const long n3 = 3L * L.N * L.N;
    {
      KScope ks(P, IB_KC_OTHER, n3 * sizeof(T));
      kv_zero<T><<<nblk(n3), TPB, 0, P.stream>>>(B.w, n3);
      IB_LAUNCH_CHECK();
    }
    for (int s = 0; s < P.prm.nu1; ++s) IB_TRY(fine_sweep<T>(P, l, false, s == 0));
    const T* rE = nullptr;
    if (has_E) {
      IB_TRY(fine_elastic<T>(P, l, B.w));
      rE = rEbuf<T>(L);
    }
    const int Nc = P.lev[l + 1].N;
    {
      KScope ks(P, IB_KC_TRANSFER, (9.0 * L.N * L.N + 3.0 * Nc * Nc) * sizeof(T));
      kv_resres<T><<<nblk((long)Nc * Nc), TPB, 0, P.stream>>>(B.w, B.b, rE, lbuf<T>(P.lev[l + 1]).b, Nc,
                                                             coefs<T>(P, l));
      IB_LAUNCH_CHECK();
    }
  }
  {
    TailArgs<T> A;
    size_t smem = 0;
    IB_TRY(build_tail_args<T>(P, lt, &A, &smem));
    KScope ks(P, IB_KC_COARSE, 0.0);
    kv_tail<T><<<1, TAIL_THREADS, smem, P.stream>>>(A);
    IB_LAUNCH_CHECK();
  }
  for (int l = lt - 1; l >= 0; --l) {
    LevelInfo& L = P.lev[l];
    LevelBuf<T>& B = lbuf<T>(L);
    {
      KScope ks(P, IB_KC_TRANSFER, (6.0 * L.N * L.N + 0.75 * L.N * L.N) * sizeof(T));
      kv_prolong<T><<<nblk((long)L.N * L.N), TPB, 0, P.stream>>>(lbuf<T>(P.lev[l + 1]).w, B.w, L.N);
      IB_LAUNCH_CHECK();
    }
    for (int s = 0; s < P.prm.nu2; ++s) IB_TRY(fine_sweep<T>(P, l, P.prm.box == 1, false));
  }
  return IB_OK;
}

}  // namespace

template <typename T>
int vcycle_run(Problem& P);

// Candidate first levels of the single-CTA tail kernel: levels with N_l <= 64
// (FP32) or <= 32 (FP64) whose arrays fit in shared memory, plus "coarsest grid
// only".  vcycle_prepare times one graph-replayed V-cycle per candidate on the
// problem's own hierarchy and keeps the fastest (the autotuner of the level
// split between grid-wide kernels and the single-CTA kernel).
template <typename T>
int vcycle_prepare(Problem& P) {
  const int nmax = sizeof(T) == 4 ? 64 : 32;
  std::vector<int> cand;
  size_t smem_max = 0;
  for (int l = 0; l < P.nlev; ++l) {
    if (P.lev[l].N > nmax) continue;
    TailArgs<T> A;
    size_t s = 0;
    IB_TRY(build_tail_args<T>(P, l, &A, &s));
    if (s <= 227u * 1024u) {
      cand.push_back(l);
      if (s > smem_max) smem_max = s;
    }
  }
  if (cand.empty() || cand.back() != P.nlev - 1) {
    TailArgs<T> A;
    size_t s = 0;
    IB_TRY(build_tail_args<T>(P, P.nlev - 1, &A, &s));
    cand.push_back(P.nlev - 1);
    if (s > smem_max) smem_max = s;
  }
  // the limit is a per-function setting shared by every problem in the process:
  // only ever raise it (problems of a batch are prepared on several threads)
  {
    static std::mutex mu;
    static size_t granted = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (smem_max > granted) {
      IB_CUDA_TRY(cudaFuncSetAttribute(kv_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
      granted = smem_max;
    }
  }
  constexpr int ix = pix<T>();
  // IB_TAIL_NMAX pins the split instead of timing it (profiler runs distort the
  // timings): the tail starts at the first candidate level with N_l <= value
  if (const char* e = std::getenv("IB_TAIL_NMAX")) {
    int nt = std::atoi(e);
    int pick = cand.back();
    for (int l : cand)
      if (P.lev[l].N <= nt) {
        pick = l;
        break;
      }
    P.tail_level[ix] = pick;
    P.graph_dirty[ix] = true;
    return IB_OK;
  }
  if (cand.size() == 1 || P.prof || !P.use_graph) {
    P.tail_level[ix] = cand.front();
    P.graph_dirty[ix] = true;
    return IB_OK;
  }
  cudaEvent_t e0, e1;
  IB_CUDA_TRY(cudaEventCreate(&e0));
  IB_CUDA_TRY(cudaEventCreate(&e1));
  long long saved[IB_KC_COUNT];
  std::memcpy(saved, P.nlaunch, sizeof(saved));
  float best = 1e30f;
  int best_l = cand.front();
  size_t n0 = 3ul * P.lev[0].N * P.lev[0].N;
  IB_CUDA_TRY(cudaMemsetAsync(lbuf<T>(P.lev[0]).b, 0, n0 * sizeof(T), P.stream));
  for (int l : cand) {
    P.tail_level[ix] = l;
    P.graph_dirty[ix] = true;
    int rc = vcycle_run<T>(P);  // capture + warm-up
    if (rc != IB_OK) return rc;
    IB_CUDA_TRY(cudaEventRecord(e0, P.stream));
    for (int r = 0; r < 3; ++r) IB_TRY(vcycle_run<T>(P));
    IB_CUDA_TRY(cudaEventRecord(e1, P.stream));
    IB_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_l = l;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::memcpy(P.nlaunch, saved, sizeof(saved));
  P.tail_level[ix] = best_l;
  P.graph_dirty[ix] = true;
  return IB_OK;
}
template int vcycle_prepare<double>(Problem&);
template int vcycle_prepare<float>(Problem&);

// One V-cycle on the fixed level-0 buffers (input lev[0].b, output lev[0].w),
// replayed from a CUDA graph unless profiling asks for individually timed launches.
template <typename T>
int vcycle_run(Problem& P) {
  if (P.prof || !P.use_graph) return vcycle_eager<T>(P);
  if (!P.gstream) {
    IB_CUDA_TRY(cudaStreamCreateWithFlags(&P.gstream, cudaStreamNonBlocking));
    IB_CUDA_TRY(cudaEventCreateWithFlags(&P.gev[0], cudaEventDisableTiming));
    IB_CUDA_TRY(cudaEventCreateWithFlags(&P.gev[1], cudaEventDisableTiming));
  }
  // the caller's stream may be the legacy default stream, which cannot be
  // captured: capture and replay on a private stream joined by events
  IB_CUDA_TRY(cudaEventRecord(P.gev[0], P.stream));
  IB_CUDA_TRY(cudaStreamWaitEvent(P.gstream, P.gev[0], 0));
  cudaStream_t user = P.stream;
  constexpr int ix = pix<T>();
  if (P.graph_dirty[ix] || !P.vgraph[ix]) {
    if (P.vgraph[ix]) {
      cudaGraphExecDestroy(P.vgraph[ix]);
      P.vgraph[ix] = nullptr;
    }
    long long before[IB_KC_COUNT];
    std::memcpy(before, P.nlaunch, sizeof(before));
    cudaGraph_t g = nullptr;
    IB_CUDA_TRY(cudaStreamBeginCapture(P.gstream, cudaStreamCaptureModeThreadLocal));
    P.stream = P.gstream;
    int rc = vcycle_eager<T>(P);
    P.stream = user;
    cudaError_t ce = cudaStreamEndCapture(P.gstream, &g);
    if (rc != IB_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ce != cudaSuccess) return fail(IB_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&P.vgraph[ix], g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return fail(IB_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
    for (int c = 0; c < IB_KC_COUNT; ++c) {
      P.graph_launches[ix][c] = P.nlaunch[c] - before[c];
      P.nlaunch[c] = before[c];
    }
    P.graph_dirty[ix] = false;
  }
  IB_CUDA_TRY(cudaGraphLaunch(P.vgraph[ix], P.gstream));
  IB_CUDA_TRY(cudaEventRecord(P.gev[1], P.gstream));
  IB_CUDA_TRY(cudaStreamWaitEvent(P.stream, P.gev[1], 0));
  for (int c = 0; c < IB_KC_COUNT; ++c) P.nlaunch[c] += P.graph_launches[ix][c];
  return IB_OK;
}
template int vcycle_run<double>(Problem&);
template int vcycle_run<float>(Problem&);

// Zero the elasticity residual buffers (their patch rows move with the points).
int vcycle_reset_rE(Problem& P) {
  for (int l = 0; l < P.nlev; ++l) {
    LevelInfo& L = P.lev[l];
    size_t n2 = 2ul * L.N * L.N;
    if (L.rE64) IB_CUDA_TRY(cudaMemsetAsync(L.rE64, 0, n2 * sizeof(double), P.stream));
    if (L.rE32) IB_CUDA_TRY(cudaMemsetAsync(L.rE32, 0, n2 * sizeof(float), P.stream));
  }
  return IB_OK;
}

}  // namespace ib
