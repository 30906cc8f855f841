// The V-cycle of Algorithm 1 as GB300 kernels.
//
// Fine levels (N_l above the tail size) run grid-wide kernels, one phase per
// launch: per colour one kernel forms the point forces -dt/h_0^2 J S*_l w (a
// quad of lanes per point) and spreads them with atomic additions into rE, on
// the rows of that colour's boxes only; then the box solves of the colour, which
// take rE back out of their structure rows (leaving rE zero).  For n x n boxes (n >= 2) the Stokes residual of a box is evaluated
// inside the box kernel: boxes of one colour are at least n >= 2 cells apart,
// farther than the 5-point stencil reaches, so no box reads an unknown another
// box of its colour writes.  1 x 1 boxes of one colour are one cell apart, so
// their residual is formed by a separate kernel first (block-Jacobi semantics).
// Residual and restriction are fused.
//
// The coarse levels run in one "tail" kernel: every sweep, transfer and the
// bordered coarsest solve, on a single CTA of 1024 threads with the arrays in
// shared memory (N_l <= 64 in FP32, <= 32 in FP64) separated by __syncthreads,
// or on one thread-block cluster of 8-16 such CTAs with the arrays in global
// memory (N_l <= 128) separated by the cluster barrier.  The split between
// grid-wide kernels and the tail, and its form, are timed per problem.
//
// The whole sequence is captured once into a CUDA graph and replayed for every
// V-cycle; the graph is re-captured when a kernel argument changes.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "ib_async.cuh"
#include "ib_ops.cuh"
#include "ib_vcycle.cuh"

namespace ib {
namespace {

constexpr int TPB = 256;
inline int nblk(long n, int t = TPB) { return (int)((n + t - 1) / t); }
constexpr int kSeq[4] = {0, 3, 1, 2};  // forward colour sequence (host)
__device__ __forceinline__ int seq_color(int cc) { return cc == 0 ? 0 : (cc == 1 ? 3 : (cc == 2 ? 1 : 2)); }
constexpr int TAIL_THREADS = 1024;

// Programmatic dependent launch.  Every V-cycle kernel is launched with
// programmatic stream serialisation and calls pdl_enter() (ib_ops.cuh) before it
// reads anything an earlier V-cycle kernel writes, so that its launch, ramp-up
// and set-up-data loads overlap the previous kernel.

template <typename... KArgs, typename... Args>
void vlaunch(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
             Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// One thread-block cluster of csize CTAs (grid = the cluster); returns the launch status.
template <typename... KArgs, typename... Args>
cudaError_t claunch(bool pdl, int csize, void (*kern)(KArgs...), dim3 block, size_t smem, cudaStream_t stream,
                    Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize);
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// PDL inside the captured graph only (eager and profiled launches are plain), and
// only for problems up to 512^2: there each V-cycle launch is latency-bound and
// PDL measured 15-20 % faster V-cycles at 256^2; on a 1024^2 grid with 16
// structures it measured 15 % slower.  IB_PDL=0 turns it off, IB_PDL=1 forces it.
bool use_pdl(const Problem& P) {
  static const int mode = [] {
    const char* e = std::getenv("IB_PDL");
    return e ? (e[0] == '0' ? 0 : 1) : -1;
  }();
  if (mode == 0 || !P.use_graph || P.prof) return false;
  return mode == 1 || P.lev[0].N <= 512;
}

template <typename T>
StokesCoef<T> coefs(const Problem& P, int l) {
  double h = P.lev[l].h;
  double reac = P.prm.rho != 0.0 ? P.prm.rho / P.prm.dt : 0.0;
  StokesCoef<T> c;
  c.diag = (T)(-4.0 * P.prm.mu / (h * h) - reac);
  c.off = (T)(P.prm.mu / (h * h));
  c.g = (T)(1.0 / h);
  c.walls = P.prm.walls;
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
const T* Ewin_of(const LevelInfo& L);
template <>
const double* Ewin_of<double>(const LevelInfo& L) { return L.Ew64; }
template <>
const float* Ewin_of<float>(const LevelInfo& L) { return L.Ew32; }

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

// rE += coef * S_l J S*_l w on the rows of colour `color` (-1: all rows): one
// quad of lanes per point.
template <typename T>
__global__ void kv_force_spread(Patches<T> pat, Springs<T> sp, const T* __restrict__ w, int N, T coef, int b,
                                int color, T* __restrict__ rE) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const int k = (int)(t >> 2), j = (int)(t & 3);
  if (k >= sp.np) return;  // whole quads: blockDim is a multiple of 4
  const int lane = threadIdx.x & 31;
  force_spread_quad<T, true>(pat, sp, w, N, coef, k, j, 0xFu << (lane & ~3), lane & ~3, b, color, rE);
}

// n x n boxes (n >= 2) of one colour, residual inline (Stokes stencil plus rE on
// structure rows, which the kernel then clears: each such row belongs to exactly
// one box of the colour).  One thread per box unknown (row
// of the box inverse), several boxes per CTA; the shared inverse of the
// structure-free box is staged in shared memory (n <= 4), the inverses of
// structure boxes are read column by column (coalesced over the box's threads).
// BPC boxes per CTA; with one box per CTA (small levels: more CTAs, so that the
// FP64 products of structure boxes spread over more SMs) the free-box inverse is
// read through the cache instead of being staged.
template <int BS, int BPC_ = (BS == 2 ? 8 : (BS == 4 ? 4 : 1))>
struct BoxShape {
  static constexpr int NB = 2 * BS * (BS + 1) + BS * BS;
  static constexpr int TPBOX = (NB + 31) / 32 * 32;
  static constexpr int BPC = BPC_;
  static constexpr int THREADS = TPBOX * BPC;
  static constexpr bool SMEM_MF = BS <= 4 && BPC > 1;
};

// T: vectors and residuals; TM: the shared inverse of the structure-free boxes
// and its products (TM = float with T = double is the mixed-precision V-cycle).
// Structure boxes (stiff: their condition number grows with the stiffness) are
// always solved in FP64, the residual cast up and the correction cast back at the
// box boundary.
template <typename T, typename TM, int BS, int BPC>
__global__ void __launch_bounds__(BoxShape<BS, BPC>::THREADS) kv_boxn(T* w, const T* __restrict__ b, T* rE, int N,
                                                                 StokesCoef<T> c, int color,
                                                                 const int* __restrict__ slot,
                                                                 const double* __restrict__ Ms,
                                                                 const TM* __restrict__ Mf) {
  using S = BoxShape<BS, BPC>;
  constexpr int NB = S::NB, NV = 2 * BS * (BS + 1);
  __shared__ TM sMf[S::SMEM_MF ? NB * NB : 1];
  __shared__ T rs[S::BPC][NB];
  const int tid = threadIdx.x;
  const int nb = N / BS, half = nb >> 1;
  if (S::SMEM_MF)
    for (int e = tid; e < NB * NB; e += S::THREADS) sMf[e] = Mf[e];  // set-up data
  // set-up data too: pull the FP64 inverses of this CTA's structure boxes towards L1
  for (int l2 = 0; l2 < S::BPC; ++l2) {
    const int t2 = blockIdx.x * S::BPC + l2;
    if (t2 >= half * half) break;
    const int s2 = slot[(2 * (t2 / half) + (color >> 1)) * nb + 2 * (t2 % half) + (color & 1)];
    if (s2 < 0) continue;
    const double* M2 = Ms + (size_t)s2 * NB * NB;
    for (int e = tid * 16; e < NB * NB; e += S::THREADS * 16) asm volatile("prefetch.global.L1 [%0];" ::"l"(M2 + e));
  }
  pdl_enter();
  const int lb = tid / S::TPBOX, q = tid - lb * S::TPBOX;
  const int t = blockIdx.x * S::BPC + lb;
  const bool valid = t < half * half && q < NB;
  int gq = 0, sl = -1;
  if (valid) {
    const int I = 2 * (t % half) + (color & 1);
    const int J = 2 * (t / half) + (color >> 1);
    sl = slot[J * nb + I];
    int cc, i, j;
    box_unknown(q, BS, I * BS, J * BS, N, &cc, &i, &j);
    gq = cc * N * N + j * N + i;
    T r = b[gq] - stokes_row(w, N, c, cc, i, j);
    if (rE && sl >= 0 && q < NV) {
      r += rE[gq];
      rE[gq] = (T)0;
    }
    rs[lb][q] = r;
  }
  __syncthreads();
  if (!valid) return;
  if (sl >= 0) {
    const double* M = Ms + (size_t)sl * NB * NB + q;
    double d = 0.0;
#pragma unroll 8
    for (int s = 0; s < NB; ++s) d += M[(size_t)s * NB] * (double)rs[lb][s];
    w[gq] += (T)d;
  } else {
    const TM* M = S::SMEM_MF ? sMf + q : Mf + q;
    TM d = 0;
#pragma unroll 8
    for (int s = 0; s < NB; ++s) d += M[s * NB] * (TM)rs[lb][s];
    w[gq] += (T)d;
  }
}

// One box per CTA (small levels, n <= 4): the box's inverse, its FP64 structure
// inverse or the shared free-box inverse, is staged in shared memory before the
// programmatic-launch wait (set-up data), so the product reads shared memory.
template <typename T, typename TM, int BS>
__global__ void __launch_bounds__(BoxShape<BS, 1>::TPBOX) kv_boxs(T* w, const T* __restrict__ b, T* rE, int N,
                                                                 StokesCoef<T> c, int color,
                                                                 const int* __restrict__ slot,
                                                                 const double* __restrict__ Ms,
                                                                 const TM* __restrict__ Mf) {
  using S = BoxShape<BS, 1>;
  constexpr int NB = S::NB, NV = 2 * BS * (BS + 1);
  __shared__ __align__(16) double sM[NB * NB];
  __shared__ T rs[NB];
  const int q = threadIdx.x;
  const int nb = N / BS, half = nb >> 1, t = blockIdx.x;
  const int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
  const int sl = slot[J * nb + I];
  if (sl >= 0) {
    const double* M = Ms + (size_t)sl * NB * NB;
    for (int e = q; e < NB * NB; e += S::TPBOX) sM[e] = M[e];
  } else {
    TM* sf = reinterpret_cast<TM*>(sM);
    for (int e = q; e < NB * NB; e += S::TPBOX) sf[e] = Mf[e];
  }
  pdl_enter();
  int gq = 0;
  if (q < NB) {
    int cc, i, j;
    box_unknown(q, BS, I * BS, J * BS, N, &cc, &i, &j);
    gq = cc * N * N + j * N + i;
    T r = b[gq] - stokes_row(w, N, c, cc, i, j);
    if (rE && sl >= 0 && q < NV) {
      r += rE[gq];
      rE[gq] = (T)0;
    }
    rs[q] = r;
  }
  __syncthreads();
  if (q >= NB) return;
  if (sl >= 0) {
    double d = 0.0;
#pragma unroll 8
    for (int s2 = 0; s2 < NB; ++s2) d += sM[s2 * NB + q] * (double)rs[s2];
    w[gq] += (T)d;
  } else {
    const TM* sf = reinterpret_cast<const TM*>(sM);
    TM d = 0;
#pragma unroll 8
    for (int s2 = 0; s2 < NB; ++s2) d += sf[s2 * NB + q] * (TM)rs[s2];
    w[gq] += (T)d;
  }
}

// Register-blocked variant for n = 2, 4: the free-box solves of the CTA's boxes are
// one small GEMM (shared inverse x the block of box residuals), each thread owning
// an RB x CB tile (rows x boxes) and reading RB inverse entries with one vector
// load; structure boxes are then solved with their own inverses.
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

template <typename T, typename TM, int BS>
__global__ void __launch_bounds__(128) kv_boxg(T* w, const T* __restrict__ b, T* rE, int N, StokesCoef<T> c,
                                               int color, const int* __restrict__ slot,
                                               const double* __restrict__ Ms, const TM* __restrict__ Mf) {
  using G = BoxGemm<TM, BS>;
  using V = typename VecOf<TM, G::RB>::type;
  constexpr int NB = G::NB, NV = 2 * BS * (BS + 1);
  __shared__ __align__(16) TM sMf[NB * NB];
  __shared__ T rs[G::BPC][NB];
  __shared__ int sslot[G::BPC];
  const int tid = threadIdx.x;
  const int nb = N / BS, half = nb >> 1, nbox = half * half;
  const int box0 = blockIdx.x * G::BPC;
  for (int e = tid; e < NB * NB; e += G::THREADS) sMf[e] = Mf[e];  // set-up data
  pdl_enter();
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
      const int g = cc * N * N + j * N + i;
      r = b[g] - stokes_row(w, N, c, cc, i, j);
      if (rE && q < NV && slot[J * nb + I] >= 0) {
        r += rE[g];
        rE[g] = (T)0;
      }
    }
    rs[lb][q] = r;
  }
  __syncthreads();
  // free boxes: delta[q][box] = sum_s Mf[s][q] r[box][s]
  const int rg = tid % G::RG, bg = tid / G::RG;
  if (bg < G::BG) {
    TM acc[G::RB][G::CB];
#pragma unroll
    for (int a = 0; a < G::RB; ++a)
#pragma unroll
      for (int k = 0; k < G::CB; ++k) acc[a][k] = 0;
#pragma unroll 4
    for (int s2 = 0; s2 < NB; ++s2) {
      const V m = *reinterpret_cast<const V*>(&sMf[s2 * NB + rg * G::RB]);
      const TM* mv = reinterpret_cast<const TM*>(&m);
#pragma unroll
      for (int k = 0; k < G::CB; ++k) {
        const TM rv = (TM)rs[bg * G::CB + k][s2];
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
        w[cc * N * N + j * N + i] += (T)acc[a][k];
      }
    }
  }
  // structure boxes: their own FP64 inverses; all threads share the (box, row) pairs
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

// Strip kernel for 4 x 4 boxes on large levels.  A CTA takes strips of W boxes of
// one colour in one box row (every other box along x, so a strip spans 8W cells),
// persistent over the strips of the colour, and for each strip:
//   1. has its w rows with their one-cell halo (u: 6 rows, v: 7, p: 6; 8W + 8
//      columns, periodic) brought into shared memory by bulk copies (one to
//      three per row, split where the row wraps) that complete on an mbarrier; the copies of the next strip go into
//      a second buffer while this one is computed;
//   2. forms the residual b - A_S w (+ the elasticity term rE on the rows of
//      structure boxes, which it clears) of every unknown of its boxes: the 56 W
//      unknowns are split into units of 32 (one component per unit), each thread
//      owns the same unknowns in every strip and keeps their positions in registers;
//   3. applies the shared free-box inverse to all W residuals as one register-
//      blocked product (RB rows x CB boxes per thread), then the FP64 inverses of
//      the strip's structure boxes, one (box, row) dot product per thread;
//   4. writes w + delta back.
// The free-box inverse is staged once per CTA before the programmatic-launch wait.
template <typename T, typename TM, int W>
struct Strip {
  static constexpr int NB = 56, THREADS = 256, WARPS = THREADS / 32;
  static constexpr int SPAN = 8 * W;            // cells of one strip
  static constexpr int LD = SPAN + 8;           // staged columns [X0 - 4, X0 + SPAN + 4)
  static constexpr int TROWS = 6 + 7 + 6;       // staged rows of u, v, p
  static constexpr int TILE = TROWS * LD;       // elements of one staging buffer
  static constexpr int RLD = W + 8;             // row stride of the residual block [q][box]
  static constexpr int QLD = 60;                // row stride of the correction block [box][q]
  static constexpr bool SPLIT = !std::is_same<T, TM>::value;  // separate TM copy of the residuals
  static constexpr int RB = sizeof(TM) == 4 ? 4 : 2;  // rows per thread (one 16-byte load of M)
  static constexpr int CB = sizeof(TM) == 4 ? 2 : 4;  // boxes per thread
  static constexpr int RG = NB / RB, BG = W / CB;
  static_assert(RG * BG <= THREADS, "product tiling");
  // units of 32 unknowns: u rows (5W unknowns each), v rows (4W), p rows (4W)
  static constexpr int UNITS = NB * W / 32, UPW = (UNITS + WARPS - 1) / WARPS;
  static_assert((5 * W) % 32 == 0 || (20 * W) % 32 == 0, "u units");
  static_assert((20 * W) % 32 == 0 && (16 * W) % 32 == 0, "unit boundaries");
  static constexpr size_t OFF_TILE = ((size_t)NB * NB * sizeof(TM) + 15) / 16 * 16;
  static constexpr size_t OFF_R = OFF_TILE + 2 * (size_t)TILE * sizeof(T);
  static constexpr size_t OFF_D = OFF_R + (size_t)NB * RLD * sizeof(T);
  static constexpr size_t OFF_RM = OFF_D + (size_t)W * QLD * sizeof(T);
  static constexpr size_t SMEM = OFF_RM + (SPLIT ? (size_t)NB * RLD * sizeof(TM) : 0);
};

template <typename TM, int n>
struct VecLoad;
template <>
struct VecLoad<float, 4> {
  __device__ static void get(const float* p, float* o) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <>
struct VecLoad<float, 2> {
  __device__ static void get(const float* p, float* o) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
};
template <>
struct VecLoad<double, 2> {
  __device__ static void get(const double* p, double* o) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
};
template <>
struct VecLoad<double, 4> {
  __device__ static void get(const double* p, double* o) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    const double2 u = *reinterpret_cast<const double2*>(p + 2);
    o[0] = v.x; o[1] = v.y; o[2] = u.x; o[3] = u.y;
  }
};

// One unknown of a strip, as a thread keeps it across strips: its offset in a
// staging buffer (toff), in the [q][box] blocks (roff = q * RLD + k), and its
// component, box-relative row, box and strip column packed in one word.
struct StripItem {
  int toff, roff, pack;  // pack = comp << 28 | jr << 24 | k << 16 | col
};

// Unknown e (0 <= e < 56 W) in the order u rows, v rows, p rows (each row: W boxes
// x 5 faces or 4 faces/cells), for a staging buffer with row stride LD and blocks
// with row stride RLD.
__device__ __forceinline__ StripItem strip_item(int e, int W, int LD, int RLD) {
  int comp, jr, k, d, q;
  if (e < 20 * W) {
    jr = e / (5 * W);
    const int t = e - jr * 5 * W;
    comp = 0; k = t / 5; d = t - k * 5; q = jr * 5 + d;
  } else if (e < 40 * W) {
    e -= 20 * W;
    jr = e / (4 * W);
    const int t = e - jr * 4 * W;
    comp = 1; k = t >> 2; d = t & 3; q = 20 + jr * 4 + d;
  } else {
    e -= 40 * W;
    jr = e / (4 * W);
    const int t = e - jr * 4 * W;
    comp = 2; k = t >> 2; d = t & 3; q = 40 + jr * 4 + d;
  }
  const int col = 8 * k + d;
  const int trow = (comp == 0 ? 0 : (comp == 1 ? 6 : 13)) + jr + 1;  // staged row of the unknown
  StripItem it;
  it.toff = trow * LD + col + 4;
  it.roff = q * RLD + k;
  it.pack = (comp << 28) | (jr << 24) | (k << 16) | col;
  return it;
}

// Issue the bulk copies of one strip's tile (rows y0 - 1 .. of u, v, p; columns
// X0 - 4 .. X0 + 8W + 3, split where they wrap) into buf: lane r < TROWS of
// the calling warp copies row r; lane 0 first announces the byte count.  The caller
// has ordered earlier generic accesses of buf before these writes (barrier + proxy
// fence).
template <typename T, int W>
__device__ __forceinline__ void strip_issue(const T* w, int N, int y0, int X0, T* buf, unsigned long long* bar,
                                            int lane) {
  constexpr int LD = 8 * W + 8, TROWS = 19;
  if (lane == 0) mbar_arrive_expect_tx(bar, (unsigned)(TROWS * LD * sizeof(T)));
  __syncwarp();
  if (lane < TROWS) {
    const int r = lane;
    const int comp = r < 6 ? 0 : (r < 13 ? 1 : 2);
    const int ry = r - (comp == 0 ? 0 : (comp == 1 ? 6 : 13));
    const int y = (y0 - 1 + ry) & (N - 1);
    const T* row = w + (size_t)comp * N * N + (size_t)y * N;
    T* dst = buf + r * LD;
    // the staged columns X0 - 4 .. X0 + 8W + 3 wrap at most twice (8W + 8 <= 2N);
    // every segment starts and ends on a multiple of 4 elements (16 bytes or more)
    int x = (X0 - 4) & (N - 1), done = 0;
    while (done < LD) {
      const int seg = min(LD - done, N - x);
      bulk_g2s(dst + done, row + x, (unsigned)(seg * sizeof(T)), bar);
      done += seg;
      x = 0;
    }
  }
}

template <typename T, typename TM, int W>
__global__ void __launch_bounds__(256, 3) kv_boxt(T* w, const T* __restrict__ b, T* rE, int N, StokesCoef<T> c,
                                               int color, const int* __restrict__ slot,
                                               const double* __restrict__ Ms, const TM* __restrict__ Mf, int* err,
                                               unsigned long long limit_ns) {
  using S = Strip<T, TM, W>;
  constexpr int NB = S::NB, LD = S::LD, RLD = S::RLD;
  extern __shared__ __align__(16) unsigned char smem[];
  TM* sMf = reinterpret_cast<TM*>(smem);
  T* tiles = reinterpret_cast<T*>(smem + S::OFF_TILE);
  T* sR = reinterpret_cast<T*>(smem + S::OFF_R);
  T* sD = reinterpret_cast<T*>(smem + S::OFF_D);
  TM* sRM = S::SPLIT ? reinterpret_cast<TM*>(smem + S::OFF_RM) : reinterpret_cast<TM*>(sR);
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ int sslot[W];
  __shared__ int slist[W];
  __shared__ int nsl;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  {
    constexpr int VM = 16 / (int)sizeof(TM);
    const float4* src = reinterpret_cast<const float4*>(Mf);
    float4* dst = reinterpret_cast<float4*>(sMf);
    for (int e = tid; e < NB * NB / VM; e += S::THREADS) dst[e] = src[e];  // set-up data
  }
  // this thread's unknowns (the same in every strip)
  StripItem items[S::UPW];
#pragma unroll
  for (int i = 0; i < S::UPW; ++i) {
    const int unit = wp + S::WARPS * i;
    items[i] = unit < S::UNITS ? strip_item(unit * 32 + lane, W, LD, RLD) : StripItem{0, 0, -1};
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  __syncthreads();
  pdl_enter();
  const int nb = N >> 2, half = nb >> 1, spr = half / W, nstrips = spr * half;
  const int cx = color & 1, cy = color >> 1, m = N - 1;
  const size_t n = (size_t)N * N;
  unsigned phase = 0u;  // bit i: parity of the next completion of bar[i]
  int st = blockIdx.x;
  if (wp == 0 && st < nstrips) {
    const int Jp = st / spr, sx = st - Jp * spr;
    strip_issue<T, W>(w, N, 4 * (2 * Jp + cy), 4 * (2 * sx * W + cx), tiles, &bar[0], lane);
  }
  for (int it = 0; st < nstrips; ++it, st += gridDim.x) {
    const int buf = it & 1;
    const int Jp = st / spr, sx = st - Jp * spr;
    const int J = 2 * Jp + cy, I0 = 2 * sx * W + cx;
    const int y0 = 4 * J, X0 = 4 * I0;
    if (tid < W) sslot[tid] = slot[J * nb + I0 + 2 * tid];
    // 1. this strip's tile has landed (bounded wait); then the next strip's copies
    const unsigned par = (phase >> buf) & 1u;
    const bool ok = mbar_wait_bounded(&bar[buf], par, limit_ns);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(err, DEV_ERR_TIMEOUT);
        mbar_wait_bounded(&bar[buf], par, DRAIN_LIMIT_NS);  // copies in flight land first
      }
      return;
    }
    phase ^= 1u << buf;
    const int nx = st + gridDim.x;
    if (wp == 0 && nx < nstrips) {
      // the other buffer was last read before the barrier that ended the previous strip
      fence_proxy_async_smem();
      const int Jn = nx / spr, sxn = nx - Jn * spr;
      strip_issue<T, W>(w, N, 4 * (2 * Jn + cy), 4 * (2 * sxn * W + cx), tiles + (buf ^ 1) * S::TILE,
                        &bar[buf ^ 1], lane);
    }
    const T* tile = tiles + buf * S::TILE;
    // 2. residuals (the component of a unit is the same for its whole warp)
    // element offsets fit 32 bits: 3 N^2 < 2^31 for N <= 16384
    auto goff = [&](int pk) -> unsigned {
      return (unsigned)(pk >> 28) * (unsigned)n + (unsigned)(((y0 + ((pk >> 24) & 15)) & m) * N) +
             (unsigned)((X0 + (pk & 0xffff)) & m);
    };
    T bv[S::UPW];
    unsigned gv[S::UPW];
#pragma unroll
    for (int i = 0; i < S::UPW; ++i) {
      gv[i] = 0u;
      bv[i] = (T)0;
      if (items[i].pack < 0) continue;
      gv[i] = goff(items[i].pack);
      bv[i] = b[gv[i]];
    }
#pragma unroll
    for (int i = 0; i < S::UPW; ++i) {
      const int pk = items[i].pack;
      if (pk < 0) continue;
      const int comp = pk >> 28, k = (pk >> 16) & 0xff;
      const T* t0 = tile + items[i].toff;
      T a;
      if (comp == 0) {  // u: staged rows 0..5 of u, p at +13 LD
        a = c.diag * t0[0] + c.off * (t0[1] + t0[-1] + t0[LD] + t0[-LD]) - c.g * (t0[13 * LD] - t0[13 * LD - 1]);
      } else if (comp == 1) {  // v: rows 6..12, p of the same row at +7 LD, the row below at +6 LD
        a = c.diag * t0[0] + c.off * (t0[1] + t0[-1] + t0[LD] + t0[-LD]) - c.g * (t0[7 * LD] - t0[6 * LD]);
      } else {  // p: rows 13..18; u of the same row at -13 LD, v at -7 LD (and -6 LD above)
        a = c.g * (t0[-13 * LD + 1] - t0[-13 * LD] + t0[-6 * LD] - t0[-7 * LD]);
      }
      T r = bv[i] - a;
      if (rE && comp < 2 && sslot[k] >= 0) {
        r += rE[gv[i]];
        rE[gv[i]] = (T)0;
      }
      sR[items[i].roff] = r;
      if (S::SPLIT) sRM[items[i].roff] = (TM)r;
    }
    __syncthreads();
    // 3a. free-box product for every box of the strip: D[k][q] = sum_s Mf[s][q] R[s][k]
    {
      const int rg = tid % S::RG, bg = tid / S::RG;
      if (bg < S::BG) {
        TM acc[S::RB][S::CB];
#pragma unroll
        for (int a = 0; a < S::RB; ++a)
#pragma unroll
          for (int kk = 0; kk < S::CB; ++kk) acc[a][kk] = (TM)0;
#pragma unroll 4
        for (int s2 = 0; s2 < NB; ++s2) {
          TM mv[S::RB], rv[S::CB];
          VecLoad<TM, S::RB>::get(sMf + s2 * NB + rg * S::RB, mv);
          VecLoad<TM, S::CB>::get(sRM + s2 * RLD + bg * S::CB, rv);
#pragma unroll
          for (int a = 0; a < S::RB; ++a)
#pragma unroll
            for (int kk = 0; kk < S::CB; ++kk) acc[a][kk] += mv[a] * rv[kk];
        }
        // each thread's RB consecutive rows of a box are contiguous in D[k][q]: one
        // 16-byte (or two) store per box
#pragma unroll
        for (int kk = 0; kk < S::CB; ++kk) {
          T* dst = sD + (bg * S::CB + kk) * S::QLD + rg * S::RB;
          if constexpr (sizeof(T) == 4 && S::RB == 4) {
            *reinterpret_cast<float4*>(dst) =
                make_float4((float)acc[0][kk], (float)acc[1][kk], (float)acc[2][kk], (float)acc[3][kk]);
          } else if constexpr (sizeof(T) == 8 && S::RB == 2) {
            *reinterpret_cast<double2*>(dst) = make_double2((double)acc[0][kk], (double)acc[1][kk]);
          } else {
#pragma unroll
            for (int a = 0; a < S::RB; ++a) dst[a] = (T)acc[a][kk];
          }
        }
      }
    }
    if (wp == 0) {  // the strip's structure boxes, in box order
      const bool isS = lane < W && sslot[lane] >= 0;
      const unsigned bal = __ballot_sync(0xffffffffu, isS);
      if (isS) slist[__popc(bal & ((1u << lane) - 1u))] = lane;
      if (lane == 0) nsl = __popc(bal);
    }
    __syncthreads();
    // 3b. structure boxes: their own FP64 inverses, one (box, row) per thread (replaces 3a)
    for (int e = tid; e < nsl * NB; e += S::THREADS) {
      const int k = slist[e / NB], q = e - (e / NB) * NB;
      const double* M = Ms + (size_t)sslot[k] * NB * NB + q;
      double d0 = 0.0, d1 = 0.0;
#pragma unroll 8
      for (int s2 = 0; s2 < NB; s2 += 2) {
        d0 += M[(size_t)s2 * NB] * (double)sR[s2 * RLD + k];
        d1 += M[(size_t)(s2 + 1) * NB] * (double)sR[(s2 + 1) * RLD + k];
      }
      sD[k * S::QLD + q] = (T)(d0 + d1);
    }
    __syncthreads();
    // 4. w += delta on the strip's unknowns
#pragma unroll
    for (int i = 0; i < S::UPW; ++i) {
      if (items[i].pack < 0) continue;
      const int k = (items[i].pack >> 16) & 0xff, q = items[i].roff / RLD;
      w[goff(items[i].pack)] = tile[items[i].toff] + sD[k * S::QLD + q];
    }
    __syncthreads();  // the buffer, the residuals and the corrections are reused next
  }
}

template <typename T, typename TM, int W>
int strip_occupancy() {
  // the dynamic shared-memory limit and the resident CTAs per SM, once per instantiation
  static std::mutex mu;
  static int occ = -1;
  std::lock_guard<std::mutex> lock(mu);
  if (occ >= 0) return occ;
  using S = Strip<T, TM, W>;
  occ = 0;
  if (cudaFuncSetAttribute(kv_boxt<T, TM, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM) !=
      cudaSuccess) {
    cudaGetLastError();
    return occ;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kv_boxt<T, TM, W>, S::THREADS, S::SMEM) == cudaSuccess)
    occ = n;
  else
    cudaGetLastError();
  return occ;
}

// Launch kv_boxt with strip width W (boxes of one colour per strip; N_l / 8 must be
// a multiple of W).  Returns false if the device cannot run it (no launch).
template <typename T, typename TM, int W>
bool launch_strip(Problem& P, bool pdl, T* w, const T* b, T* E, int N, StokesCoef<T> c, int color, const int* slot,
                  const double* Ms, const TM* Mf) {
  const int occ = strip_occupancy<T, TM, W>();
  if (occ <= 0) return false;
  const long half = N / 8, strips = half * half / W;
  const int grid = (int)std::min<long>(strips, (long)P.n_sm * occ);
  vlaunch(pdl, kv_boxt<T, TM, W>, grid, Strip<T, TM, W>::THREADS, Strip<T, TM, W>::SMEM, P.stream, w, b, E, N, c,
          color, slot, Ms, Mf, P.dev_err, P.wait_limit_ns);
  return true;
}

// Strip width: the widest of 32, 16, 8 that divides N_l / 8 and still gives at
// least 2 strips per SM, else the narrowest that divides it (most CTAs).
inline int strip_width(const Problem& P, int N) {
  const long half = N / 8, nbox = half * half;
  if (P.box_strip_w > 0) return half % P.box_strip_w == 0 ? P.box_strip_w : 0;
  int pick = 0;
  for (int W : {32, 16, 8}) {
    if (half % W) continue;
    pick = W;
    if (nbox / W >= 2L * P.n_sm) break;
  }
  return pick;
}

// FP32 4 x 4 boxes, eight per CTA of 64 threads: the residuals of the eight boxes
// first (7 rows a thread), then thread q forms row q of all eight free-box solves
// together, one entry of the shared inverse (read through L1) against the eight
// residuals read as two vectors, so that a thread spends 11 instructions per 8
// FMAs instead of 3 per FMA; a structure box's row is then formed again from its
// FP64 inverse.  The same sums, in the same order, as kv_boxn.
constexpr int OCT_BPC = 8;
__global__ void __launch_bounds__(64) kv_boxo(float* w, const float* __restrict__ b, float* rE, int N,
                                              StokesCoef<float> c, int color, const int* __restrict__ slot,
                                              const double* __restrict__ Ms, const float* __restrict__ Mf) {
  constexpr int BS = 4, NB = 2 * BS * (BS + 1) + BS * BS, NV = 2 * BS * (BS + 1);
  __shared__ __align__(16) float rs[NB][OCT_BPC];
  __shared__ int sg[OCT_BPC][NB];
  __shared__ int ssl[OCT_BPC];
  const int tid = threadIdx.x;
  const int nb = N / BS, half = nb >> 1, nbox = half * half;
  const int t0 = blockIdx.x * OCT_BPC;
  if (tid < OCT_BPC) {
    const int t = t0 + tid;
    ssl[tid] = t < nbox ? slot[(2 * (t / half) + (color >> 1)) * nb + 2 * (t % half) + (color & 1)] : -2;
  }
  __syncthreads();
  pdl_enter();
  for (int e = tid; e < OCT_BPC * NB; e += 64) {
    const int lb = e / NB, q = e - lb * NB, t = t0 + lb;
    if (t >= nbox) {
      rs[q][lb] = 0.f;
      sg[lb][q] = -1;
      continue;
    }
    const int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
    int cc, i, j;
    box_unknown(q, BS, I * BS, J * BS, N, &cc, &i, &j);
    const int gq = cc * N * N + j * N + i;
    float r = b[gq] - stokes_row(w, N, c, cc, i, j);
    if (rE && ssl[lb] >= 0 && q < NV) {
      r += rE[gq];
      rE[gq] = 0.f;
    }
    rs[q][lb] = r;
    sg[lb][q] = gq;
  }
  __syncthreads();
  const int q = tid;
  if (q >= NB) return;
  float d[OCT_BPC];
#pragma unroll
  for (int k = 0; k < OCT_BPC; ++k) d[k] = 0.f;
  const float* M = Mf + q;
#pragma unroll 4
  for (int s2 = 0; s2 < NB; ++s2) {
    const float m = __ldg(M + s2 * NB);
    const float4 r0 = *reinterpret_cast<const float4*>(&rs[s2][0]);
    const float4 r1 = *reinterpret_cast<const float4*>(&rs[s2][4]);
    d[0] = fmaf(m, r0.x, d[0]);
    d[1] = fmaf(m, r0.y, d[1]);
    d[2] = fmaf(m, r0.z, d[2]);
    d[3] = fmaf(m, r0.w, d[3]);
    d[4] = fmaf(m, r1.x, d[4]);
    d[5] = fmaf(m, r1.y, d[5]);
    d[6] = fmaf(m, r1.z, d[6]);
    d[7] = fmaf(m, r1.w, d[7]);
  }
#pragma unroll
  for (int lb = 0; lb < OCT_BPC; ++lb) {
    const int gq = sg[lb][q];
    if (gq < 0) continue;
    const int sl = ssl[lb];
    float dv = d[lb];
    if (sl >= 0) {
      const double* Mb = Ms + (size_t)sl * NB * NB + q;
      double dd = 0.0;
#pragma unroll 8
      for (int s2 = 0; s2 < NB; ++s2) dd += Mb[(size_t)s2 * NB] * (double)rs[s2][lb];
      dv = (float)dd;
    }
    w[gq] += dv;
  }
}

// Forms of the n x n box kernel (n = 2, 4) the set-up autotuner chooses from.
enum : int { BOXF_RULE = 0, BOXF_ONE = 1, BOXF_ROWS = 2, BOXF_GEMM = 3, BOXF_STRIP8 = 4, BOXF_STRIP16 = 5,
             BOXF_STRIP32 = 6, BOXF_OCT = 7 };

template <typename T>
constexpr int pix();

// Launch one colour phase of level l's boxes in the given form (BOXF_RULE: the size
// rule).  Returns false if the form does not apply to the level (nothing launched).
template <typename T, typename TM>
bool launch_box_form(Problem& P, int l, int form, T* w, const T* b, T* E, int color) {
  LevelInfo& L = P.lev[l];
  const StokesCoef<T> c = coefs<T>(P, l);
  const int half = L.nb / 2;
  const long nbox = (long)half * half;
  const double* Ms = L.Mstruct;
  const TM* Mf = Mfree_of<TM>(L);
  const bool pdl = use_pdl(P);
  const int bs = P.prm.box;
  if (bs != 2 && bs != 4) return false;
  switch (form) {
    case BOXF_ONE:
      if (bs == 2)
        vlaunch(pdl, kv_boxs<T, TM, 2>, (int)nbox, BoxShape<2, 1>::TPBOX, 0, P.stream, w, b, E, L.N, c, color, L.flag,
                Ms, Mf);
      else
        vlaunch(pdl, kv_boxs<T, TM, 4>, (int)nbox, BoxShape<4, 1>::TPBOX, 0, P.stream, w, b, E, L.N, c, color, L.flag,
                Ms, Mf);
      return true;
    case BOXF_ROWS:
      if (bs == 2)
        vlaunch(pdl, kv_boxn<T, TM, 2, 8>, nblk(nbox, 8), BoxShape<2, 8>::THREADS, 0, P.stream, w, b, E, L.N, c, color,
                L.flag, Ms, Mf);
      else
        vlaunch(pdl, kv_boxn<T, TM, 4, 4>, nblk(nbox, 4), BoxShape<4, 4>::THREADS, 0, P.stream, w, b, E, L.N, c, color,
                L.flag, Ms, Mf);
      return true;
    case BOXF_GEMM:
      if (bs == 2)
        vlaunch(pdl, kv_boxg<T, TM, 2>, nblk(nbox, BoxGemm<TM, 2>::BPC), 128, 0, P.stream, w, b, E, L.N, c, color,
                L.flag, Ms, Mf);
      else
        vlaunch(pdl, kv_boxg<T, TM, 4>, nblk(nbox, BoxGemm<TM, 4>::BPC), 128, 0, P.stream, w, b, E, L.N, c, color,
                L.flag, Ms, Mf);
      return true;
    case BOXF_STRIP8:  // the strip kernel stages periodic rows: not with walls
      return bs == 4 && !P.prm.walls && half % 8 == 0 && launch_strip<T, TM, 8>(P, pdl, w, b, E, L.N, c, color, L.flag, Ms, Mf);
    case BOXF_STRIP16:
      return bs == 4 && !P.prm.walls && half % 16 == 0 && launch_strip<T, TM, 16>(P, pdl, w, b, E, L.N, c, color, L.flag, Ms, Mf);
    case BOXF_STRIP32:
      return bs == 4 && !P.prm.walls && half % 32 == 0 && launch_strip<T, TM, 32>(P, pdl, w, b, E, L.N, c, color, L.flag, Ms, Mf);
    case BOXF_OCT:
      if constexpr (std::is_same<T, float>::value && std::is_same<TM, float>::value) {
        if (bs != 4) return false;
        vlaunch(pdl, kv_boxo, nblk(nbox, OCT_BPC), 64, 0, P.stream, w, b, E, L.N, c, color, (const int*)L.flag, Ms,
                Mf);
        return true;
      }
      return false;
    default:
      return false;
  }
}

// Big boxes (8 x 8 and 16 x 16: 208 and 800 unknowns) in two launches per colour:
// kv_bigres takes the residuals of the colour's boxes (one CTA per box, into
// rbox), then kv_bigsolve multiplies them by the box inverses with the rows of a
// box split over CTAs of 32 rows (8 warps share the sum over the columns), so that
// a structure box's FP64 product (n_B^2 FMAs) spreads over n_B / 32 SMs instead of
// one.  Boxes of one colour share no unknowns, so every residual of the colour can
// be taken before any update, as in the other forms.
constexpr int BIG_NB_MAX = 800;

template <typename T>
__global__ void __launch_bounds__(256) kv_bigres(const T* __restrict__ w, const T* __restrict__ b, T* rE,
                                                 T* __restrict__ rbox, int N, StokesCoef<T> c, int color, int bs,
                                                 int nB, const int* __restrict__ slot) {
  pdl_enter();
  const int nb = N / bs, half = nb >> 1, t = blockIdx.x;
  const int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
  const int sl = slot[J * nb + I];
  const int nV = 2 * bs * (bs + 1);
  for (int q = threadIdx.x; q < nB; q += blockDim.x) {
    int cc, i, j;
    box_unknown(q, bs, I * bs, J * bs, N, &cc, &i, &j);
    const int gq = cc * N * N + j * N + i;
    T r = b[gq] - stokes_row(w, N, c, cc, i, j);
    if (rE && sl >= 0 && q < nV) {
      r += rE[gq];
      rE[gq] = (T)0;
    }
    rbox[(size_t)t * nB + q] = r;
  }
}

// grid (row chunks of 32, boxes of the colour)
template <typename T, typename TM>
__global__ void __launch_bounds__(256) kv_bigsolve(T* w, const T* __restrict__ rbox, int N, int color, int bs,
                                                   int nB, const int* __restrict__ slot,
                                                   const double* __restrict__ Ms, const TM* __restrict__ Mf) {
  __shared__ T rs[BIG_NB_MAX];
  __shared__ double part[8][32];
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int nb = N / bs, half = nb >> 1, t = blockIdx.y;
  const int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
  const int sl = slot[J * nb + I];
  const int q = blockIdx.x * 32 + lane;
  pdl_enter();
  for (int s2 = tid; s2 < nB; s2 += 256) rs[s2] = rbox[(size_t)t * nB + s2];
  __syncthreads();
  double d = 0.0;
  if (q < nB) {
    if (sl >= 0) {
      const double* M = Ms + (size_t)sl * nB * nB + q;
      for (int s2 = wp; s2 < nB; s2 += 8) d += M[(size_t)s2 * nB] * (double)rs[s2];
    } else {
      const TM* M = Mf + q;
      TM dm = 0;
      for (int s2 = wp; s2 < nB; s2 += 8) dm += M[(size_t)s2 * nB] * (TM)rs[s2];
      d = (double)dm;
    }
  }
  part[wp][lane] = d;
  __syncthreads();
  if (wp == 0 && q < nB) {
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += part[k][lane];
    int cc, i, j;
    box_unknown(q, bs, I * bs, J * bs, N, &cc, &i, &j);
    w[cc * N * N + j * N + i] += (T)sum;
  }
}

template <typename T, typename TM>
int launch_bigbox(Problem& P, int l, T* w, const T* b, T* E, int color) {
  LevelInfo& L = P.lev[l];
  const StokesCoef<T> c = coefs<T>(P, l);
  const int half = L.nb / 2, nbox = half * half, nB = P.nB, bs = P.prm.box;
  if (nB > BIG_NB_MAX) return fail(IB_ERR_INVALID_ARG, "box too large for the split box kernel");
  T* rbox = lbuf<T>(L).r;  // 3 N^2 >= nbox * n_B: free during a sweep
  const bool pdl = use_pdl(P);
  vlaunch(pdl, kv_bigres<T>, nbox, 256, 0, P.stream, (const T*)w, b, E, rbox, L.N, c, color, bs, nB,
          (const int*)L.flag);
  IB_LAUNCH_CHECK();
  vlaunch(pdl, kv_bigsolve<T, TM>, dim3((nB + 31) / 32, nbox), 256, 0, P.stream, w, (const T*)rbox, L.N, color,
          bs, nB, (const int*)L.flag, (const double*)L.Mstruct, Mfree_of<TM>(L));
  IB_LAUNCH_CHECK();
  return IB_OK;
}

template <typename T, typename TM>
int launch_boxn(Problem& P, int l, T* w, const T* b, T* E, int color) {
  LevelInfo& L = P.lev[l];
  const StokesCoef<T> c = coefs<T>(P, l);
  const int half = L.nb / 2;
  const long nbox = (long)half * half;
  const double* Ms = L.Mstruct;
  const TM* Mf = Mfree_of<TM>(L);
  // the form the set-up timed fastest on this level, else the size rule
  // 16 x 16 boxes, and 8 x 8 boxes on levels with fewer boxes per colour than SMs:
  // the split form
  if (P.prm.box == 16 || (P.prm.box == 8 && nbox < P.n_sm)) return launch_bigbox<T, TM>(P, l, w, b, E, color);
  const int tuned = l < 32 ? P.box_form[pix<T>()][l] : 0;
  if (tuned != BOXF_RULE && launch_box_form<T, TM>(P, l, tuned, w, b, E, color)) {
    IB_LAUNCH_CHECK();
    return IB_OK;
  }
  // the GEMM form pays off on large levels, one box per CTA on small ones
  const bool gemm = nbox >= P.box_gemm_min;
  const bool one = nbox <= P.box_one_max;
  const bool pdl = use_pdl(P);
  if (P.prm.box == 4 && P.box_strip && !P.prm.walls && nbox >= P.box_strip_min) {
    bool done = false;
    switch (strip_width(P, L.N)) {
      case 32: done = launch_strip<T, TM, 32>(P, pdl, w, b, E, L.N, c, color, L.flag, Ms, Mf); break;
      case 16: done = launch_strip<T, TM, 16>(P, pdl, w, b, E, L.N, c, color, L.flag, Ms, Mf); break;
      case 8: done = launch_strip<T, TM, 8>(P, pdl, w, b, E, L.N, c, color, L.flag, Ms, Mf); break;
      default: break;
    }
    if (done) {
      IB_LAUNCH_CHECK();
      return IB_OK;
    }
  }
#define IB_BOXN(BS_, BPC_)                                                                                    \
  vlaunch(pdl, kv_boxn<T, TM, BS_, BPC_>, nblk(nbox, BPC_), BoxShape<BS_, BPC_>::THREADS, 0, P.stream, w, b, E, \
          L.N, c, color, L.flag, Ms, Mf)
  switch (P.prm.box) {
    case 2:
      if (gemm)
        vlaunch(pdl, kv_boxg<T, TM, 2>, nblk(nbox, BoxGemm<TM, 2>::BPC), 128, 0, P.stream, w, b, E, L.N, c, color,
                L.flag, Ms, Mf);
      else if (one)
        vlaunch(pdl, kv_boxs<T, TM, 2>, (int)nbox, BoxShape<2, 1>::TPBOX, 0, P.stream, w, b, E, L.N, c, color,
                L.flag, Ms, Mf);
      else
        IB_BOXN(2, 8);
      break;
    case 4:
      if (gemm)
        vlaunch(pdl, kv_boxg<T, TM, 4>, nblk(nbox, BoxGemm<TM, 4>::BPC), 128, 0, P.stream, w, b, E, L.N, c, color,
                L.flag, Ms, Mf);
      else if (one)
        vlaunch(pdl, kv_boxs<T, TM, 4>, (int)nbox, BoxShape<4, 1>::TPBOX, 0, P.stream, w, b, E, L.N, c, color,
                L.flag, Ms, Mf);
      else
        IB_BOXN(4, 4);
      break;
    case 8:
      IB_BOXN(8, 1);
      break;
    default:  // 16 x 16 boxes: 800 unknowns, one CTA of 800 threads per box
      IB_BOXN(16, 1);
      break;
  }
#undef IB_BOXN
  IB_LAUNCH_CHECK();
  return IB_OK;
}

// 1 x 1 boxes: residual of the colour's boxes first, then the solves.
// rE rows of the colour's structure boxes are taken out (cleared).
template <typename T>
__global__ void kv_colres1(const T* __restrict__ w, const T* __restrict__ b, T* rE, T* __restrict__ r, int N,
                           StokesCoef<T> c, int color, const int* __restrict__ slot) {
  pdl_enter();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int half = N >> 1;
  if (t >= half * half) return;
  int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
  int n = N * N, m = N - 1;
  int I1 = (I + 1) & m, J1 = (J + 1) & m;
  const bool st = rE && slot[J * N + I] >= 0;  // only structure rows carry rE
  const T* e = st ? rE : nullptr;
  r[J * N + I] = resid_at(w, b, e, N, c, 0, I, J);
  r[J * N + I1] = resid_at(w, b, e, N, c, 0, I1, J);
  r[n + J * N + I] = resid_at(w, b, e, N, c, 1, I, J);
  r[n + J1 * N + I] = resid_at(w, b, e, N, c, 1, I, J1);
  r[2 * n + J * N + I] = resid_at(w, b, e, N, c, 2, I, J);
  if (st) {
    rE[J * N + I] = (T)0;
    rE[J * N + I1] = (T)0;
    rE[n + J * N + I] = (T)0;
    rE[n + J1 * N + I] = (T)0;
  }
}

template <typename T, typename TM>
__global__ void kv_box1(const T* __restrict__ r, T* __restrict__ w, int N, int color,
                        const int* __restrict__ slot, const double* __restrict__ Ms,
                        const TM* __restrict__ Mf) {
  pdl_enter();
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

// b_{l+1} = R (b - A_l w + rE); rE (all rows, may be NULL) is cleared by kv_prolong.
// Also zeroes the coarse correction w_{l+1} (the coarse level's initial guess),
// one cell per thread like b_{l+1}.
template <typename T>
__global__ void kv_resres(const T* __restrict__ w, const T* __restrict__ b, const T* __restrict__ rE,
                          T* __restrict__ bc, T* __restrict__ wc, int Nc, StokesCoef<T> c) {
  pdl_enter();
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int nc = Nc * Nc;
  if (idx >= nc) return;
  T ru, rv, rp;
  restrict_resid_cell(w, b, rE, 2 * Nc, c, idx % Nc, idx / Nc, &ru, &rv, &rp);
  bc[idx] = ru;
  bc[nc + idx] = rv;
  bc[2 * nc + idx] = rp;
  wc[idx] = (T)0;
  wc[nc + idx] = (T)0;
  wc[2 * nc + idx] = (T)0;
}

// w += P e; also clears rE (the restriction's elasticity term; may be NULL).
template <typename T>
__global__ void kv_prolong(const T* __restrict__ ec, T* __restrict__ wf, int N, T* __restrict__ rE, int walls) {
  pdl_enter();
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int n = N * N;
  if (idx >= n) return;
  T cu, cv, cp;
  prolong_cell(ec, N, idx & (N - 1), idx / N, &cu, &cv, &cp, walls);
  wf[idx] += cu;
  wf[n + idx] += cv;
  wf[2 * n + idx] += cp;
  if (rE) {
    rE[idx] = (T)0;
    rE[n + idx] = (T)0;
  }
}

template <typename T>
__global__ void kv_zero(T* x, long n) {
  pdl_enter();
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) x[i] = (T)0;
}

// ------------------------------------------------------------------ tail kernel
//
// Two forms of the same code.  CL = false: one CTA, every array of the tail
// levels in shared memory, phases separated by __syncthreads.  CL = true: the
// CTAs of one thread-block cluster, the arrays in global memory (the levels' own
// w and b buffers, L2-resident at these sizes), loops strided over every thread of
// the cluster and phases separated by the cluster barrier, whose arrive/wait pair
// has release/acquire semantics at cluster scope (a hardware barrier: no spin).
// Every loop below has the same trip count in all threads, and the kernel has no
// early exit, so every thread reaches every barrier.

template <bool CL>
struct TailCtx;
template <>
struct TailCtx<false> {
  __device__ static int id() { return threadIdx.x; }
  __device__ static int n() { return blockDim.x; }
  __device__ static void sync() { __syncthreads(); }
};
template <>
struct TailCtx<true> {
  __device__ static unsigned rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
  }
  __device__ static unsigned size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
  }
  // warps interleaved over the CTAs (work item k of a strided loop runs in CTA
  // (k / 32) mod size), so that small phases spread over every SM of the cluster
  __device__ static int id() { return (int)((((threadIdx.x >> 5) * size() + rank()) << 5) + (threadIdx.x & 31)); }
  __device__ static int n() { return (int)(size() * blockDim.x); }
  // release/acquire at cluster scope (the defaults of arrive and wait)
  __device__ static void sync() { asm volatile("barrier.cluster.arrive;\n\tbarrier.cluster.wait;" ::: "memory"); }
};

// rE = -dt E_l w of a tail level, all rows, into the velocity part of r: clear,
// then force + spread per point quad with atomic additions.
// One structure row of the assembled elasticity (window slot t) applied to w: the
// row index and sum_e Ew[t][e] w[column of e].
template <typename T, typename TM>
__device__ __forceinline__ T window_row(const TailLevel<T, TM>& L, const T* w, int t, int* row) {
  const int N = L.N, n = N * N, r = L.wrow[t], c = r / n, rr = r - c * n, i = rr % N, j = rr / N;
  *row = r;
  const T* e0 = L.Ew + (size_t)t * WIN;
  // differences from the component's value at the row's index: each row of E_l sums
  // to zero over each column component (uniform velocities are in its kernel); with
  // no-slip walls the plain sum (the wall prolongation does not keep constants)
  const T ref[2] = {L.c.walls ? (T)0 : w[j * N + i], L.c.walls ? (T)0 : w[n + j * N + i]};
  T acc = 0;
  for (int e = 0; e < WIN; ++e) {
    const int cc = e / WSQ, rem = e - cc * WSQ;
    acc += e0[e] * (w[cc * n + wrapi(j + rem / WD - WR, N) * N + wrapi(i + rem % WD - WR, N)] - ref[cc]);
  }
  return acc;
}

template <typename T, typename TM, bool CL>
__device__ void tail_elastic(const TailLevel<T, TM>& L, const TailArgs<T, TM>& A, const T* w, T* r) {
  using C = TailCtx<CL>;
  const int tid = C::id(), nt = C::n();
  const int n2 = 2 * L.N * L.N, np = A.sp.np, lane = threadIdx.x & 31;
  for (int e = tid; e < n2; e += nt) r[e] = (T)0;
  C::sync();
  if (L.Ew) {  // assembled rows: one row per thread, each written once
    const int nr = *L.wn;
    for (int t = tid; t < nr; t += nt) {
      int row;
      const T v = window_row(L, w, t, &row);
      r[row] = A.coefE * v;
    }
    C::sync();
    return;
  }
  // 4 np is a multiple of 4: the four lanes of a quad run the same iterations
  for (int t = tid; t < 4 * np; t += nt)
    force_spread_quad<T, false>(L.pat, A.sp, w, L.N, A.coefE, t >> 2, t & 3, 0xFu << (lane & ~3), lane & ~3, A.box,
                                -1, r);
  C::sync();
}

// Full residual r = b - A_l w of a tail level (for the restriction).
template <typename T, typename TM, bool CL>
__device__ void tail_residual(const TailLevel<T, TM>& L, const TailArgs<T, TM>& A, const T* w, const T* b, T* r) {
  using C = TailCtx<CL>;
  const int tid = C::id(), nt = C::n();
  const bool hasE = A.has_E;
  if (hasE) tail_elastic<T, TM, CL>(L, A, w, r);
  const int N = L.N, n = N * N;
  for (int e = tid; e < n; e += nt) {
    const int i = e & (N - 1), j = e / N;
    r[e] = (hasE ? r[e] : (T)0) + b[e] - stokes_row(w, N, L.c, 0, i, j);
    r[n + e] = (hasE ? r[n + e] : (T)0) + b[n + e] - stokes_row(w, N, L.c, 1, i, j);
    r[2 * n + e] = b[2 * n + e] - stokes_row(w, N, L.c, 2, i, j);
  }
  C::sync();
}

// One colour of box solves on a tail level: every residual of the colour's boxes
// is staged first (1 x 1 boxes of one colour are neighbours, so all residuals
// must be taken before any update), then each (box, row) product of the box
// inverse is split over G lanes (G as large as the thread count allows, at most 32).
// rE: the level's elasticity term, or NULL.
template <typename T, typename TM, bool CL>
__device__ void tail_boxes(const TailLevel<T, TM>& L, const TailArgs<T, TM>& A, const T* b, const T* rE, T* w,
                           int color, T* sr, int* sg) {
  using C = TailCtx<CL>;
  const int tid = C::id(), nt = C::n();
  const int N = L.N, n = N * N, bs = A.box, nB = A.nB;
  const int nb = N / bs, half = nb >> 1, nbox = half * half;
  const int items = nbox * nB;
  for (int e = tid; e < items; e += nt) {
    const int t = e / nB, q = e - t * nB;
    const int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
    int cc, i, j;
    box_unknown(q, bs, I * bs, J * bs, N, &cc, &i, &j);
    const int gq = cc * n + j * N + i;
    T r = b[gq] - stokes_row(w, N, L.c, cc, i, j);
    if (rE && cc < 2) r += rE[gq];
    sr[e] = r;
    sg[e] = gq;
  }
  C::sync();
  int G = 32;
  while (G > 1 && items * G > nt) G >>= 1;
  const int total = items * G;
  for (int base = 0; base < total; base += nt) {  // same trip count in every thread
    const int e = base + tid, it = e / G, gl = e - it * G;
    T d = 0;
    if (it < items) {
      const int t = it / nB, q = it - t * nB;
      const int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
      const int sl = L.slot[J * nb + I];
      const T* rs = sr + t * nB;
      if (sl >= 0) {
        const double* M = L.Ms + (size_t)sl * nB * nB + q;
        double dd = 0.0;
        for (int s = gl; s < nB; s += G) dd += M[(size_t)s * nB] * (double)rs[s];
        d = (T)dd;
      } else {
        const TM* M = L.Mf + q;
        TM dm = 0;
        for (int s = gl; s < nB; s += G) dm += M[(size_t)s * nB] * (TM)rs[s];
        d = (T)dm;
      }
    }
    for (int o = G >> 1; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (it < items && gl == 0) w[sg[it]] += d;
  }
  C::sync();
}

template <typename T, typename TM, bool CL>
__device__ void tail_sweep(const TailLevel<T, TM>& L, const TailArgs<T, TM>& A, T* w, const T* b, T* r, bool rev,
                           T* sr, int* sg) {
  for (int cc = 0; cc < 4; ++cc) {
    const int color = rev ? seq_color(3 - cc) : seq_color(cc);
    if (A.has_E) tail_elastic<T, TM, CL>(L, A, w, r);
    tail_boxes<T, TM, CL>(L, A, b, A.has_E ? r : nullptr, w, color, sr, sg);
  }
}

// ---- cluster form: two cluster barriers per colour
//
// The elasticity term is spread with the colour filter into rE (the tail's finest
// level's own buffer, zero between phases), and each box takes its rows back out
// and clears them, as the grid-wide kernels do.  CTA r owns the boxes r, r + C,
// r + 2C, ... of the colour (C CTAs): it stages their residuals in its shared
// memory and applies their inverses behind a CTA barrier (n x n boxes, n >= 2, of
// one colour are farther apart than the stencil reaches; 1 x 1 boxes need the
// cluster barrier there).

template <typename T, typename TM>
__device__ void ctail_spread(const TailLevel<T, TM>& L, const TailArgs<T, TM>& A, const T* w, int color, T* re) {
  using C = TailCtx<true>;
  const int tid = C::id(), nt = C::n(), np = A.sp.np, lane = threadIdx.x & 31;
  if (L.Ew) {  // assembled rows of the colour (re is zero there: one writer per row)
    const int nr = *L.wn, N = L.N, n = N * N;
    for (int t = tid; t < nr; t += nt) {
      const int r = L.wrow[t], c = r / n, rr = r - c * n;
      if (!row_in_color(c, rr % N, rr / N, A.box, color)) continue;
      int row;
      const T v = window_row(L, w, t, &row);
      re[row] += A.coefE * v;
    }
    C::sync();
    return;
  }
  for (int t = tid; t < 4 * np; t += nt)
    force_spread_quad<T, false>(L.pat, A.sp, w, L.N, A.coefE, t >> 2, t & 3, 0xFu << (lane & ~3), lane & ~3, A.box,
                                color, re);
  C::sync();
}

template <typename T, typename TM>
__device__ void ctail_boxes(const TailLevel<T, TM>& L, const TailArgs<T, TM>& A, const T* b, T* re, T* w, int color,
                            T* sr, int* sg) {
  using C = TailCtx<true>;
  const int N = L.N, n = N * N, bs = A.box, nB = A.nB;
  const int nb = N / bs, half = nb >> 1, nbox = half * half;
  const int cs = (int)C::size(), rk = (int)C::rank();
  const int mine = nbox > rk ? (nbox - rk + cs - 1) / cs : 0;  // boxes rk + cs k, k < mine
  const int items = mine * nB;
  for (int e = threadIdx.x; e < items; e += blockDim.x) {
    const int k = e / nB, q = e - k * nB, t = rk + cs * k;
    const int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
    int cc, i, j;
    box_unknown(q, bs, I * bs, J * bs, N, &cc, &i, &j);
    const int gq = cc * n + j * N + i;
    T r = b[gq] - stokes_row(w, N, L.c, cc, i, j);
    if (re && cc < 2) {
      r += re[gq];
      re[gq] = (T)0;
    }
    sr[e] = r;
    sg[e] = gq;
  }
  if (bs == 1) {
    C::sync();
  } else {
    __syncthreads();
  }
  int G = 32;
  while (G > 1 && items * G > (int)blockDim.x) G >>= 1;
  const int total = items * G;
  for (int base = 0; base < total; base += blockDim.x) {  // same trip count in every thread of the CTA
    const int e = base + threadIdx.x, it = e / G, gl = e - it * G;
    T d = 0;
    if (it < items) {
      const int k = it / nB, q = it - k * nB, t = rk + cs * k;
      const int I = 2 * (t % half) + (color & 1), J = 2 * (t / half) + (color >> 1);
      const int sl = L.slot[J * nb + I];
      const T* rs = sr + k * nB;
      if (sl >= 0) {
        const double* M = L.Ms + (size_t)sl * nB * nB + q;
        double dd = 0.0;
        for (int s = gl; s < nB; s += G) dd += M[(size_t)s * nB] * (double)rs[s];
        d = (T)dd;
      } else {
        const TM* M = L.Mf + q;
        TM dm = 0;
        for (int s = gl; s < nB; s += G) dm += M[(size_t)s * nB] * (TM)rs[s];
        d = (T)dm;
      }
    }
    for (int o = G >> 1; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (it < items && gl == 0) w[sg[it]] += d;
  }
  C::sync();
}

template <typename T, typename TM>
__device__ void ctail_sweep(const TailLevel<T, TM>& L, const TailArgs<T, TM>& A, T* w, const T* b, T* re, bool rev,
                            T* sr, int* sg) {
  for (int cc = 0; cc < 4; ++cc) {
    const int color = rev ? seq_color(3 - cc) : seq_color(cc);
    if (A.has_E) ctail_spread(L, A, w, color, re);
    ctail_boxes(L, A, b, A.has_E ? re : nullptr, w, color, sr, sg);
  }
}

// r = b - A_l w, all rows; rE is read once per row and cleared.
template <typename T, typename TM>
__device__ void ctail_residual(const TailLevel<T, TM>& L, const TailArgs<T, TM>& A, const T* w, const T* b, T* re,
                               T* r) {
  using C = TailCtx<true>;
  const int tid = C::id(), nt = C::n();
  const bool hasE = A.has_E;
  if (hasE) ctail_spread(L, A, w, -1, re);
  const int N = L.N, n = N * N;
  for (int e = tid; e < n; e += nt) {
    const int i = e & (N - 1), j = e / N;
    T eu = 0, ev = 0;
    if (hasE) {
      eu = re[e];
      ev = re[n + e];
      re[e] = (T)0;
      re[n + e] = (T)0;
    }
    r[e] = eu + b[e] - stokes_row(w, N, L.c, 0, i, j);
    r[n + e] = ev + b[n + e] - stokes_row(w, N, L.c, 1, i, j);
    r[2 * n + e] = b[2 * n + e] - stokes_row(w, N, L.c, 2, i, j);
  }
  C::sync();
}

template <typename T, typename TM, bool CL>
__global__ void __launch_bounds__(TAIL_THREADS) kv_tail(TailArgs<T, TM> A) {
  pdl_enter();
  using C = TailCtx<CL>;
  const int tid = C::id(), nt = C::n();
  extern __shared__ __align__(16) unsigned char smem[];
  T* W[MAX_LEVELS];
  T* B[MAX_LEVELS];
  const int nl = A.nlev;
  T *r, *sr;
  int* sg;
  T* re = nullptr;
  if (CL) {
    for (int l = 0; l < nl; ++l) {
      W[l] = A.gw[l];
      B[l] = A.gb[l];  // B[0] is the input b_in itself, W[0] the output w_out
    }
    r = A.gr;
    re = A.gre;
    sr = (T*)(smem + A.off_sr);  // this CTA's boxes
    sg = (int*)(smem + A.off_sg);
  } else {
    for (int l = 0; l < nl; ++l) {
      W[l] = (T*)(smem + A.off_w[l]);
      B[l] = (T*)(smem + A.off_b[l]);
    }
    r = (T*)(smem + A.off_r);
    sr = (T*)(smem + A.off_sr);
    sg = (int*)(smem + A.off_sg);
    const int n0 = 3 * A.lev[0].N * A.lev[0].N;
    for (int e = tid; e < n0; e += nt) B[0][e] = A.b_in[e];
  }
  C::sync();
  for (int l = 0; l < nl - 1; ++l) {
    const TailLevel<T, TM>& L = A.lev[l];
    const int n3 = 3 * L.N * L.N;
    for (int e = tid; e < n3; e += nt) W[l][e] = (T)0;
    C::sync();
    if constexpr (CL) {
      for (int s = 0; s < A.nu1; ++s) ctail_sweep<T, TM>(L, A, W[l], B[l], re, false, sr, sg);
      ctail_residual<T, TM>(L, A, W[l], B[l], re, r);
    } else {
      for (int s = 0; s < A.nu1; ++s) tail_sweep<T, TM, CL>(L, A, W[l], B[l], r, false, sr, sg);
      tail_residual<T, TM, CL>(L, A, W[l], B[l], r);
    }
    const int Nc = L.N / 2, ncell = Nc * Nc;
    for (int e = tid; e < ncell; e += nt) {
      T ru, rv, rp;
      restrict_cell(r, L.N, e % Nc, e / Nc, &ru, &rv, &rp, L.c.walls);
      B[l + 1][e] = ru;
      B[l + 1][ncell + e] = rv;
      B[l + 1][2 * ncell + e] = rp;
    }
    C::sync();
  }
  {
    // exact bordered solve on the coarsest grid: w = (M^{-1})[0:nc, 0:nc] b
    const T* bc = B[nl - 1];
    T* wc = W[nl - 1];
    for (int q = tid; q < A.nc; q += nt) {
      double acc = 0.0;
      for (int s = 0; s < A.nc; ++s) acc += A.Mc[(size_t)s * A.ldc + q] * (double)bc[s];
      wc[q] = (T)acc;
    }
    C::sync();
  }
  for (int l = nl - 2; l >= 0; --l) {
    const TailLevel<T, TM>& L = A.lev[l];
    const int N = L.N, n = N * N;
    for (int e = tid; e < n; e += nt) {
      T cu, cv, cp;
      prolong_cell(W[l + 1], N, e & (N - 1), e / N, &cu, &cv, &cp, L.c.walls);
      W[l][e] += cu;
      W[l][n + e] += cv;
      W[l][2 * n + e] += cp;
    }
    C::sync();
    for (int s = 0; s < A.nu2; ++s) {
      if constexpr (CL) {
        ctail_sweep<T, TM>(L, A, W[l], B[l], re, A.post_rev != 0, sr, sg);
      } else {
        tail_sweep<T, TM, CL>(L, A, W[l], B[l], r, A.post_rev != 0, sr, sg);
      }
    }
  }
  if (!CL) {
    const int n0 = 3 * A.lev[0].N * A.lev[0].N;
    for (int e = tid; e < n0; e += nt) A.w_out[e] = W[0][e];
  }
}

// ------------------------------------------------------------------ host side

template <typename T, typename TM>
int build_tail_args(Problem& P, int lt, TailArgs<T, TM>* A, size_t* smem_bytes, int cluster = 0) {
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
  A->has_E = op_elastic(P);
  for (int q = 0; q < A->nlev; ++q) {
    int l = lt + q;
    LevelInfo& L = P.lev[l];
    TailLevel<T, TM>& t = A->lev[q];
    t.N = L.N;
    t.c = coefs<T>(P, l);
    t.pat = pats<T>(L);
    t.slot = L.flag;
    t.Ms = L.Mstruct;
    t.Mf = Mfree_of<TM>(L);
    t.wrow = P.win_step ? L.slot_row : nullptr;
    t.wn = P.win_step ? P.count + 1 + l : nullptr;
    t.Ew = P.win_step ? Ewin_of<T>(L) : nullptr;
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
  A->off_sr = (int)take((size_t)max_boxes * P.nB * sizeof(T));
  A->off_sg = (int)take((size_t)max_boxes * P.nB * sizeof(int));
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
  if (cluster > 0) {
    for (int q = 0; q < A->nlev; ++q) {
      A->gw[q] = lbuf<T>(P.lev[lt + q]).w;
      A->gb[q] = lbuf<T>(P.lev[lt + q]).b;
    }
    A->gr = lbuf<T>(P.lev[lt]).r;
    A->gre = rEbuf<T>(P.lev[lt]);
    // shared memory: the staged residuals of one CTA's boxes on the finest tail level
    const size_t half = (size_t)P.lev[lt].N / P.prm.box / 2;
    const size_t items = (half * half + cluster - 1) / cluster * (size_t)P.nB;
    off = 0;
    A->off_sr = (int)take(items * sizeof(T));
    A->off_sg = (int)take(items * sizeof(int));
    *smem_bytes = off;
  }
  return IB_OK;
}

// rE += -dt E_l w on the rows of colour `color` (-1: all rows) of a fine level.
template <typename T>
int fine_elastic(Problem& P, int l, const T* w, int color) {
  LevelInfo& L = P.lev[l];
  if (P.win_step)  // assembled rows: one gather per structure row of the colour
    return launch_window_apply<T>(P, l, w, rEbuf<T>(L), -P.prm.dt / (P.lev[0].h * P.lev[0].h), color, use_pdl(P));
  const double sT = sizeof(T);
  double deg = P.np ? 2.0 * P.ns / P.np : 0.0;
  // algorithmic bytes per point (the re-interpolation of neighbours is redundant
  // work, not data): its interpolation patch for both components (16 values, 8
  // weights, 2 bases each), half of its springs' K and adjacency, its spread
  // patch (8 weights, 2 bases per component) and the read-modify-write of the
  // spread entries (32 for all rows, about 8 on the rows of one colour)
  const double upd = (color < 0 ? 32.0 : 8.0) * 2 * sT;
  KScope ks(P, IB_KC_SPREAD,
            P.np * (2.0 * (24 * sT + 8) + 0.5 * deg * (3 * sT + 8) + 8 + 2.0 * (8 * sT + 8) + upd));
  // FP64: small CTAs so that the interpolation FMAs spread over many SMs (the FP64
  // pipe is narrow); FP32: the usual block size (a multiple of 4 either way)
  const int tpb = sizeof(T) == 8 ? 64 : TPB;
  vlaunch(use_pdl(P), kv_force_spread<T>, nblk(4L * P.np, tpb), tpb, 0, P.stream, pats<T>(L), sview<T>(P), w,
          L.N, (T)(-P.prm.dt / (P.lev[0].h * P.lev[0].h)), P.prm.box, color, rEbuf<T>(L));
  IB_LAUNCH_CHECK();
  return IB_OK;
}

template <typename T, typename TM>
int fine_sweep(Problem& P, int l, bool rev, bool w_is_zero) {
  LevelInfo& L = P.lev[l];
  LevelBuf<T>& B = lbuf<T>(L);
  const int N = L.N, bs = P.prm.box;
  const bool has_E = op_elastic(P);
  const StokesCoef<T> c = coefs<T>(P, l);
  const int half = L.nb / 2;
  const long nbox = (long)half * half;
  const int nB = P.nB;
  const double sT = sizeof(T);
  for (int cc = 0; cc < 4; ++cc) {
    const int color = rev ? kSeq[3 - cc] : kSeq[cc];
    const bool with_E = has_E && !(w_is_zero && cc == 0);  // w = 0: no elasticity term
    if (with_E) IB_TRY(fine_elastic<T>(P, l, B.w, color));
    T* E = with_E ? rEbuf<T>(L) : nullptr;
    // rE read and cleared on the velocity rows of the colour's structure boxes
    const double e_bytes = with_E ? 0.25 * L.n_struct * 2.0 * bs * (bs + 1) * 2 * sT : 0.0;
    if (bs == 1) {
      {
        KScope ks(P, IB_KC_STOKES, nbox * 5.0 * (6 * sT + 2 * sT) + e_bytes);
        vlaunch(use_pdl(P), kv_colres1<T>, nblk(nbox), TPB, 0, P.stream, B.w, B.b, E, B.r, N, c, color, L.flag);
        IB_LAUNCH_CHECK();
      }
      KScope ks(P, IB_KC_BOX, nbox * (15.0 * sT + 4) + 0.25 * L.n_struct * 25 * sT + 25 * sT);
      vlaunch(use_pdl(P), kv_box1<T, TM>, nblk(nbox), TPB, 0, P.stream, B.r, B.w, N, color, L.flag, L.Mstruct,
              Mfree_of<TM>(L));
      IB_LAUNCH_CHECK();
    } else {
      // per box: its unknowns' rows read w (5-point stencils, counted once per
      // unknown plus the one-cell halo), b, write w
      const double box_bytes = sT * (3.0 * nB + (4.0 * bs + 4)) + 4;
      KScope ks(P, IB_KC_BOX, nbox * box_bytes + 0.25 * L.n_struct * nB * nB * sT + (double)nB * nB * sT + e_bytes);
      IB_TRY((launch_boxn<T, TM>(P, l, B.w, B.b, E, color)));
    }
  }
  return IB_OK;
}

template <typename T>
constexpr int pix() { return sizeof(T) == 8 ? 1 : 0; }

template <typename T, typename TM>
int vcycle_eager_t(Problem& P) {
  const int lt = P.tail_level[pix<T>()];
  const bool has_E = op_elastic(P);
  for (int l = 0; l < lt; ++l) {
    LevelInfo& L = P.lev[l];
    LevelBuf<T>& B = lbuf<T>(L);
    const long n3 = 3L * L.N * L.N;
    if (l == 0) {  // coarser levels are zeroed by the restriction that fills their b
      KScope ks(P, IB_KC_OTHER, n3 * sizeof(T));
      vlaunch(use_pdl(P), kv_zero<T>, nblk(n3), TPB, 0, P.stream, B.w, n3);
      IB_LAUNCH_CHECK();
    }
    for (int s = 0; s < P.prm.nu1; ++s) IB_TRY((fine_sweep<T, TM>(P, l, false, s == 0)));
    if (has_E) IB_TRY(fine_elastic<T>(P, l, B.w, -1));
    const T* E = has_E ? rEbuf<T>(L) : nullptr;
    const int Nc = P.lev[l + 1].N;
    {
      // w read once per stencil (9 fine values per coarse cell incl. the halo), b, rE
      const double e_bytes = has_E ? 2.0 * L.N * L.N * sizeof(T) : 0.0;
      KScope ks(P, IB_KC_TRANSFER, (9.0 * L.N * L.N + 6.0 * Nc * Nc) * sizeof(T) + e_bytes);
      vlaunch(use_pdl(P), kv_resres<T>, nblk((long)Nc * Nc), TPB, 0, P.stream, B.w, B.b, E,
              lbuf<T>(P.lev[l + 1]).b, lbuf<T>(P.lev[l + 1]).w, Nc, coefs<T>(P, l));
      IB_LAUNCH_CHECK();
    }
  }
  {
    const int csize = P.tail_cluster[pix<T>()];
    TailArgs<T, TM> A;
    size_t smem = 0;
    IB_TRY((build_tail_args<T, TM>(P, lt, &A, &smem, csize)));
    KScope ks(P, IB_KC_COARSE, 0.0);
    if (csize > 0) {
      if (smem > 48u * 1024u) return fail(IB_ERR_INVALID_ARG, "cluster tail staging above 48 KB");
      IB_CUDA_TRY(claunch(use_pdl(P), csize, kv_tail<T, TM, true>, TAIL_THREADS, smem, P.stream, A));
    } else {
      vlaunch(use_pdl(P), kv_tail<T, TM, false>, 1, TAIL_THREADS, smem, P.stream, A);
      IB_LAUNCH_CHECK();
    }
  }
  for (int l = lt - 1; l >= 0; --l) {
    LevelInfo& L = P.lev[l];
    LevelBuf<T>& B = lbuf<T>(L);
    {
      const double e_bytes = has_E ? 2.0 * L.N * L.N * sizeof(T) : 0.0;
      KScope ks(P, IB_KC_TRANSFER, (6.0 * L.N * L.N + 0.75 * L.N * L.N) * sizeof(T) + e_bytes);
      vlaunch(use_pdl(P), kv_prolong<T>, nblk((long)L.N * L.N), TPB, 0, P.stream,
              (const T*)lbuf<T>(P.lev[l + 1]).w, B.w, L.N, has_E ? rEbuf<T>(L) : (T*)nullptr, (int)P.prm.walls);
      IB_LAUNCH_CHECK();
    }
    for (int s = 0; s < P.prm.nu2; ++s) IB_TRY((fine_sweep<T, TM>(P, l, P.prm.box == 1, false)));
  }
  return IB_OK;
}

// The FP64 V-cycle applies the FP32 free-box inverse unless the problem asked for
// FP64 throughout (the mixed-precision V-cycle: FP64 vectors, residuals,
// transfers, elasticity and structure-box solves; FP32 free-box solves).
template <typename T>
int vcycle_eager(Problem& P) {
  if constexpr (sizeof(T) == 8) {
    if (P.prm.precision != IB_FP64) return vcycle_eager_t<double, float>(P);
    return vcycle_eager_t<double, double>(P);
  } else {
    return vcycle_eager_t<float, float>(P);
  }
}

// Shared-memory bytes of the tail kernel starting at level lt, and raising the
// kernel's dynamic shared-memory limit to smem_max.
template <typename T, typename TM>
int tail_smem_t(Problem& P, int lt, size_t* bytes) {
  TailArgs<T, TM> A;
  return build_tail_args<T, TM>(P, lt, &A, bytes);
}

template <typename T, typename TM>
int tail_raise_smem_t(size_t smem_max) {
  // the limit is a per-function setting shared by every problem in the process:
  // only ever raise it (problems of a batch are prepared on several threads)
  static std::mutex mu;
  static size_t granted = 0;
  std::lock_guard<std::mutex> lock(mu);
  if (smem_max > granted) {
    IB_CUDA_TRY(
        cudaFuncSetAttribute(kv_tail<T, TM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
    granted = smem_max;
  }
  return IB_OK;
}

template <typename T>
int tail_smem(Problem& P, int lt, size_t* bytes) {
  if constexpr (sizeof(T) == 8) {
    if (P.prm.precision != IB_FP64) return tail_smem_t<double, float>(P, lt, bytes);
    return tail_smem_t<double, double>(P, lt, bytes);
  } else {
    return tail_smem_t<float, float>(P, lt, bytes);
  }
}

// CTAs per cluster of the cluster tail (16 where the device can co-schedule a
// non-portable cluster of 16 CTAs of 1024 threads, else 8, else 0 = no cluster
// form), found once per process.
template <typename T, typename TM>
int tail_cluster_size_t() {
  static std::mutex mu;
  static int cs = -1;
  std::lock_guard<std::mutex> lock(mu);
  if (cs >= 0) return cs;
  cs = 0;
  cudaFuncSetAttribute(kv_tail<T, TM, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int c : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(TAIL_THREADS);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kv_tail<T, TM, true>, &cfg) == cudaSuccess && n > 0) {
      cs = c;
      break;
    }
    cudaGetLastError();
  }
  return cs;
}

template <typename T>
int tail_cluster_size(const Problem& P) {
  if constexpr (sizeof(T) == 8) {
    if (P.prm.precision != IB_FP64) return tail_cluster_size_t<double, float>();
    return tail_cluster_size_t<double, double>();
  } else {
    return tail_cluster_size_t<float, float>();
  }
}

template <typename T>
int tail_raise_smem(Problem& P, size_t smem_max) {
  if constexpr (sizeof(T) == 8) {
    if (P.prm.precision != IB_FP64) return tail_raise_smem_t<double, float>(smem_max);
    return tail_raise_smem_t<double, double>(smem_max);
  } else {
    return tail_raise_smem_t<float, float>(smem_max);
  }
}

}  // namespace

template <typename T>
int vcycle_run(Problem& P);

// Box-kernel autotuner: on every smoothing level with n x n boxes (n = 2, 4), time one
// colour phase of each applicable form (one box per CTA, a thread per box row, the
// register-blocked product, the strip kernel at widths 8, 16, 32, eight FP32 boxes
// per 64-thread CTA) on the problem's
// own hierarchy with w = b = 0 (the same products and memory traffic, no change of
// state) and keep the fastest.  Skipped when an IB_BOX_* variable pins the forms.
template <typename T, typename TM>
int tune_box_forms_t(Problem& P) {
  constexpr int ix = pix<T>();
  for (int l = 0; l < 32; ++l) P.box_form[ix][l] = BOXF_RULE;
  if (P.box_form_pinned) {  // forms given by hand (profiler runs distort the timings)
    for (int l = 0; l < 32; ++l) P.box_form[ix][l] = P.box_form_pin[l];
    P.graph_dirty[ix] = true;
    return IB_OK;
  }
  if (!P.box_autotune || (P.prm.box != 2 && P.prm.box != 4) || P.prof) return IB_OK;
  cudaEvent_t e0, e1;
  IB_CUDA_TRY(cudaEventCreate(&e0));
  IB_CUDA_TRY(cudaEventCreate(&e1));
  long long saved[IB_KC_COUNT];
  std::memcpy(saved, P.nlaunch, sizeof(saved));
  int rc = IB_OK;
  for (int l = 0; l < P.nlev - 1 && l < 32 && rc == IB_OK; ++l) {
    LevelInfo& L = P.lev[l];
    LevelBuf<T>& B = lbuf<T>(L);
    const size_t n3 = 3ul * L.N * L.N;
    if (cudaMemsetAsync(B.w, 0, n3 * sizeof(T), P.stream) != cudaSuccess ||
        cudaMemsetAsync(B.b, 0, n3 * sizeof(T), P.stream) != cudaSuccess) {
      rc = fail(IB_ERR_CUDA, "box autotuner: memset");
      break;
    }
    float best = 1e30f;
    int best_f = BOXF_RULE;
    for (int f = BOXF_ONE; f <= BOXF_OCT; ++f) {
      if (!launch_box_form<T, TM>(P, l, f, B.w, B.b, (T*)nullptr, 0)) continue;  // warm-up (and applicability)
      cudaEventRecord(e0, P.stream);
      for (int r = 0; r < 4; ++r) launch_box_form<T, TM>(P, l, f, B.w, B.b, (T*)nullptr, r);
      cudaEventRecord(e1, P.stream);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        rc = fail(IB_ERR_CUDA, "box autotuner: timing launch failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_f = f;
      }
    }
    P.box_form[ix][l] = best_f;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::memcpy(P.nlaunch, saved, sizeof(saved));
  P.graph_dirty[ix] = true;
  return rc;
}

template <typename T>
int tune_box_forms(Problem& P) {
  if constexpr (sizeof(T) == 8) {
    if (P.prm.precision != IB_FP64) return tune_box_forms_t<double, float>(P);
    return tune_box_forms_t<double, double>(P);
  } else {
    return tune_box_forms_t<float, float>(P);
  }
}

// Candidate forms of the tail: the single-CTA kernel from levels with N_l <= 64
// (FP32) or <= 32 (FP64) whose arrays fit in shared memory, plus "coarsest grid
// only"; and the cluster kernel from levels with 16 <= N_l <= 128.
// vcycle_prepare times one graph-replayed V-cycle per candidate on the problem's
// own hierarchy and keeps the fastest (the autotuner of the level split between
// grid-wide kernels and the tail kernel).
template <typename T>
int vcycle_prepare(Problem& P) {
  IB_TRY(tune_box_forms<T>(P));
  const int nmax = sizeof(T) == 4 ? 64 : 32;
  struct Cand {
    int l, cs;
  };
  std::vector<Cand> cand;
  size_t smem_max = 0;
  for (int l = 0; l < P.nlev; ++l) {
    if (P.lev[l].N > nmax) continue;
    size_t s = 0;
    IB_TRY(tail_smem<T>(P, l, &s));
    if (s <= 227u * 1024u) {
      cand.push_back({l, 0});
      if (s > smem_max) smem_max = s;
    }
  }
  if (cand.empty() || cand.back().l != P.nlev - 1) {
    size_t s = 0;
    IB_TRY(tail_smem<T>(P, P.nlev - 1, &s));
    cand.push_back({P.nlev - 1, 0});
    if (s > smem_max) smem_max = s;
  }
  IB_TRY(tail_raise_smem<T>(P, smem_max));
  const int cs = P.use_graph ? tail_cluster_size<T>(P) : 0;
  if (cs > 0)
    for (int l = 0; l < P.nlev - 1; ++l)
      if (P.lev[l].N <= 128 && P.lev[l].N >= 16) cand.push_back({l, cs});
  constexpr int ix = pix<T>();
  // IB_TAIL_NMAX pins the split instead of timing it (profiler runs distort the
  // timings): the tail starts at the first candidate level with N_l <= value, in
  // the single-CTA form where that level has one unless IB_TAIL_CLUSTER=1 (and
  // IB_TAIL_CLUSTER=0 excludes the cluster form)
  const char* ecl = std::getenv("IB_TAIL_CLUSTER");
  const int want_cl = ecl ? (ecl[0] == '1' ? 1 : 0) : -1;
  if (want_cl == 0) {
    std::vector<Cand> keep;
    for (const Cand& c : cand)
      if (c.cs == 0) keep.push_back(c);
    cand.swap(keep);
  }
  if (const char* e = std::getenv("IB_TAIL_NMAX")) {
    const int nt = std::atoi(e);
    Cand pick = {-1, 0};
    for (int pass = 0; pass < 2 && pick.l < 0; ++pass)
      for (const Cand& c : cand) {
        if (P.lev[c.l].N > nt) continue;
        if (pass == 0 && want_cl == 1 && c.cs == 0) continue;
        if (pass == 0 && want_cl != 1 && c.cs != 0) continue;
        if (pick.l < 0 || c.l < pick.l) pick = c;
      }
    if (pick.l < 0) pick = {P.nlev - 1, 0};
    P.tail_level[ix] = pick.l;
    P.tail_cluster[ix] = pick.cs;
    P.graph_dirty[ix] = true;
    return IB_OK;
  }
  if (cand.size() == 1 || P.prof || !P.use_graph) {
    P.tail_level[ix] = cand.front().l;
    P.tail_cluster[ix] = 0;
    P.graph_dirty[ix] = true;
    return IB_OK;
  }
  cudaEvent_t e0, e1;
  IB_CUDA_TRY(cudaEventCreate(&e0));
  IB_CUDA_TRY(cudaEventCreate(&e1));
  long long saved[IB_KC_COUNT];
  std::memcpy(saved, P.nlaunch, sizeof(saved));
  float best = 1e30f;
  Cand best_c = cand.front();
  size_t n0 = 3ul * P.lev[0].N * P.lev[0].N;
  IB_CUDA_TRY(cudaMemsetAsync(lbuf<T>(P.lev[0]).b, 0, n0 * sizeof(T), P.stream));
  for (const Cand& c : cand) {
    P.tail_level[ix] = c.l;
    P.tail_cluster[ix] = c.cs;
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
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::memcpy(P.nlaunch, saved, sizeof(saved));
  P.tail_level[ix] = best_c.l;
  P.tail_cluster[ix] = best_c.cs;
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
  // the caller's stream may be the legacy default stream, which cannot be
  // captured: capture on a private stream (capture runs nothing), replay on the
  // caller's stream
  if (!P.gstream) IB_CUDA_TRY(cudaStreamCreateWithFlags(&P.gstream, cudaStreamNonBlocking));
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
  cudaEvent_t ta = nullptr, tb = nullptr;
  if (P.vt_on) {
    for (cudaEvent_t* e : {&ta, &tb}) {
      if (!P.ev_pool.empty()) {
        *e = P.ev_pool.back();
        P.ev_pool.pop_back();
      } else {
        IB_CUDA_TRY(cudaEventCreate(e));
      }
    }
    IB_CUDA_TRY(cudaEventRecord(ta, P.stream));
  }
  IB_CUDA_TRY(cudaGraphLaunch(P.vgraph[ix], P.stream));
  if (P.vt_on) {
    IB_CUDA_TRY(cudaEventRecord(tb, P.stream));
    P.vt_pending.emplace_back(ta, tb);
    P.vt_kind.push_back(ix);
  }
  for (int c = 0; c < IB_KC_COUNT; ++c) P.nlaunch[c] += P.graph_launches[ix][c];
  return IB_OK;
}
template int vcycle_run<double>(Problem&);
template int vcycle_run<float>(Problem&);

// rE must be zero when a V-cycle starts (every use clears what it consumed).
int vcycle_reset_rE(Problem& P) {
  for (int l = 0; l < P.nlev; ++l) {
    LevelInfo& L = P.lev[l];
    const size_t n2 = 2ul * L.N * L.N;
    if (L.rE64) IB_CUDA_TRY(cudaMemsetAsync(L.rE64, 0, n2 * sizeof(double), P.stream));
    if (L.rE32) IB_CUDA_TRY(cudaMemsetAsync(L.rE32, 0, n2 * sizeof(float), P.stream));
  }
  return IB_OK;
}

// Zero the elasticity residual buffers (their patch rows move with the points).

}  // namespace ib
