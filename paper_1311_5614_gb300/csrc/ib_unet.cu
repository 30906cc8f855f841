// The learned preconditioner stage: a small convolutional U-Net that maps the
// residual left by one V-cycle to an estimate of the remaining error.  It is
// not part of the paper's method; it is added as an extra stage inside flexible
// GMRES (which admits any preconditioner), with the plain V-cycle kept when the
// stage does not lower the residual.
//
// Network (periodic / circular padding, activations [C][N][N] FP32, weights
// BF16 with FP32 master copies, FP32 accumulation):
//   level 1 (N):   conv3x3 4->16, GELU, conv3x3 16->16, GELU          -> s1
//   level 2 (N/2): avgpool(s1), conv 16->32, GELU, conv 32->32, GELU  -> s2
//   level 3 (N/4): avgpool(s2), conv 32->64, GELU, conv 64->64, GELU
//   up to N/2:     nearest-upsample, concat [up | s2] (96), conv 96->32, GELU, conv 32->32, GELU
//   up to N:       nearest-upsample, concat [up | s1] (48), conv 48->16, GELU, conv 16->16, GELU
//   head:          conv1x1 16->3
// Direct convolution on CUDA cores: a CTA computes a 16 x 16 pixel tile for 16
// output channels, staging an 18 x 18 input halo and the weights in shared memory.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "ib_internal.cuh"

namespace ib {

// ---------------------------------------------------------------- network description

struct UConv {
  int ci, co, k, H;   // channels in/out, kernel size, grid size
  long w_off, b_off;  // offsets into the parameter vector
  int act;            // GELU after the conv
};

// The fixed architecture: parameter layout [W0 b0 W1 b1 ...], W in [co][ci][k][k].
static std::vector<UConv> unet_layers(int N) {
  std::vector<UConv> L;
  auto add = [&](int ci, int co, int k, int H, int act) { L.push_back(UConv{ci, co, k, H, 0, 0, act}); };
  add(4, 16, 3, N, 1);
  add(16, 16, 3, N, 1);
  add(16, 32, 3, N / 2, 1);
  add(32, 32, 3, N / 2, 1);
  add(32, 64, 3, N / 4, 1);
  add(64, 64, 3, N / 4, 1);
  add(96, 32, 3, N / 2, 1);
  add(32, 32, 3, N / 2, 1);
  add(48, 16, 3, N, 1);
  add(16, 16, 3, N, 1);
  add(16, 3, 1, N, 0);
  long off = 0;
  for (auto& c : L) {
    c.w_off = off;
    off += (long)c.co * c.ci * c.k * c.k;
    c.b_off = off;
    off += c.co;
  }
  return L;
}

static long unet_param_count() {
  auto L = unet_layers(64);
  const auto& c = L.back();
  return c.b_off + c.co;
}

}  // namespace ib

struct ib_unet {
  int N = 0;
  cudaStream_t stream = nullptr;
  std::vector<ib::UConv> L;
  long np = 0;
  float* w = nullptr;            // FP32 master
  __nv_bfloat16* wb = nullptr;   // BF16 used by the kernels
  float* g = nullptr;            // gradient
  float* m = nullptr;            // Adam moments
  float* v = nullptr;
  long step = 0;
  // activations: a[k] = output of layer k (post-activation), pre[k] = pre-activation
  std::vector<float*> a, pre, ga;
  float* x_in = nullptr;      // [4][N][N]
  float* p1 = nullptr;        // pool(a1) [16][N/2]^2
  float* p2 = nullptr;        // pool(a3) [32][N/4]^2
  float* c2 = nullptr;        // concat [64 up | 32 s2] at N/2 = 96 channels
  float* c1 = nullptr;        // concat [32 up | 16 s1] at N = 48 channels
  float* gp1 = nullptr, * gp2 = nullptr, * gc2 = nullptr, * gc1 = nullptr, * gx = nullptr;
  double* red = nullptr;      // reductions
  double* red_host = nullptr;
  std::vector<void*> allocs;
  bool tc = true;  // convolutions on the tensor cores (IB_UNET_TC=0: CUDA cores)
};

namespace ib {
namespace {

constexpr int TILE = 16;  // pixel tile side
constexpr int COT = 16;   // output channels per CTA
constexpr int CIT = 8;    // input channels staged per pass

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * __expf(-0.5f * x * x);
  return cdf + x * pdf;
}

// out[co][p] (+)= bias[co] + sum_ci sum_tap W(co, ci, tap) in[ci][p + off(tap)], K = 1 or 3.
// mode 0: forward weights W[co][ci][tap];  mode 1: data gradient, the transposed
// and flipped kernel W[ci][co][8 - tap] (in = dOut, out = dIn, "co" = forward ci).
// pre (optional) receives the pre-activation, act applies GELU to the output.
template <int K>
__global__ void __launch_bounds__(TILE * TILE) k_conv(const float* __restrict__ in, int Ci, const __nv_bfloat16* __restrict__ Wt,
                                                      const float* __restrict__ bias, float* __restrict__ out, int Co,
                                                      int out_cstride_off, float* __restrict__ pre, int H, int act,
                                                      int mode, int Wco, int Wci, int accumulate) {
  __shared__ float s_in[CIT][TILE + 2][TILE + 2];
  __shared__ float s_w[COT][CIT][K * K];
  const int tx = threadIdx.x & (TILE - 1), ty = threadIdx.x / TILE;
  const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE, co0 = blockIdx.z * COT;
  const int HW = H * H, m = H - 1;
  float acc[COT];
#pragma unroll
  for (int c = 0; c < COT; ++c) acc[c] = 0.f;
  const int R = K / 2;
  for (int ci0 = 0; ci0 < Ci; ci0 += CIT) {
    // input tile with a halo of R (circular)
    for (int e = threadIdx.x; e < CIT * (TILE + 2) * (TILE + 2); e += TILE * TILE) {
      const int c = e / ((TILE + 2) * (TILE + 2)), r = e % ((TILE + 2) * (TILE + 2));
      const int yy = r / (TILE + 2), xx = r % (TILE + 2);
      const int gy = (y0 + yy - 1) & m, gx = (x0 + xx - 1) & m;
      s_in[c][yy][xx] = (ci0 + c < Ci) ? in[(size_t)(ci0 + c) * HW + gy * H + gx] : 0.f;
    }
    for (int e = threadIdx.x; e < COT * CIT * K * K; e += TILE * TILE) {
      const int co = e / (CIT * K * K), r = e % (CIT * K * K);
      const int ci = r / (K * K), tap = r % (K * K);
      const int gco = co0 + co, gci = ci0 + ci;
      float v = 0.f;
      if (gco < Co && gci < Ci) {
        if (mode == 0) v = __bfloat162float(Wt[((size_t)gco * Wci + gci) * K * K + tap]);
        else v = __bfloat162float(Wt[((size_t)gci * Wci + gco) * K * K + (K * K - 1 - tap)]);
      }
      s_w[co][ci][tap] = v;
    }
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < CIT; ++c) {
#pragma unroll
      for (int tap = 0; tap < K * K; ++tap) {
        const int dy = tap / K, dx = tap % K;
        const float v = s_in[c][ty + 1 + dy - R][tx + 1 + dx - R];
#pragma unroll
        for (int co = 0; co < COT; ++co) acc[co] += s_w[co][c][tap] * v;
      }
    }
    __syncthreads();
  }
  const int p = (y0 + ty) * H + x0 + tx;
#pragma unroll
  for (int co = 0; co < COT; ++co) {
    const int gco = co0 + co;
    if (gco >= Co) break;
    float v = acc[co] + (bias ? bias[gco] : 0.f);
    const size_t o = (size_t)(gco + out_cstride_off) * HW + p;
    if (pre) pre[(size_t)gco * HW + p] = v;
    if (act) v = gelu_f(v);
    if (accumulate) out[o] += v;
    else out[o] = v;
  }
  (void)Wco;
}

// ---------------------------------------------------------------- tensor-core convolution
//
// The same convolution as an implicit GEMM on the tensor cores (mma.sync
// m16n8k16, BF16 operands, FP32 accumulation): rows = output channels (MT tiles of
// 16), columns = pixels, and the reduction runs over blocks of 16 input channels at
// each tap.  A CTA computes a 16 x 16 pixel tile for all its output channels; warp w
// takes pixel rows 2w and 2w + 1 (four column tiles of 8 pixels).  Each block of 16
// input channels is staged with its one-pixel halo in two planes of 8 channels
// ([pixel][8], 16 bytes per pixel), so the 32 lanes of a fragment load read 32
// consecutive words; the weights likewise ([tap][plane][co][8]).  The FP32
// activations enter as two BF16 terms, hi = bf16(v) and lo = bf16(v - hi), and both
// are multiplied by the BF16 weight (two products per fragment), so the result is the
// BF16-weight convolution of the FP32 activations to about 2^-16 relative, as the
// CUDA-core kernel computes it.
__device__ __forceinline__ void mma_bf16_16816(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int K, int MT>
struct ConvTC {
  static constexpr int HALO = TILE + 2, HP = HALO * HALO;  // staged pixels (18 x 18)
  static constexpr int COP = MT * 16;                      // output channels (padded)
  // shared memory: input hi / lo [2 planes][HP][8] bf16, weights [K*K][2 planes][COP][8] bf16
  static constexpr size_t IN_BYTES = 2ul * HP * 8 * 2;
  static constexpr size_t W_BYTES = (size_t)K * K * 2 * COP * 8 * 2;
  static constexpr size_t SMEM = 2 * IN_BYTES + W_BYTES;
};

template <int K, int MT>
__global__ void __launch_bounds__(TILE * TILE) k_conv_tc(const float* __restrict__ in, int Ci,
                                                         const __nv_bfloat16* __restrict__ Wt,
                                                         const float* __restrict__ bias, float* __restrict__ out,
                                                         int Co, int out_cstride_off, float* __restrict__ pre, int H,
                                                         int act, int mode, int Wci, int accumulate) {
  using S = ConvTC<K, MT>;
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* s_hi = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* s_lo = reinterpret_cast<__nv_bfloat16*>(smem + S::IN_BYTES);
  __nv_bfloat16* s_w = reinterpret_cast<__nv_bfloat16*>(smem + 2 * S::IN_BYTES);
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5, gid = lane >> 2, tig = lane & 3;
  const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE;
  const int HW = H * H, m = H - 1, R = K / 2, KK = K * K;
  float acc[MT][4][4];
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  for (int ci0 = 0; ci0 < Ci; ci0 += 16) {
    // input block: pixel fastest across threads (coalesced), split into hi / lo
    for (int e = tid; e < 16 * S::HP; e += TILE * TILE) {
      const int c = e / S::HP, px = e - c * S::HP;
      const int yy = px / S::HALO, xx = px - yy * S::HALO;
      const int gy = (y0 + yy - 1) & m, gx = (x0 + xx - 1) & m;
      const float v = (ci0 + c < Ci) ? in[(size_t)(ci0 + c) * HW + gy * H + gx] : 0.f;
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
      const int o = ((c >> 3) * S::HP + px) * 8 + (c & 7);
      s_hi[o] = hi;
      s_lo[o] = lo;
    }
    // weights of this block (mode 1: the transposed, flipped kernel of the data gradient)
    for (int e = tid; e < KK * 16 * S::COP; e += TILE * TILE) {
      const int tap = e / (16 * S::COP), r = e - tap * 16 * S::COP;
      const int co = r >> 4, c = r & 15;
      const int gco = co, gci = ci0 + c;
      __nv_bfloat16 v = __float2bfloat16_rn(0.f);
      if (gco < Co && gci < Ci) {
        v = (mode == 0) ? Wt[((size_t)gco * Wci + gci) * KK + tap] : Wt[((size_t)gci * Wci + gco) * KK + (KK - 1 - tap)];
      }
      s_w[((tap * 2 + (c >> 3)) * S::COP + co) * 8 + (c & 7)] = v;
    }
    __syncthreads();
#pragma unroll 1
    for (int tap = 0; tap < KK; ++tap) {
      const int dy = tap / K - R + 1, dx = tap % K - R + 1;  // halo offsets of the tap
      unsigned bh[4][2], bl[4][2];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int y = 2 * wp + (nt >> 1), x = (nt & 1) * 8 + gid;
        const int px = (y + dy) * S::HALO + (x + dx);
        bh[nt][0] = *reinterpret_cast<const unsigned*>(s_hi + (size_t)px * 8 + 2 * tig);
        bh[nt][1] = *reinterpret_cast<const unsigned*>(s_hi + (size_t)(S::HP + px) * 8 + 2 * tig);
        bl[nt][0] = *reinterpret_cast<const unsigned*>(s_lo + (size_t)px * 8 + 2 * tig);
        bl[nt][1] = *reinterpret_cast<const unsigned*>(s_lo + (size_t)(S::HP + px) * 8 + 2 * tig);
      }
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const __nv_bfloat16* w0 = s_w + ((size_t)(tap * 2 + 0) * S::COP + mt * 16) * 8;
        const __nv_bfloat16* w1 = s_w + ((size_t)(tap * 2 + 1) * S::COP + mt * 16) * 8;
        unsigned a[4];
        a[0] = *reinterpret_cast<const unsigned*>(w0 + gid * 8 + 2 * tig);
        a[1] = *reinterpret_cast<const unsigned*>(w0 + (gid + 8) * 8 + 2 * tig);
        a[2] = *reinterpret_cast<const unsigned*>(w1 + gid * 8 + 2 * tig);
        a[3] = *reinterpret_cast<const unsigned*>(w1 + (gid + 8) * 8 + 2 * tig);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          mma_bf16_16816(acc[mt][nt], a, bh[nt]);
          mma_bf16_16816(acc[mt][nt], a, bl[nt]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int co = mt * 16 + gid + (q >> 1) * 8;
        if (co >= Co) continue;
        const int y = 2 * wp + (nt >> 1), x = (nt & 1) * 8 + 2 * tig + (q & 1);
        const int p = (y0 + y) * H + x0 + x;
        float v = acc[mt][nt][q] + (bias ? bias[co] : 0.f);
        const size_t o = (size_t)(co + out_cstride_off) * HW + p;
        if (pre) pre[(size_t)co * HW + p] = v;
        if (act) v = gelu_f(v);
        if (accumulate) out[o] += v;
        else out[o] = v;
      }
}

// dW[co][ci][tap] += sum_p g[co][p] in[ci][p + off(tap)] over a chunk of tiles.
template <int K>
__global__ void __launch_bounds__(TILE * TILE) k_conv_wgrad(const float* __restrict__ in, int Ci, const float* __restrict__ g,
                                                            int Co, int H, float* __restrict__ dW, int tiles_per_block) {
  __shared__ float s_in[CIT][TILE + 2][TILE + 2];
  __shared__ float s_g[COT][TILE][TILE];
  const int co0 = blockIdx.y * COT, ci0 = blockIdx.z * CIT;
  const int HW = H * H, m = H - 1, tpr = H / TILE, ntiles = tpr * tpr;
  const int R = K / 2;
  // each thread owns up to ceil(COT*CIT*K*K / 256) weight entries
  constexpr int NW = (COT * CIT * K * K + TILE * TILE - 1) / (TILE * TILE);
  float acc[NW];
#pragma unroll
  for (int q = 0; q < NW; ++q) acc[q] = 0.f;
  for (int t = blockIdx.x * tiles_per_block; t < min(ntiles, (blockIdx.x + 1) * tiles_per_block); ++t) {
    const int x0 = (t % tpr) * TILE, y0 = (t / tpr) * TILE;
    for (int e = threadIdx.x; e < CIT * (TILE + 2) * (TILE + 2); e += TILE * TILE) {
      const int c = e / ((TILE + 2) * (TILE + 2)), r = e % ((TILE + 2) * (TILE + 2));
      const int yy = r / (TILE + 2), xx = r % (TILE + 2);
      const int gy = (y0 + yy - 1) & m, gx = (x0 + xx - 1) & m;
      s_in[c][yy][xx] = (ci0 + c < Ci) ? in[(size_t)(ci0 + c) * HW + gy * H + gx] : 0.f;
    }
    for (int e = threadIdx.x; e < COT * TILE * TILE; e += TILE * TILE) {
      const int c = e / (TILE * TILE), r = e % (TILE * TILE);
      s_g[c][r / TILE][r % TILE] = (co0 + c < Co) ? g[(size_t)(co0 + c) * HW + (y0 + r / TILE) * H + x0 + r % TILE] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      const int e = threadIdx.x + q * TILE * TILE;
      if (e >= COT * CIT * K * K) break;
      const int co = e / (CIT * K * K), r = e % (CIT * K * K);
      const int ci = r / (K * K), tap = r % (K * K);
      const int dy = tap / K, dx = tap % K;
      float s = 0.f;
      for (int yy = 0; yy < TILE; ++yy)
#pragma unroll 4
        for (int xx = 0; xx < TILE; ++xx) s += s_g[co][yy][xx] * s_in[ci][yy + 1 + dy - R][xx + 1 + dx - R];
      acc[q] += s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NW; ++q) {
    const int e = threadIdx.x + q * TILE * TILE;
    if (e >= COT * CIT * K * K) break;
    const int co = e / (CIT * K * K), r = e % (CIT * K * K);
    const int ci = r / (K * K), tap = r % (K * K);
    if (co0 + co < Co && ci0 + ci < Ci) atomicAdd(&dW[((size_t)(co0 + co) * Ci + ci0 + ci) * K * K + tap], acc[q]);
  }
}

// Weight gradient on the tensor cores: for each tap, dW[co][ci] += sum_p g[co][p]
// in[ci][p + off(tap)], a product with rows = output channels (MT tiles of 16),
// columns = 16 input channels (two tiles of 8) and the reduction over pixels (one
// row of 16 pixels per mma).  A CTA owns all output channels and one block of 16
// input channels and sweeps a chunk of 16 x 16 pixel tiles; warp w takes the
// (tap, column tile) pairs w, w + 8, w + 16.  Both operands are FP32 and enter as
// hi + lo BF16 pairs; hi*hi + hi*lo + lo*hi keeps the products to about 2^-16.
// Shared memory: g [co][256 + 8] and the input halo [16][18 * 18 + 4], hi and lo.
template <int K, int MT>
struct WgradTC {
  static constexpr int COP = MT * 16;
  static constexpr int LDA = TILE * TILE + 8;          // 264: rows of g 4 banks apart
  static constexpr int LDB = (TILE + 2) * (TILE + 2) + 4;  // 328: input channels 4 banks apart
  static constexpr int PAIRS = K * K * 2;
  static constexpr int PPW = (PAIRS + 7) / 8;          // pairs per warp
  static constexpr size_t A_BYTES = (size_t)COP * LDA * 2;
  static constexpr size_t B_BYTES = (size_t)16 * LDB * 2;
  static constexpr size_t SMEM = 2 * A_BYTES + 2 * B_BYTES;
};

__device__ __forceinline__ unsigned pack_bf16(__nv_bfloat16 lo_k, __nv_bfloat16 hi_k) {
  return (unsigned)__bfloat16_as_ushort(lo_k) | ((unsigned)__bfloat16_as_ushort(hi_k) << 16);
}

template <int K, int MT>
__global__ void __launch_bounds__(TILE * TILE) k_conv_wgrad_tc(const float* __restrict__ in, int Ci,
                                                               const float* __restrict__ g, int Co, int H,
                                                               float* __restrict__ dW, int tiles_per_block) {
  using S = WgradTC<K, MT>;
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* a_hi = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* a_lo = reinterpret_cast<__nv_bfloat16*>(smem + S::A_BYTES);
  __nv_bfloat16* b_hi = reinterpret_cast<__nv_bfloat16*>(smem + 2 * S::A_BYTES);
  __nv_bfloat16* b_lo = reinterpret_cast<__nv_bfloat16*>(smem + 2 * S::A_BYTES + S::B_BYTES);
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5, gid = lane >> 2, tig = lane & 3;
  const int ci0 = blockIdx.y * 16;
  const int HW = H * H, m = H - 1, tpr = H / TILE, ntiles = tpr * tpr, R = K / 2, KK = K * K;
  constexpr int HALO = TILE + 2;
  float acc[MT][S::PPW][4];
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int b = 0; b < S::PPW; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const int t_end = min(ntiles, (blockIdx.x + 1) * tiles_per_block);
  for (int t = blockIdx.x * tiles_per_block; t < t_end; ++t) {
    const int x0 = (t % tpr) * TILE, y0 = (t / tpr) * TILE;
    for (int e = tid; e < S::COP * TILE * TILE; e += TILE * TILE) {
      const int co = e >> 8, px = e & 255;
      const float v = co < Co ? g[(size_t)co * HW + (y0 + (px >> 4)) * H + x0 + (px & 15)] : 0.f;
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      a_hi[co * S::LDA + px] = hi;
      a_lo[co * S::LDA + px] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
    for (int e = tid; e < 16 * HALO * HALO; e += TILE * TILE) {
      const int c = e / (HALO * HALO), px = e - c * HALO * HALO;
      const int yy = px / HALO, xx = px - yy * HALO;
      const float v = (ci0 + c < Ci) ? in[(size_t)(ci0 + c) * HW + ((y0 + yy - 1) & m) * H + ((x0 + xx - 1) & m)] : 0.f;
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      b_hi[c * S::LDB + px] = hi;
      b_lo[c * S::LDB + px] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
    __syncthreads();
#pragma unroll 1
    for (int y = 0; y < TILE; ++y) {  // reduction step: pixel row y (16 pixels)
      unsigned ah[MT][4], al[MT][4];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const int r0 = (mt * 16 + gid) * S::LDA + y * TILE + 2 * tig, r1 = r0 + 8 * S::LDA;
        ah[mt][0] = *reinterpret_cast<const unsigned*>(a_hi + r0);
        ah[mt][1] = *reinterpret_cast<const unsigned*>(a_hi + r1);
        ah[mt][2] = *reinterpret_cast<const unsigned*>(a_hi + r0 + 8);
        ah[mt][3] = *reinterpret_cast<const unsigned*>(a_hi + r1 + 8);
        al[mt][0] = *reinterpret_cast<const unsigned*>(a_lo + r0);
        al[mt][1] = *reinterpret_cast<const unsigned*>(a_lo + r1);
        al[mt][2] = *reinterpret_cast<const unsigned*>(a_lo + r0 + 8);
        al[mt][3] = *reinterpret_cast<const unsigned*>(a_lo + r1 + 8);
      }
#pragma unroll
      for (int q = 0; q < S::PPW; ++q) {
        const int pair = wp + 8 * q;
        if (pair >= S::PAIRS) break;
        const int tap = pair >> 1, nt = pair & 1;
        const int dy = tap / K - R + 1, dx = tap % K - R + 1;
        // column gid of the tile: input channel nt * 8 + gid; rows: pixels x = 2 tig (+1), (+8)
        const int base = (nt * 8 + gid) * S::LDB + (y + dy) * HALO + dx + 2 * tig;
        unsigned bh[2], bl[2];
        bh[0] = pack_bf16(b_hi[base], b_hi[base + 1]);
        bh[1] = pack_bf16(b_hi[base + 8], b_hi[base + 9]);
        bl[0] = pack_bf16(b_lo[base], b_lo[base + 1]);
        bl[1] = pack_bf16(b_lo[base + 8], b_lo[base + 9]);
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          mma_bf16_16816(acc[mt][q], ah[mt], bh);
          mma_bf16_16816(acc[mt][q], ah[mt], bl);
          mma_bf16_16816(acc[mt][q], al[mt], bh);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < S::PPW; ++q) {
    const int pair = wp + 8 * q;
    if (pair >= S::PAIRS) break;
    const int tap = pair >> 1, nt = pair & 1;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int co = mt * 16 + gid + (r >> 1) * 8, ci = ci0 + nt * 8 + 2 * tig + (r & 1);
        if (co < Co && ci < Ci) atomicAdd(&dW[((size_t)co * Ci + ci) * KK + tap], acc[mt][q][r]);
      }
  }
}

// db[c] += sum_p g[c][p]  (one CTA per channel)
__global__ void k_bias_grad(const float* __restrict__ g, int HW, float* db) {
  __shared__ float sh[32];
  float s = 0.f;
  const float* gc = g + (size_t)blockIdx.x * HW;
  for (int p = threadIdx.x; p < HW; p += blockDim.x) s += gc[p];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    atomicAdd(&db[blockIdx.x], t);
  }
}

// g *= gelu'(pre)
__global__ void k_gelu_bwd(float* g, const float* __restrict__ pre, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) g[i] *= gelu_d(pre[i]);
}

// 2x2 average pool of C channels of an H grid (out H/2); bwd spreads g/4.
__global__ void k_pool(const float* __restrict__ in, float* __restrict__ out, int C, int H) {
  const int h = H / 2;
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)C * h * h) return;
  const int c = (int)(i / (h * h)), r = (int)(i % (h * h)), y = r / h, x = r % h;
  const float* a = in + (size_t)c * H * H + 2 * y * H + 2 * x;
  out[i] = 0.25f * (a[0] + a[1] + a[H] + a[H + 1]);
}
__global__ void k_pool_bwd(const float* __restrict__ g, float* __restrict__ gin, int C, int H) {
  const int h = H / 2;
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)C * H * H) return;
  const int c = (int)(i / (H * H)), r = (int)(i % (H * H)), y = r / H, x = r % H;
  gin[i] += 0.25f * g[(size_t)c * h * h + (y / 2) * h + x / 2];
}
// nearest upsample of C channels from h to 2h, written at channel offset 0 of out;
// bwd sums the 2x2 gradients.
__global__ void k_up(const float* __restrict__ in, float* __restrict__ out, int C, int h) {
  const int H = 2 * h;
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)C * H * H) return;
  const int c = (int)(i / (H * H)), r = (int)(i % (H * H)), y = r / H, x = r % H;
  out[i] = in[(size_t)c * h * h + (y / 2) * h + x / 2];
}
__global__ void k_up_bwd(const float* __restrict__ g, float* __restrict__ gin, int C, int h) {
  const int H = 2 * h;
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)C * h * h) return;
  const int c = (int)(i / (h * h)), r = (int)(i % (h * h)), y = r / h, x = r % h;
  const float* a = g + (size_t)c * H * H + 2 * y * H + 2 * x;
  gin[i] += a[0] + a[1] + a[H] + a[H + 1];
}

// relative squared error L = sum (o - t)^2 / sum t^2, gradient 2 (o - t) / sum t^2
__global__ void k_sq_partial(const float* __restrict__ a, const float* __restrict__ b, long n, double* out) {
  __shared__ double sh[32];
  double s = 0.0, t = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double d = (double)a[i] - (b ? (double)b[i] : 0.0);
    s += d * d;
  }
  (void)t;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double q = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) q += sh[w];
    atomicAdd(out, q);
  }
}
__global__ void k_loss_grad(const float* __restrict__ o, const float* __restrict__ t, const double* tnorm2, long n,
                            float* g) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) g[i] = (float)(2.0 * ((double)o[i] - (double)t[i]) / *tnorm2);
}

// Adam on the FP32 master weights, then the BF16 copy used by the forward pass.
__global__ void k_adam(float* w, const float* __restrict__ g, float* m, float* v, __nv_bfloat16* wb, long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  wb[i] = __float2bfloat16_rn(wi);
}
__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* wb, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

inline int nb(long n, int t = 256) { return (int)((n + t - 1) / t); }


// structure channel: s = log(1 + dt / (mu h^2) * sum_k Kbar_k phi_x phi_y), Kbar_k the
// summed stiffness of the springs at point k, spread with the level-0 u-grid weights
__global__ void k_struct_density(Patches<double> pat, const int* __restrict__ adj_ptr, const int* __restrict__ adj_spring,
                                 const double* __restrict__ kappa, int np, int N, double* s) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  double kb = 0.0;
  for (int q = adj_ptr[k]; q < adj_ptr[k + 1]; ++q) kb += kappa[adj_spring[q]];
  const int x0 = pat.b_at(0, 0, 0, k), y0 = pat.b_at(0, 0, 1, k);
  for (int b = 0; b < PATCH; ++b)
    for (int a = 0; a < PATCH; ++a) {
      double w = pat.w_at(0, 0, 0, a, k) * pat.w_at(0, 0, 1, b, k) * kb;
      if (w != 0.0) atomicAdd(&s[((y0 + b) & (N - 1)) * N + ((x0 + a) & (N - 1))], w);
    }
}
__global__ void k_log1p_scale(const double* __restrict__ s, float* out, long n, double scale) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)log1p(scale * s[i]);
}
// Physical scaling of the stage: the residual is brought to velocity-error units
// (u, v rows times h^2/mu, p rows times h) before normalisation, and the pressure
// output is scaled by mu/h.  rs = sigma_in r.
__global__ void k_scaled_copy(const double* __restrict__ r, double* rs, long n1, double su, double sp) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < 3 * n1) rs[i] = r[i] * (i < 2 * n1 ? su : sp);
}
// x[0..2] = rs / ||rs|| (FP32), x[3] = the structure channel
__global__ void k_features(const double* __restrict__ rs, const double* __restrict__ nrm2,
                           const float* __restrict__ sch, float* x, long n1) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= 4 * n1) return;
  if (i < 3 * n1) {
    const double nr = sqrt(*nrm2);
    x[i] = nr > 0.0 ? (float)(rs[i] / nr) : 0.f;
  } else {
    x[i] = sch[i - 3 * n1];
  }
}
// dz = ||rs|| y, pressure rows also times mu/h (FP64)
__global__ void k_scale_out(const float* __restrict__ y, const double* __restrict__ nrm2, double* dz, long n1,
                            double po) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < 3 * n1) dz[i] = sqrt(*nrm2) * (i < 2 * n1 ? 1.0 : po) * (double)y[i];
}
// target = e / ||rs||, pressure rows also divided by mu/h
__global__ void k_target(const double* __restrict__ e, const double* __restrict__ nrm2, float* t, long n1,
                         double po) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= 3 * n1) return;
  const double nr = sqrt(*nrm2);
  t[i] = nr > 0.0 ? (float)(e[i] / (nr * (i < 2 * n1 ? 1.0 : po))) : 0.f;
}

}  // namespace

namespace {
int ualloc(ib_unet* U, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(IB_ERR_OOM, "cudaMalloc failed in the U-Net");
  }
  U->allocs.push_back(*p);
  return IB_OK;
}
template <typename T>
int ualloc_t(ib_unet* U, T** p, size_t count) {
  return ualloc(U, (void**)p, count * sizeof(T));
}

// Tensor-core launch of one convolution: MT tiles of 16 output channels (Co <= 96).
template <int K, int MT>
int conv_tc_launch(cudaStream_t st, int H, const float* in, int Ci, const __nv_bfloat16* Wt, const float* bias,
                   float* out, int Co, int off, float* pre, int act, int mode, int Wci, int accumulate) {
  static bool ready = false;  // raise the dynamic shared-memory limit once per instantiation
  if (!ready) {
    IB_CUDA_TRY(cudaFuncSetAttribute(k_conv_tc<K, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)ConvTC<K, MT>::SMEM));
    ready = true;
  }
  dim3 grid(H / TILE, H / TILE);
  k_conv_tc<K, MT><<<grid, TILE * TILE, ConvTC<K, MT>::SMEM, st>>>(in, Ci, Wt, bias, out, Co, off, pre, H, act, mode,
                                                                   Wci, accumulate);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

template <int K>
int conv_tc(cudaStream_t st, int H, const float* in, int Ci, const __nv_bfloat16* Wt, const float* bias, float* out,
            int Co, int off, float* pre, int act, int mode, int Wci, int accumulate) {
  switch ((Co + 15) / 16) {
    case 1: return conv_tc_launch<K, 1>(st, H, in, Ci, Wt, bias, out, Co, off, pre, act, mode, Wci, accumulate);
    case 2: return conv_tc_launch<K, 2>(st, H, in, Ci, Wt, bias, out, Co, off, pre, act, mode, Wci, accumulate);
    case 3: return conv_tc_launch<K, 3>(st, H, in, Ci, Wt, bias, out, Co, off, pre, act, mode, Wci, accumulate);
    case 4: return conv_tc_launch<K, 4>(st, H, in, Ci, Wt, bias, out, Co, off, pre, act, mode, Wci, accumulate);
    case 6: return conv_tc_launch<K, 6>(st, H, in, Ci, Wt, bias, out, Co, off, pre, act, mode, Wci, accumulate);
    default: return fail(IB_ERR_INVALID_ARG, "convolution channel count not supported on the tensor-core path");
  }
}

template <int K, int MT>
int wgrad_tc_launch(cudaStream_t st, dim3 grid, const float* in, int Ci, const float* g, int Co, int H, float* dW,
                    int tpb) {
  static bool ready = false;
  if (!ready) {
    IB_CUDA_TRY(cudaFuncSetAttribute(k_conv_wgrad_tc<K, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)WgradTC<K, MT>::SMEM));
    ready = true;
  }
  k_conv_wgrad_tc<K, MT><<<grid, TILE * TILE, WgradTC<K, MT>::SMEM, st>>>(in, Ci, g, Co, H, dW, tpb);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

template <int K>
int wgrad_tc(cudaStream_t st, dim3 grid, const float* in, int Ci, const float* g, int Co, int H, float* dW, int tpb) {
  switch ((Co + 15) / 16) {
    case 1: return wgrad_tc_launch<K, 1>(st, grid, in, Ci, g, Co, H, dW, tpb);
    case 2: return wgrad_tc_launch<K, 2>(st, grid, in, Ci, g, Co, H, dW, tpb);
    case 4: return wgrad_tc_launch<K, 4>(st, grid, in, Ci, g, Co, H, dW, tpb);
    default: return fail(IB_ERR_INVALID_ARG, "weight-gradient channel count not supported on the tensor-core path");
  }
}

int conv_fwd(ib_unet* U, int li, const float* in, float* out, int out_off, bool keep_pre) {
  const UConv& c = U->L[li];
  dim3 grid(c.H / TILE, c.H / TILE, (c.co + COT - 1) / COT);
  float* pre = keep_pre ? U->pre[li] : nullptr;
  if (U->tc) {
    if (c.k == 3)
      return conv_tc<3>(U->stream, c.H, in, c.ci, U->wb + c.w_off, U->w + c.b_off, out, c.co, out_off, pre, c.act, 0,
                        c.ci, 0);
    return conv_tc<1>(U->stream, c.H, in, c.ci, U->wb + c.w_off, U->w + c.b_off, out, c.co, out_off, pre, c.act, 0,
                      c.ci, 0);
  }
  if (c.k == 3)
    k_conv<3><<<grid, TILE * TILE, 0, U->stream>>>(in, c.ci, U->wb + c.w_off, U->w + c.b_off, out, c.co, out_off, pre,
                                                   c.H, c.act, 0, c.co, c.ci, 0);
  else
    k_conv<1><<<grid, TILE * TILE, 0, U->stream>>>(in, c.ci, U->wb + c.w_off, U->w + c.b_off, out, c.co, out_off, pre,
                                                   c.H, c.act, 0, c.co, c.ci, 0);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

// gradient of layer li: g_out is d loss / d post-activation (modified in place to
// the pre-activation gradient); accumulates d in into g_in (if not NULL) and the
// parameter gradients.
int conv_bwd(ib_unet* U, int li, const float* in, float* g_out, float* g_in) {
  const UConv& c = U->L[li];
  const long HW = (long)c.H * c.H;
  if (c.act) {
    k_gelu_bwd<<<nb(c.co * HW), 256, 0, U->stream>>>(g_out, U->pre[li], c.co * HW);
    IB_LAUNCH_CHECK();
  }
  const int ntiles = (c.H / TILE) * (c.H / TILE);
  const int tpb = ntiles >= 64 ? 16 : 1;
  dim3 gw((ntiles + tpb - 1) / tpb, (c.co + COT - 1) / COT, (c.ci + CIT - 1) / CIT);
  if (U->tc) {
    const dim3 gt((ntiles + tpb - 1) / tpb, (c.ci + 15) / 16);
    if (c.k == 3) IB_TRY(wgrad_tc<3>(U->stream, gt, in, c.ci, g_out, c.co, c.H, U->g + c.w_off, tpb));
    else IB_TRY(wgrad_tc<1>(U->stream, gt, in, c.ci, g_out, c.co, c.H, U->g + c.w_off, tpb));
  } else if (c.k == 3)
    k_conv_wgrad<3><<<gw, TILE * TILE, 0, U->stream>>>(in, c.ci, g_out, c.co, c.H, U->g + c.w_off, tpb);
  else
    k_conv_wgrad<1><<<gw, TILE * TILE, 0, U->stream>>>(in, c.ci, g_out, c.co, c.H, U->g + c.w_off, tpb);
  IB_LAUNCH_CHECK();
  k_bias_grad<<<c.co, 256, 0, U->stream>>>(g_out, (int)HW, U->g + c.b_off);
  IB_LAUNCH_CHECK();
  if (g_in && U->tc) {
    if (c.k == 3) return conv_tc<3>(U->stream, c.H, g_out, c.co, U->wb + c.w_off, nullptr, g_in, c.ci, 0, nullptr, 0, 1,
                                    c.ci, 1);
    return conv_tc<1>(U->stream, c.H, g_out, c.co, U->wb + c.w_off, nullptr, g_in, c.ci, 0, nullptr, 0, 1, c.ci, 1);
  }
  if (g_in) {
    dim3 grid(c.H / TILE, c.H / TILE, (c.ci + COT - 1) / COT);
    if (c.k == 3)
      k_conv<3><<<grid, TILE * TILE, 0, U->stream>>>(g_out, c.co, U->wb + c.w_off, nullptr, g_in, c.ci, 0, nullptr, c.H,
                                                     0, 1, c.co, c.ci, 1);
    else
      k_conv<1><<<grid, TILE * TILE, 0, U->stream>>>(g_out, c.co, U->wb + c.w_off, nullptr, g_in, c.ci, 0, nullptr, c.H,
                                                     0, 1, c.co, c.ci, 1);
    IB_LAUNCH_CHECK();
  }
  return IB_OK;
}

int unet_forward(ib_unet* U, const float* x, float* y) {
  const int N = U->N;
  const long n1 = (long)N * N, n2 = n1 / 4, n4 = n1 / 16;
  IB_TRY(conv_fwd(U, 0, x, U->a[0], 0, true));
  // layer 1 writes s1 into the concat buffer c1 at channels 32..47 and a[1]
  IB_TRY(conv_fwd(U, 1, U->a[0], U->a[1], 0, true));
  k_pool<<<nb(16 * n2), 256, 0, U->stream>>>(U->a[1], U->p1, 16, N);
  IB_LAUNCH_CHECK();
  IB_TRY(conv_fwd(U, 2, U->p1, U->a[2], 0, true));
  IB_TRY(conv_fwd(U, 3, U->a[2], U->a[3], 0, true));
  k_pool<<<nb(32 * n4), 256, 0, U->stream>>>(U->a[3], U->p2, 32, N / 2);
  IB_LAUNCH_CHECK();
  IB_TRY(conv_fwd(U, 4, U->p2, U->a[4], 0, true));
  IB_TRY(conv_fwd(U, 5, U->a[4], U->a[5], 0, true));
  k_up<<<nb(64 * n2), 256, 0, U->stream>>>(U->a[5], U->c2, 64, N / 4);
  IB_LAUNCH_CHECK();
  IB_CUDA_TRY(cudaMemcpyAsync(U->c2 + 64 * n2, U->a[3], sizeof(float) * 32 * n2, cudaMemcpyDeviceToDevice, U->stream));
  IB_TRY(conv_fwd(U, 6, U->c2, U->a[6], 0, true));
  IB_TRY(conv_fwd(U, 7, U->a[6], U->a[7], 0, true));
  k_up<<<nb(32 * n1), 256, 0, U->stream>>>(U->a[7], U->c1, 32, N / 2);
  IB_LAUNCH_CHECK();
  IB_CUDA_TRY(cudaMemcpyAsync(U->c1 + 32 * n1, U->a[1], sizeof(float) * 16 * n1, cudaMemcpyDeviceToDevice, U->stream));
  IB_TRY(conv_fwd(U, 8, U->c1, U->a[8], 0, true));
  IB_TRY(conv_fwd(U, 9, U->a[8], U->a[9], 0, true));
  IB_TRY(conv_fwd(U, 10, U->a[9], y, 0, false));
  return IB_OK;
}

__global__ void k_axpy_f(float* y, const float* __restrict__ x, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) y[i] += x[i];
}

// backward of the whole network from g_y (d loss / d output; overwritten), into U->g.
int unet_backward(ib_unet* U, const float* x, float* g_y) {
  const int N = U->N;
  const long n1 = (long)N * N, n2 = n1 / 4, n4 = n1 / 16;
  std::vector<float*>& ga = U->ga;
  for (int k = 0; k < 10; ++k)
    IB_CUDA_TRY(cudaMemsetAsync(ga[k], 0, sizeof(float) * U->L[k].co * U->L[k].H * U->L[k].H, U->stream));
  IB_CUDA_TRY(cudaMemsetAsync(U->gc1, 0, sizeof(float) * 48 * n1, U->stream));
  IB_CUDA_TRY(cudaMemsetAsync(U->gc2, 0, sizeof(float) * 96 * n2, U->stream));
  IB_CUDA_TRY(cudaMemsetAsync(U->gp1, 0, sizeof(float) * 16 * n2, U->stream));
  IB_CUDA_TRY(cudaMemsetAsync(U->gp2, 0, sizeof(float) * 32 * n4, U->stream));
  IB_TRY(conv_bwd(U, 10, U->a[9], g_y, ga[9]));
  IB_TRY(conv_bwd(U, 9, U->a[8], ga[9], ga[8]));
  IB_TRY(conv_bwd(U, 8, U->c1, ga[8], U->gc1));
  // concat [up(a7) | a1]: channels [0, 32) go back through the upsample, [32, 48) to a1
  k_up_bwd<<<nb(32 * n2), 256, 0, U->stream>>>(U->gc1, ga[7], 32, N / 2);
  IB_LAUNCH_CHECK();
  k_axpy_f<<<nb(16 * n1), 256, 0, U->stream>>>(ga[1], U->gc1 + 32 * n1, 16 * n1);
  IB_LAUNCH_CHECK();
  IB_TRY(conv_bwd(U, 7, U->a[6], ga[7], ga[6]));
  IB_TRY(conv_bwd(U, 6, U->c2, ga[6], U->gc2));
  // concat [up(a5) | a3]
  k_up_bwd<<<nb(64 * n4), 256, 0, U->stream>>>(U->gc2, ga[5], 64, N / 4);
  IB_LAUNCH_CHECK();
  k_axpy_f<<<nb(32 * n2), 256, 0, U->stream>>>(ga[3], U->gc2 + 64 * n2, 32 * n2);
  IB_LAUNCH_CHECK();
  IB_TRY(conv_bwd(U, 5, U->a[4], ga[5], ga[4]));
  IB_TRY(conv_bwd(U, 4, U->p2, ga[4], U->gp2));
  k_pool_bwd<<<nb(32 * n2), 256, 0, U->stream>>>(U->gp2, ga[3], 32, N / 2);
  IB_LAUNCH_CHECK();
  IB_TRY(conv_bwd(U, 3, U->a[2], ga[3], ga[2]));
  IB_TRY(conv_bwd(U, 2, U->p1, ga[2], U->gp1));
  k_pool_bwd<<<nb(16 * n1), 256, 0, U->stream>>>(U->gp1, ga[1], 16, N);
  IB_LAUNCH_CHECK();
  IB_TRY(conv_bwd(U, 1, U->a[0], ga[1], ga[0]));
  IB_TRY(conv_bwd(U, 0, x, ga[0], nullptr));
  return IB_OK;
}

// loss = sum (y - t)^2 / sum t^2 and, in U->ga_y, its gradient with respect to y.
int unet_loss(ib_unet* U, const float* y, const float* t, float* gy, double* loss) {
  const long n = 3L * U->N * U->N;
  IB_CUDA_TRY(cudaMemsetAsync(U->red, 0, 2 * sizeof(double), U->stream));
  k_sq_partial<<<256, 256, 0, U->stream>>>(t, nullptr, n, U->red);
  IB_LAUNCH_CHECK();
  k_sq_partial<<<256, 256, 0, U->stream>>>(y, t, n, U->red + 1);
  IB_LAUNCH_CHECK();
  k_loss_grad<<<nb(n), 256, 0, U->stream>>>(y, t, U->red, n, gy);
  IB_LAUNCH_CHECK();
  IB_CUDA_TRY(cudaMemcpyAsync(U->red_host, U->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, U->stream));
  IB_CUDA_TRY(cudaStreamSynchronize(U->stream));
  *loss = U->red_host[0] > 0 ? U->red_host[1] / U->red_host[0] : 0.0;
  return IB_OK;
}


}  // namespace

// Structure channel of a problem (after its set-up); allocates the channel once.
int learned_struct_channel(Problem& P) {
  const int N = P.lev[0].N;
  const long n1 = (long)N * N;
  if (!P.nn_sch) {
    cudaError_t e = cudaMalloc(&P.nn_sch, n1 * sizeof(float));
    if (e != cudaSuccess) return fail(IB_ERR_OOM, "structure channel");
  }
  double* tmp = P.t64b;  // n1 doubles of scratch
  IB_CUDA_TRY(cudaMemsetAsync(tmp, 0, n1 * sizeof(double), P.stream));
  if (P.np > 0 && P.ns > 0) {
    KScope ks(P, IB_KC_OTHER, P.np * 200.0);
    k_struct_density<<<nb(P.np), 128, 0, P.stream>>>(P.lev[0].pat64, P.adj_ptr, P.adj_spring, P.kappa, P.np, N, tmp);
    IB_LAUNCH_CHECK();
  }
  KScope ks(P, IB_KC_OTHER, n1 * 12.0);
  k_log1p_scale<<<nb(n1), 256, 0, P.stream>>>(tmp, P.nn_sch, n1, P.prm.dt / (P.prm.mu * P.lev[0].h * P.lev[0].h));
  IB_LAUNCH_CHECK();
  return IB_OK;
}

// NN input from a residual r (FP64, 3N^2): rs = sigma_in r in scratch, ||rs||^2 into
// nrm2 (device), x = [rs / ||rs||; structure channel].
int learned_features(Problem& P, const double* r, double* scratch, double* nrm2, float* x) {
  const long n1 = (long)P.lev[0].N * P.lev[0].N;
  const double h = P.lev[0].h;
  {
    KScope ks(P, IB_KC_OTHER, n1 * 48.0);
    k_scaled_copy<<<nb(3 * n1), 256, 0, P.stream>>>(r, scratch, n1, h * h / P.prm.mu, h);
    IB_LAUNCH_CHECK();
  }
  IB_TRY(launch_dot(P, scratch, scratch, nrm2));
  KScope ks(P, IB_KC_OTHER, n1 * 32.0);
  k_features<<<nb(4 * n1), 256, 0, P.stream>>>(scratch, nrm2, P.nn_sch, x, n1);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int learned_scale_out(Problem& P, const float* y, const double* nrm2, double* dz) {
  const long n1 = (long)P.lev[0].N * P.lev[0].N;
  KScope ks(P, IB_KC_OTHER, n1 * 36.0);
  k_scale_out<<<nb(3 * n1), 256, 0, P.stream>>>(y, nrm2, dz, n1, P.prm.mu / P.lev[0].h);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int learned_target(Problem& P, const double* e, const double* nrm2, float* t) {
  const long n1 = (long)P.lev[0].N * P.lev[0].N;
  KScope ks(P, IB_KC_OTHER, n1 * 36.0);
  k_target<<<nb(3 * n1), 256, 0, P.stream>>>(e, nrm2, t, n1, P.prm.mu / P.lev[0].h);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int learned_unet_size(const ib_unet* U) { return U ? U->N : 0; }

int learned_forward(ib_unet* U, cudaStream_t s, const float* x, float* y) {
  cudaStream_t old = U->stream;
  U->stream = s;
  int rc = unet_forward(U, x, y);
  U->stream = old;
  return rc;
}


}  // namespace ib

using namespace ib;

// ---------------------------------------------------------------- C ABI

extern "C" {

int64_t ib_unet_num_params(void) { return unet_param_count(); }

int ib_unet_create(int32_t N, const float* params, void* stream, ib_unet** out) {
  set_error("");
  if (!out) return fail(IB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (N < 64 || N > 4096 || (N & (N - 1)) != 0)
    return fail(IB_ERR_INVALID_ARG, "the U-Net grid must be a power of two in 64..4096");
  ib_unet* U = new (std::nothrow) ib_unet();
  if (!U) return fail(IB_ERR_OOM, "host allocation failed");
  U->N = N;
  U->stream = (cudaStream_t)stream;
  if (const char* e = std::getenv("IB_UNET_TC")) U->tc = e[0] != '0';
  U->L = unet_layers(N);
  U->np = unet_param_count();
  auto bail = [&](int code) {
    std::string msg = ib_last_error();
    ib_unet_destroy(U);
    set_error(msg);
    return code;
  };
  const long n1 = (long)N * N;
  int rc = IB_OK;
  rc = rc ? rc : ualloc_t(U, &U->w, U->np);
  rc = rc ? rc : ualloc_t(U, &U->wb, U->np);
  rc = rc ? rc : ualloc_t(U, &U->g, U->np);
  rc = rc ? rc : ualloc_t(U, &U->m, U->np);
  rc = rc ? rc : ualloc_t(U, &U->v, U->np);
  U->a.assign(10, nullptr);
  U->pre.assign(11, nullptr);
  U->ga.assign(10, nullptr);
  for (int k = 0; k < 11 && rc == IB_OK; ++k) {
    const long sz = (long)U->L[k].co * U->L[k].H * U->L[k].H;
    if (k < 10) {
      rc = ualloc_t(U, &U->a[k], sz);
      if (rc == IB_OK) rc = ualloc_t(U, &U->ga[k], sz);
    }
    if (rc == IB_OK) rc = ualloc_t(U, &U->pre[k], sz);
  }
  rc = rc ? rc : ualloc_t(U, &U->x_in, 4 * n1);
  rc = rc ? rc : ualloc_t(U, &U->p1, 16 * n1 / 4);
  rc = rc ? rc : ualloc_t(U, &U->p2, 32 * n1 / 16);
  rc = rc ? rc : ualloc_t(U, &U->c2, 96 * n1 / 4);
  rc = rc ? rc : ualloc_t(U, &U->c1, 48 * n1);
  rc = rc ? rc : ualloc_t(U, &U->gp1, 16 * n1 / 4);
  rc = rc ? rc : ualloc_t(U, &U->gp2, 32 * n1 / 16);
  rc = rc ? rc : ualloc_t(U, &U->gc2, 96 * n1 / 4);
  rc = rc ? rc : ualloc_t(U, &U->gc1, 48 * n1);
  rc = rc ? rc : ualloc_t(U, &U->gx, 3 * n1);
  rc = rc ? rc : ualloc_t(U, &U->red, 4);
  if (rc != IB_OK) return bail(rc);
  if (cudaMallocHost((void**)&U->red_host, 4 * sizeof(double)) != cudaSuccess)
    return bail(fail(IB_ERR_OOM, "pinned allocation failed"));
  cudaMemsetAsync(U->w, 0, U->np * sizeof(float), U->stream);
  cudaMemsetAsync(U->m, 0, U->np * sizeof(float), U->stream);
  cudaMemsetAsync(U->v, 0, U->np * sizeof(float), U->stream);
  if (params) {
    if (cudaMemcpyAsync(U->w, params, U->np * sizeof(float), cudaMemcpyHostToDevice, U->stream) != cudaSuccess)
      return bail(fail(IB_ERR_CUDA, "parameter upload failed"));
  }
  k_to_bf16<<<nb(U->np), 256, 0, U->stream>>>(U->w, U->wb, U->np);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(U->stream) != cudaSuccess)
    return bail(fail(IB_ERR_CUDA, "U-Net initialisation failed"));
  *out = U;
  return IB_OK;
}

int ib_unet_set_params(ib_unet* U, const float* params) {
  set_error("");
  if (!U || !params) return fail(IB_ERR_INVALID_ARG, "NULL argument");
  IB_CUDA_TRY(cudaMemcpyAsync(U->w, params, U->np * sizeof(float), cudaMemcpyHostToDevice, U->stream));
  k_to_bf16<<<nb(U->np), 256, 0, U->stream>>>(U->w, U->wb, U->np);
  IB_LAUNCH_CHECK();
  IB_CUDA_TRY(cudaStreamSynchronize(U->stream));
  return IB_OK;
}

int ib_unet_get_params(ib_unet* U, float* params) {
  set_error("");
  if (!U || !params) return fail(IB_ERR_INVALID_ARG, "NULL argument");
  IB_CUDA_TRY(cudaMemcpyAsync(params, U->w, U->np * sizeof(float), cudaMemcpyDeviceToHost, U->stream));
  IB_CUDA_TRY(cudaStreamSynchronize(U->stream));
  return IB_OK;
}

int ib_unet_forward(ib_unet* U, const float* x, float* y) {
  set_error("");
  if (!U || !x || !y) return fail(IB_ERR_INVALID_ARG, "NULL argument");
  IB_TRY(unet_forward(U, x, y));
  IB_CUDA_TRY(cudaStreamSynchronize(U->stream));
  return IB_OK;
}

int ib_unet_loss_grad(ib_unet* U, const float* x, const float* t, double* loss, float* grad) {
  set_error("");
  if (!U || !x || !t) return fail(IB_ERR_INVALID_ARG, "NULL argument");
  float* y = U->pre[10];  // the head has no activation: its pre-activation buffer holds y
  IB_CUDA_TRY(cudaMemsetAsync(U->g, 0, U->np * sizeof(float), U->stream));
  IB_TRY(unet_forward(U, x, y));
  double l = 0.0;
  IB_TRY(unet_loss(U, y, t, U->gx, &l));
  IB_TRY(unet_backward(U, x, U->gx));
  if (grad) IB_CUDA_TRY(cudaMemcpyAsync(grad, U->g, U->np * sizeof(float), cudaMemcpyDeviceToHost, U->stream));
  IB_CUDA_TRY(cudaStreamSynchronize(U->stream));
  if (loss) *loss = l;
  return IB_OK;
}

int ib_unet_train_step(ib_unet* U, const float* x, const float* t, float lr, double* loss) {
  IB_TRY(ib_unet_loss_grad(U, x, t, loss, nullptr));
  U->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)U->step), c2 = 1.f - powf(b2, (float)U->step);
  k_adam<<<nb(U->np), 256, 0, U->stream>>>(U->w, U->g, U->m, U->v, U->wb, U->np, lr, b1, b2, 1e-8f, c1, c2);
  IB_LAUNCH_CHECK();
  IB_CUDA_TRY(cudaStreamSynchronize(U->stream));
  return IB_OK;
}

void ib_unet_destroy(ib_unet* U) {
  if (!U) return;
  for (void* p : U->allocs) cudaFree(p);
  if (U->red_host) cudaFreeHost(U->red_host);
  delete U;
}

}  // extern "C"
