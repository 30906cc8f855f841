// Assembled rows of the elasticity operator E_l = S_l J S_l^* (sec. 3.2: the
// elasticity block of every level, Galerkin-coarsened, E_{l+1} = R E_l P, Eq. 27).
//
// Every velocity row r = (c, i, j) of level l that a spread patch touches (a
// "structure row") keeps a dense window of its entries: the columns (cc, i + di,
// j + dj) with |di|, |dj| <= WR, for both column components, 2 (2 WR + 1)^2 values.
// The offsets are geometric (a column is wrapped onto the periodic grid only when
// it is read), so on grids smaller than the window two offsets may name the same
// column; the operator is the sum of both, which every consumer forms.
//
// Level 0 is assembled from the points: row node of point k's spread patch x
// J_kl x column node of point l's interpolation patch (J_kk and the spring blocks),
// with atomic additions.  A point pair farther apart than the window allows (a
// spring longer than about 1.5 cells in x or y) sets DEV_ERR_WINDOW; the set-up then
// keeps the point-based path for that step.  Coarse levels are exact Galerkin
// products of the level above, in two gathers with one writer per result (no
// atomics): T = E_l P per fine row, then E_{l+1} = R T per coarse row.  The box
// matrices of structure boxes and the coarsest dense matrix are read out of the
// windows, and the V-cycle and the FP64 operator apply E_l w as one gather per row.
#include "ib_internal.cuh"
#include "ib_ops.cuh"

namespace ib {

namespace {

constexpr int TPB = 256;
inline int nblk(long n, int t = TPB) { return (int)((n + t - 1) / t); }

// a - b for two indices of a periodic grid of size N, as the representative in
// [-N/2, N/2) (every representative names the same column; on grids of 16 or more
// cells the level-0 offsets of one point pair lie well inside that range)
__device__ __forceinline__ int sdiff(int a, int b, int N) { return ((a - b + N / 2) & (N - 1)) - N / 2; }

// Rows touched by the level's spread patches (the same nonzero test as the
// structure-box marking).
__global__ void k_mark_rows(Patches<double> pat, int np, int N, int* rowslot) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * np) return;
  const int comp = t / np, k = t - comp * np;
  const int x0 = pat.b_at(0, comp, 0, k), y0 = pat.b_at(0, comp, 1, k);
  for (int bb = 0; bb < PATCH; ++bb) {
    if (pat.w_at(0, comp, 1, bb, k) == 0.0) continue;
    const int j = wrapi(y0 + bb, N);
    for (int a = 0; a < PATCH; ++a)
      if (pat.w_at(0, comp, 0, a, k) != 0.0) rowslot[(size_t)comp * N * N + (size_t)j * N + wrapi(x0 + a, N)] = 1;
  }
}

// Marked rows get consecutive slots (in an arbitrary order) and their row index.
__global__ void k_assign_rows(int* rowslot, long nrow, int* slot_row, int* count) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= nrow) return;
  if (rowslot[t]) {
    const int s = atomicAdd(count, 1);
    rowslot[t] = s;
    slot_row[s] = (int)t;
  } else {
    rowslot[t] = -1;
  }
}

// Level-0 windows from the points.  Thread = (point k, coupling q, row component
// c, row node of k's spread patch): q = 0 the diagonal block J_kk = -sum K_s, q >= 1
// the block K_s of the q-th spring at k (coupling to its other end l).
__global__ void k_window_points(Patches<double> pat, Springs<double> sp, int N, const int* __restrict__ rowslot,
                                double* __restrict__ Ew, int* err) {
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
      const int s = sp.adj_spring[a];
      J[0][0] -= sp.K[s];
      J[0][1] -= sp.K[ns + s];
      J[1][1] -= sp.K[2 * ns + s];
    }
  } else {
    const int a = sp.adj_ptr[k] + q - 1;
    const int s = sp.adj_spring[a];
    l = sp.adj_other[a];
    J[0][0] = sp.K[s];
    J[0][1] = sp.K[ns + s];
    J[1][1] = sp.K[2 * ns + s];
  }
  J[1][0] = J[0][1];
  const int ri = wrapi(pat.b_at(0, c, 0, k) + ra, N), rj = wrapi(pat.b_at(0, c, 1, k) + rb, N);
  const int slot = rowslot[(size_t)c * N * N + (size_t)rj * N + ri];
  if (slot < 0) {
    atomicOr(err, DEV_ERR_INDEX);
    return;
  }
  double* row = Ew + (size_t)slot * WIN;
  for (int cc = 0; cc < 2; ++cc) {
    const double jv = ws * J[c][cc];
    if (jv == 0.0) continue;
    const int ix0 = pat.b_at(1, cc, 0, l), iy0 = pat.b_at(1, cc, 1, l);
    for (int cb = 0; cb < PATCH; ++cb) {
      const double wiy = pat.w_at(1, cc, 1, cb, l);
      if (wiy == 0.0) continue;
      const int dj = sdiff(wrapi(iy0 + cb, N), rj, N);
      for (int ca = 0; ca < PATCH; ++ca) {
        const double wi = pat.w_at(1, cc, 0, ca, l) * wiy;
        if (wi == 0.0) continue;
        const int di = sdiff(wrapi(ix0 + ca, N), ri, N);
        if (di < -WR || di > WR || dj < -WR || dj > WR) {
          atomicOr(err, DEV_ERR_WINDOW);
          continue;
        }
        atomicAdd(&row[cc * WSQ + (dj + WR) * WD + di + WR], jv * wi);
      }
    }
  }
}

// ---- level-0 row lists: for each structure row, the points whose spread patch
// covers it.  Thread = (point k, row component c, spread node): count, then fill
// after a scan, then sort each row's entries by point (a point covers a row once).
__global__ void k_rc_count(Patches<double> pat, int np, int N, const int* __restrict__ rowslot, int* cnt,
                           int* err) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= 32L * np) return;
  const int k = (int)(t >> 5), rem = (int)(t & 31), c = rem >> 4, a = rem & 3, bb = (rem >> 2) & 3;
  const double ws = pat.w_at(0, c, 0, a, k) * pat.w_at(0, c, 1, bb, k);
  if (ws == 0.0) return;
  const int ri = wrapi(pat.b_at(0, c, 0, k) + a, N), rj = wrapi(pat.b_at(0, c, 1, k) + bb, N);
  const int s = rowslot[(size_t)c * N * N + (size_t)rj * N + ri];
  if (s < 0) {
    atomicOr(err, DEV_ERR_INDEX);
    return;
  }
  atomicAdd(&cnt[s], 1);
}

// Exclusive scan of cnt[0, n) into start[0, n] by one block: each thread sums a
// contiguous chunk, the chunk sums are scanned in shared memory, then each thread
// writes its chunk's offsets.
__global__ void __launch_bounds__(1024) k_scan_block(const int* __restrict__ cnt, int n, int* __restrict__ start) {
  __shared__ int part[1024];
  const int t = threadIdx.x, per = (n + 1023) / 1024;
  const int b0 = min(n, t * per), b1 = min(n, b0 + per);
  int s = 0;
  for (int i = b0; i < b1; ++i) s += cnt[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = t ? part[t - 1] : 0;
  for (int i = b0; i < b1; ++i) {
    start[i] = run;
    run += cnt[i];
  }
  if (t == 1023) start[n] = part[1023];
}

__global__ void k_rc_fill(Patches<double> pat, int np, int N, const int* __restrict__ rowslot,
                          const int* __restrict__ start, int* fill, int* pt, double* wt) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= 32L * np) return;
  const int k = (int)(t >> 5), rem = (int)(t & 31), c = rem >> 4, a = rem & 3, bb = (rem >> 2) & 3;
  const double ws = pat.w_at(0, c, 0, a, k) * pat.w_at(0, c, 1, bb, k);
  if (ws == 0.0) return;
  const int ri = wrapi(pat.b_at(0, c, 0, k) + a, N), rj = wrapi(pat.b_at(0, c, 1, k) + bb, N);
  const int s = rowslot[(size_t)c * N * N + (size_t)rj * N + ri];
  if (s < 0) return;
  const int pos = start[s] + atomicAdd(&fill[s], 1);
  pt[pos] = k;
  wt[pos] = ws;
}

__global__ void k_rc_sort(const int* __restrict__ start, int nrows, int* pt, double* wt) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nrows) return;
  const int e0 = start[s], e1 = start[s + 1];
  for (int e = e0 + 1; e < e1; ++e) {
    const int k = pt[e];
    const double w = wt[e];
    int q = e - 1;
    while (q >= e0 && pt[q] > k) {
      pt[q + 1] = pt[q];
      wt[q + 1] = wt[q];
      --q;
    }
    pt[q + 1] = k;
    wt[q + 1] = w;
  }
}

// y[row] += scale * sum over the row's entries of weight * vals[k sk + c sc] (c the
// row's component), one thread per structure row: the spread S of a per-point
// field as a gather in a fixed order.
__global__ void k_spread_rows(const int* __restrict__ slot_row, int nrows, int N, const int* __restrict__ start,
                              const int* __restrict__ pt, const double* __restrict__ wt,
                              const double* __restrict__ vals, long sk, long sc, double scale, double* y) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nrows) return;
  const int r = slot_row[s], c = r / (N * N);
  double acc = 0.0;
  for (int e = start[s]; e < start[s + 1]; ++e) acc += wt[e] * vals[(size_t)pt[e] * sk + (size_t)c * sc];
  y[r] += scale * acc;
}

// Level-0 windows by rows: one warp per structure row, each half-warp one column
// component cc of the row's window and each of its 16 lanes one node (a, b) of
// the 4 x 4 interpolation patch.  The row's entries (points k in order), each
// coupling of k (J_kk, then its springs' blocks in adjacency order) add, in that
// fixed order, into the row window kept in shared memory; within a coupling every
// lane adds to a cell of its own, so each cell's sum runs in the same order as in
// k_window_points, without atomics.  A block holds WROWS consecutive rows, whose
// windows are contiguous in Ew.
constexpr int WROWS = 8;
__global__ void __launch_bounds__(32 * WROWS) k_window_rows(const int* __restrict__ slot_row, int nrows, int N,
                                                            const int* __restrict__ start, const int* __restrict__ pt,
                                                            const double* __restrict__ wt, Patches<double> pat,
                                                            Springs<double> sp, double* __restrict__ Ew, int* err) {
  __shared__ double sw[WROWS * WIN];
  const int tid = threadIdx.x, lane = tid & 31, wr = tid >> 5;
  const int s0 = blockIdx.x * WROWS, s = s0 + wr;
  const int cc = lane >> 4, pa = lane & 3, pb = (lane >> 2) & 3;
  double* mine = sw + wr * WIN + cc * WSQ;  // the half-window (row s, component cc)
  for (int e = lane; e < WIN; e += 32) sw[wr * WIN + e] = 0.0;
  __syncwarp();
  bool outside = false;
  if (s < nrows) {
    const int r = slot_row[s], n = N * N, c = r / n, rr = r - c * n, ri = rr % N, rj = rr / N;
    const int ns = sp.ns;
    const int koff = (c == cc) ? (c == 0 ? 0 : 2) * ns : ns;  // J[c][cc] in K's [3][ns] layout
    for (int e = start[s]; e < start[s + 1]; ++e) {
      const int k = pt[e];
      const double ws = wt[e];
      const int a0 = sp.adj_ptr[k], deg = sp.adj_ptr[k + 1] - a0;
      // the couplings of k: q = 0 the point itself (J_kk = -sum of its springs'
      // blocks), q = 1..deg its springs' other ends; up to WQ of them have their
      // loads issued together, then add in the order q = 0, 1, ...
      constexpr int WQ = 4;
      int lq[WQ];
      double jq[WQ];
      lq[0] = k;
      jq[0] = 0.0;
      if (deg < WQ) {
#pragma unroll
        for (int q = 1; q < WQ; ++q) {
          if (q > deg) break;
          lq[q] = sp.adj_other[a0 + q - 1];
          jq[q] = sp.K[koff + sp.adj_spring[a0 + q - 1]];
        }
#pragma unroll
        for (int q = 1; q < WQ; ++q)
          if (q <= deg) jq[0] -= jq[q];
      } else {
        for (int a = a0; a < a0 + deg; ++a) jq[0] -= sp.K[koff + sp.adj_spring[a]];
      }
      for (int q0 = 0; q0 <= deg; q0 += WQ) {
        double wiq[WQ];
        int cell[WQ];
#pragma unroll
        for (int u = 0; u < WQ; ++u) {
          const int q = q0 + u;
          wiq[u] = 0.0;
          cell[u] = -1;
          if (q > deg) continue;
          int l;
          if (q0 == 0 && deg < WQ) {
            l = lq[u];
          } else if (q == 0) {
            l = k;
          } else {
            l = sp.adj_other[a0 + q - 1];
            jq[u] = sp.K[koff + sp.adj_spring[a0 + q - 1]];
          }
          if (q == 0) jq[u] = jq[0];
          wiq[u] = pat.w_at(1, cc, 0, pa, l) * pat.w_at(1, cc, 1, pb, l);
          const int di = sdiff(wrapi(pat.b_at(1, cc, 0, l) + pa, N), ri, N);
          const int dj = sdiff(wrapi(pat.b_at(1, cc, 1, l) + pb, N), rj, N);
          cell[u] = (di < -WR || di > WR || dj < -WR || dj > WR) ? -2 : (dj + WR) * WD + di + WR;
        }
#pragma unroll
        for (int u = 0; u < WQ; ++u) {
          const int q = q0 + u;
          if (q > deg) break;
          const double jv = ws * jq[u];
          if (jv == 0.0 || wiq[u] == 0.0) continue;
          if (cell[u] < 0) {
            outside = true;
            continue;
          }
          mine[cell[u]] += jv * wiq[u];
        }
      }
    }
  }
  if (outside) atomicOr(err, DEV_ERR_WINDOW);
  __syncthreads();
  const int rows = nrows - s0 < WROWS ? nrows - s0 : WROWS;
  double* dst = Ew + (size_t)s0 * WIN;
  for (int e = tid; e < rows * WIN; e += 32 * WROWS) dst[e] = sw[e];
}

// Prolongation weights of coarse column C along one direction (sec. 3.1): fine
// index 2C + o, o in [-1, 2].  Normal direction (faces): 1/2, 1, 1/2 at o = -1, 0, 1;
// centred direction (cell rows): 1/4, 3/4, 3/4, 1/4 at o = -1, 0, 1, 2.
__device__ __forceinline__ double pw(bool normal, int o) {
  if (normal) return o == 0 ? 1.0 : ((o == -1 || o == 1) ? 0.5 : 0.0);
  return (o == 0 || o == 1) ? 0.75 : ((o == -1 || o == 2) ? 0.25 : 0.0);
}

// Galerkin step 1: T = E_f P for every fine structure row (one thread per entry).
// T[s][cc][dJ + TR][dI + TR] is the entry at coarse column (cc, I0 + dI, J0 + dJ),
// (I0, J0) = (i >> 1, j >> 1) of the fine row (i, j); |dI|, |dJ| <= TR = 3 covers
// every coarse column P reaches from the row's window.
// With no-slip walls (walls = 1) P is the wall prolongation: coarse columns beyond
// the grid and coarse wall faces have no entries, and next to a wall the ghost folds
// the far row's 1/4 onto the near one (fine row 0 takes 1/2 of coarse row 0).
__global__ void k_window_EP(const int* __restrict__ slot_row, int nrows, int Nf, const double* __restrict__ Ef,
                            double* __restrict__ T, int walls) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)nrows * TWIN) return;
  const int s = (int)(t / TWIN), e = (int)(t - (long)s * TWIN);
  const int cc = e / (TD * TD), rem = e - cc * TD * TD;
  const int dJ = rem / TD - TR, dI = rem - (rem / TD) * TD - TR;
  const int r = slot_row[s];
  const int nf = Nf * Nf;
  const int rr = r % nf, i = rr % Nf, j = rr / Nf;
  const int I0 = i >> 1, J0 = j >> 1;
  // coarse column (cc, I0 + dI, J0 + dJ): fine columns 2 (I0 + dI) + ox, 2 (J0 + dJ) + oy
  const bool nx = cc == 0, ny = cc == 1;  // u: normal in x; v: normal in y
  const double* row = Ef + (size_t)s * WIN + cc * WSQ;
  const int Nc = Nf / 2, Cx = I0 + dI, Cy = J0 + dJ;
  double acc = 0.0;
  if (walls && (Cx < 0 || Cx >= Nc || Cy < 0 || Cy >= Nc || (nx && Cx == 0) || (ny && Cy == 0))) {
    T[(size_t)s * TWIN + e] = 0.0;
    return;
  }
  for (int oy = -1; oy <= 2; ++oy) {
    double wy = pw(ny, oy);
    if (wy == 0.0) continue;
    const int dj = 2 * Cy + oy - j;
    if (dj < -WR || dj > WR) continue;
    if (walls) {
      const int F = 2 * Cy + oy;
      if (F < 0 || F >= Nf) continue;
      if (!ny && ((Cy == 0 && oy == 0) || (Cy == Nc - 1 && oy == 1))) wy = 0.5;
    }
    for (int ox = -1; ox <= 2; ++ox) {
      double wx = pw(nx, ox);
      if (wx == 0.0) continue;
      const int di = 2 * Cx + ox - i;
      if (di < -WR || di > WR) continue;
      if (walls) {
        const int F = 2 * Cx + ox;
        if (F < 0 || F >= Nf) continue;
        if (!nx && ((Cx == 0 && ox == 0) || (Cx == Nc - 1 && ox == 1))) wx = 0.5;
      }
      acc += row[(dj + WR) * WD + di + WR] * wx * wy;
    }
  }
  T[(size_t)s * TWIN + e] = acc;
}

// Galerkin step 2: E_c = R T for every coarse structure row (one thread per window
// entry).  R (sec. 3.1, Eqs. 25-26): u at coarse (I, J) from fine faces 2I - 1, 2I,
// 2I + 1 (weights 1, 2, 1) on rows 2J, 2J + 1, times 1/8; v transposed.
// With no-slip walls a coarse wall face has no row (its entries are zero).
__global__ void k_window_R(const int* __restrict__ slot_row_c, int nrows_c, int Nc,
                           const int* __restrict__ rowslot_f, const double* __restrict__ T,
                           double* __restrict__ Ec, int walls) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)nrows_c * WIN) return;
  const int S = (int)(t / WIN), e = (int)(t - (long)S * WIN);
  const int cc = e / WSQ, rem = e - cc * WSQ;
  const int dJ = rem / WD - WR, dI = rem - (rem / WD) * WD - WR;
  const int R = slot_row_c[S];
  const int nc = Nc * Nc, c = R / nc, Rr = R - c * nc, I = Rr % Nc, J = Rr / Nc;
  const int Nf = 2 * Nc, nf = Nf * Nf;
  double acc = 0.0;
  if (walls && wall_face(c, I, J)) {
    Ec[(size_t)S * WIN + e] = 0.0;
    return;
  }
  for (int a = -1; a <= 1; ++a) {      // normal direction offset: weights 1, 2, 1
    for (int bb = 0; bb <= 1; ++bb) {  // centred direction: rows 2J, 2J + 1 (v: columns)
      const double wr = (a == 0 ? 0.25 : 0.125);
      const int iu = c == 0 ? 2 * I + a : 2 * I + bb;  // unwrapped fine row position
      const int ju = c == 0 ? 2 * J + bb : 2 * J + a;
      const int fs = rowslot_f[(size_t)c * nf + (size_t)wrapi(ju, Nf) * Nf + wrapi(iu, Nf)];
      if (fs < 0) continue;
      // coarse column (cc, I + dI, J + dJ) relative to the fine row's anchor
      const int tI = I + dI - (iu >> 1), tJ = J + dJ - (ju >> 1);
      if (tI < -TR || tI > TR || tJ < -TR || tJ > TR) continue;
      acc += wr * T[(size_t)fs * TWIN + cc * TD * TD + (tJ + TR) * TD + tI + TR];
    }
  }
  Ec[(size_t)S * WIN + e] = acc;
}

// Structure-box matrices: add coef * E_BB to the Stokes blocks already there.  One
// thread per (box slot, velocity row q) adds the window entries of that row whose
// columns are unknowns of the box (column-major n_B x n_B blocks).
__global__ void k_struct_from_windows(const int* __restrict__ box_of_slot, int nslot, int N, int b,
                                      const int* __restrict__ rowslot, const double* __restrict__ Ew, double coef,
                                      double* __restrict__ M, int nB) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const int nv = 2 * b * (b + 1);
  if (t >= (long)nslot * nv) return;
  const int s = (int)(t / nv), q = (int)(t - (long)s * nv);
  const int nb = N / b, box = box_of_slot[s], x0 = (box % nb) * b, y0 = (box / nb) * b;
  int comp, i, j;
  box_unknown(q, b, x0, y0, N, &comp, &i, &j);
  const int ws = rowslot[(size_t)comp * N * N + (size_t)j * N + i];
  if (ws < 0) return;
  const double* row = Ew + (size_t)ws * WIN;
  double* Mb = M + (size_t)s * nB * nB;
  // the box's velocity columns, each at the window offsets congruent to its
  // distance from the row modulo N (more than one only on grids narrower than the
  // window), in the window's order: the same additions as walking the window
  for (int cq = 0; cq < nv; ++cq) {
    int cc, ci, cj;
    box_unknown(cq, b, x0, y0, N, &cc, &ci, &cj);
    int dx = sdiff(ci, i, N), dy = sdiff(cj, j, N);
    while (dy - N >= -WR) dy -= N;
    while (dx - N >= -WR) dx -= N;
    for (int oy = dy; oy <= WR; oy += N) {
      if (oy < -WR) continue;
      for (int ox = dx; ox <= WR; ox += N) {
        if (ox < -WR) continue;
        const double v = row[cc * WSQ + (oy + WR) * WD + ox + WR];
        if (v != 0.0) Mb[(size_t)cq * nB + q] += coef * v;
      }
    }
  }
}

// Coarsest dense matrix (column-major, leading dimension ld): add coef * E_c.  One
// thread per structure row adds that row's entries.
__global__ void k_coarse_from_windows(const int* __restrict__ slot_row, int nrows, int N,
                                      const double* __restrict__ Ew, double coef, double* __restrict__ M, int ld) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nrows) return;
  const int r = slot_row[s], n = N * N;
  const int rr = r % n, i = rr % N, j = rr / N;
  const double* row = Ew + (size_t)s * WIN;
  for (int e = 0; e < WIN; ++e) {
    const double v = row[e];
    if (v == 0.0) continue;
    const int cc = e / WSQ, rem = e - cc * WSQ;
    const int col = cc * n + wrapi(j + rem / WD - WR, N) * N + wrapi(i + rem % WD - WR, N);
    M[(size_t)col * ld + r] += coef * v;
  }
}

__global__ void k_window_cast(const double* __restrict__ a, float* __restrict__ b, long n) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t < n) b[t] = (float)a[t];
}

}  // namespace

// y[r] += coef * (E_l w)[r] on the structure rows of colour `color` (-1: all rows),
// formed from differences of w (see below): one warp per row, the lanes take the window entries in turn and the warp sums
// them.  The row count is read from the device (the set-up's counter), so that a
// captured launch, sized by the storage capacity, stays valid when the count
// changes from step to step.  Only the programmatic-launch wait orders the reads of w.
// The colour lists of a level's structure rows: each slot whose row belongs to
// colour c (a face on a box edge belongs to the boxes on both sides) and is not a
// no-slip wall face is appended to colour c's list.  The order within a list does
// not matter: every row is applied by one warp, into its own entry.
__global__ void k_color_append(const int* __restrict__ slot_row, int nr, int N, int b, int walls, int cap,
                               int* __restrict__ crow, int* __restrict__ ccount) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nr) return;
  const int r = slot_row[s], n = N * N, c = r / n, rr = r - c * n, i = rr % N, j = rr / N;
  if (walls && wall_face(c, i, j)) return;
#pragma unroll
  for (int col = 0; col < 4; ++col)
    if (row_in_color(c, i, j, b, col)) crow[(size_t)col * cap + atomicAdd(&ccount[col], 1)] = s;
}

// rE (or y) += coef * E_l w on the structure rows of colour `color` (-1: all
// rows): a warp per row, each lane its window entries e = lane + 32 t; the
// entries' offsets from the row are decoded once per warp, and rows at least WR
// cells from the grid's edges gather without wrapping.  The warps stride over the
// colour's list (or over all slots).
template <typename T>
__global__ void __launch_bounds__(256) kv_window_apply(const int* __restrict__ slot_row, const int* __restrict__ nrows_dev,
                                                       const int* __restrict__ crow, const int* __restrict__ ccount,
                                                       int cap, const T* __restrict__ Ew, const T* __restrict__ w,
                                                       int N, T coef, int color, int walls, T* __restrict__ y) {
  constexpr int NT = (WIN + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * (long)blockDim.x) >> 5);
  const size_t n = (size_t)N * N;
  int offc[NT], offd[NT];  // per entry: component and row/column offsets (dj * N + di), -1: none
  int dis[NT], djs[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int e = lane + 32 * t;
    const int cc = e / WSQ, rem = e - cc * WSQ;
    djs[t] = rem / WD - WR;
    dis[t] = rem - (rem / WD) * WD - WR;
    offc[t] = e < WIN ? cc : -1;
    offd[t] = djs[t] * N + dis[t];
  }
  const int k1 = color < 0 ? *nrows_dev : ccount[color];
  const int* list = color < 0 ? nullptr : crow + (size_t)color * cap;
  pdl_enter();
  for (int k = warp; k < k1; k += nwarps) {
    const int s = color < 0 ? k : list[k];
    const int r = slot_row[s], c = (int)(r / n), rr = r - c * (int)n, i = rr % N, j = rr / N;
    if (color < 0 && walls && wall_face(c, i, j)) continue;  // the whole warp: one row
    const T* row = Ew + (size_t)s * WIN;
    // every row of E_l sums to zero over each column component (a uniform velocity
    // is in the kernel of E_l: J annihilates translations, P reproduces constants),
    // so the entries multiply differences from the component's value at the row's
    // own index; a structure moving almost rigidly then keeps the accuracy of the
    // per-point form, which works on velocity differences.  With no-slip walls the
    // prolongation does not reproduce constants next to a wall, so the coarse rows
    // need not sum to zero there: the plain sum is taken.
    const T ref0 = walls ? (T)0 : w[(size_t)j * N + i], ref1 = walls ? (T)0 : w[n + (size_t)j * N + i];
    const bool inner = i >= WR && i < N - WR && j >= WR && j < N - WR;
    const long base = (long)j * N + i;
    T acc = 0;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int cc = offc[t];
      if (cc < 0) continue;
      const size_t idx = inner ? (size_t)(cc * (long)n + base + offd[t])
                               : cc * n + (size_t)wrapi(j + djs[t], N) * N + wrapi(i + dis[t], N);
      acc += row[lane + 32 * t] * (w[idx] - (cc == 0 ? ref0 : ref1));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[r] += coef * acc;
  }
}
template __global__ void kv_window_apply<double>(const int*, const int*, const int*, const int*, int, const double*,
                                                 const double*, int, double, int, int, double*);
template __global__ void kv_window_apply<float>(const int*, const int*, const int*, const int*, int, const float*,
                                                const float*, int, float, int, int, float*);

// ---------------------------------------------------------------- launchers

int launch_mark_rows(Problem& P, int level) {
  LevelInfo& L = P.lev[level];
  const long nrow = 2L * L.N * L.N;
  IB_CUDA_TRY(cudaMemsetAsync(L.rowslot, 0, sizeof(int) * nrow, P.stream));
  IB_CUDA_TRY(cudaMemsetAsync(P.count + 1 + level, 0, sizeof(int), P.stream));
  {
    KScope ks(P, IB_KC_SETUP, 2.0 * P.np * (8 * 8 + 8 + 32 * 4));
    k_mark_rows<<<nblk(2L * P.np), TPB, 0, P.stream>>>(L.pat64, P.np, L.N, L.rowslot);
    IB_LAUNCH_CHECK();
  }
  KScope ks(P, IB_KC_SETUP, nrow * 8.0);
  k_assign_rows<<<nblk(nrow), TPB, 0, P.stream>>>(L.rowslot, nrow, L.slot_row, P.count + 1 + level);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_window_points(Problem& P) {
  LevelInfo& L = P.lev[0];
  if (L.n_rows == 0) return IB_OK;
  if (!P.rows_ready)  // the row form writes every entry; the point form adds into zeros
    IB_CUDA_TRY(cudaMemsetAsync(L.Ew64, 0, sizeof(double) * WIN * (size_t)L.n_rows, P.stream));
  Springs<double> sp;
  sp.np = P.np; sp.ns = P.ns; sp.adj_ptr = P.adj_ptr; sp.adj_spring = P.adj_spring;
  sp.adj_other = P.adj_other; sp.K = P.K64;
  KScope ks(P, IB_KC_SETUP, 0.0);
  if (P.rows_ready)  // one writer per row half: a fixed summation order
    k_window_rows<<<(L.n_rows + WROWS - 1) / WROWS, 32 * WROWS, 0, P.stream>>>(L.slot_row, L.n_rows, L.N, P.rc_start, P.rc_pt,
                                                             P.rc_w, L.pat64, sp, L.Ew64, P.dev_err);
  else
    k_window_points<<<nblk(256L * P.np), TPB, 0, P.stream>>>(L.pat64, sp, L.N, L.rowslot, L.Ew64, P.dev_err);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

// Level-0 row lists (Problem::rows_ready): count the entries of each structure row,
// scan, fill, sort each row by point.
int launch_row_lists(Problem& P) {
  LevelInfo& L = P.lev[0];
  P.rows_ready = false;
  if (!P.row_lists || !P.rc_pt || L.n_rows == 0) return IB_OK;
  if (P.cap_rc < L.n_rows) {
    dfree(P.rc_start);
    dfree(P.rc_cnt);
    P.cap_rc = L.cap_rows > L.n_rows ? L.cap_rows : L.n_rows;
    IB_TRY(dalloc(&P.rc_start, (size_t)P.cap_rc + 1));
    IB_TRY(dalloc(&P.rc_cnt, (size_t)P.cap_rc));
  }
  const int nr = L.n_rows;
  KScope ks(P, IB_KC_SETUP, 32.0 * P.np * 40.0);
  IB_CUDA_TRY(cudaMemsetAsync(P.rc_cnt, 0, sizeof(int) * nr, P.stream));
  k_rc_count<<<nblk(32L * P.np), TPB, 0, P.stream>>>(L.pat64, P.np, L.N, L.rowslot, P.rc_cnt, P.dev_err);
  IB_LAUNCH_CHECK();
  k_scan_block<<<1, 1024, 0, P.stream>>>(P.rc_cnt, nr, P.rc_start);
  IB_LAUNCH_CHECK();
  IB_CUDA_TRY(cudaMemsetAsync(P.rc_cnt, 0, sizeof(int) * nr, P.stream));
  k_rc_fill<<<nblk(32L * P.np), TPB, 0, P.stream>>>(L.pat64, P.np, L.N, L.rowslot, P.rc_start, P.rc_cnt,
                                                    P.rc_pt, P.rc_w);
  IB_LAUNCH_CHECK();
  k_rc_sort<<<nblk(nr), TPB, 0, P.stream>>>(P.rc_start, nr, P.rc_pt, P.rc_w);
  IB_LAUNCH_CHECK();
  P.rows_ready = true;
  return IB_OK;
}

// y[row] += scale * (S vals)[row] on the level-0 structure rows by the row lists.
int launch_spread_rows(Problem& P, const double* vals, long sk, long sc, double scale, double* y) {
  LevelInfo& L = P.lev[0];
  if (L.n_rows == 0) return IB_OK;
  KScope ks(P, IB_KC_SPREAD, (double)L.n_rows * 24.0 + 32.0 * P.np * 20.0);
  k_spread_rows<<<nblk(L.n_rows), TPB, 0, P.stream>>>(L.slot_row, L.n_rows, L.N, P.rc_start, P.rc_pt, P.rc_w,
                                                       vals, sk, sc, scale, y);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_window_galerkin(Problem& P, int level) {
  LevelInfo& F = P.lev[level - 1];
  LevelInfo& C = P.lev[level];
  if (C.n_rows == 0) return IB_OK;
  if (F.n_rows > 0) {
    KScope ks(P, IB_KC_SETUP, (double)F.n_rows * (WIN + TWIN) * 8.0);
    k_window_EP<<<nblk((long)F.n_rows * TWIN), TPB, 0, P.stream>>>(F.slot_row, F.n_rows, F.N, F.Ew64, P.Twin,
                                                                    P.prm.walls);
    IB_LAUNCH_CHECK();
  }
  KScope ks(P, IB_KC_SETUP, (double)C.n_rows * (6.0 * TWIN + WIN) * 8.0);
  k_window_R<<<nblk((long)C.n_rows * WIN), TPB, 0, P.stream>>>(C.slot_row, C.n_rows, C.N, F.rowslot, P.Twin,
                                                                C.Ew64, P.prm.walls);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_struct_from_windows(Problem& P, int level) {
  LevelInfo& L = P.lev[level];
  if (L.n_form == 0 || L.n_rows == 0) return IB_OK;
  const int nv = 2 * P.prm.box * (P.prm.box + 1);
  const double coef = P.prm.dt / (P.lev[0].h * P.lev[0].h);
  KScope ks(P, IB_KC_SETUP, (double)L.n_form * nv * (WIN * 8.0 + 8.0 * nv));
  k_struct_from_windows<<<nblk((long)L.n_form * nv), TPB, 0, P.stream>>>(
      L.box_of_slot, L.n_form, L.N, P.prm.box, L.rowslot, L.Ew64, coef, L.Mstruct, P.nB);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_coarse_from_windows(Problem& P) {
  LevelInfo& L = P.lev[P.nlev - 1];
  if (L.n_rows == 0) return IB_OK;
  const double coef = P.prm.dt / (P.lev[0].h * P.lev[0].h);
  KScope ks(P, IB_KC_SETUP, (double)L.n_rows * WIN * 16.0);
  k_coarse_from_windows<<<nblk(L.n_rows), TPB, 0, P.stream>>>(L.slot_row, L.n_rows, L.N, L.Ew64, coef, P.Mcoarse,
                                                               P.nc + P.nborder);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

int launch_window_cast(Problem& P, int level) {
  LevelInfo& L = P.lev[level];
  if (L.n_rows == 0 || !L.Ew32) return IB_OK;
  const long n = (long)L.n_rows * WIN;
  KScope ks(P, IB_KC_SETUP, n * 12.0);
  k_window_cast<<<nblk(n), TPB, 0, P.stream>>>(L.Ew64, L.Ew32, n);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

template <typename T>
const T* window_of(const LevelInfo& L);
template <>
const double* window_of<double>(const LevelInfo& L) { return L.Ew64; }
template <>
const float* window_of<float>(const LevelInfo& L) { return L.Ew32; }

// y += coef * E_l w on the structure rows of colour `color` (-1: all).  A colour
// holds about a third of the rows (those of its boxes and the faces it shares):
// half the row capacity in warps, striding when a colour holds more.
template <typename T>
int launch_window_apply(Problem& P, int level, const T* w, T* y, double coef, int color, bool pdl) {
  LevelInfo& L = P.lev[level];
  if (L.cap_rows == 0) return IB_OK;
  const double sT = sizeof(T);
  // per row: its window, the gathered w values and the read-modify-write of y
  const double rows = color < 0 ? L.n_rows : L.n_rows / 3.0;
  KScope ks(P, IB_KC_SPREAD, rows * (WIN * 2.0 * sT + 2 * sT + 4));
  const long warps = color < 0 ? (long)L.cap_rows : ((long)L.cap_rows + 1) / 2;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nblk(32L * warps));
  cfg.blockDim = dim3(TPB);
  cfg.stream = P.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  IB_CUDA_TRY(cudaLaunchKernelEx(&cfg, kv_window_apply<T>, (const int*)L.slot_row, (const int*)(P.count + 1 + level),
                                 (const int*)L.crow, (const int*)L.ccount, L.cap_rows, window_of<T>(L), w, L.N,
                                 (T)coef, color, (int)P.prm.walls, y));
  return IB_OK;
}

int launch_color_rows(Problem& P, int level) {
  LevelInfo& L = P.lev[level];
  const int nr = L.n_rows;
  if (!L.crow) return IB_OK;
  IB_CUDA_TRY(cudaMemsetAsync(L.ccount, 0, 4 * sizeof(int), P.stream));
  if (nr == 0) return IB_OK;
  KScope ks(P, IB_KC_SETUP, nr * 24.0);
  k_color_append<<<nblk(nr), TPB, 0, P.stream>>>(L.slot_row, nr, L.N, P.prm.box, (int)P.prm.walls, L.cap_rows,
                                                 L.crow, L.ccount);
  IB_LAUNCH_CHECK();
  return IB_OK;
}

template int launch_window_apply<double>(Problem&, int, const double*, double*, double, int, bool);
template int launch_window_apply<float>(Problem&, int, const float*, float*, double, int, bool);

}  // namespace ib
