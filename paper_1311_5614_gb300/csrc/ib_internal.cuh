// Internal declarations shared by the translation units of the library.
//
// Grid conventions (periodic N x N MAC grid, vector [u | v | p], x fastest):
//   u[j*N + i] at (i h, (j + 1/2) h)      -- face normal to x
//   v[j*N + i] at ((i + 1/2) h, j h)      -- face normal to y
//   p[j*N + i] at ((i + 1/2) h, (j + 1/2) h)
// For u the x direction is "normal" (faces on integer positions) and y is
// "centred"; for v the roles are exchanged.  All index arithmetic wraps with
// & (N - 1) because every level size is a power of two.
#pragma once

#include <cstdlib>

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/ib.h"

namespace ib {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
#define IB_CUDA_TRY(expr)                                                        \
  do {                                                                           \
    cudaError_t _e = (expr);                                                     \
    if (_e != cudaSuccess)                                                       \
      return ::ib::fail(IB_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)
#define IB_TRY(...)                \
  do {                             \
    int _s = (__VA_ARGS__);        \
    if (_s != IB_OK) return _s;    \
  } while (0)
#define IB_LAUNCH_CHECK() IB_CUDA_TRY(cudaGetLastError())

// Device error flags (bit mask, one word per problem).
enum : int {
  DEV_ERR_SINGULAR = 1,
  DEV_ERR_INDEX = 2,
  DEV_ERR_NONFINITE = 4,
  DEV_ERR_TIMEOUT = 8,
  DEV_ERR_WINDOW = 16,  // a coupling outside the assembled rows' windows (not an error: point path)
  DEV_ERR_WALL = 32     // a point whose kernel support reaches a no-slip wall
};

// Assembled elasticity rows (ib_windows.cu): per structure row, the entries at
// column offsets |di|, |dj| <= WR for both column components; the Galerkin product
// keeps E_l P per fine row at coarse offsets |dI|, |dJ| <= TR.
constexpr int WR = 5, WD = 2 * WR + 1, WSQ = WD * WD, WIN = 2 * WSQ;
constexpr int TR = 3, TD = 2 * TR + 1, TWIN = 2 * TD * TD;

// ---------------------------------------------------------------- patches
// Per level and point: for kind (0 spread, 1 interp) and component (0 u, 1 v)
// a 4 x 4 tensor-product patch: base (x0, y0) and 1-D weights wx[4], wy[4].
// Level 0 weights are phi(.) (dimensionless); coarse levels hold R applied to
// the spread weights and P^T applied to the interp weights (Galerkin, sec. 3.2).
constexpr int PATCH = 4;
template <typename T>
struct Patches {
  int np = 0;
  int* base = nullptr;  // [kind][comp][xy][np]
  T* w = nullptr;       // [kind][comp][xy][4][np]
  __host__ __device__ int b_at(int kind, int comp, int xy, int k) const {
    return base[((kind * 2 + comp) * 2 + xy) * np + k];
  }
  __host__ __device__ T w_at(int kind, int comp, int xy, int a, int k) const {
    return w[((((kind * 2 + comp) * 2 + xy) * PATCH) + a) * np + k];
  }
  __host__ __device__ int* b_ptr(int kind, int comp, int xy, int k) {
    return base + ((kind * 2 + comp) * 2 + xy) * np + k;
  }
  __host__ __device__ T* w_ptr(int kind, int comp, int xy, int a, int k) {
    return w + ((((kind * 2 + comp) * 2 + xy) * PATCH) + a) * np + k;
  }
};

// Springs in the point-adjacency form used by J U:  (J U)_k = sum over springs s
// at k of K_s (U_other - U_k), K_s the symmetric 2 x 2 block (kxx, kxy, kyy).
template <typename T>
struct Springs {
  int np = 0, ns = 0;
  const int* adj_ptr = nullptr;    // [np + 1]
  const int* adj_spring = nullptr; // [2 ns]
  const int* adj_other = nullptr;  // [2 ns]
  const T* K = nullptr;            // [3][ns]
};

// Stokes coefficients of one level: diag = -4 mu / h^2 - rho / dt, off = mu / h^2, g = 1 / h.
// walls = 1: the no-slip square (IB_WALLS_NOSLIP): the faces u(0, j) and v(i, 0) are
// the walls x = 0 (= x = 1 after the wrap) and y = 0 (= y = 1); they hold zero and
// their rows are the identity.  A tangential row next to a wall sees the ghost value
// minus itself instead of the wrapped neighbour.
template <typename T>
struct StokesCoef {
  T diag, off, g;
  int walls = 0;
};

// Whether (comp, i, j) is a wall face of a level with no-slip walls.
__host__ __device__ inline bool wall_face(int comp, int i, int j) {
  return (comp == 0 && i == 0) || (comp == 1 && j == 0);
}

// ---------------------------------------------------------------- device helpers
__host__ __device__ inline int wrapi(int i, int N) { return i & (N - 1); }

// Box-local unknown numbering of a b x b box with lower-left cell (x0, y0):
//   u faces (ir in [0, b], jr in [0, b)):  q = jr (b + 1) + ir
//   v faces (ir in [0, b), jr in [0, b]):  q = b (b + 1) + jr b + ir
//   cells   (ir, jr in [0, b)):            q = 2 b (b + 1) + jr b + ir
__host__ __device__ inline int box_nunk(int b) { return 2 * b * (b + 1) + b * b; }
__device__ inline int box_local(int comp, int i, int j, int x0, int y0, int b, int N) {
  int ir = (i - x0) & (N - 1), jr = (j - y0) & (N - 1);
  if (comp == 0) return (ir <= b && jr < b) ? jr * (b + 1) + ir : -1;
  if (comp == 1) return (ir < b && jr <= b) ? b * (b + 1) + jr * b + ir : -1;
  return (ir < b && jr < b) ? 2 * b * (b + 1) + jr * b + ir : -1;
}
__device__ inline void box_unknown(int q, int b, int x0, int y0, int N, int* comp, int* i, int* j) {
  int nu = b * (b + 1);
  if (q < nu) {
    *comp = 0; *i = x0 + q % (b + 1); *j = y0 + q / (b + 1);
  } else if (q < 2 * nu) {
    q -= nu; *comp = 1; *i = x0 + q % b; *j = y0 + q / b;
  } else {
    q -= 2 * nu; *comp = 2; *i = x0 + q % b; *j = y0 + q / b;
  }
  *i &= (N - 1);
  *j &= (N - 1);
}

// Entry A_S[(ca, ia, ja), (cb, ib, jb)] of the MAC Stokes operator
// [[mu Lap - rho/dt, -G], [D, 0]] of one level (N >= 4): periodic, or with no-slip
// walls (c.walls), where a wall face's row is the identity, no other row reads a
// wall face, and a tangential row next to a wall takes -off onto its diagonal (the
// ghost) instead of the wrapped neighbour.
__device__ inline double stokes_entry(const StokesCoef<double>& c, int N, int ca, int ia, int ja,
                                      int cb, int ib, int jb) {
  if (c.walls) {
    if (ca < 2 && wall_face(ca, ia, ja)) return (cb == ca && ib == ia && jb == ja) ? 1.0 : 0.0;
    if (cb < 2 && wall_face(cb, ib, jb)) return 0.0;
  }
  int di = (ib - ia) & (N - 1), dj = (jb - ja) & (N - 1);
  double v = 0.0;
  if (ca < 2) {
    if (cb == ca) {
      // tangential neighbours across a wall: u rows j = 0 and N - 1, v rows i = 0 and N - 1
      const int t = (ca == 0) ? ja : ia;
      const bool lo_wall = c.walls && t == 0, hi_wall = c.walls && t == N - 1;
      const int dn = (ca == 0) ? di : dj, dt = (ca == 0) ? dj : di;  // normal / tangential offsets
      if (dn == 0 && dt == 0) v += c.diag - (lo_wall ? c.off : 0.0) - (hi_wall ? c.off : 0.0);
      if (dt == 0 && dn == 1) v += c.off;
      if (dt == 0 && dn == N - 1) v += c.off;
      if (dn == 0 && dt == 1 && !hi_wall) v += c.off;
      if (dn == 0 && dt == N - 1 && !lo_wall) v += c.off;
    } else if (cb == 2) {
      // (G p) on a u face (i, j) = (p_{i,j} - p_{i-1,j}) / h; on a v face with j - 1.
      if (di == 0 && dj == 0) v -= c.g;
      if (ca == 0 && di == N - 1 && dj == 0) v += c.g;
      if (ca == 1 && di == 0 && dj == N - 1) v += c.g;
    }
  } else {
    // (D w)_{i,j} = (u_{i+1,j} - u_{i,j} + v_{i,j+1} - v_{i,j}) / h
    if (cb == 0 && dj == 0) {
      if (di == 1) v += c.g;
      if (di == 0) v -= c.g;
    } else if (cb == 1 && di == 0) {
      if (dj == 1) v += c.g;
      if (dj == 0) v -= c.g;
    }
  }
  return v;
}

constexpr int MAX_LEVELS_ALLOC = 32;  // per-level device counters

// ---------------------------------------------------------------- problem state
template <typename T>
struct LevelBuf {
  T* w = nullptr;  // iterate / correction
  T* b = nullptr;  // right-hand side
  T* r = nullptr;  // residual scratch
};

struct LevelInfo {
  int N = 0;
  double h = 0.0;
  int nb = 0;          // boxes per side (smoothing levels)
  int n_struct = 0;    // structure boxes found at the last set-up (slots in use)
  int n_form = 0;      // of them formed and inverted at each set-up: slots [0, n_form); slots
                       // [n_form, n_struct) are no-slip wall boxes without elasticity, whose
                       // inverses are copied from Mring
  int cap_struct = 0;  // allocated structure-box slots
  double* Mring = nullptr;  // no-slip walls: [4 (nb - 1)][nB * nB] inverses of the wall boxes
  int nring = 0;            // (their blocks depend on the grid only: computed once)
  int* flag = nullptr;        // [nb * nb] structure flag -> slot (-1 free)
  double* Mstruct = nullptr;  // [cap][nB * nB] inverse (column-major), FP64
  double* Sfree = nullptr;    // [nB * nB] Stokes block of a box (column-major), FP64
  double* Mfree = nullptr;    // [nB * nB] shared inverse of structure-free boxes, FP64
  float* Mfree32 = nullptr;   // FP32 copy for the FP32 V-cycle
  // elasticity residual part -dt E_l w of the V-cycle, [2 N^2]: zero between
  // uses (each colour phase adds to its own rows and the box solves take the
  // values back out; prolongation clears what the restriction used)
  double* rE64 = nullptr;
  float* rE32 = nullptr;
  Patches<double> pat64;      // FP64 patches (operator path)
  Patches<float> pat32;       // FP32 patches (FP32 V-cycle)
  LevelBuf<double> v64;
  LevelBuf<float> v32;
  int* box_of_slot = nullptr;  // [cap_struct] box index of each structure slot
  // assembled elasticity rows: rowslot [2 N^2] (row -> slot or -1), slot_row [2 N^2]
  // (slot -> row c N^2 + j N + i), windows [cap_rows][WIN] in FP64 and FP32
  int* rowslot = nullptr;
  int* slot_row = nullptr;
  int n_rows = 0, cap_rows = 0;
  // the structure rows (slots) of each colour, rebuilt at every set-up: colour c's
  // list is crow[c cap_rows ...], ccount[c] long
  int* crow = nullptr;
  int* ccount = nullptr;
  double* Ew64 = nullptr;
  float* Ew32 = nullptr;
};

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
  double bytes;
};

struct Problem {
  ib_params prm{};
  // launch accounting / event timing
  long long nlaunch[IB_KC_COUNT] = {};
  bool prof = false;
  long long prof_n[IB_KC_COUNT] = {};
  double prof_ms[IB_KC_COUNT] = {};
  double prof_bytes[IB_KC_COUNT] = {};
  std::vector<cudaEvent_t> ev_pool;
  std::vector<ProfRec> pending;
  // V-cycle timer: an event pair around every V-cycle replayed from its graph
  bool vt_on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> vt_pending;
  long long vt_n[2] = {0, 0};   // timed V-cycles: [0] FP32 V-cycle, [1] V-cycle on FP64 vectors
  double vt_ms[2] = {0.0, 0.0};
  std::vector<int> vt_kind;
  // V-cycle engine
  // index [0] = FP32 V-cycle, [1] = FP64 V-cycle
  int tail_level[2] = {0, 0};    // first level handled by the tail kernel
  int tail_cluster[2] = {0, 0};  // CTAs of its cluster (0: one CTA, arrays in shared memory)
  bool use_graph = true;
  bool graph_dirty[2] = {true, true};
  cudaGraphExec_t vgraph[2] = {nullptr, nullptr};
  bool has64 = false, has32 = false;  // hierarchies available for the V-cycle
  long box_gemm_min = 2048;           // boxes per colour from which n x n boxes use the GEMM kernel
  long box_one_max = 512;             // boxes per colour up to which each box gets its own CTA
  bool box_strip = true;             // 4 x 4 boxes: strip kernel on levels with N_l / 8 a multiple of 32
  long box_strip_min = 2048;          // ... and at least this many boxes per colour
  int box_strip_w = 0;                // strip width (8, 16 or 32; 0: chosen per level)
  // box-kernel form per V-cycle ([0] FP32, [1] on FP64 vectors) and level, chosen by timing
  // at set-up (0: the size rule above; see IB_BOXF_* in ib_vcycle.cu)
  bool box_autotune = true;
  int box_form[2][32] = {};
  int box_form_pin[32] = {};  // IB_BOX_FORMS: forms given per level (0: none given)
  bool box_form_pinned = false;
  double sigma = 0.0;                 // stiffness ratio dt * max(kappa) / mu of the structure
  double stiff_sigma = 3000.0;        // FP32 mode: from this sigma on, precondition with the mixed V-cycle
  bool inv32 = true;                  // IB_INV32=0 (read at ib_setup): structure boxes always inverted in FP64
  bool struct_inv32 = false;          // this set-up's structure-box inverses came from an FP32 elimination
  cudaStream_t gstream = nullptr;                 // private stream the graph is captured on
  long long graph_launches[2][IB_KC_COUNT] = {};
  cudaStream_t stream = nullptr;
  int np = 0, ns = 0;
  int nlev = 0;
  int nB = 0;  // unknowns per box
  bool free_ready = false;  // free-box inverses computed (they do not depend on the points)
  bool ring_ready = false;  // no-slip wall-box inverses computed (likewise)
  std::vector<LevelInfo> lev;

  // structure (device)
  double* X = nullptr;        // [np][2]
  int* springs = nullptr;     // [ns][2]
  double* kappa = nullptr;    // [ns]
  double* rest = nullptr;     // [ns]
  int* adj_ptr = nullptr;     // [np + 1]
  int* adj_spring = nullptr;  // [2 ns]
  int* adj_other = nullptr;   // [2 ns]
  double* K64 = nullptr;      // [3][ns]
  float* K32 = nullptr;       // [3][ns]
  double* F = nullptr;        // [np][2] spring force at X (gathered per point from Fs)
  double* Fs = nullptr;       // [ns][2] force of each spring on its first end
  // Newton steps (ib_solve_step_newton): the points the springs are evaluated at
  // (NULL: X), X^n, the iterate X^k, and per-point scratch
  const double* Xs = nullptr;
  double* Xn = nullptr;       // [np][2]
  double* Xk = nullptr;       // [np][2]
  double* Dk = nullptr;       // [2][np] X^k - X^n
  double* Gk = nullptr;       // [2][np] J(X^k) (X^k - X^n)
  double* U64 = nullptr;      // [2][np] interpolated velocity scratch
  double* G64 = nullptr;      // [2][np] J U per point (the operator's spread by row lists)
  // Level-0 row lists, rebuilt at every set-up with the assembled rows: for each
  // structure row (slot), the points whose spread patch covers it, in point order,
  // with their spread weight.  The right-hand side's spread, the FP64 operator's
  // spread and the level-0 row assembly gather through them, one writer per row,
  // so their sums run in a fixed order (no floating-point atomics).
  bool rows_ready = false;
  bool row_lists = true;      // IB_ROW_LISTS=0 (read at ib_setup): the scatter forms with atomics
  int cap_rc = 0;             // rows the count/start arrays hold
  int* rc_start = nullptr;    // [cap_rc + 1]
  int* rc_cnt = nullptr;      // [cap_rc]
  int* rc_pt = nullptr;       // [32 np] point of each entry
  double* rc_w = nullptr;     // [32 np] its weight phi_x phi_y
  float* U32 = nullptr;       // [2][np]

  // coarsest level
  int nc = 0;                 // 3 Nc^2
  int nborder = 0;            // null-space border columns (1 or 3)
  double* Mcoarse = nullptr;  // [(nc + nborder)^2] bordered inverse, column-major
  double* inv_ws = nullptr;   // blocked inversion: saved pivot rows, [count][16][n]
  size_t inv_ws_cap = 0;
  int* inv_perm = nullptr;    // blocked inversion: pivot rows, [count][n]
  size_t inv_perm_cap = 0;

  // Krylov (FP64)
  double* V = nullptr;        // [m + 1][n]
  void* Z = nullptr;          // [m][n] in the preconditioner precision
  double* Z64 = nullptr;      // [m][n] FP64 directions after an FP32 -> FP64 escalation
  double* H = nullptr;        // [(m + 1) * m] column-major Hessenberg
  double* givens = nullptr;   // cs[m], sn[m], g[m + 1], y[m]
  double* dots = nullptr;     // partial sums [blocks][m + 2]
  double* scal = nullptr;     // small scalars on the device
  double* scal_host = nullptr;// pinned host mirror
  double* x64 = nullptr;      // [n] solution
  double* b64 = nullptr;      // [n] rhs
  double* t64 = nullptr;      // [n] scratch
  double* t64b = nullptr;     // [n] scratch
  int* dev_err = nullptr;     // device error flags
  // learned stage
  ib_unet* net = nullptr;     // attached network (not owned)
  float* nn_sch = nullptr;    // [N^2] structure channel
  float* nn_x = nullptr;      // [4 N^2] network input
  float* nn_y = nullptr;      // [3 N^2] network output
  double* nn_r = nullptr;     // [3 N^2] residual v - A z
  double* nn_dz = nullptr;    // [3 N^2] proposed correction
  double* nn_adz = nullptr;   // [3 N^2] A dz
  int max_m = 0;
  int dot_blocks = 0;         // rows of the partial-sum buffer
  int n_sm = 0;               // SMs of the device
  int cgs_smem_max = 0;       // dynamic shared memory limit of the fused Gram-Schmidt pass
  int occ_multidot = 0;       // resident blocks per SM of the partial-dot kernel
  int occ_subnorm = 0;        // ... and of the last Gram-Schmidt subtraction
  std::vector<int> occ_cgs;   // resident blocks per SM of the fused pass, by basis size
  int occ_cgs_reg[2] = {0, 0};  // ... of its register form for bases of <= 8 and <= 16 vectors
  bool cgs_reg = true;          // register form for bases of <= 16 vectors (IB_CGS_REG=0: off)
  bool cgs_fused = true;      // middle Gram-Schmidt step as one fused pass
  unsigned long long wait_limit_ns = 1000000000ull;  // bounded device-side waits (IB_WAIT_LIMIT_NS)
  int* count = nullptr;       // device counters: [0] structure boxes, [1 + l] structure rows of level l
  bool windows = true;        // assembled elasticity rows available (IB_WINDOWS=0: point path only)
  bool win_step = false;      // this step's hierarchy uses them (no coupling fell outside a window)
  double* Twin = nullptr;     // Galerkin scratch [cap_twin][TWIN]
  int cap_twin = 0;
  int* count_host = nullptr;  // pinned

  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t pev[2] = {nullptr, nullptr};  // FGMRES pipeline: scalars of iterations j, j - 1
};

// Launch scope: counts the launch of one kernel of class cls and, while
// profiling is on, brackets it with CUDA events on the problem's stream.
struct KScope {
  Problem& P;
  int cls;
  double bytes;
  cudaEvent_t a = nullptr;
  KScope(Problem& P_, int cls_, double bytes_);
  ~KScope();
};

// Whether new device allocations are filled with all-ones bytes (NaN as float or
// double, -1 as int): IB_POISON=1 in the environment, for tests that look for
// reads of memory nothing has written.
inline bool poison_allocations() {
  static const bool on = [] {
    const char* e = std::getenv("IB_POISON");
    return e && e[0] == '1';
  }();
  return on;
}

// Device allocation with the library's error reporting (count 0: NULL).
template <typename T>
int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return IB_OK;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaSuccess && poison_allocations()) e = cudaMemset((void*)*p, 0xFF, count * sizeof(T));
  if (e != cudaSuccess) {
    if (*p) cudaFree((void*)*p);
    *p = nullptr;
    cudaGetLastError();
    return fail(IB_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  return IB_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// ---------------------------------------------------------------- launchers (points)
int launch_fine_patches(Problem& P);
int launch_coarse_patches(Problem& P, int level);
int launch_cast_patches(Problem& P, int level);
int launch_spring_force_jacobian(Problem& P);
// F <- F - J (X^k - X^n) at the Newton iterate (F and J evaluated at P.Xs = X^k).
int launch_newton_force(Problem& P);
int launch_spread_force(Problem& P, double* b);  // b_vel -= S F
int launch_move_points(Problem& P, const double* up);
template <typename T>
int launch_elastic(Problem& P, int level, const T* w, T* y, double coef, T* U);
int launch_mark_struct(Problem& P, int level);

int launch_assemble_struct(Problem& P, int level);
int launch_mark_rows(Problem& P, int level);
int launch_window_points(Problem& P);
int launch_window_galerkin(Problem& P, int level);
int launch_struct_from_windows(Problem& P, int level);
int launch_coarse_from_windows(Problem& P);
int launch_window_cast(Problem& P, int level);
// The colour lists of a level's structure rows (LevelInfo::crow, ccount).
int launch_color_rows(Problem& P, int level);
template <typename T>
int launch_window_apply(Problem& P, int level, const T* w, T* y, double coef, int color, bool pdl);
int launch_assemble_coarse(Problem& P);

// ---------------------------------------------------------------- launchers (grid)
template <typename T>
int launch_stokes(Problem& P, int level, const T* w, const T* b, T* out, bool residual);
int launch_free_box(Problem& P, int level);
int launch_struct_fill(Problem& P, int level);
// fp32: matrices too large for shared memory are eliminated in FP32 (the inverses
// stored in FP64); the others in FP64 regardless.
int launch_invert(Problem& P, double* M, int n, int count, bool fp32 = false);
int launch_invert_struct_all(Problem& P, bool* done, bool fp32 = false);
int launch_coarse_fill(Problem& P);
template <typename T>
int launch_fill(Problem& P, T* x, size_t n, T v);
template <typename A, typename B>
int launch_cast(Problem& P, const A* x, B* y, size_t n);

// ---------------------------------------------------------------- learned stage
int learned_struct_channel(Problem& P);
int learned_features(Problem& P, const double* r, double* scratch, double* nrm2, float* x);
int learned_scale_out(Problem& P, const float* y, const double* nrm2, double* dz);
int learned_target(Problem& P, const double* e, const double* nrm2, float* t);
int learned_forward(ib_unet* U, cudaStream_t s, const float* x, float* y);
int learned_unet_size(const ib_unet* U);

// ---------------------------------------------------------------- launchers (krylov)
int launch_multidot(Problem& P, const double* V, int nvec, const double* w, double* out);
int launch_multiaxpy(Problem& P, const double* V, int nvec, const double* coef, double* w);
int launch_dot(Problem& P, const double* a, const double* b, double* out);
int launch_scale_copy(Problem& P, const double* x, const double* s, double* y, bool invert);
int launch_cgs_sub_dot(Problem& P, const double* V, int nvec, const double* coef, double* w, double* out);
int launch_cgs_finish(Problem& P, const double* V, int nvec, double* w, int j);
int krylov_init(Problem& P);
int launch_backsolve(Problem& P, int k);
template <typename T>
int launch_update_x(Problem& P, const T* Z, int k, double* x, int first = 0);
int launch_axpby(Problem& P, double a, const double* x, double b, const double* y, double* z);
int launch_pressure_mean_remove(Problem& P, double* w);
// Whether the operator carries the elasticity block: a structure, and the implicit
// method (IB_EXPLICIT keeps the structure's force on the right-hand side only).
inline bool op_elastic(const Problem& P) { return P.np > 0 && P.ns > 0 && P.prm.time_method == IB_IMPLICIT; }
int launch_zero_walls(Problem& P, double* w);  // no-slip walls: w = 0 on the wall faces
int launch_ring_prepare(Problem& P, int level); // ... the wall boxes' inverses (once)
int launch_row_lists(Problem& P);               // level-0 row lists (see Problem::rows_ready)
int launch_spread_rows(Problem& P, const double* vals, long sk, long sc, double scale, double* y);
int launch_ring_copy(Problem& P, int level);    // ... into their slots (every set-up)
int launch_wall_rhs(Problem& P, double* b);    // ... and the moving lid's ghost term

}  // namespace ib
