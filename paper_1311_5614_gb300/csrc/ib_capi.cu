// Host side of the C ABI: validation, workspace, hierarchy set-up, the V-cycle
// of Algorithm 1 and the flexible GMRES driver of sec. 3.3.  Every arithmetic
// step runs in the kernels of the other translation units; this file only
// orders launches on the problem's stream and reads back the few scalars that
// decide control flow (structure-box counts, Krylov residual estimates).
#include <algorithm>
#include <atomic>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "ib_internal.cuh"
#include "ib_vcycle.cuh"

namespace ib {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

KScope::KScope(Problem& P_, int cls_, double bytes_) : P(P_), cls(cls_), bytes(bytes_) {
  ++P.nlaunch[cls];
  if (!P.prof) return;
  if (P.ev_pool.empty()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    P.ev_pool.push_back(e);
  }
  a = P.ev_pool.back();
  P.ev_pool.pop_back();
  cudaEventRecord(a, P.stream);
}

KScope::~KScope() {
  if (!P.prof || !a) return;
  cudaEvent_t b;
  if (!P.ev_pool.empty()) {
    b = P.ev_pool.back();
    P.ev_pool.pop_back();
  } else if (cudaEventCreate(&b) != cudaSuccess) {
    P.ev_pool.push_back(a);
    return;
  }
  cudaEventRecord(b, P.stream);
  P.pending.push_back(ProfRec{cls, a, b, bytes});
}

// Fold the pending event pairs into the per-class accumulators.
static int resolve_profile(Problem& P) {
  if (P.pending.empty()) return IB_OK;
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  for (auto& r : P.pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    P.prof_n[r.cls] += 1;
    P.prof_ms[r.cls] += ms;
    P.prof_bytes[r.cls] += r.bytes;
    P.ev_pool.push_back(r.a);
    P.ev_pool.push_back(r.b);
  }
  P.pending.clear();
  return IB_OK;
}
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

namespace {


bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// The elastic block dt S J S^* scales like dt kappa / h^2 against mu / h^2 for
// the viscous one, so sigma = dt max(kappa) / mu measures how stiff the step is,
// independently of h.  Measured on the 256^2 sweep: sigma = 1e3 converges with
// the FP32 V-cycle like FP64, sigma = 1e4 stalls it.
double stiffness(const ib_params& p, int n_springs, const double* kappa) {
  double kmax = 0.0;
  for (int s = 0; s < n_springs; ++s) kmax = std::max(kmax, kappa[s]);
  return p.dt * kmax / p.mu;
}

double stiff_threshold() {
  const char* e = std::getenv("IB_STIFF_SIGMA");
  return e ? std::atof(e) : 3000.0;
}

int validate(const ib_params* p) {
  if (!p) return fail(IB_ERR_INVALID_ARG, "params is NULL");
  if (!(p->box == 1 || p->box == 2 || p->box == 4 || p->box == 8 || p->box == 16))
    return fail(IB_ERR_INVALID_ARG, "box must be 1, 2, 4, 8 or 16");
  int nc = p->box > 4 ? p->box : 4;
  if (!is_pow2(p->N) || p->N < 2 * nc || p->N > (1 << 14))
    return fail(IB_ERR_INVALID_ARG, "N must be a power of two with 2*max(4, box) <= N <= 16384");
  if (!(std::isfinite(p->L) && p->L > 0)) return fail(IB_ERR_INVALID_ARG, "L must be > 0");
  if (!(std::isfinite(p->mu) && p->mu > 0)) return fail(IB_ERR_INVALID_ARG, "mu must be > 0");
  if (!(std::isfinite(p->dt) && p->dt > 0)) return fail(IB_ERR_INVALID_ARG, "dt must be > 0");
  if (!(std::isfinite(p->rho) && p->rho >= 0)) return fail(IB_ERR_INVALID_ARG, "rho must be >= 0");
  if (p->delta != IB_DELTA_PESKIN4 && p->delta != IB_DELTA_COS4)
    return fail(IB_ERR_INVALID_ARG, "unknown delta kernel");
  if (p->precision != IB_FP64 && p->precision != IB_FP32_PRECOND && p->precision != IB_MIXED_PRECOND)
    return fail(IB_ERR_INVALID_ARG, "unknown precision");
  if (p->jacobian != IB_JAC_CLAMPED && p->jacobian != IB_JAC_EXACT)
    return fail(IB_ERR_INVALID_ARG, "unknown jacobian variant");
  if (p->nu1 < 0 || p->nu1 > 8 || p->nu2 < 0 || p->nu2 > 8)
    return fail(IB_ERR_INVALID_ARG, "nu1, nu2 must be in 0..8");
  if (!(std::isfinite(p->tol) && p->tol > 0)) return fail(IB_ERR_INVALID_ARG, "tol must be > 0");
  if (p->max_iters < 1 || p->max_iters > 512)
    return fail(IB_ERR_INVALID_ARG, "max_iters must be in 1..512");
  if (p->escalate != 0 && p->escalate != 1) return fail(IB_ERR_INVALID_ARG, "escalate must be 0 or 1");
  if (p->restart < 0 || p->restart > 512) return fail(IB_ERR_INVALID_ARG, "restart must be in 0..512");
  if (p->time_method != IB_IMPLICIT && p->time_method != IB_EXPLICIT)
    return fail(IB_ERR_INVALID_ARG, "time_method must be IB_IMPLICIT or IB_EXPLICIT");
  if (p->walls != IB_WALLS_PERIODIC && p->walls != IB_WALLS_NOSLIP)
    return fail(IB_ERR_INVALID_ARG, "walls must be IB_WALLS_PERIODIC or IB_WALLS_NOSLIP");
  if (!std::isfinite(p->lid) || (p->lid != 0.0 && p->walls != IB_WALLS_NOSLIP))
    return fail(IB_ERR_INVALID_ARG, "lid must be finite, and 0 without no-slip walls");
  return IB_OK;
}

double efac(const Problem& P) { return P.prm.dt / (P.lev[0].h * P.lev[0].h); }

__global__ void k_set(double* dst, double v) { *dst = v; }

__global__ void k_axpy_n(double a, const double* __restrict__ x, double* y, long n) {
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e < n) y[e] += a * x[e];
}

// y = A_l w in FP64.  The elasticity of a coarse level with no-slip walls comes from
// its assembled rows (the per-point coarse patches are periodic Galerkin products).
int apply64(Problem& P, int l, const double* w, double* y) {
  IB_TRY(launch_stokes<double>(P, l, w, nullptr, y, false));
  if (P.prm.walls && l > 0) {
    if (op_elastic(P)) IB_TRY(launch_window_apply<double>(P, l, w, y, efac(P), -1, false));
    return IB_OK;
  }
  IB_TRY(launch_elastic<double>(P, l, w, y, efac(P), P.U64));
  return IB_OK;
}

int check_dev_err(Problem& P) {
  int h = 0;
  IB_CUDA_TRY(cudaMemcpyAsync(P.count_host + 64, P.dev_err, sizeof(int), cudaMemcpyDeviceToHost,
                              P.stream));
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  h = P.count_host[64];
  if (h) {
    IB_CUDA_TRY(cudaMemsetAsync(P.dev_err, 0, sizeof(int), P.stream));
    if (h & DEV_ERR_NONFINITE)
      return fail(IB_ERR_INVALID_ARG, "a spring has coincident or non-finite end points");
    if (h & DEV_ERR_SINGULAR) return fail(IB_ERR_SINGULAR, "zero pivot in a box or coarsest factorisation");
    if (h & DEV_ERR_TIMEOUT) return fail(IB_ERR_TIMEOUT, "a bulk copy of the Krylov basis did not complete");
    if (h & DEV_ERR_WALL)
      return fail(IB_ERR_INVALID_ARG, "a point is closer than 2h to a no-slip wall (its kernel reaches the wall)");
    return fail(IB_ERR_INVALID_ARG, "internal index check failed (too many springs at a point?)");
  }
  return IB_OK;
}

// IB_INV32=2: the FP32 elimination for every step of the FP32 and mixed V-cycles,
// stiff ones included, and no FP64 re-forming when a solve escalates.
bool inv32_always() {
  const char* e = std::getenv("IB_INV32");
  return e && e[0] == '2';
}

// Re-form S, J and everything that depends on them (per step, sec. 8).  With the
// assembled elasticity rows (ib_windows.cu): mark the structure boxes and rows of
// every level and read their counts (one synchronisation), assemble the level-0 rows
// from the points, check that no coupling fell outside a row's window (a second
// synchronisation; otherwise this step keeps the point-based path), coarsen the rows
// level by level, and read the structure-box blocks and the coarsest matrix out of
// them.
int setup_hierarchy(Problem& P) {
  IB_TRY(launch_fine_patches(P));
  IB_TRY(launch_spring_force_jacobian(P));
  for (int l = 1; l < P.nlev; ++l) IB_TRY(launch_coarse_patches(P, l));
  if (P.prm.precision == IB_FP32_PRECOND)
    for (int l = 0; l < P.nlev; ++l) IB_TRY(launch_cast_patches(P, l));
  const int ns = P.nlev - 1;  // smoothing levels
  const bool win = P.windows && op_elastic(P);
  for (int l = 0; l < ns; ++l) {
    IB_TRY(launch_mark_struct(P, l));
    IB_CUDA_TRY(cudaMemcpyAsync(P.count_host + l, P.count, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
  }
  if (P.prm.walls)  // wall boxes without elasticity, per level
    IB_CUDA_TRY(cudaMemcpyAsync(P.count_host + 65, P.count + 1 + MAX_LEVELS_ALLOC, sizeof(int) * ns,
                                cudaMemcpyDeviceToHost, P.stream));
  if (win) {
    for (int l = 0; l < P.nlev; ++l) IB_TRY(launch_mark_rows(P, l));
    IB_CUDA_TRY(cudaMemcpyAsync(P.count_host + 32, P.count + 1, sizeof(int) * P.nlev, cudaMemcpyDeviceToHost,
                                P.stream));
  }
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  const int nB = P.nB;
  for (int l = 0; l < ns; ++l) {
    LevelInfo& L = P.lev[l];
    const int ring = P.prm.walls ? P.count_host[65 + l] : 0;
    int cnt = P.count_host[l] + ring;
    L.n_form = P.count_host[l];
    if (cnt > L.cap_struct) {
      P.graph_dirty[0] = P.graph_dirty[1] = true;  // the box kernels take the new pointer
      dfree(L.Mstruct);
      int cap = cnt + cnt / 4 + 16;
      if (cap > L.nb * L.nb) cap = L.nb * L.nb;
      IB_TRY(dalloc(&L.Mstruct, (size_t)cap * nB * nB));
      L.cap_struct = cap;
    }
    L.n_struct = cnt;
  }
  int max_rows = 0;
  if (win) {
    for (int l = 0; l < P.nlev; ++l) {
      LevelInfo& L = P.lev[l];
      const int cnt = P.count_host[32 + l];
      if (cnt > L.cap_rows) {  // new storage: the captured V-cycle takes the new pointers
        P.graph_dirty[0] = P.graph_dirty[1] = true;
        dfree(L.Ew64);
        dfree(L.Ew32);
        dfree(L.crow);
        const int cap = cnt + cnt / 4 + 64;
        IB_TRY(dalloc(&L.Ew64, (size_t)cap * WIN));
        if (P.has32 || P.prm.precision == IB_FP32_PRECOND) IB_TRY(dalloc(&L.Ew32, (size_t)cap * WIN));
        IB_TRY(dalloc(&L.crow, 4ul * cap));
        if (!L.ccount) IB_TRY(dalloc(&L.ccount, 4));
        L.cap_rows = cap;
      }
      L.n_rows = cnt;
      max_rows = std::max(max_rows, cnt);
    }
    if (max_rows > P.cap_twin) {
      dfree(P.Twin);
      P.cap_twin = max_rows + max_rows / 4 + 64;
      IB_TRY(dalloc(&P.Twin, (size_t)P.cap_twin * TWIN));
    }
  }
  for (int l = 0; l < ns; ++l) {
    if (!P.free_ready) IB_TRY(launch_free_box(P, l));
    if (P.prm.walls && !P.ring_ready) IB_TRY(launch_ring_prepare(P, l));
    IB_TRY(launch_struct_fill(P, l));
  }
  if (P.prm.walls) P.ring_ready = true;
  P.rows_ready = false;
  if (win) IB_TRY(launch_row_lists(P));
  bool use_win = false;
  if (win) {
    IB_TRY(launch_window_points(P));
    IB_CUDA_TRY(cudaMemcpyAsync(P.count_host + 64, P.dev_err, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
    IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
    use_win = (P.count_host[64] & DEV_ERR_WINDOW) == 0;
    if (!use_win) {  // a coupling outside a window: this step keeps the point path
      P.count_host[64] &= ~DEV_ERR_WINDOW;
      IB_CUDA_TRY(cudaMemcpyAsync(P.dev_err, &P.count_host[64], sizeof(int), cudaMemcpyHostToDevice, P.stream));
      IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
    }
  }
  if (P.prm.walls && op_elastic(P) && !use_win)
    return fail(IB_ERR_INVALID_ARG,
                "no-slip walls need the assembled elasticity rows: a coupling leaves the row window "
                "(springs longer than about 1.5 cells) or IB_WINDOWS=0");
  if (use_win != P.win_step) P.graph_dirty[0] = P.graph_dirty[1] = true;
  P.win_step = use_win;
  if (use_win) {
    for (int l = 1; l < P.nlev; ++l) IB_TRY(launch_window_galerkin(P, l));
    for (int l = 0; l < ns; ++l) IB_TRY(launch_struct_from_windows(P, l));
    for (int l = 0; l < P.nlev; ++l) IB_TRY(launch_window_cast(P, l));
    for (int l = 0; l < P.nlev; ++l) IB_TRY(launch_color_rows(P, l));
  } else {
    for (int l = 0; l < ns; ++l) IB_TRY(launch_assemble_struct(P, l));
  }
  // a step of the FP32 V-cycle that is not stiff eliminates its structure boxes in
  // FP32 (the inverses are stored, and applied, in FP64); an escalation to the
  // mixed V-cycle re-forms them in FP64 (reform_struct64)
  const bool inv32 = P.inv32 && P.prm.precision != IB_FP64 &&
                     (inv32_always() || (P.prm.precision == IB_FP32_PRECOND && P.sigma < P.stiff_sigma));
  bool all_done = false;
  IB_TRY(launch_invert_struct_all(P, &all_done, inv32));
  const bool big = (size_t)nB * nB * sizeof(double) > 160u * 1024u;  // the blocked form (8 x 8, 16 x 16 boxes)
  P.struct_inv32 = inv32 && (all_done || big);
  if (!all_done)
    for (int l = 0; l < ns; ++l) IB_TRY(launch_invert(P, P.lev[l].Mstruct, nB, P.lev[l].n_form, inv32 && big));
  if (P.prm.walls)
    for (int l = 0; l < ns; ++l) IB_TRY(launch_ring_copy(P, l));
  P.free_ready = true;
  IB_TRY(launch_coarse_fill(P));
  if (use_win) IB_TRY(launch_coarse_from_windows(P));
  else IB_TRY(launch_assemble_coarse(P));
  IB_TRY(launch_invert(P, P.Mcoarse, P.nc + P.nborder, 1));
  IB_TRY(vcycle_reset_rE(P));
  if (P.nn_sch) IB_TRY(learned_struct_channel(P));
  return check_dev_err(P);
}

// The structure-box blocks of this step formed again and inverted in FP64, for a
// solve that escalates from the FP32 V-cycle to the mixed one after a set-up that
// eliminated them in FP32 (the same sequence as in setup_hierarchy).
int reform_struct64(Problem& P) {
  const int ns = P.nlev - 1;
  for (int l = 0; l < ns; ++l) IB_TRY(launch_struct_fill(P, l));
  if (P.win_step) {
    for (int l = 0; l < ns; ++l) IB_TRY(launch_struct_from_windows(P, l));
  } else {
    for (int l = 0; l < ns; ++l) IB_TRY(launch_assemble_struct(P, l));
  }
  bool all_done = false;
  IB_TRY(launch_invert_struct_all(P, &all_done, false));
  if (!all_done)
    for (int l = 0; l < ns; ++l) IB_TRY(launch_invert(P, P.lev[l].Mstruct, P.nB, P.lev[l].n_form));
  if (P.prm.walls)
    for (int l = 0; l < ns; ++l) IB_TRY(launch_ring_copy(P, l));
  P.struct_inv32 = false;
  return check_dev_err(P);
}

void free_problem(Problem* P) {
  if (!P) return;
  for (auto& L : P->lev) {
    dfree(L.flag); dfree(L.Mstruct); dfree(L.Sfree); dfree(L.Mfree); dfree(L.Mfree32);
    dfree(L.pat64.base); dfree(L.pat64.w); dfree(L.pat32.base); dfree(L.pat32.w);
    dfree(L.v64.w); dfree(L.v64.b); dfree(L.v64.r);
    dfree(L.v32.w); dfree(L.v32.b); dfree(L.v32.r);
    dfree(L.rE64); dfree(L.rE32);
    dfree(L.box_of_slot); dfree(L.rowslot); dfree(L.slot_row); dfree(L.Ew64); dfree(L.Ew32);
    dfree(L.crow); dfree(L.ccount);
    dfree(L.Mring);
  }
  dfree(P->Twin);
  for (auto& g : P->vgraph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
  if (P->gstream) cudaStreamDestroy(P->gstream);
  P->gstream = nullptr;
  dfree(P->X); dfree(P->springs); dfree(P->kappa); dfree(P->rest);
  dfree(P->adj_ptr); dfree(P->adj_spring); dfree(P->adj_other);
  dfree(P->K64); dfree(P->K32); dfree(P->F); dfree(P->Fs); dfree(P->U64); dfree(P->U32);
  dfree(P->Xn); dfree(P->Xk); dfree(P->Dk); dfree(P->Gk);
  dfree(P->G64); dfree(P->rc_pt); dfree(P->rc_w); dfree(P->rc_start); dfree(P->rc_cnt);
  dfree(P->Mcoarse); dfree(P->inv_ws); dfree(P->inv_perm); dfree(P->V); dfree(P->Z); dfree(P->Z64); dfree(P->H); dfree(P->givens);
  dfree(P->dots); dfree(P->scal); dfree(P->x64); dfree(P->b64); dfree(P->t64); dfree(P->t64b);
  dfree(P->dev_err); dfree(P->count);
  dfree(P->nn_sch); dfree(P->nn_x); dfree(P->nn_y); dfree(P->nn_r); dfree(P->nn_dz); dfree(P->nn_adz);
  if (P->scal_host) cudaFreeHost(P->scal_host);
  if (P->count_host) cudaFreeHost(P->count_host);
  for (auto& e : P->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : P->pev)
    if (e) cudaEventDestroy(e);
  for (auto& r : P->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto& r : P->vt_pending) {
    cudaEventDestroy(r.first);
    cudaEventDestroy(r.second);
  }
  P->vt_pending.clear();
  for (auto& e : P->ev_pool) cudaEventDestroy(e);
  P->pending.clear();
  P->ev_pool.clear();
}

int allocate(Problem& P) {
  const int nl = P.nlev;
  const bool fp32 = P.prm.precision == IB_FP32_PRECOND;
  for (int l = 0; l < nl; ++l) {
    LevelInfo& L = P.lev[l];
    size_t n3 = 3ul * L.N * L.N;
    if (P.windows && op_elastic(P)) {
      IB_TRY(dalloc(&L.rowslot, 2ul * L.N * L.N));
      IB_TRY(dalloc(&L.slot_row, 2ul * L.N * L.N));
    }
    if (l < nl - 1) {
      IB_TRY(dalloc(&L.flag, (size_t)L.nb * L.nb));
      IB_TRY(dalloc(&L.box_of_slot, (size_t)L.nb * L.nb));
      IB_TRY(dalloc(&L.Sfree, (size_t)P.nB * P.nB));
      IB_TRY(dalloc(&L.Mfree, (size_t)P.nB * P.nB));
      if (P.prm.precision != IB_FP64) IB_TRY(dalloc(&L.Mfree32, (size_t)P.nB * P.nB));
    }
    if (P.np > 0) {
      L.pat64.np = P.np;
      IB_TRY(dalloc(&L.pat64.base, 8ul * P.np));
      IB_TRY(dalloc(&L.pat64.w, 32ul * P.np));
      if (fp32) {
        L.pat32.np = P.np;
        IB_TRY(dalloc(&L.pat32.base, 8ul * P.np));
        IB_TRY(dalloc(&L.pat32.w, 32ul * P.np));
      }
    }
    if (fp32) {
      IB_TRY(dalloc(&L.v32.w, n3)); IB_TRY(dalloc(&L.v32.b, n3)); IB_TRY(dalloc(&L.v32.r, n3));
      IB_TRY(dalloc(&L.rE32, 2ul * L.N * L.N));
    }
    if (!fp32 || P.prm.escalate) {
      IB_TRY(dalloc(&L.v64.w, n3)); IB_TRY(dalloc(&L.v64.b, n3)); IB_TRY(dalloc(&L.v64.r, n3));
      IB_TRY(dalloc(&L.rE64, 2ul * L.N * L.N));
    }
  }
  int np = P.np, ns = P.ns;
  if (np > 0) {
    IB_TRY(dalloc(&P.X, 2ul * np));
    IB_TRY(dalloc(&P.F, 2ul * np));
    if (ns > 0) IB_TRY(dalloc(&P.Fs, 2ul * ns));
    IB_TRY(dalloc(&P.U64, 2ul * np));
    if (P.windows && ns > 0) {
      IB_TRY(dalloc(&P.G64, 2ul * np));
      IB_TRY(dalloc(&P.rc_pt, 32ul * np));
      IB_TRY(dalloc(&P.rc_w, 32ul * np));
    }
    if (fp32) IB_TRY(dalloc(&P.U32, 2ul * np));
    IB_TRY(dalloc(&P.adj_ptr, (size_t)np + 1));
  }
  if (ns > 0) {
    IB_TRY(dalloc(&P.springs, 2ul * ns));
    IB_TRY(dalloc(&P.kappa, (size_t)ns));
    IB_TRY(dalloc(&P.rest, (size_t)ns));
    IB_TRY(dalloc(&P.adj_spring, 2ul * ns));
    IB_TRY(dalloc(&P.adj_other, 2ul * ns));
    IB_TRY(dalloc(&P.K64, 3ul * ns));
    if (fp32) IB_TRY(dalloc(&P.K32, 3ul * ns));
  }
  int ldc = P.nc + P.nborder;
  IB_TRY(dalloc(&P.Mcoarse, (size_t)ldc * ldc));
  int m = P.max_m;
  size_t n = 3ul * P.prm.N * P.prm.N;
  IB_TRY(dalloc(&P.V, (size_t)(m + 1) * n));
  if (fp32) {
    float* z;
    IB_TRY(dalloc(&z, (size_t)m * n));
    P.Z = z;
    if (P.prm.escalate) IB_TRY(dalloc(&P.Z64, (size_t)m * n));
  } else {
    double* z;
    IB_TRY(dalloc(&z, (size_t)m * n));
    P.Z = z;
  }
  IB_TRY(dalloc(&P.H, (size_t)(m + 1) * m));
  IB_TRY(dalloc(&P.givens, 4ul * m + 1));
  IB_TRY(krylov_init(P));
  IB_TRY(dalloc(&P.dots, (size_t)P.dot_blocks * (m + 2)));
  IB_TRY(dalloc(&P.scal, 16ul + 2ul * (m + 2) + 8));
  IB_TRY(dalloc(&P.x64, n));
  IB_TRY(dalloc(&P.b64, n));
  IB_TRY(dalloc(&P.t64, n));
  IB_TRY(dalloc(&P.t64b, n));
  IB_TRY(dalloc(&P.dev_err, 1));
  IB_TRY(dalloc(&P.count, 1 + 2 * MAX_LEVELS_ALLOC));
  IB_CUDA_TRY(cudaMemsetAsync(P.dev_err, 0, sizeof(int), P.stream));
  IB_CUDA_TRY(cudaMallocHost((void**)&P.scal_host, 64 * sizeof(double)));
  IB_CUDA_TRY(cudaMallocHost((void**)&P.count_host, 128 * sizeof(int)));
  for (auto& e : P.ev) IB_CUDA_TRY(cudaEventCreate(&e));
  for (auto& e : P.pev) IB_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return IB_OK;
}

int read_scalars(Problem& P, int count) {
  IB_CUDA_TRY(cudaMemcpyAsync(P.scal_host, P.scal, sizeof(double) * count, cudaMemcpyDeviceToHost,
                              P.stream));
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  return IB_OK;
}

// FP64 residual r = b - A_0 x.
int residual64(Problem& P, const double* x, const double* b, double* r) {
  IB_TRY(launch_stokes<double>(P, 0, x, b, r, true));
  IB_TRY(launch_elastic<double>(P, 0, x, r, -efac(P), P.U64));
  return IB_OK;
}

__global__ void k_add_d2t_f(float* z, const double* __restrict__ dz, const double* __restrict__ alpha, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) z[i] += (float)((*alpha) * dz[i]);
}
__global__ void k_add_d2t_d(double* z, const double* __restrict__ dz, const double* __restrict__ alpha, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) z[i] += (*alpha) * dz[i];
}

// Learned stage of one FGMRES iteration: with P.t64 = A z_j and r = v_j - A z_j,
// d = the network's correction for r, alpha = <r, A d> / <A d, A d> (exact line
// search along d); z_j + alpha d is kept when alpha > 0 and it lowers ||r||^2 by at
// least 0.1%, then P.t64 = A (stored z_j).  z64 (if not NULL) is the FP64 copy of z_j
// used after an FP32 -> FP64 escalation.
template <typename T>
int learned_step(Problem& P, const double* vj, T* zj, double* z64, ib_stats* st, bool* accepted) {
  *accepted = false;
  const size_t n = 3ul * P.prm.N * P.prm.N;
  double* sc = P.scal + 8 + 2 * (P.max_m + 2) + 1;  // free scalars after ||w||^2
  IB_TRY(launch_axpby(P, 1.0, vj, -1.0, P.t64, P.nn_r));
  IB_TRY(learned_features(P, P.nn_r, P.nn_dz, sc, P.nn_x));
  {
    KScope ks(P, IB_KC_OTHER, 0.0);  // the network's own launches are not counted per class
    IB_TRY(learned_forward(P.net, P.stream, P.nn_x, P.nn_y));
  }
  IB_TRY(learned_scale_out(P, P.nn_y, sc, P.nn_dz));
  IB_TRY(apply64(P, 0, P.nn_dz, P.nn_adz));
  IB_TRY(launch_dot(P, P.nn_r, P.nn_adz, sc + 1));
  IB_TRY(launch_dot(P, P.nn_adz, P.nn_adz, sc + 2));
  IB_TRY(launch_dot(P, P.nn_r, P.nn_r, sc + 3));
  IB_CUDA_TRY(cudaMemcpyAsync(P.scal_host + 16, sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  const double ra = P.scal_host[17], aa = P.scal_host[18], rr = P.scal_host[19];
  if (!(std::isfinite(ra) && std::isfinite(aa) && aa > 0.0 && ra > 0.0)) return IB_OK;
  const double gain = ra * ra / aa;  // ||r||^2 - ||r - alpha A d||^2
  if (!(gain >= 1e-3 * rr)) return IB_OK;  // keep the V-cycle direction
  const double alpha = ra / aa;
  {
    KScope ks(P, IB_KC_OTHER, 8.0);
    k_set<<<1, 1, 0, P.stream>>>(sc + 4, alpha);
    IB_LAUNCH_CHECK();
  }
  st->learned_used += 1;
  *accepted = true;
  const int tpb = 256;
  const int nbk = (int)((n + tpb - 1) / tpb);
  KScope ks(P, IB_KC_OTHER, n * 20.0);
  if (z64) {
    k_add_d2t_d<<<nbk, tpb, 0, P.stream>>>(z64, P.nn_dz, sc + 4, (long)n);
    IB_LAUNCH_CHECK();
    return apply64(P, 0, z64, P.t64);
  }
  if constexpr (std::is_same<T, double>::value) {
    k_add_d2t_d<<<nbk, tpb, 0, P.stream>>>(zj, P.nn_dz, sc + 4, (long)n);
    IB_LAUNCH_CHECK();
    return apply64(P, 0, zj, P.t64);
  } else {
    k_add_d2t_f<<<nbk, tpb, 0, P.stream>>>(zj, P.nn_dz, sc + 4, (long)n);
    IB_LAUNCH_CHECK();
    IB_TRY((launch_cast<float, double>(P, zj, P.t64b, n)));
    return apply64(P, 0, P.t64b, P.t64);
  }
}

// Flexible GMRES with the V-cycle as right preconditioner (sec. 3.3), zero
// initial guess, classical Gram-Schmidt applied twice, Givens rotations; stop
// when the estimate reaches tol ||b||, confirm with the true FP64 residual and
// restart from the iterate if needed.
//
// The iterations are pipelined on the host: iteration j is launched before the
// residual estimate of iteration j - 1 is read, so the device never waits for
// the host between iterations.  When j - 1 turns out to be the last one, the
// work of iteration j is discarded: it only touched column j of H, g[j], g[j+1],
// V[j+1] and Z[j], none of which the update with k = j directions reads.  An
// escalation to the mixed V-cycle also ends the cycle: FGMRES restarts from the
// iterate, so a cycle's directions are all FP32 (Z) or all FP64 (Z64).
template <typename T>
int fgmres(Problem& P, const double* b, double* x, ib_stats* st) {
  const size_t n = 3ul * P.prm.N * P.prm.N;
  const int m = P.max_m;
  const double tol = P.prm.tol;
  T* Z = (T*)P.Z;
  double* s = P.scal;
  IB_TRY(launch_dot(P, b, b, s + 4));
  IB_TRY(read_scalars(P, 8));
  double bnorm = std::sqrt(P.scal_host[4]);
  IB_TRY(launch_fill<double>(P, x, n, 0.0));
  st->iters = 0;
  st->restarts = 0;
  st->rel_res_true = 0.0;
  st->rel_res_est = 0.0;
  if (!(bnorm > 0.0)) {
    if (!std::isfinite(bnorm)) return fail(IB_ERR_BREAKDOWN, "non-finite right-hand side");
    return IB_OK;
  }
  int total = 0;
  std::vector<double> hist;
  int nn_rejected = 0;  // consecutive rejections of the learned stage
  st->escalated_at = -1;
  // a step stiff enough to stall the FP32 V-cycle starts on the mixed one
  if (!std::is_same<T, double>::value && P.has64 && P.sigma >= P.stiff_sigma) st->escalated_at = 0;
  double* h1 = s + 8;
  double* h2 = h1 + m + 2;
  double* g = P.givens + 2 * m;
  for (int restart = 0;; ++restart) {
    if (total == 0) {
      IB_CUDA_TRY(cudaMemcpyAsync(P.V, b, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
    } else {
      IB_TRY(residual64(P, x, b, P.V));
    }
    IB_TRY(launch_dot(P, P.V, P.V, s + 5));
    IB_TRY(read_scalars(P, 8));
    double beta = std::sqrt(P.scal_host[5]);
    if (!std::isfinite(beta)) return fail(IB_ERR_BREAKDOWN, "non-finite residual");
    if (beta <= tol * bnorm) {
      st->rel_res_true = beta / bnorm;
      return IB_OK;
    }
    if (total >= P.prm.max_iters) break;
    if (st->escalated_at >= 0 && P.struct_inv32 && !inv32_always()) IB_TRY(reform_struct64(P));
    int mav = std::min(P.max_m, P.prm.max_iters - total);
    const int cycle_start = total;
    IB_TRY(launch_fill<double>(P, g, (size_t)m + 1, 0.0));
    {
      KScope ks(P, IB_KC_KRYLOV, 8.0);
      k_set<<<1, 1, 0, P.stream>>>(g, beta);
    }
    {
      KScope ks(P, IB_KC_KRYLOV, 8.0);
      k_set<<<1, 1, 0, P.stream>>>(s + 6, beta);
    }
    IB_LAUNCH_CHECK();
    IB_TRY(launch_scale_copy(P, P.V, s + 6, P.V, true));
    int k = 0;
    bool stopped = false;
    // Reads the scalars of iteration jj (waiting for them): 1 = stop after jj
    // (converged, lucky breakdown, or escalation: the cycle ends and FGMRES restarts
    // from the iterate with the mixed V-cycle and a fresh basis), 0 = continue,
    // -1 = non-finite or CUDA error.
    auto check = [&](int jj) -> int {
      if (cudaEventSynchronize(P.pev[jj & 1]) != cudaSuccess) return -1;
      const double* h = P.scal_host + 24 + 4 * (jj & 1);
      const double est = h[0];
      st->rel_res_est = est / bnorm;
      if (h[2] != 0.0) return -1;
      if (est <= tol * bnorm) return 1;
      hist.push_back(est);
      if (!(h[1] > 0.0)) return 1;  // lucky breakdown: exact solution in the space
      // stagnation of the FP32-preconditioned iteration: less than a factor 2 in
      // the last 4 iterations -> restart with the mixed-precision V-cycle (FP64
      // residuals, which the stiff cancellation needs)
      if (!std::is_same<T, double>::value && P.has64 && st->escalated_at < 0 && hist.size() > 4 &&
          est > 0.5 * hist[hist.size() - 5]) {
        st->escalated_at = cycle_start + jj + 1;
        return 1;
      }
      return 0;
    };
    for (int j = 0; j < mav; ++j) {
      double* vj = P.V + (size_t)j * n;
      T* zj = Z + (size_t)j * n;
      if constexpr (std::is_same<T, double>::value) {
        LevelBuf<double>& B0 = P.lev[0].v64;
        IB_CUDA_TRY(cudaMemcpyAsync(B0.b, vj, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
        IB_TRY(vcycle_run<double>(P));
        IB_CUDA_TRY(cudaMemcpyAsync(zj, B0.w, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
        IB_TRY(apply64(P, 0, zj, P.t64));
      } else if (st->escalated_at < 0) {
        LevelBuf<float>& B0 = P.lev[0].v32;
        IB_TRY((launch_cast<double, float>(P, vj, B0.b, n)));
        IB_TRY(vcycle_run<float>(P));
        IB_CUDA_TRY(cudaMemcpyAsync(zj, B0.w, n * sizeof(float), cudaMemcpyDeviceToDevice, P.stream));
        IB_TRY((launch_cast<float, double>(P, zj, P.t64b, n)));
        IB_TRY(apply64(P, 0, P.t64b, P.t64));
      } else {
        // escalated: the mixed-precision V-cycle (FP64 vectors and residuals, FP32
        // box solves) preconditions and its directions are kept in
        // FP64 (flexible GMRES combines the two bases in the update of x)
        LevelBuf<double>& B0 = P.lev[0].v64;
        double* zj64 = P.Z64 + (size_t)j * n;
        IB_CUDA_TRY(cudaMemcpyAsync(B0.b, vj, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
        IB_TRY(vcycle_run<double>(P));
        IB_CUDA_TRY(cudaMemcpyAsync(zj64, B0.w, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
        IB_TRY(apply64(P, 0, zj64, P.t64));
      }
      if (P.net) {
        bool esc = !std::is_same<T, double>::value && st->escalated_at >= 0;
        if (nn_rejected < 3) {
          bool acc = false;
          IB_TRY(learned_step<T>(P, vj, zj, esc ? P.Z64 + (size_t)j * n : nullptr, st, &acc));
          nn_rejected = acc ? 0 : nn_rejected + 1;
        }
      }
      // classical Gram-Schmidt applied twice: h1 = V^T w; w -= V h1 and h2 = V^T w in
      // one pass over V; w -= V h2 with ||w||^2 and the Givens step
      IB_TRY(launch_multidot(P, P.V, j + 1, P.t64, h1));
      IB_TRY(launch_cgs_sub_dot(P, P.V, j + 1, h1, P.t64, h2));
      IB_TRY(launch_cgs_finish(P, P.V, j + 1, P.t64, j));
      IB_TRY(launch_scale_copy(P, P.t64, s + 1, P.V + (size_t)(j + 1) * n, true));
      IB_CUDA_TRY(cudaMemcpyAsync(P.scal_host + 24 + 4 * (j & 1), P.scal, 3 * sizeof(double),
                                  cudaMemcpyDeviceToHost, P.stream));
      IB_CUDA_TRY(cudaEventRecord(P.pev[j & 1], P.stream));
      ++total;
      k = j + 1;
      if (j > 0) {
        int rc = check(j - 1);
        if (rc < 0) {
          IB_TRY(check_dev_err(P));  // a device-side error explains what followed it
          return P.scal_host[24 + 4 * ((j - 1) & 1) + 2] != 0.0 ? fail(IB_ERR_BREAKDOWN, "non-finite value in FGMRES")
                                                                 : fail(IB_ERR_CUDA, "FGMRES pipeline");
        }
        if (rc == 1) {  // iteration j - 1 was the last of the cycle: drop iteration j
          k = j;
          --total;
          stopped = true;
          break;
        }
      }
    }
    if (!stopped && k > 0) {
      int rc = check(k - 1);
      if (rc < 0) {
        IB_TRY(check_dev_err(P));
        return P.scal_host[24 + 4 * ((k - 1) & 1) + 2] != 0.0 ? fail(IB_ERR_BREAKDOWN, "non-finite value in FGMRES")
                                                               : fail(IB_ERR_CUDA, "FGMRES pipeline");
      }
    }
    IB_TRY(launch_backsolve(P, k));
    if constexpr (std::is_same<T, double>::value) {
      IB_TRY(launch_update_x<T>(P, Z, k, x));
    } else {
      // directions j < e are FP32 (Z), j >= e FP64 (Z64); e = k in the cycle that
      // escalates, 0 in the cycles after it
      int e = k;
      if (st->escalated_at >= 0) e = std::max(0, std::min(k, st->escalated_at - cycle_start));
      IB_TRY(launch_update_x<float>(P, Z, e, x, 0));
      if (e < k) IB_TRY(launch_update_x<double>(P, P.Z64, k - e, x, e));
    }
    IB_TRY(residual64(P, x, b, P.t64));
    IB_TRY(launch_dot(P, P.t64, P.t64, s + 7));
    IB_TRY(read_scalars(P, 8));
    IB_TRY(check_dev_err(P));
    double rt = std::sqrt(P.scal_host[7]) / bnorm;
    st->rel_res_true = rt;
    st->iters = total;
    st->restarts = restart;
    if (!std::isfinite(rt)) return fail(IB_ERR_BREAKDOWN, "non-finite true residual");
    if (rt <= tol) return IB_OK;
    if (total >= P.prm.max_iters) break;
  }
  return fail(IB_ERR_NOT_CONVERGED, "FGMRES reached max_iters above tol");
}

// One implicit IB step on the problem's stream (the body of ib_solve_step).
int solve_step_impl(Problem& P, const double* u_n, double* up, double* X, ib_stats* stats) {
  if (P.np > 0 && !X) return fail(IB_ERR_INVALID_ARG, "X is NULL");
  ib_stats local;
  std::memset(&local, 0, sizeof(local));
  ib_stats* st = stats ? stats : &local;
  std::memset(st, 0, sizeof(*st));
  st->escalated_at = -1;
  size_t n = 3ul * P.prm.N * P.prm.N;
  IB_CUDA_TRY(cudaEventRecord(P.ev[0], P.stream));
  if (P.np > 0)
    IB_CUDA_TRY(cudaMemcpyAsync(P.X, X, sizeof(double) * 2 * P.np, cudaMemcpyDeviceToDevice, P.stream));
  int rc = setup_hierarchy(P);
  if (rc != IB_OK) { st->status = rc; return rc; }
  IB_TRY(launch_fill<double>(P, P.b64, n, 0.0));
  IB_TRY(launch_spread_force(P, P.b64));
  if (u_n && P.prm.rho != 0.0) {
    long n2 = 2L * P.prm.N * P.prm.N;
    KScope ks(P, IB_KC_OTHER, 3.0 * n2 * 8.0);
    k_axpy_n<<<(int)((n2 + 255) / 256), 256, 0, P.stream>>>(-P.prm.rho / P.prm.dt, u_n, P.b64, n2);
    IB_LAUNCH_CHECK();
  }
  if (P.prm.walls) IB_TRY(launch_wall_rhs(P, P.b64));
  IB_CUDA_TRY(cudaEventRecord(P.ev[1], P.stream));
  if (P.prm.precision != IB_FP32_PRECOND) rc = fgmres<double>(P, P.b64, P.x64, st);
  else rc = fgmres<float>(P, P.b64, P.x64, st);
  IB_CUDA_TRY(cudaEventRecord(P.ev[2], P.stream));
  if (rc != IB_OK && rc != IB_ERR_NOT_CONVERGED) { st->status = rc; return rc; }
  std::string msg = g_err;
  IB_TRY(launch_pressure_mean_remove(P, P.x64));
  IB_CUDA_TRY(cudaMemcpyAsync(up, P.x64, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
  if (P.np > 0) {
    IB_TRY(launch_move_points(P, P.x64));
    IB_CUDA_TRY(cudaMemcpyAsync(X, P.X, sizeof(double) * 2 * P.np, cudaMemcpyDeviceToDevice, P.stream));
  }
  IB_CUDA_TRY(cudaEventRecord(P.ev[3], P.stream));
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  float t0 = 0, t1 = 0;
  cudaEventElapsedTime(&t0, P.ev[0], P.ev[1]);
  cudaEventElapsedTime(&t1, P.ev[1], P.ev[2]);
  st->t_setup_ms = t0;
  st->t_solve_ms = t1;
  int nsb = 0;
  for (int l = 0; l < P.nlev - 1; ++l) nsb += P.lev[l].n_struct;
  st->n_struct_boxes = nsb;
  st->status = rc;
  g_err = msg;
  return rc;
}

// One implicit step with the spring force taken at the new positions (a nonlinear
// backward-Euler step, the body of ib_solve_step_newton), solved by Newton's method:
// S and S* stay at X^n (lagged, as in the linearised step), the springs' force and
// Jacobian are evaluated at the iterate X^k = X^n + dt S*^n u^k, and iteration k
// solves the linearised step's system with J(X^k) and the right-hand side
// -(rho/dt) u^n - S [F(X^k) - J(X^k)(X^k - X^n)].  u^0 = 0: the first iterate is the
// linearised step.  Stops when max |X^{k+1} - X^k| <= tol h (k >= 1) or after
// max_newton solves.
int newton_step_impl(Problem& P, const double* u_n, double* up, double* X, int max_newton, double tol,
                     ib_stats* stats, double* newton) {
  if (max_newton < 1) return fail(IB_ERR_INVALID_ARG, "max_newton must be >= 1");
  if (!(tol >= 0.0)) return fail(IB_ERR_INVALID_ARG, "tol_newton must be >= 0");
  if (P.prm.time_method == IB_EXPLICIT)
    return fail(IB_ERR_INVALID_ARG, "the Newton step needs the implicit-time method");
  if (P.np > 0 && !X) return fail(IB_ERR_INVALID_ARG, "X is NULL");
  ib_stats local;
  ib_stats* st = stats ? stats : &local;
  std::memset(st, 0, sizeof(*st));
  st->escalated_at = -1;
  const size_t n = 3ul * P.prm.N * P.prm.N, np2 = 2ul * P.np;
  if (P.np == 0 || P.ns == 0) {  // no springs: nothing nonlinear
    const int rc = solve_step_impl(P, u_n, up, X, st);
    if (newton) { newton[0] = 1.0; newton[1] = 0.0; }
    return rc;
  }
  if (!P.Xn) IB_TRY(dalloc(&P.Xn, np2));
  if (!P.Xk) IB_TRY(dalloc(&P.Xk, np2));
  if (!P.Dk) IB_TRY(dalloc(&P.Dk, np2));
  if (!P.Gk) IB_TRY(dalloc(&P.Gk, np2));
  IB_CUDA_TRY(cudaMemcpyAsync(P.Xn, X, sizeof(double) * np2, cudaMemcpyDeviceToDevice, P.stream));
  std::vector<double> xa(np2), xb(np2);
  const double h = P.prm.L / P.prm.N, Lp = P.prm.L;
  double change = 0.0, t_setup = 0.0, t_solve = 0.0;
  int k = 0, total_iters = 0, rc = IB_OK;
  struct ClearXs {  // the springs go back to P.X on every exit
    Problem& P;
    ~ClearXs() { P.Xs = nullptr; }
  } clear_xs{P};
  for (; k < max_newton; ++k) {
    IB_CUDA_TRY(cudaMemcpyAsync(P.X, P.Xn, sizeof(double) * np2, cudaMemcpyDeviceToDevice, P.stream));
    P.Xs = k == 0 ? nullptr : P.Xk;
    IB_CUDA_TRY(cudaEventRecord(P.ev[0], P.stream));
    rc = setup_hierarchy(P);
    if (rc != IB_OK) { st->status = rc; return rc; }
    IB_TRY(launch_fill<double>(P, P.b64, n, 0.0));
    if (k > 0) IB_TRY(launch_newton_force(P));
    IB_TRY(launch_spread_force(P, P.b64));
    if (u_n && P.prm.rho != 0.0) {
      const long n2 = 2L * P.prm.N * P.prm.N;
      KScope ks(P, IB_KC_OTHER, 3.0 * n2 * 8.0);
      k_axpy_n<<<(int)((n2 + 255) / 256), 256, 0, P.stream>>>(-P.prm.rho / P.prm.dt, u_n, P.b64, n2);
      IB_LAUNCH_CHECK();
    }
    if (P.prm.walls) IB_TRY(launch_wall_rhs(P, P.b64));
    IB_CUDA_TRY(cudaEventRecord(P.ev[1], P.stream));
    ib_stats sk;
    std::memset(&sk, 0, sizeof(sk));
    sk.escalated_at = -1;
    rc = P.prm.precision != IB_FP32_PRECOND ? fgmres<double>(P, P.b64, P.x64, &sk)
                                            : fgmres<float>(P, P.b64, P.x64, &sk);
    IB_CUDA_TRY(cudaEventRecord(P.ev[2], P.stream));
    total_iters += sk.iters;
    st->restarts += sk.restarts;
    st->rel_res_true = sk.rel_res_true;
    st->rel_res_est = sk.rel_res_est;
    st->escalated_at = sk.escalated_at;
    if (rc != IB_OK && rc != IB_ERR_NOT_CONVERGED) { st->status = rc; return rc; }
    IB_TRY(launch_pressure_mean_remove(P, P.x64));
    IB_TRY(launch_move_points(P, P.x64));  // P.X = X^{k+1} (interpolation at X^n)
    IB_CUDA_TRY(cudaMemcpyAsync(xa.data(), P.X, sizeof(double) * np2, cudaMemcpyDeviceToHost, P.stream));
    IB_CUDA_TRY(cudaMemcpyAsync(xb.data(), k == 0 ? P.Xn : P.Xk, sizeof(double) * np2, cudaMemcpyDeviceToHost,
                                P.stream));
    IB_CUDA_TRY(cudaMemcpyAsync(P.Xk, P.X, sizeof(double) * np2, cudaMemcpyDeviceToDevice, P.stream));
    IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, P.ev[0], P.ev[1]);
    cudaEventElapsedTime(&b, P.ev[1], P.ev[2]);
    t_setup += a;
    t_solve += b;
    change = 0.0;
    for (size_t i = 0; i < np2; ++i) {
      double d = xa[i] - xb[i];
      d -= Lp * std::rint(d / Lp);
      change = std::max(change, std::fabs(d));
    }
    change /= h;
    if (rc == IB_ERR_NOT_CONVERGED) { ++k; break; }
    if (k >= 1 && change <= tol) { ++k; break; }
  }
  std::string msg = g_err;
  IB_CUDA_TRY(cudaMemcpyAsync(up, P.x64, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
  IB_CUDA_TRY(cudaMemcpyAsync(X, P.X, sizeof(double) * np2, cudaMemcpyDeviceToDevice, P.stream));
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  st->iters = total_iters;
  st->t_setup_ms = (float)t_setup;
  st->t_solve_ms = (float)t_solve;
  int nsb = 0;
  for (int l = 0; l < P.nlev - 1; ++l) nsb += P.lev[l].n_struct;
  st->n_struct_boxes = nsb;
  st->status = rc;
  if (newton) {
    newton[0] = (double)k;
    newton[1] = change;
  }
  g_err = msg;
  return rc;
}

}  // namespace
}  // namespace ib

struct ib_problem {
  ib::Problem P;
};

using namespace ib;

extern "C" {

const char* ib_version(void) { return "ibmg-gb300 0.1 (sm_103a)"; }

const char* ib_last_error(void) { return g_err.c_str(); }

void ib_default_params(ib_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->N = 64;
  p->L = 1.0;
  p->rho = 1.0;
  p->mu = 1.0;
  p->dt = 1e-2;
  p->delta = IB_DELTA_PESKIN4;
  p->box = 1;
  p->nu1 = 1;
  p->nu2 = 1;
  p->precision = IB_FP64;
  p->jacobian = IB_JAC_CLAMPED;
  p->tol = 1e-8;
  p->max_iters = 100;
  p->escalate = 1;
  p->restart = 0;
}

int ib_setup(const ib_params* params, int32_t n_points, const double* X, int32_t n_springs,
             const int32_t* springs, const double* kappa, const double* rest, void* stream,
             ib_problem** out) {
  g_err.clear();
  if (!out) return fail(IB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  IB_TRY(validate(params));
  if (n_points < 0 || n_springs < 0) return fail(IB_ERR_INVALID_ARG, "negative counts");
  if (n_points == 0 && n_springs > 0) return fail(IB_ERR_INVALID_ARG, "springs without points");
  if (n_points > 0 && !X) return fail(IB_ERR_INVALID_ARG, "X is NULL");
  if (n_springs > 0 && (!springs || !kappa || !rest))
    return fail(IB_ERR_INVALID_ARG, "spring arrays are NULL");
  for (int k = 0; k < 2 * n_points; ++k)
    if (!std::isfinite(X[k])) return fail(IB_ERR_INVALID_ARG, "non-finite point position");
  if (params->walls == IB_WALLS_NOSLIP) {
    const double h = params->L / params->N;
    for (int k = 0; k < 2 * n_points; ++k)
      if (X[k] < 2.0 * h || X[k] > params->L - 2.0 * h)
        return fail(IB_ERR_INVALID_ARG, "with no-slip walls every point must lie at least 2h from the walls");
  }
  std::vector<int> deg(n_points + 1, 0);
  for (int s = 0; s < n_springs; ++s) {
    int i = springs[2 * s], j = springs[2 * s + 1];
    if (i < 0 || j < 0 || i >= n_points || j >= n_points || i == j)
      return fail(IB_ERR_INVALID_ARG, "spring end points out of range or equal");
    if (!(std::isfinite(kappa[s]) && kappa[s] >= 0) || !(std::isfinite(rest[s]) && rest[s] >= 0))
      return fail(IB_ERR_INVALID_ARG, "kappa and rest length must be finite and >= 0");
    ++deg[i];
    ++deg[j];
  }
  for (int k = 0; k < n_points; ++k)
    if (deg[k] > 7) return fail(IB_ERR_INVALID_ARG, "at most 7 springs per point are supported");

  ib_problem* H = new (std::nothrow) ib_problem();
  if (!H) return fail(IB_ERR_OOM, "host allocation failed");
  Problem& P = H->P;
  P.prm = *params;
  P.stream = (cudaStream_t)stream;
  P.np = n_points;
  P.ns = n_springs;
  P.nB = box_nunk(params->box);
  // the explicit method's operator is Stokes alone: nothing stiff to escalate for
  P.sigma = params->time_method == IB_EXPLICIT ? 0.0 : stiffness(*params, n_springs, kappa);
  P.stiff_sigma = stiff_threshold();
  if (const char* e = std::getenv("IB_WINDOWS")) P.windows = e[0] != '0';
  if (const char* e = std::getenv("IB_ROW_LISTS")) P.row_lists = e[0] != '0';
  if (const char* e = std::getenv("IB_INV32")) P.inv32 = e[0] != '0';
  int Nc = params->box > 4 ? params->box : 4;
  for (int N = params->N; N >= Nc; N /= 2) {
    LevelInfo L;
    L.N = N;
    L.h = params->L / N;
    L.nb = N / params->box;
    P.lev.push_back(L);
  }
  P.nlev = (int)P.lev.size();
  P.nc = 3 * Nc * Nc;
  // bordered null space of the coarsest solve: the constant pressure, and with
  // rho = 0 on the periodic square also the constant velocities
  P.nborder = (params->rho == 0.0 && params->walls == IB_WALLS_PERIODIC) ? 3 : 1;
  P.max_m = (params->restart > 0 && params->restart < params->max_iters) ? params->restart : params->max_iters;
  int st = allocate(P);
  if (st != IB_OK) {
    std::string msg = g_err;
    free_problem(&H->P);
    delete H;
    g_err = msg;
    return st;
  }
  // spring adjacency (host-side bookkeeping of the input graph)
  std::vector<int> ptr(n_points + 1, 0), sp_idx(2 * n_springs), other(2 * n_springs);
  for (int s = 0; s < n_springs; ++s) {
    ++ptr[springs[2 * s] + 1];
    ++ptr[springs[2 * s + 1] + 1];
  }
  for (int k = 0; k < n_points; ++k) ptr[k + 1] += ptr[k];
  std::vector<int> fillp(ptr.begin(), ptr.end() - (n_points > 0 ? 1 : 0));
  for (int s = 0; s < n_springs; ++s) {
    int i = springs[2 * s], j = springs[2 * s + 1];
    sp_idx[fillp[i]] = s; other[fillp[i]++] = j;
    sp_idx[fillp[j]] = s; other[fillp[j]++] = i;
  }
  cudaStream_t s = P.stream;
  auto fail_free = [&](int code) {
    std::string msg = g_err;
    free_problem(&H->P);
    delete H;
    g_err = msg;
    return code;
  };
#define IB_SETUP_CUDA(expr)                                                   \
  do {                                                                        \
    cudaError_t _e = (expr);                                                  \
    if (_e != cudaSuccess) {                                                  \
      fail(IB_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));  \
      return fail_free(IB_ERR_CUDA);                                          \
    }                                                                         \
  } while (0)
  if (n_points > 0) {
    IB_SETUP_CUDA(cudaMemcpyAsync(P.X, X, sizeof(double) * 2 * n_points, cudaMemcpyHostToDevice, s));
    IB_SETUP_CUDA(cudaMemcpyAsync(P.adj_ptr, ptr.data(), sizeof(int) * (n_points + 1),
                                  cudaMemcpyHostToDevice, s));
  }
  if (n_springs > 0) {
    IB_SETUP_CUDA(cudaMemcpyAsync(P.springs, springs, sizeof(int) * 2 * n_springs,
                                  cudaMemcpyHostToDevice, s));
    IB_SETUP_CUDA(cudaMemcpyAsync(P.kappa, kappa, sizeof(double) * n_springs, cudaMemcpyHostToDevice, s));
    IB_SETUP_CUDA(cudaMemcpyAsync(P.rest, rest, sizeof(double) * n_springs, cudaMemcpyHostToDevice, s));
    IB_SETUP_CUDA(cudaMemcpyAsync(P.adj_spring, sp_idx.data(), sizeof(int) * 2 * n_springs,
                                  cudaMemcpyHostToDevice, s));
    IB_SETUP_CUDA(cudaMemcpyAsync(P.adj_other, other.data(), sizeof(int) * 2 * n_springs,
                                  cudaMemcpyHostToDevice, s));
  }
  IB_SETUP_CUDA(cudaStreamSynchronize(s));
  st = setup_hierarchy(P);
  if (st != IB_OK) return fail_free(st);
  for (const char* v : {"IB_BOX_GEMM_MIN", "IB_BOX_ONE_MAX", "IB_BOX_STRIP", "IB_BOX_STRIP_MIN", "IB_BOX_STRIP_W"})
    if (std::getenv(v)) P.box_autotune = false;  // the forms are pinned by hand
  if (const char* e = std::getenv("IB_BOX_TUNE")) P.box_autotune = P.box_autotune && e[0] != '0';
  if (const char* e = std::getenv("IB_BOX_FORMS")) {  // comma-separated forms, finest level first
    int l = 0;
    for (const char* c = e; *c && l < 32;) {
      P.box_form_pin[l++] = std::atoi(c);
      while (*c && *c != ',') ++c;
      if (*c == ',') ++c;
    }
    P.box_form_pinned = true;
  }
  if (const char* e = std::getenv("IB_BOX_GEMM_MIN")) P.box_gemm_min = std::atol(e);
  if (const char* e = std::getenv("IB_BOX_ONE_MAX")) P.box_one_max = std::atol(e);
  if (const char* e = std::getenv("IB_WAIT_LIMIT_NS")) P.wait_limit_ns = std::strtoull(e, nullptr, 10);
  if (const char* e = std::getenv("IB_BOX_STRIP")) P.box_strip = e[0] != '0';
  if (const char* e = std::getenv("IB_BOX_STRIP_MIN")) P.box_strip_min = std::atol(e);
  if (const char* e = std::getenv("IB_BOX_STRIP_W")) {
    const int wv = std::atoi(e);
    P.box_strip_w = (wv == 8 || wv == 16 || wv == 32) ? wv : 0;
  }
  P.has32 = params->precision == IB_FP32_PRECOND;
  P.has64 = params->precision != IB_FP32_PRECOND || params->escalate != 0;
  if (P.has32) {
    st = vcycle_prepare<float>(P);
    if (st != IB_OK) return fail_free(st);
  }
  if (P.has64) {
    st = vcycle_prepare<double>(P);
    if (st != IB_OK) return fail_free(st);
  }
  *out = H;
  return IB_OK;
}

int ib_update_points(ib_problem* H, const double* X_dev) {
  g_err.clear();
  if (!H) return fail(IB_ERR_INVALID_ARG, "problem is NULL");
  Problem& P = H->P;
  if (P.np > 0) {
    if (!X_dev) return fail(IB_ERR_INVALID_ARG, "X is NULL");
    IB_CUDA_TRY(cudaMemcpyAsync(P.X, X_dev, sizeof(double) * 2 * P.np, cudaMemcpyDeviceToDevice,
                                P.stream));
  }
  return setup_hierarchy(P);
}

int ib_num_levels(const ib_problem* H) { return H ? H->P.nlev : 0; }

int ib_level_size(const ib_problem* H, int32_t level) {
  if (!H || level < 0 || level >= H->P.nlev) return 0;
  return H->P.lev[level].N;
}

int ib_tail_grid(const ib_problem* H, int32_t precision) {
  if (!H || (precision != IB_FP64 && precision != IB_FP32_PRECOND && precision != IB_MIXED_PRECOND)) return 0;
  const Problem& P = H->P;
  const int ix = precision == IB_FP32_PRECOND ? 0 : 1;
  if ((ix == 1 && !P.has64) || (ix == 0 && !P.has32)) return 0;
  return P.lev[P.tail_level[ix]].N;
}

int ib_tail_cluster(const ib_problem* H, int32_t precision) {
  if (!H || (precision != IB_FP64 && precision != IB_FP32_PRECOND && precision != IB_MIXED_PRECOND)) return 0;
  const Problem& P = H->P;
  const int ix = precision == IB_FP32_PRECOND ? 0 : 1;
  if ((ix == 1 && !P.has64) || (ix == 0 && !P.has32)) return 0;
  return P.tail_cluster[ix];
}

int ib_box_form(const ib_problem* H, int32_t precision, int32_t level) {
  if (!H || (precision != IB_FP64 && precision != IB_FP32_PRECOND && precision != IB_MIXED_PRECOND)) return -1;
  const Problem& P = H->P;
  if (level < 0 || level >= P.nlev - 1 || level >= 32) return -1;
  return P.box_form[precision == IB_FP32_PRECOND ? 0 : 1][level];
}

int ib_num_struct_boxes(const ib_problem* H, int32_t level) {
  if (!H || level < 0 || level >= H->P.nlev - 1) return 0;
  return H->P.lev[level].n_struct;
}

int ib_apply(ib_problem* H, int32_t level, const double* w, double* y) {
  g_err.clear();
  if (!H || !w || !y) return fail(IB_ERR_INVALID_ARG, "NULL argument");
  Problem& P = H->P;
  if (level < 0 || level >= P.nlev) return fail(IB_ERR_INVALID_ARG, "level out of range");
  if (w == y) return fail(IB_ERR_INVALID_ARG, "w and y must not alias");
  IB_TRY(apply64(P, level, w, y));
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  return IB_OK;
}

int ib_vcycle(ib_problem* H, const double* b, double* w) {
  g_err.clear();
  if (!H || !b || !w) return fail(IB_ERR_INVALID_ARG, "NULL argument");
  if (b == w) return fail(IB_ERR_INVALID_ARG, "b and w must not alias");
  Problem& P = H->P;
  size_t n = 3ul * P.prm.N * P.prm.N;
  if (P.prm.precision != IB_FP32_PRECOND) {
    LevelBuf<double>& B0 = P.lev[0].v64;
    IB_CUDA_TRY(cudaMemcpyAsync(B0.b, b, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
    IB_TRY(vcycle_run<double>(P));
    IB_CUDA_TRY(cudaMemcpyAsync(w, B0.w, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
  } else {
    LevelBuf<float>& B0 = P.lev[0].v32;
    IB_TRY((launch_cast<double, float>(P, b, B0.b, n)));
    IB_TRY(vcycle_run<float>(P));
    IB_TRY((launch_cast<float, double>(P, B0.w, w, n)));
  }
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  return IB_OK;
}

int ib_rhs(ib_problem* H, const double* u_n, double* b) {
  g_err.clear();
  if (!H || !b) return fail(IB_ERR_INVALID_ARG, "NULL argument");
  Problem& P = H->P;
  size_t n = 3ul * P.prm.N * P.prm.N;
  IB_TRY(launch_fill<double>(P, b, n, 0.0));
  IB_TRY(launch_spread_force(P, b));
  if (u_n && P.prm.rho != 0.0) {
    long n2 = 2L * P.prm.N * P.prm.N;
    KScope ks(P, IB_KC_OTHER, 3.0 * n2 * 8.0);
    k_axpy_n<<<(int)((n2 + 255) / 256), 256, 0, P.stream>>>(-P.prm.rho / P.prm.dt, u_n, b, n2);
    IB_LAUNCH_CHECK();
  }
  if (P.prm.walls) IB_TRY(launch_wall_rhs(P, b));
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  return IB_OK;
}

int ib_solve_step(ib_problem* H, const double* u_n, double* up, double* X, ib_stats* stats) {
  g_err.clear();
  if (!H || !up) return fail(IB_ERR_INVALID_ARG, "NULL argument");
  return solve_step_impl(H->P, u_n, up, X, stats);
}

int ib_solve_step_newton(ib_problem* H, const double* u_n, double* up, double* X, int32_t max_newton,
                         double tol_newton, ib_stats* stats, double* newton) {
  g_err.clear();
  if (!H || !up) return fail(IB_ERR_INVALID_ARG, "NULL argument");
  return newton_step_impl(H->P, u_n, up, X, max_newton, tol_newton, stats, newton);
}

int ib_solve(ib_problem* H, const double* b, double* x, ib_stats* stats) {
  g_err.clear();
  if (!H || !b || !x) return fail(IB_ERR_INVALID_ARG, "NULL argument");
  Problem& P = H->P;
  ib_stats local;
  ib_stats* st = stats ? stats : &local;
  std::memset(st, 0, sizeof(*st));
  st->escalated_at = -1;
  const size_t n = 3ul * P.prm.N * P.prm.N;
  IB_CUDA_TRY(cudaMemcpyAsync(P.b64, b, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
  if (P.prm.walls) IB_TRY(launch_zero_walls(P, P.b64));
  IB_CUDA_TRY(cudaEventRecord(P.ev[1], P.stream));
  int rc = (P.prm.precision != IB_FP32_PRECOND) ? fgmres<double>(P, P.b64, P.x64, st)
                                                : fgmres<float>(P, P.b64, P.x64, st);
  IB_CUDA_TRY(cudaEventRecord(P.ev[2], P.stream));
  if (rc != IB_OK && rc != IB_ERR_NOT_CONVERGED) { st->status = rc; return rc; }
  std::string msg = g_err;
  IB_TRY(launch_pressure_mean_remove(P, P.x64));
  IB_CUDA_TRY(cudaMemcpyAsync(x, P.x64, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  float t1 = 0;
  cudaEventElapsedTime(&t1, P.ev[1], P.ev[2]);
  st->t_solve_ms = t1;
  int nsb = 0;
  for (int l = 0; l < P.nlev - 1; ++l) nsb += P.lev[l].n_struct;
  st->n_struct_boxes = nsb;
  st->status = rc;
  g_err = msg;
  return rc;
}

static int learned_buffers(Problem& P) {
  const size_t n1 = (size_t)P.prm.N * P.prm.N;
  if (!P.nn_x) {
    IB_TRY(dalloc(&P.nn_x, 4 * n1));
    IB_TRY(dalloc(&P.nn_y, 3 * n1));
    IB_TRY(dalloc(&P.nn_r, 3 * n1));
    IB_TRY(dalloc(&P.nn_dz, 3 * n1));
    IB_TRY(dalloc(&P.nn_adz, 3 * n1));
  }
  if (!P.nn_sch) IB_TRY(learned_struct_channel(P));
  return IB_OK;
}

int ib_set_learned_stage(ib_problem* H, ib_unet* net) {
  g_err.clear();
  if (!H) return fail(IB_ERR_INVALID_ARG, "problem is NULL");
  Problem& P = H->P;
  if (net && learned_unet_size(net) != P.prm.N)
    return fail(IB_ERR_INVALID_ARG, "the network's grid size differs from the problem's");
  if (net && P.prm.walls != IB_WALLS_PERIODIC)
    return fail(IB_ERR_INVALID_ARG, "the learned stage's convolutions are periodic: not with no-slip walls");
  if (net) IB_TRY(learned_buffers(P));
  P.net = net;
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  return IB_OK;
}

int ib_learned_chain(ib_problem* H, double* e, float* in4, float* target) {
  g_err.clear();
  if (!H || !e || !in4 || !target) return fail(IB_ERR_INVALID_ARG, "NULL argument");
  IB_TRY(ib_learned_pair(H, e, in4, target));
  Problem& P = H->P;
  const size_t n = 3ul * P.prm.N * P.prm.N;
  // ib_learned_pair left e - MG(A e) in nn_dz
  IB_CUDA_TRY(cudaMemcpyAsync(e, P.nn_dz, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  return IB_OK;
}

int ib_learned_pair(ib_problem* H, const double* x, float* in4, float* target) {
  g_err.clear();
  if (!H || !x || !in4 || !target) return fail(IB_ERR_INVALID_ARG, "NULL argument");
  Problem& P = H->P;
  IB_TRY(learned_buffers(P));
  const size_t n = 3ul * P.prm.N * P.prm.N;
  double* sc = P.scal + 8 + 2 * (P.max_m + 2) + 1;
  // b = A x into nn_r; z = MG(b) into nn_dz; r = b - A z into nn_r; e = x - z into nn_dz
  IB_TRY(apply64(P, 0, x, P.nn_r));
  if (P.prm.precision != IB_FP32_PRECOND) {
    LevelBuf<double>& B0 = P.lev[0].v64;
    IB_CUDA_TRY(cudaMemcpyAsync(B0.b, P.nn_r, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
    IB_TRY(vcycle_run<double>(P));
    IB_CUDA_TRY(cudaMemcpyAsync(P.nn_dz, B0.w, n * sizeof(double), cudaMemcpyDeviceToDevice, P.stream));
  } else {
    LevelBuf<float>& B0 = P.lev[0].v32;
    IB_TRY((launch_cast<double, float>(P, P.nn_r, B0.b, n)));
    IB_TRY(vcycle_run<float>(P));
    IB_TRY((launch_cast<float, double>(P, B0.w, P.nn_dz, n)));
  }
  IB_TRY(apply64(P, 0, P.nn_dz, P.nn_adz));
  IB_TRY(launch_axpby(P, 1.0, P.nn_r, -1.0, P.nn_adz, P.nn_r));
  IB_TRY(launch_axpby(P, 1.0, x, -1.0, P.nn_dz, P.nn_dz));
  IB_TRY(learned_features(P, P.nn_r, P.t64, sc, in4));
  IB_TRY(learned_target(P, P.nn_dz, sc, target));
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  return IB_OK;
}

int64_t ib_launch_count(const ib_problem* H, int32_t kclass) {
  if (!H) return -1;
  const Problem& P = H->P;
  if (kclass >= 0 && kclass < IB_KC_COUNT) return P.nlaunch[kclass];
  int64_t t = 0;
  for (int c = 0; c < IB_KC_COUNT; ++c) t += P.nlaunch[c];
  return t;
}

int ib_profile(ib_problem* H, int32_t enable) {
  g_err.clear();
  if (!H) return fail(IB_ERR_INVALID_ARG, "problem is NULL");
  Problem& P = H->P;
  IB_TRY(resolve_profile(P));
  for (int c = 0; c < IB_KC_COUNT; ++c) {
    P.prof_n[c] = 0;
    P.prof_ms[c] = 0.0;
    P.prof_bytes[c] = 0.0;
  }
  P.prof = enable != 0;
  return IB_OK;
}

int ib_profile_read(ib_problem* H, int32_t kclass, int64_t* launches, double* ms, double* bytes) {
  g_err.clear();
  if (!H) return fail(IB_ERR_INVALID_ARG, "problem is NULL");
  if (kclass < 0 || kclass >= IB_KC_COUNT) return fail(IB_ERR_INVALID_ARG, "kernel class out of range");
  Problem& P = H->P;
  IB_TRY(resolve_profile(P));
  if (launches) *launches = P.prof_n[kclass];
  if (ms) *ms = P.prof_ms[kclass];
  if (bytes) *bytes = P.prof_bytes[kclass];
  return IB_OK;
}

}  // extern "C"

namespace ib {
namespace {
int resolve_vtimer(Problem& P) {
  if (P.vt_pending.empty()) return IB_OK;
  IB_CUDA_TRY(cudaStreamSynchronize(P.stream));
  for (size_t i = 0; i < P.vt_pending.size(); ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, P.vt_pending[i].first, P.vt_pending[i].second);
    P.vt_n[P.vt_kind[i]] += 1;
    P.vt_ms[P.vt_kind[i]] += ms;
    P.ev_pool.push_back(P.vt_pending[i].first);
    P.ev_pool.push_back(P.vt_pending[i].second);
  }
  P.vt_pending.clear();
  P.vt_kind.clear();
  return IB_OK;
}
}  // namespace
}  // namespace ib

extern "C" {

int ib_vcycle_timer(ib_problem* H, int32_t enable) {
  g_err.clear();
  if (!H) return fail(IB_ERR_INVALID_ARG, "problem is NULL");
  Problem& P = H->P;
  IB_TRY(resolve_vtimer(P));
  P.vt_n[0] = P.vt_n[1] = 0;
  P.vt_ms[0] = P.vt_ms[1] = 0.0;
  P.vt_on = enable != 0;
  return IB_OK;
}

int ib_vcycle_timer_read(ib_problem* H, int32_t precision, int64_t* count, double* ms) {
  g_err.clear();
  if (!H) return fail(IB_ERR_INVALID_ARG, "problem is NULL");
  if (precision != IB_FP64 && precision != IB_FP32_PRECOND && precision != IB_MIXED_PRECOND)
    return fail(IB_ERR_INVALID_ARG, "unknown precision");
  Problem& P = H->P;
  IB_TRY(resolve_vtimer(P));
  const int ix = precision == IB_FP32_PRECOND ? 0 : 1;
  if (count) *count = P.vt_n[ix];
  if (ms) *ms = P.vt_ms[ix];
  return IB_OK;
}

void ib_destroy(ib_problem* H) {
  if (!H) return;
  free_problem(&H->P);
  delete H;
}

}  // extern "C"

// ---------------------------------------------------------------- batches of independent problems

struct ib_batch {
  std::vector<ib_problem*> probs;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  std::vector<size_t> up_off, x_off;
  cudaStream_t caller = nullptr;
  cudaEvent_t start = nullptr;
  int threads = 1;
};

namespace {

// Run f(k) for k in [0, n) on up to `threads` host threads; returns the first
// failing status (IB_ERR_NOT_CONVERGED only if nothing worse happened) and its message.
// ids (may be NULL) names the problem of each k in the messages.
// Every worker makes the caller's current device its own before it runs f: a
// new host thread starts on device 0, whatever device the caller had selected.
template <typename F>
int parallel_for(int n, int threads, F f, std::string* msg, const std::vector<int>* ids = nullptr) {
  std::atomic<int> next(0);
  std::vector<int> codes(n, IB_OK);
  std::vector<std::string> msgs(n);
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    *msg = "cudaGetDevice failed";
    return IB_ERR_CUDA;
  }
  auto work = [&]() {
    if (cudaSetDevice(device) != cudaSuccess) {
      for (;;) {  // this worker cannot run anything: mark the items it takes
        int k = next.fetch_add(1);
        if (k >= n) return;
        codes[k] = IB_ERR_CUDA;
        msgs[k] = "problem " + std::to_string(ids ? (*ids)[k] : k) + ": cudaSetDevice failed";
      }
    }
    for (;;) {
      int k = next.fetch_add(1);
      if (k >= n) break;
      codes[k] = f(k);
      if (codes[k] != IB_OK) msgs[k] = "problem " + std::to_string(ids ? (*ids)[k] : k) + ": " + g_err;
    }
  };
  int nt = std::max(1, std::min(threads, n));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
  int worst = IB_OK;
  for (int k = 0; k < n; ++k) {
    if (codes[k] == IB_OK) continue;
    if (worst == IB_OK || (worst == IB_ERR_NOT_CONVERGED && codes[k] != IB_ERR_NOT_CONVERGED)) {
      worst = codes[k];
      *msg = msgs[k];
    }
  }
  return worst;
}

// Work order and worker count of a batch solve.  Order: longest first by the cost
// estimate N^2 g(sigma), g = min(1 + sigma / 1000, max_iters / 8) (the iteration
// count grows with the stiffness ratio sigma = dt kappa_max / mu: on the 256^2
// sweep 7-8 iterations up to sigma = 100, 15 at 1e3, ~105 at 1e4).  Workers: the
// fewest (up to the batch's thread count) whose longest-first schedule of these
// estimates ends within 5 % of the costliest problem, so that the long stiff
// runs, which set the makespan, share the GPU with as few other streams as the
// rest of the batch allows.
void batch_schedule(const ib_batch* B, std::vector<int>* order, int* workers) {
  const int n = (int)B->probs.size();
  std::vector<double> cost(n);
  for (int k = 0; k < n; ++k) {
    const Problem& P = B->probs[k]->P;
    const double g = std::min(1.0 + P.sigma / 1000.0, std::max(1.0, P.prm.max_iters / 8.0));
    cost[k] = (double)P.prm.N * P.prm.N * g;
  }
  order->resize(n);
  for (int k = 0; k < n; ++k) (*order)[k] = k;
  std::stable_sort(order->begin(), order->end(), [&](int a, int b) { return cost[a] > cost[b]; });
  const double cmax = n ? cost[(*order)[0]] : 0.0;
  *workers = std::max(1, B->threads);
  for (int w = 1; w < B->threads; ++w) {
    std::vector<double> load(w, 0.0);
    for (int k : *order) *std::min_element(load.begin(), load.end()) += cost[k];
    if (*std::max_element(load.begin(), load.end()) <= 1.05 * cmax) {
      *workers = w;
      break;
    }
  }
}

void free_batch(ib_batch* B) {
  if (!B) return;
  for (auto* p : B->probs)
    if (p) ib_destroy(p);
  for (auto s : B->streams)
    if (s) cudaStreamDestroy(s);
  for (auto e : B->done)
    if (e) cudaEventDestroy(e);
  if (B->start) cudaEventDestroy(B->start);
  delete B;
}

}  // namespace

extern "C" {

int ib_setup_batch(int32_t nprob, const ib_params* params, const int32_t* pt_off, const double* X,
                   const int32_t* sp_off, const int32_t* springs, const double* kappa, const double* rest,
                   void* stream, ib_batch** out) {
  g_err.clear();
  if (!out) return fail(IB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nprob < 1 || !params || !pt_off || !sp_off) return fail(IB_ERR_INVALID_ARG, "bad batch description");
  for (int k = 0; k < nprob; ++k) {
    if (pt_off[k + 1] < pt_off[k] || sp_off[k + 1] < sp_off[k])
      return fail(IB_ERR_INVALID_ARG, "batch offsets must be non-decreasing");
    IB_TRY(validate(&params[k]));
  }
  if (pt_off[0] != 0 || sp_off[0] != 0) return fail(IB_ERR_INVALID_ARG, "batch offsets must start at 0");
  ib_batch* B = new (std::nothrow) ib_batch();
  if (!B) return fail(IB_ERR_OOM, "host allocation failed");
  B->caller = (cudaStream_t)stream;
  B->probs.assign(nprob, nullptr);
  B->streams.assign(nprob, nullptr);
  B->done.assign(nprob, nullptr);
  unsigned hw = std::thread::hardware_concurrency();
  B->threads = (int)std::max(1u, std::min(hw ? hw : 4u, 16u));
  if (const char* e = std::getenv("IB_BATCH_THREADS")) {  // host worker threads (>= 1)
    int t = std::atoi(e);
    if (t >= 1) B->threads = std::min(t, 64);
  }
  size_t uo = 0, xo = 0;
  for (int k = 0; k < nprob; ++k) {
    B->up_off.push_back(uo);
    B->x_off.push_back(xo);
    uo += 3ul * params[k].N * params[k].N;
    xo += 2ul * (pt_off[k + 1] - pt_off[k]);
  }
  cudaError_t e = cudaEventCreateWithFlags(&B->start, cudaEventDisableTiming);
  // stiff problems (the long FGMRES runs that set the batch's makespan) get the
  // highest stream priority, so their latency-bound V-cycles are scheduled first
  int prio_low = 0, prio_high = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  const double sig_c = stiff_threshold();
  for (int k = 0; k < nprob && e == cudaSuccess; ++k) {
    const int s0 = sp_off[k], nsk = sp_off[k + 1] - s0;
    const bool stiff = kappa && stiffness(params[k], nsk, kappa + s0) >= sig_c;
    e = cudaStreamCreateWithPriority(&B->streams[k], cudaStreamNonBlocking, stiff ? prio_high : prio_low);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->done[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    free_batch(B);
    return fail(IB_ERR_CUDA, std::string("batch streams: ") + cudaGetErrorString(e));
  }
  std::string msg;
  int rc = parallel_for(nprob, B->threads, [&](int k) {
    const int p0 = pt_off[k], s0 = sp_off[k];
    return ib_setup(&params[k], pt_off[k + 1] - p0, X ? X + 2 * p0 : nullptr, sp_off[k + 1] - s0,
                    springs ? springs + 2 * s0 : nullptr, kappa ? kappa + s0 : nullptr,
                    rest ? rest + s0 : nullptr, B->streams[k], &B->probs[k]);
  }, &msg);
  if (rc != IB_OK) {
    free_batch(B);
    return fail(rc, msg);
  }
  *out = B;
  return IB_OK;
}

int ib_batch_size(const ib_batch* B) { return B ? (int)B->probs.size() : 0; }

ib_problem* ib_batch_problem(ib_batch* B, int32_t k) {
  if (!B || k < 0 || k >= (int)B->probs.size()) return nullptr;
  return B->probs[k];
}

int ib_solve_step_batch(ib_batch* B, const double* u_n_all, double* up_all, double* X_all, ib_stats* stats) {
  g_err.clear();
  if (!B || !up_all) return fail(IB_ERR_INVALID_ARG, "NULL argument");
  const int nprob = (int)B->probs.size();
  IB_CUDA_TRY(cudaEventRecord(B->start, B->caller));
  for (int k = 0; k < nprob; ++k) IB_CUDA_TRY(cudaStreamWaitEvent(B->streams[k], B->start, 0));
  std::vector<int> order;
  int workers = 1;
  batch_schedule(B, &order, &workers);
  std::string msg;
  int rc = parallel_for(nprob, workers, [&](int i) {
    const int k = order[i];
    Problem& P = B->probs[k]->P;
    const double* un = u_n_all ? u_n_all + (B->up_off[k] / 3) * 2 : nullptr;
    double* Xk = (X_all && P.np > 0) ? X_all + B->x_off[k] : nullptr;
    int c = solve_step_impl(P, un, up_all + B->up_off[k], Xk, stats ? &stats[k] : nullptr);
    cudaEventRecord(B->done[k], B->streams[k]);
    return c;
  }, &msg, &order);
  for (int k = 0; k < nprob; ++k) IB_CUDA_TRY(cudaStreamWaitEvent(B->caller, B->done[k], 0));
  if (rc != IB_OK) return fail(rc, msg);
  return IB_OK;
}

void ib_destroy_batch(ib_batch* B) { free_batch(B); }

}  // extern "C"
