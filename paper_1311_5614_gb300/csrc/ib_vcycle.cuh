// Launch arguments of the coarse-level ("tail") kernel, on one CTA or one
// thread-block cluster, and the
// host entry points of the V-cycle engine.
#pragma once

#include "ib_internal.cuh"

namespace ib {

constexpr int MAX_LEVELS = 16;

// T: vectors of the V-cycle; TM: the free-box inverse (float with T = double in
// the mixed-precision V-cycle).  Structure-box inverses are FP64 in every mode.
template <typename T, typename TM = T>
struct TailLevel {
  int N;
  StokesCoef<T> c;
  Patches<T> pat;
  const int* slot;  // box -> structure slot (-1 free)
  const double* Ms; // structure-box inverses (FP64)
  const TM* Mf;     // shared inverse of the structure-free boxes
  // assembled elasticity rows of the level (NULL Ew: the point path)
  const int* wrow;  // slot -> row
  const int* wn;    // row count (device)
  const T* Ew;      // windows [rows][WIN]
};

template <typename T, typename TM = T>
struct TailArgs {
  int nlev;  // levels in the tail: lev[0] is the finest of them, lev[nlev-1] the coarsest grid
  TailLevel<T, TM> lev[MAX_LEVELS];
  const T* b_in;  // right-hand side of lev[0] (global)
  T* w_out;       // correction of lev[0] (global)
  Springs<T> sp;
  T coefE;        // -dt / h_0^2: residual sign of the elasticity term
  const double* Mc;
  int nc, ldc;
  int nu1, nu2, box, nB, post_rev, has_E;
  int off_w[MAX_LEVELS], off_b[MAX_LEVELS], off_r, off_sr, off_sg;  // shared-memory offsets (bytes)
  // cluster form (the tail spread over the CTAs of one thread-block cluster): the
  // same arrays in global memory, W and B the levels' own buffers
  T* gw[MAX_LEVELS];
  T* gb[MAX_LEVELS];
  T* gr;    // residual scratch (3 N^2 of the tail's finest level)
  T* gre;   // elasticity term (2 N^2 of the tail's finest level; zero between phases)
};

template <typename T>
int vcycle_prepare(Problem& P);
template <typename T>
int vcycle_run(Problem& P);
int vcycle_reset_rE(Problem& P);

}  // namespace ib
