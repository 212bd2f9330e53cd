// Internal definitions shared by the host runtime's translation units: the
// problem and batch handles of include/to.h, and the core launch.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "launch.cuh"
#include "to.h"

struct to_problem_s {
  int sys, n, m, T_max, device;
  const to::SysOps* ops;
  std::vector<double> params;
  void* d_params[2] = {nullptr, nullptr};   // parameter struct in float64, float32
  float* d_actor = nullptr;
  size_t n_actor = 0;
  size_t knot_scratch[2] = {0, 0};   // per-knot derivative scratch elements (FP64, mixed); 0 = none
  int tuned_G[2] = {0, 0};     // autotuned launch shape per precision (FP64, mixed); 0 = none
  int tuned_gpb[2] = {0, 0};
  int tuned_depth[2] = {0, 0};
  unsigned long long* chk = nullptr;   // bounds-check report of the checked build (4 words), else null
};

struct to_batch_s {
  to_problem p = nullptr;
  int B_max = 0;
  long long knots_max = 0;
  int elem_bytes = 0;
  size_t bytes = 0;
  size_t budget = 0;
  // inputs
  double* x0 = nullptr;
  int* T = nullptr;
  double* U_init = nullptr;
  int* forced = nullptr;
  size_t forced_cap = 0;
  bool has_uinit = false;
  // scheduling
  long long* toff = nullptr;
  int* order = nullptr;
  int* hist = nullptr;
  int* err = nullptr;
  int* queue = nullptr;
  // workspace
  void* traj = nullptr;
  void* gains = nullptr;
  void* dscr = nullptr;      // per-knot derivative scratch (systems with knot_scratch)
  double* vx = nullptr;
  // results
  double* J = nullptr;
  int* iters = nullptr;
  int* status = nullptr;
  int* slot = nullptr;
  int* ahist = nullptr;
  double* Jhist = nullptr;
  int hist_iter_cap = -1;
  // gather staging
  double* gX = nullptr;
  double* gU = nullptr;
  double* gV = nullptr;
  double* gK = nullptr;
  unsigned long long* prof = nullptr;   // 8 per-phase cycle counters
  // last solve
  int B = 0, max_iter = 0, prec = TO_MIXED, want_vx = 0, launches = 0, G = 8;
  const int* last_T = nullptr;
  cudaStream_t stream = nullptr;
  double grid_frac = 1.0;      // share of the resident CTAs a solve of this batch may take
};

// record the calling thread's error message and return code
int to_fail(int code, const std::string& msg);

// prepare + solver launch of one batch (serve != nullptr: serving mode, the
// solver claims requests from the serving ring and no prepare kernel runs)
int to_launch_core(to_batch b, int B, const double* d_x0, const int* d_T, const double* d_U, const int* d_forced,
                   const to_solver_opts* o, cudaStream_t s, const to::ServeArgs* serve);

// option validation (TO_ERR_ARG on a bad value)
int to_check_opts(const to_solver_opts* o);

// launch shape of a solve of B instances allowed frac of the resident CTAs
// (depth may be null: the shape's staging depth)
int to_resolve_shape(to_problem p, const to_solver_opts* o, int B, double frac, int* G, int* gpb, int* grid,
                     int* ctas_per_sm, int* depth = nullptr);

// grow the option-dependent workspace (per-iteration history; with
// want_traj, the X / U gather staging) so that a solve allocates nothing
int to_ensure_workspace(to_batch b, const to_solver_opts* o, bool want_traj);

// gather the last solve's X (B x (T_max+1) x n) and U (B x T_max x m) as
// float64 into device buffers (either may be null) on stream s
int to_enqueue_gather(to_batch b, int B, const int* d_T, double* d_X, double* d_U, cudaStream_t s);
