// Launch-shape autotuner and CUDA-graph solves of multi-system batches
// (include/to.h: totune, tograph_*).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "handles.h"

using namespace to;

#define GR_CK(x)                                                                                \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) return to_fail(TO_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace {

// owns the calibration batch, its stream and events
struct TuneScratch {
  to_batch b = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~TuneScratch() {
    if (s) cudaStreamSynchronize(s);
    if (b) tofree_batch(b);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
  }
};

// The persisted choice of the autotuner: when the environment variable
// TO_TUNE_CACHE names a file, each tuned shape is appended to it as one line
//   <key> <group_lanes> <groups_per_block> <ms> <stage_depth>
// and a later totune with the same key (in any process) takes the shape from
// the file instead of timing again.  The key holds what the best shape
// depends on: the system and its sizes, T_max, the batch size and the mean
// horizon (powers of two), the precision and LM mode, the GPU's name and SM
// count, and the library's build time (a rebuilt kernel is tuned again).
std::string tune_key(to_problem p, int B, const int* T, const to_solver_opts* o) {
  long long sum = 0;
  for (int i = 0; i < B; ++i) sum += T[i];
  const int meanT = (int)(sum / std::max(B, 1));
  int dev = 0;
  cudaDeviceProp prop{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "";
  std::string name(prop.name);
  for (char& c : name) if (c == ' ' || c == '\t') c = '_';
  auto log2i = [](long long v) { int l = 0; while (v > 1) { v >>= 1; ++l; } return l; };
  char buf[512];
  snprintf(buf, sizeof buf, "sys%d_n%d_m%d_Tmax%d_B2^%d_T2^%d_prec%d_reg%d_%s_sm%d_build%s_%s", p->sys, p->n, p->m,
           p->T_max, log2i(B), log2i(meanT), o->prec, o->reg, name.c_str(), prop.multiProcessorCount, __DATE__, __TIME__);
  std::string key(buf);
  for (char& c : key) if (c == ' ') c = '_';
  return key;
}

bool tune_cache_lookup(const std::string& key, int* G, int* gpb, double* ms, int* depth) {
  const char* path = std::getenv("TO_TUNE_CACHE");
  if (!path || !*path || key.empty()) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (std::fgets(line, sizeof line, f)) {
    char k[600];
    int g = 0, b = 0, d = 1;
    double t = 0;
    const int got = std::sscanf(line, "%599s %d %d %lf %d", k, &g, &b, &t, &d);
    if (got >= 4 && key == k) {
      *G = g; *gpb = b; *ms = t;          // the last entry for a key wins
      *depth = got == 5 ? d : 1;
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void tune_cache_store(const std::string& key, int G, int gpb, double ms, int depth) {
  const char* path = std::getenv("TO_TUNE_CACHE");
  if (!path || !*path || key.empty()) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %.6f %d\n", key.c_str(), G, gpb, ms, depth);
  std::fclose(f);
}

}  // namespace

int totune(to_problem p, int B, const double* x0, const int* T, to_solver_opts* opts, to_tune_row* rows,
           int max_rows, int* n_rows) {
  if (n_rows) *n_rows = 0;
  if (!p || !opts || B < 1 || !x0 || !T) return to_fail(TO_ERR_ARG, "totune: bad arguments");
  if (opts->forced_alpha || opts->want_vx || opts->profile_phases)
    return to_fail(TO_ERR_UNSUPPORTED, "totune: forced steps, want_vx and profiling are not tuned");
  int rc = to_check_opts(opts);
  if (rc) return rc;
  long long knots = 0;
  for (int i = 0; i < B; ++i) {
    if (T[i] < 1 || T[i] > p->T_max) return to_fail(TO_ERR_ARG, "totune: horizon outside [1, T_max]");
    knots += (long long)T[i] + 1;
  }
  const int prec0 = opts->prec == TO_FP64 ? PREC_FP64 : PREC_MIXED;
  const std::string key = tune_key(p, B, T, opts);
  {
    int G = 0, gpb = 0, depth = 1;
    double ms = 0;
    if (tune_cache_lookup(key, &G, &gpb, &ms, &depth)) {
      to_solver_opts o = *opts;
      o.group_lanes = G;
      o.groups_per_block = gpb;
      o.stage_depth = depth;
      int g2 = 0, b2 = 0, grid = 0, bps = 0;
      if (to_resolve_shape(p, &o, B, 1.0, &g2, &b2, &grid, &bps) == TO_OK) {
        opts->group_lanes = G;
        opts->groups_per_block = gpb;
        opts->stage_depth = depth;
        p->tuned_G[prec0] = G;
        p->tuned_gpb[prec0] = gpb;
        p->tuned_depth[prec0] = depth;
        if (rows && max_rows > 0) rows[0] = to_tune_row{G, gpb, grid, bps, ms, depth};
        if (n_rows) *n_rows = max_rows > 0 ? 1 : 0;
        return TO_OK;
      }
    }
  }
  TuneScratch w;
  to_solver_opts base = *opts;
  base.group_lanes = 0;
  base.groups_per_block = 0;
  base.stage_depth = 0;
  rc = tocreate_batch(p, B, knots, &base, &w.b);
  if (rc) return rc;
  rc = to_ensure_workspace(w.b, &base, false);
  if (rc) return rc;
  GR_CK(cudaStreamCreateWithFlags(&w.s, cudaStreamNonBlocking));
  GR_CK(cudaEventCreate(&w.e0));
  GR_CK(cudaEventCreate(&w.e1));
  GR_CK(cudaMemcpyAsync(w.b->x0, x0, sizeof(double) * B * p->n, cudaMemcpyHostToDevice, w.s));
  GR_CK(cudaMemcpyAsync(w.b->T, T, sizeof(int) * B, cudaMemcpyHostToDevice, w.s));

  const SysOps* ops = p->ops;
  const int prec = opts->prec == TO_FP64 ? PREC_FP64 : PREC_MIXED;
  int best_G = 0, best_gpb = 0, best_depth = 1, n = 0;
  double best_ms = INFINITY;
  const int cta_threads[] = {32, 64, 128, 256};
  for (int gi = 0; gi < ops->n_groups; ++gi) {
    const int G = ops->groups[gi];
    for (int depth = 1; depth <= (G > 1 ? ops->max_depth : 1); ++depth)
    for (int threads : cta_threads) {
      if (G > 32 && threads != 32) continue;            // one group per CTA: a single shape
      const int gpb = G > 32 ? 1 : threads / G;
      if (G * gpb > kMaxCtaThreads) continue;
      to_solver_opts o = base;
      o.group_lanes = G;
      o.groups_per_block = gpb;
      o.stage_depth = depth;
      int g2 = 0, b2 = 0, grid = 0, bps = 0;
      if (to_resolve_shape(p, &o, B, 1.0, &g2, &b2, &grid, &bps) != TO_OK) continue;   // does not fit an SM
      // one untimed solve (first launch of this instantiation), then the timed one
      rc = to_launch_core(w.b, B, w.b->x0, w.b->T, nullptr, nullptr, &o, w.s, nullptr);
      if (rc) return rc;
      GR_CK(cudaEventRecord(w.e0, w.s));
      rc = to_launch_core(w.b, B, w.b->x0, w.b->T, nullptr, nullptr, &o, w.s, nullptr);
      if (rc) return rc;
      GR_CK(cudaEventRecord(w.e1, w.s));
      GR_CK(cudaEventSynchronize(w.e1));
      float ms = 0;
      GR_CK(cudaEventElapsedTime(&ms, w.e0, w.e1));
      if (rows && n < max_rows) rows[n] = to_tune_row{G, gpb, grid, bps, (double)ms, depth};
      ++n;
      if (ms < best_ms) {
        best_ms = ms;
        best_G = G;
        best_gpb = gpb;
        best_depth = depth;
      }
    }
  }
  if (!best_G) return to_fail(TO_ERR_ARG, "totune: no launch shape fits an SM");
  tune_cache_store(key, best_G, best_gpb, best_ms, best_depth);
  opts->group_lanes = best_G;
  opts->groups_per_block = best_gpb;
  opts->stage_depth = best_depth;
  p->tuned_G[prec] = best_G;
  p->tuned_gpb[prec] = best_gpb;
  p->tuned_depth[prec] = best_depth;
  if (n_rows) *n_rows = std::min(n, max_rows);
  return TO_OK;
}

// ---------------------------------------------------------------------------
// CUDA graphs
// ---------------------------------------------------------------------------
struct to_graph_s {
  struct Member {
    to_batch b = nullptr;
    int B = 0;
    double* x0 = nullptr;   // pinned staging
    int* T = nullptr;
    double* X = nullptr;
    double* U = nullptr;
    double* J = nullptr;
    int* iters = nullptr;
    int* status = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
  };
  std::vector<Member> m;
  cudaStream_t stream = nullptr, last = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;
};

void tograph_destroy(to_graph g) {
  if (!g) return;
  if (g->last) cudaStreamSynchronize(g->last);
  // the members' batches must not keep a stream this graph is about to destroy
  for (auto& mm : g->m)
    if (mm.b && (mm.b->stream == g->stream || mm.b->stream == mm.s)) mm.b->stream = nullptr;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  for (auto& mm : g->m) {
    void* hp[] = {mm.x0, mm.T, mm.X, mm.U, mm.J, mm.iters, mm.status};
    for (void* q : hp)
      if (q) cudaFreeHost(q);
    if (mm.done) cudaEventDestroy(mm.done);
    if (mm.s) cudaStreamDestroy(mm.s);
  }
  if (g->fork) cudaEventDestroy(g->fork);
  if (g->stream) cudaStreamDestroy(g->stream);
  delete g;
}

template <class T>
static cudaError_t pinned(T** p, size_t count) {
  return cudaHostAlloc((void**)p, std::max<size_t>(count, 1) * sizeof(T), cudaHostAllocDefault);
}

// enqueue one member's branch on its stream (inside the capture)
static int record_member(to_graph_s::Member& mm, const to_solver_opts* opts, double frac, bool want_traj) {
  to_batch b = mm.b;
  to_problem p = b->p;
  const int B = mm.B;
  GR_CK(cudaMemcpyAsync(b->x0, mm.x0, sizeof(double) * B * p->n, cudaMemcpyHostToDevice, mm.s));
  GR_CK(cudaMemcpyAsync(b->T, mm.T, sizeof(int) * B, cudaMemcpyHostToDevice, mm.s));
  b->grid_frac = frac;
  int rc = to_launch_core(b, B, b->x0, b->T, nullptr, nullptr, opts, mm.s, nullptr);
  b->grid_frac = 1.0;
  if (rc) return rc;
  if (want_traj) {
    rc = to_enqueue_gather(b, B, b->T, b->gX, b->gU, mm.s);
    if (rc) return rc;
    GR_CK(cudaMemcpyAsync(mm.X, b->gX, sizeof(double) * B * (p->T_max + 1) * p->n, cudaMemcpyDeviceToHost, mm.s));
    GR_CK(cudaMemcpyAsync(mm.U, b->gU, sizeof(double) * B * p->T_max * p->m, cudaMemcpyDeviceToHost, mm.s));
  }
  GR_CK(cudaMemcpyAsync(mm.J, b->J, sizeof(double) * B, cudaMemcpyDeviceToHost, mm.s));
  GR_CK(cudaMemcpyAsync(mm.iters, b->iters, sizeof(int) * B, cudaMemcpyDeviceToHost, mm.s));
  GR_CK(cudaMemcpyAsync(mm.status, b->status, sizeof(int) * B, cudaMemcpyDeviceToHost, mm.s));
  GR_CK(cudaEventRecord(mm.done, mm.s));
  return TO_OK;
}

int tograph_create(const to_batch* batches, const int* B, const double* shares, int n, const to_solver_opts* opts,
                   int want_traj, to_graph* out) {
  if (!batches || !B || n < 1 || !out) return to_fail(TO_ERR_ARG, "tograph_create: bad arguments");
  *out = nullptr;
  to_solver_opts def;
  to_default_opts(&def);
  if (!opts) opts = &def;
  if (opts->forced_alpha || opts->want_vx || opts->profile_phases)
    return to_fail(TO_ERR_UNSUPPORTED, "tograph_create: forced steps, want_vx and profiling cannot be captured");
  int rc = to_check_opts(opts);
  if (rc) return rc;
  double total = 0;
  for (int i = 0; i < n; ++i) {
    if (!batches[i] || B[i] < 1 || B[i] > batches[i]->B_max)
      return to_fail(TO_ERR_ARG, "tograph_create: member " + std::to_string(i) + ": null batch or B outside [1, B_max]");
    if ((long long)B[i] * (batches[i]->p->T_max + 1) > batches[i]->knots_max)
      return to_fail(TO_ERR_BUDGET, "tograph_create: member " + std::to_string(i) +
                                        ": knots_max must hold B (T_max + 1) knots (horizons change between launches)");
    for (int j = 0; j < i; ++j)
      if (batches[j] == batches[i]) return to_fail(TO_ERR_ARG, "tograph_create: a batch appears twice");
    const double sh = shares ? shares[i] : 1.0;
    if (!(sh > 0)) return to_fail(TO_ERR_ARG, "tograph_create: shares must be > 0");
    total += sh;
  }
  to_graph g = new to_graph_s();
  g->m.resize(n);
  auto bail = [&](int code) { tograph_destroy(g); return code; };
  // workspace and staging first: nothing may allocate inside the capture
  for (int i = 0; i < n; ++i) {
    auto& mm = g->m[i];
    mm.b = batches[i];
    mm.B = B[i];
    to_problem p = mm.b->p;
    rc = to_ensure_workspace(mm.b, opts, want_traj != 0);
    if (rc) return bail(rc);
    cudaError_t e = pinned(&mm.x0, (size_t)mm.B * p->n);
    if (e == cudaSuccess) e = pinned(&mm.T, (size_t)mm.B);
    if (e == cudaSuccess && want_traj) e = pinned(&mm.X, (size_t)mm.B * (p->T_max + 1) * p->n);
    if (e == cudaSuccess && want_traj) e = pinned(&mm.U, (size_t)mm.B * p->T_max * p->m);
    if (e == cudaSuccess) e = pinned(&mm.J, (size_t)mm.B);
    if (e == cudaSuccess) e = pinned(&mm.iters, (size_t)mm.B);
    if (e == cudaSuccess) e = pinned(&mm.status, (size_t)mm.B);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&mm.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&mm.done, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(to_fail(TO_ERR_CUDA, std::string("tograph_create: ") + cudaGetErrorString(e)));
    for (int k = 0; k < mm.B; ++k) mm.T[k] = p->T_max;   // valid horizons until the caller fills them
  }
  cudaError_t e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return bail(to_fail(TO_ERR_CUDA, std::string("tograph_create: ") + cudaGetErrorString(e)));
  // fork: every member stream joins the capture through the fork event
  e = cudaEventRecord(g->fork, g->stream);
  int crc = e == cudaSuccess ? TO_OK : to_fail(TO_ERR_CUDA, std::string("tograph_create: ") + cudaGetErrorString(e));
  for (int i = 0; i < n && crc == TO_OK; ++i) {
    auto& mm = g->m[i];
    e = cudaStreamWaitEvent(mm.s, g->fork, 0);
    if (e != cudaSuccess) { crc = to_fail(TO_ERR_CUDA, std::string("tograph_create: ") + cudaGetErrorString(e)); break; }
    crc = record_member(mm, opts, (shares ? shares[i] : 1.0) / total, want_traj != 0);
    if (crc == TO_OK) {
      e = cudaStreamWaitEvent(g->stream, mm.done, 0);   // join
      if (e != cudaSuccess) crc = to_fail(TO_ERR_CUDA, std::string("tograph_create: ") + cudaGetErrorString(e));
    }
    g->launches += 2 + (want_traj ? 1 : 0);
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(g->stream, &graph);
  g->graph = graph;
  for (auto& mm : g->m) mm.b->stream = nullptr;   // nothing of the capture ran; no stream to wait for
  if (crc != TO_OK) return bail(crc);
  if (e != cudaSuccess) return bail(to_fail(TO_ERR_CUDA, std::string("tograph_create: capture: ") + cudaGetErrorString(e)));
  e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) return bail(to_fail(TO_ERR_CUDA, std::string("tograph_create: instantiate: ") + cudaGetErrorString(e)));
  *out = g;
  return TO_OK;
}

int tograph_staging(to_graph g, int member, double** x0, int** T, double** X, double** U, double** J, int** iters,
                    int** status) {
  if (!g || member < 0 || member >= (int)g->m.size()) return to_fail(TO_ERR_ARG, "tograph_staging: bad member");
  auto& mm = g->m[member];
  if (x0) *x0 = mm.x0;
  if (T) *T = mm.T;
  if (X) *X = mm.X;
  if (U) *U = mm.U;
  if (J) *J = mm.J;
  if (iters) *iters = mm.iters;
  if (status) *status = mm.status;
  return TO_OK;
}

int tograph_launch(to_graph g, void* cuda_stream) {
  if (!g || !g->exec) return to_fail(TO_ERR_ARG, "tograph_launch: null graph");
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : g->stream;
  for (auto& mm : g->m) {
    for (int k = 0; k < mm.B; ++k)
      if (mm.T[k] < 1 || mm.T[k] > mm.b->p->T_max) return to_fail(TO_ERR_ARG, "tograph_launch: horizon outside [1, T_max]");
  }
  GR_CK(cudaGraphLaunch(g->exec, s));
  g->last = s;
  for (auto& mm : g->m) {
    mm.b->stream = s;   // toget_trajectories on a member waits for this replay
    mm.b->launches = 2;
  }
  return TO_OK;
}

int tograph_sync(to_graph g) {
  if (!g) return to_fail(TO_ERR_ARG, "tograph_sync: null graph");
  if (g->last) GR_CK(cudaStreamSynchronize(g->last));
  return TO_OK;
}

int tograph_launch_count(to_graph g) { return g ? g->launches : 0; }
