// Host runtime of libto.so: the C ABI of include/to.h.
//
// Problems own their parsed device parameters and actor weights; batches own
// the device workspace (knot records, gains, per-instance results).  A solve
// is two launches on the caller's stream: a one-CTA prepare kernel (horizon
// validation, knot offsets, longest-first order, queue reset) and the
// persistent solver kernel.  Nothing in a solve allocates once the batch has
// the capacity it needs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "launch.cuh"
#include "to.h"

namespace to {

const SysOps& pointmass_ops();
const SysOps& planar3_ops();
const SysOps& arm7_ops();
const SysOps& quad_ops();
const SysOps& dubins_ops();

const SysOps* sys_ops(int sys) {
  switch (sys) {
    case TO_SYS_POINTMASS2D: return &pointmass_ops();
    case TO_SYS_PLANAR3: return &planar3_ops();
    case TO_SYS_ARM7: return &arm7_ops();
    case TO_SYS_QUAD18: return &quad_ops();
    case TO_SYS_DUBINS: return &dubins_ops();
    default: return nullptr;
  }
}

// ---------------------------------------------------------------------------
// prepare: validate horizons, exclusive scan of (T+1), counting sort by T
// (longest first), reset the queue.  One CTA of 1024 threads.
// ---------------------------------------------------------------------------
__device__ long long block_exclusive_scan(long long v, long long* part, long long* total) {
  const int tid = threadIdx.x, nt = blockDim.x;
  part[tid] = v;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    long long a = tid >= off ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += a;
    __syncthreads();
  }
  long long incl = part[tid];
  *total = part[nt - 1];
  __syncthreads();
  return incl - v;
}

__global__ void prepare_kernel(int B, const int* __restrict__ T, int T_max, long long knots_max,
                               long long* __restrict__ toff, int* __restrict__ order, int* __restrict__ hist,
                               int* __restrict__ err, int* __restrict__ status_out, int* __restrict__ queue,
                               double* __restrict__ J_out, int* __restrict__ iters_out) {
  __shared__ long long part[1024];
  __shared__ int bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) { bad = 0; *queue = 0; }
  for (int i = tid; i <= T_max; i += nt) hist[i] = 0;
  __syncthreads();
  // knot offsets in instance order
  const int chunk = (B + nt - 1) / nt;
  const int lo = min(B, tid * chunk), hi = min(B, lo + chunk);
  long long s = 0;
  for (int i = lo; i < hi; ++i) {
    const int t = T[i];
    if (t < 1 || t > T_max) bad = 1;
    else atomicAdd(&hist[T_max - t], 1);
    s += (long long)t + 1;
  }
  long long total = 0;
  long long run = block_exclusive_scan(s, part, &total);
  for (int i = lo; i < hi; ++i) {
    toff[i] = run;
    run += (long long)T[i] + 1;
  }
  if (tid == 0 && total > knots_max) bad = 1;
  __syncthreads();
  // bucket starts (bins in decreasing horizon)
  const int nb = T_max + 1;
  const int bchunk = (nb + nt - 1) / nt;
  const int blo = min(nb, tid * bchunk), bhi = min(nb, blo + bchunk);
  long long bs = 0;
  for (int i = blo; i < bhi; ++i) bs += hist[i];
  long long btot = 0;
  long long brun = block_exclusive_scan(bs, part, &btot);
  for (int i = blo; i < bhi; ++i) {
    const int c = hist[i];
    hist[i] = (int)brun;
    brun += c;
  }
  __syncthreads();
  if (!bad) {
    for (int i = tid; i < B; i += nt) {
      const int pos = atomicAdd(&hist[T_max - T[i]], 1);
      order[pos] = i;
    }
  } else {
    for (int i = tid; i < B; i += nt) {
      status_out[i] = ST_NONFINITE;
      iters_out[i] = 0;
      J_out[i] = __longlong_as_double(0x7ff8000000000000LL);
    }
  }
  if (tid == 0) *err = bad;
}

// results to instance-major float64 arrays with the padding of include/to.h.
// A batch that the prepare kernel rejected (*err set: a horizon outside
// [1, T_max] or more knots than the workspace) ran no solve, so its offsets
// and slots are not valid: every output is NaN and nothing is read.  The
// horizon and slot are clamped to their ranges before use either way.
__global__ void gather_kernel(int B, int T_max, int n, int m, int RS, int GS, int NS, int rbytes,
                              const long long* __restrict__ toff, const int* __restrict__ T,
                              const int* __restrict__ slot,
                              const void* __restrict__ traj, const void* __restrict__ gains,
                              const double* __restrict__ vx, double* __restrict__ X, double* __restrict__ U,
                              double* __restrict__ Vx, double* __restrict__ K, const int* __restrict__ err) {
  const long long total = (long long)B * (T_max + 1);
  const bool rejected = err && *err;
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / (T_max + 1));
    const int k = (int)(t % (T_max + 1));
    if (rejected) {
      if (X) for (int i = 0; i < n; ++i) X[t * n + i] = qnan;
      if (U && k < T_max) for (int i = 0; i < m; ++i) U[((long long)b * T_max + k) * m + i] = qnan;
      if (Vx) for (int i = 0; i < n; ++i) Vx[t * n + i] = qnan;
      if (K && k < T_max) for (int i = 0; i < m * n; ++i) K[((long long)b * T_max + k) * m * n + i] = qnan;
      continue;
    }
    const int Tb = min(max(T[b], 0), T_max);
    const long long base = toff[b];
    const int sl = min(max(slot[b], 0), NS - 1);
    const long long xr = ((base + min(k, Tb)) * NS + sl) * RS;
    auto rd = [&](const void* p, long long idx) -> double {
      return rbytes == 8 ? reinterpret_cast<const double*>(p)[idx] : (double)reinterpret_cast<const float*>(p)[idx];
    };
    if (X)   // float32 records carry the state's low parts after u
      for (int i = 0; i < n; ++i) X[t * n + i] = rd(traj, xr + i) + (rbytes == 4 ? rd(traj, xr + n + m + i) : 0.0);
    if (U && k < T_max)
      for (int i = 0; i < m; ++i)
        U[((long long)b * T_max + k) * m + i] = k < Tb ? rd(traj, ((base + k) * NS + sl) * RS + n + i) : 0.0;
    if (Vx)
      for (int i = 0; i < n; ++i) Vx[t * n + i] = (vx && k <= Tb) ? vx[(base + k) * n + i] : 0.0;
    if (K && k < T_max)
      for (int i = 0; i < m * n; ++i)
        K[((long long)b * T_max + k) * m * n + i] = k < Tb ? rd(gains, (base + k) * GS + i) : 0.0;
  }
}

// Vbar_k = sum_{j=k}^{min(k+K,T)-1} l_j + [k + K >= T] l_T over the per-knot
// costs l (B x (T_max+1)); 0 past T.  One thread per knot, summed in order.
__global__ void window_kernel(int B, int T_max, int K, const int* __restrict__ T, const double* __restrict__ l,
                              double* __restrict__ Vbar) {
  const long long total = (long long)B * (T_max + 1);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / (T_max + 1)), k = (int)(t % (T_max + 1));
    const int Tb = T[b];
    if (k > Tb) {
      Vbar[t] = 0.0;
      continue;
    }
    const double* lb = l + (long long)b * (T_max + 1);
    const int end = min(k + K, Tb);
    double s = 0.0;
    for (int j = k; j < end; ++j) s += lb[j];
    if (k + K >= Tb) s += lb[Tb];
    Vbar[t] = s;
  }
}

}  // namespace to

// ===========================================================================
// C ABI
// ===========================================================================
using namespace to;

static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define TO_CK(x)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess) return fail(TO_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#include "handles.h"

// Exported functions take C linkage from their declarations in to.h.

const char* tolast_error(void) { return g_err.c_str(); }

void to_default_opts(to_solver_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_iter = 100;
  o->tol_rel = 1e-8;
  o->eps_clip = 1e-8;
  o->n_alpha = 16;
  o->alpha_decay = 0.5;
  o->prec = TO_MIXED;
  o->refine = 1;
  o->forced_alpha = nullptr;
  o->want_vx = 0;
  o->hbm_budget_bytes = 0;
  o->group_lanes = 0;
  o->groups_per_block = 0;
}

int tocreate_problem(const to_problem_desc* d, to_problem* out) {
  if (!d || !out) return fail(TO_ERR_ARG, "tocreate_problem: null argument");
  *out = nullptr;
  const SysOps* ops = sys_ops(d->sys);
  if (!ops) return fail(TO_ERR_ARG, "tocreate_problem: unknown system id");
  if (d->n != ops->n || d->m != ops->m) return fail(TO_ERR_ARG, "tocreate_problem: n, m do not match the system");
  if (d->T_max < 1) return fail(TO_ERR_ARG, "tocreate_problem: T_max must be >= 1");
  if (!d->params || d->n_params < 1) return fail(TO_ERR_ARG, "tocreate_problem: params missing");
  if (d->params[0] != d->dt || !(d->dt > 0)) return fail(TO_ERR_ARG, "tocreate_problem: dt must be > 0 and equal params[0]");
  if (!std::isinf(d->u_max) || d->u_max < 0) return fail(TO_ERR_UNSUPPORTED, "tocreate_problem: control bounds are not supported (u_max must be +inf)");
  if (d->actor_w && !ops->accepts_actor) return fail(TO_ERR_ARG, "tocreate_problem: this system takes no actor weights");
  std::vector<unsigned char> blob64, blob32;
  std::string err;
  if (ops->parse(d->params, d->n_params, blob64, blob32, err) != 0) return fail(TO_ERR_ARG, "tocreate_problem: " + err);
  to_problem p = new to_problem_s();
  p->sys = d->sys; p->n = d->n; p->m = d->m; p->T_max = d->T_max;
  p->ops = ops;
  p->params.assign(d->params, d->params + d->n_params);
  if (ops->knot_scratch)
    for (int pi = 0; pi < 2; ++pi) p->knot_scratch[pi] = ops->knot_scratch(d->params, d->n_params, pi);
  cudaGetDevice(&p->device);
  cudaError_t e = cudaMalloc(&p->d_params[0], blob64.size());
  if (e == cudaSuccess) e = cudaMemcpy(p->d_params[0], blob64.data(), blob64.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_params[1], blob32.size());
  if (e == cudaSuccess) e = cudaMemcpy(p->d_params[1], blob32.data(), blob32.size(), cudaMemcpyHostToDevice);
#ifdef TO_CHECKED
  if (e == cudaSuccess) e = cudaMalloc(&p->chk, 4 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(p->chk, 0, 4 * sizeof(unsigned long long));
#endif
  if (e == cudaSuccess && d->actor_w) {
    // W1 b1 W2 b2 W3 b3 with every W (out x in, row-major) stored transposed
    const int H = 256, n = d->n, m = d->m;
    const size_t expect = (size_t)n * H + H + (size_t)H * H + H + (size_t)H * m + m;
    if (d->n_actor_w != expect) {
      todestroy_problem(p);
      return fail(TO_ERR_ARG, "tocreate_problem: actor weights must be 36x256, 256, 256x256, 256, 12x256, 12");
    }
    std::vector<float> t(expect);
    const float* s = d->actor_w;
    size_t o = 0;
    auto transpose = [&](int rows, int cols) {   // source rows x cols -> cols x rows
      for (int i = 0; i < cols; ++i)
        for (int j = 0; j < rows; ++j) t[o + (size_t)i * rows + j] = s[o + (size_t)j * cols + i];
      o += (size_t)rows * cols;
    };
    auto copy = [&](int k) {
      for (int i = 0; i < k; ++i) t[o + i] = s[o + i];
      o += k;
    };
    transpose(H, n); copy(H); transpose(H, H); copy(H); transpose(m, H); copy(m);
    p->n_actor = expect;
    e = cudaMalloc(&p->d_actor, p->n_actor * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_actor, t.data(), p->n_actor * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    todestroy_problem(p);
    return fail(TO_ERR_CUDA, std::string("tocreate_problem: ") + cudaGetErrorString(e));
  }
  *out = p;
  return TO_OK;
}

int tobounds_checked(void) {
#ifdef TO_CHECKED
  return 1;
#else
  return 0;
#endif
}

int toget_bounds_report(to_problem p, long long* out4, int reset) {
  if (!p || !out4) return fail(TO_ERR_ARG, "toget_bounds_report: null argument");
  if (!p->chk) return fail(TO_ERR_UNSUPPORTED, "toget_bounds_report: the library was built without bounds checks");
  unsigned long long h[4];
  TO_CK(cudaDeviceSynchronize());
  TO_CK(cudaMemcpy(h, p->chk, sizeof(h), cudaMemcpyDeviceToHost));
  for (int i = 0; i < 4; ++i) out4[i] = (long long)h[i];
  if (reset) TO_CK(cudaMemset(p->chk, 0, sizeof(h)));
  return TO_OK;
}

void todestroy_problem(to_problem p) {
  if (!p) return;
  for (void* q : p->d_params)
    if (q) cudaFree(q);
  if (p->d_actor) cudaFree(p->d_actor);
  if (p->chk) cudaFree(p->chk);
  delete p;
}

static void free_batch_buffers(to_batch b) {
  void* ptrs[] = {b->x0, b->T, b->U_init, b->forced, b->toff, b->order, b->hist, b->err, b->queue, b->traj,
                  b->gains, b->dscr, b->vx, b->J, b->iters, b->status, b->slot, b->ahist, b->Jhist, b->gX, b->gU,
                  b->gV, b->gK, b->prof};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

void tofree_batch(to_batch b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  free_batch_buffers(b);
  delete b;
}

template <class T>
static cudaError_t grow(T*& ptr, size_t count, size_t& bytes) {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes += count * sizeof(T);
  return cudaMalloc(&ptr, std::max<size_t>(count, 1) * sizeof(T));
}

static size_t workspace_bytes(const to_problem p, int B, long long knots, int elem, int prec_idx) {
  const SysOps* o = p->ops;
  size_t s = (size_t)B * (p->n * 8 + 4 + 8 + 4 + 8 + 4 + 4) + (size_t)(p->T_max + 2) * 4 + 8;
  s += (size_t)knots * (kMaxSlots * o->rs[prec_idx] + o->gs[prec_idx] + p->knot_scratch[prec_idx]) * elem;
  return s;
}

int tocreate_batch(to_problem p, int B_max, long long knots_max, const to_solver_opts* opts, to_batch* out) {
  if (!p || !out || B_max < 1 || knots_max < 2) return fail(TO_ERR_ARG, "tocreate_batch: bad arguments");
  to_solver_opts def;
  to_default_opts(&def);
  if (!opts) opts = &def;
  const int prec_idx = opts->prec == TO_FP64 ? 0 : 1;
  const int elem = opts->prec == TO_FP64 ? 8 : 4;
  const size_t need = workspace_bytes(p, B_max, knots_max, elem, prec_idx);
  if (opts->hbm_budget_bytes && need > opts->hbm_budget_bytes)
    return fail(TO_ERR_BUDGET, "tocreate_batch: workspace of " + std::to_string(need) + " bytes exceeds the HBM budget");
  to_batch b = new to_batch_s();
  b->p = p;
  b->B_max = B_max;
  b->knots_max = knots_max;
  b->elem_bytes = elem;
  b->budget = opts->hbm_budget_bytes;
  size_t bytes = 0;
  cudaError_t e = cudaSuccess;
  const SysOps* o = p->ops;
  if (e == cudaSuccess) e = grow(b->x0, (size_t)B_max * p->n, bytes);
  if (e == cudaSuccess) e = grow(b->T, (size_t)B_max, bytes);
  if (e == cudaSuccess) e = grow(b->toff, (size_t)B_max, bytes);
  if (e == cudaSuccess) e = grow(b->order, (size_t)B_max, bytes);
  if (e == cudaSuccess) e = grow(b->hist, (size_t)p->T_max + 2, bytes);
  if (e == cudaSuccess) e = grow(b->err, (size_t)1, bytes);
  if (e == cudaSuccess) e = grow(b->queue, (size_t)1, bytes);
  if (e == cudaSuccess) e = grow(b->J, (size_t)B_max, bytes);
  if (e == cudaSuccess) e = grow(b->iters, (size_t)B_max, bytes);
  if (e == cudaSuccess) e = grow(b->status, (size_t)B_max, bytes);
  if (e == cudaSuccess) e = grow(b->slot, (size_t)B_max, bytes);
  if (e == cudaSuccess) {
    bytes += (size_t)knots_max * (kMaxSlots * o->rs[prec_idx] + o->gs[prec_idx]) * elem;
    e = cudaMalloc(&b->traj, (size_t)knots_max * kMaxSlots * o->rs[prec_idx] * elem);
    if (e == cudaSuccess) e = cudaMalloc(&b->gains, (size_t)knots_max * o->gs[prec_idx] * elem);
  }
  if (e == cudaSuccess && p->knot_scratch[prec_idx]) {
    bytes += (size_t)knots_max * p->knot_scratch[prec_idx] * elem;
    e = cudaMalloc(&b->dscr, (size_t)knots_max * p->knot_scratch[prec_idx] * elem);
  }
  b->bytes = bytes;
  if (e != cudaSuccess) {
    free_batch_buffers(b);
    delete b;
    return fail(TO_ERR_CUDA, std::string("tocreate_batch: ") + cudaGetErrorString(e));
  }
  *out = b;
  return TO_OK;
}

// grow the parts of the workspace that depend on the solve's options
static int ensure_options(to_batch b, const to_solver_opts* o, bool need_uinit, bool need_forced) {
  to_problem p = b->p;
  const int elem = o->prec == TO_FP64 ? 8 : 4;
  if (elem > b->elem_bytes) return fail(TO_ERR_ARG, "solve: batch was created for mixed precision; FP64 needs a batch created with prec = TO_FP64");
  size_t extra = 0;
  cudaError_t e = cudaSuccess;
  if (b->hist_iter_cap < o->max_iter) {
    e = grow(b->ahist, (size_t)b->B_max * std::max(o->max_iter, 1), extra);
    if (e == cudaSuccess) e = grow(b->Jhist, (size_t)b->B_max * (o->max_iter + 1), extra);
    if (e != cudaSuccess) return fail(TO_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(e));
    b->hist_iter_cap = o->max_iter;
  }
  if (o->want_vx && !b->vx) {
    e = grow(b->vx, (size_t)b->knots_max * p->n, extra);
    if (e != cudaSuccess) return fail(TO_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(e));
  }
  if (need_uinit && !b->U_init) {
    e = grow(b->U_init, (size_t)b->B_max * p->T_max * p->m, extra);
    if (e != cudaSuccess) return fail(TO_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(e));
  }
  if (need_forced && b->forced_cap < (size_t)b->B_max * o->max_iter) {
    e = grow(b->forced, (size_t)b->B_max * o->max_iter, extra);
    if (e != cudaSuccess) return fail(TO_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(e));
    b->forced_cap = (size_t)b->B_max * o->max_iter;
  }
  b->bytes += extra;
  if (b->budget && b->bytes > b->budget) return fail(TO_ERR_BUDGET, "solve: workspace exceeds the HBM budget");
  return TO_OK;
}

static int check_opts(const to_solver_opts* o) {
  if (o->max_iter < 0) return fail(TO_ERR_ARG, "opts: max_iter must be >= 0");
  if (o->n_alpha < 1 || o->n_alpha > kMaxAlpha) return fail(TO_ERR_ARG, "opts: n_alpha must be in [1, 32]");
  if (!(o->alpha_decay > 0 && o->alpha_decay <= 1)) return fail(TO_ERR_ARG, "opts: alpha_decay must be in (0, 1]");
  if (!(o->eps_clip >= 0)) return fail(TO_ERR_ARG, "opts: eps_clip must be >= 0");
  if (o->prec != TO_FP64 && o->prec != TO_MIXED) return fail(TO_ERR_ARG, "opts: prec must be TO_FP64 or TO_MIXED");
  if (o->reg != TO_REG_CLIP && o->reg != TO_REG_LM) return fail(TO_ERR_ARG, "opts: reg must be TO_REG_CLIP or TO_REG_LM");
  if (o->stage_depth < 0 || o->stage_depth > 2) return fail(TO_ERR_ARG, "opts: stage_depth must be 0, 1 or 2");
  return TO_OK;
}

// launch shape of a solve: group size, groups per CTA, staging depth, CTAs
// (persistent: at most frac of the CTAs the GPU holds resident at once)
static int resolve_shape(to_problem p, const to_solver_opts* o, int B, double frac, int* G_out, int* gpb_out,
                         int* grid_out, int* bps_out, int* depth_out) {
  const SysOps* ops = p->ops;
  const int prec = o->prec == TO_FP64 ? PREC_FP64 : PREC_MIXED;
  int G = o->group_lanes, gpb = o->groups_per_block, depth = o->stage_depth;
  if (!G && !gpb && !depth && p->tuned_G[prec]) {
    G = p->tuned_G[prec];
    gpb = p->tuned_gpb[prec];
    depth = p->tuned_depth[prec];
  }
  if (!depth) depth = 1;
  if (!G) G = ops->default_G;
  if (!gpb) {
    gpb = ops->default_gpb[prec];
    if (G <= 32 && (G * gpb) % 32 != 0) gpb = 64 / G;   // a group size other than the default: 64-thread CTAs
  }
  bool okG = false;
  for (int i = 0; i < ops->n_groups; ++i) okG |= ops->groups[i] == G;
  if (!okG) return fail(TO_ERR_ARG, "opts: group_lanes not supported by this system");
  if (G <= 32 && (G * gpb) % 32 != 0) return fail(TO_ERR_ARG, "opts: groups_per_block * group_lanes must be a multiple of 32");
  if (G > 32 && gpb != 1) return fail(TO_ERR_ARG, "opts: groups_per_block must be 1 when group_lanes > 32");
  if (G * gpb > kMaxCtaThreads) return fail(TO_ERR_ARG, "opts: CTA larger than 256 threads");
  if (depth > ops->max_depth || (depth > 1 && G == 1))
    return fail(TO_ERR_ARG, "opts: stage_depth not offered by this system at this group size");
  size_t smem = 0;
  int bps = 0;
  TO_CK(ops->occupancy(prec, G, depth, gpb, &smem, &bps));
  if (bps < 1) return fail(TO_ERR_ARG, "opts: launch shape does not fit on an SM");
  int dev = 0, sms = 0;
  TO_CK(cudaGetDevice(&dev));
  TO_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int cap = std::max(1, (int)(bps * sms * std::min(1.0, std::max(frac, 0.0))));
  *G_out = G;
  *gpb_out = gpb;
  *grid_out = std::max(1, std::min((B + gpb - 1) / gpb, cap));
  if (bps_out) *bps_out = bps;
  if (depth_out) *depth_out = depth;
  return TO_OK;
}

// the solver arguments of one batch (everything but the serving ring and the
// phase counters)
static int fill_solve_args(to_batch b, int B, const double* d_x0, const int* d_T, const double* d_U, const int* d_forced,
                           const to_solver_opts* o, SolveArgs& a) {
  to_problem p = b->p;
  const int prec = o->prec == TO_FP64 ? PREC_FP64 : PREC_MIXED;
  a.B = B; a.T_max = p->T_max; a.max_iter = o->max_iter; a.n_alpha = o->n_alpha;
  a.refine = o->refine; a.want_vx = o->want_vx;
  a.tol = o->tol_rel; a.eps = o->eps_clip;
  a.lm = o->reg == TO_REG_LM ? 1 : 0;
  if (a.lm) a.eps = -1e30;   // no clipping: every eigenvalue is above the floor
  double al = 1.0;
  for (int j = 0; j < kMaxAlpha; ++j) {
    a.alpha_d[j] = al;
    a.alpha_f[j] = (float)al;
    al *= o->alpha_decay;
  }
  a.x0 = d_x0; a.T = d_T; a.U_init = d_U; a.forced = d_forced;
  a.toff = b->toff; a.order = b->order; a.queue = b->queue;
  a.traj = b->traj; a.gains = b->gains; a.vx = o->want_vx ? b->vx : nullptr;
  a.kscr = (long long)p->knot_scratch[prec == PREC_FP64 ? 0 : 1];
  a.dscr = b->dscr;
  if (a.kscr && !a.dscr) return fail(TO_ERR_ARG, "solve: the batch has no derivative scratch for this precision");
  a.J_out = b->J; a.iters_out = b->iters; a.status_out = b->status; a.slot_out = b->slot;
  a.ahist = b->ahist; a.Jhist = b->Jhist;
  a.params = p->d_params[prec == PREC_FP64 ? 0 : 1]; a.actor_w = p->d_actor; a.err = b->err;
  a.prof = nullptr;
  a.knots_cap = b->knots_max;
  a.chk = p->chk;
  return TO_OK;
}

static int launch_solve(to_batch b, int B, const double* d_x0, const int* d_T, const double* d_U, const int* d_forced,
                        const to_solver_opts* o, cudaStream_t s, const ServeArgs* serve = nullptr) {
  to_problem p = b->p;
  const SysOps* ops = p->ops;
  const int prec = o->prec == TO_FP64 ? PREC_FP64 : PREC_MIXED;
  // the problem's parameters and actor weights live on the device that was
  // current when it was created; a launch from another device would hand the
  // kernel another GPU's pointers
  int cur_dev = -1;
  TO_CK(cudaGetDevice(&cur_dev));
  if (cur_dev != p->device)
    return fail(TO_ERR_ARG, "solve: the current device is " + std::to_string(cur_dev) + ", the problem was created on " +
                                std::to_string(p->device));
  // a serving kernel, or a member of a multi-system graph, takes its share of
  // the resident CTAs, so the kernels of the other problems run beside it
  const double frac = serve ? serve->grid_frac : b->grid_frac;
  int G = 0, gpb = 0, grid = 0, depth = 1;
  int rc = resolve_shape(p, o, B, frac, &G, &gpb, &grid, nullptr, &depth);
  if (rc) return rc;

  SolveArgs a{};
  rc = fill_solve_args(b, B, d_x0, d_T, d_U, d_forced, o, a);
  if (rc) return rc;
  if (o->profile_phases) {
    if (!b->prof) TO_CK(cudaMalloc(&b->prof, 8 * sizeof(unsigned long long)));
    TO_CK(cudaMemsetAsync(b->prof, 0, 8 * sizeof(unsigned long long), s));
    a.prof = b->prof;
  }

  if (serve) {
    a.serve = *serve;    // seats replace the batch; nothing to sort or offset
  } else {
    prepare_kernel<<<1, 1024, 0, s>>>(B, d_T, p->T_max, b->knots_max, b->toff, b->order, b->hist, b->err, b->status,
                                      b->queue, b->J, b->iters);
    TO_CK(cudaGetLastError());
  }
  TO_CK(ops->launch(prec, G, depth, gpb, grid, s, a));
  b->B = B;
  b->max_iter = o->max_iter;
  b->prec = o->prec;
  b->want_vx = o->want_vx;
  b->stream = s;
  b->launches = 2;
  b->G = G;
  b->last_T = d_T;
  return TO_OK;
}

int to_fail(int code, const std::string& msg) { return fail(code, msg); }

int to_check_opts(const to_solver_opts* o) { return check_opts(o); }

int to_resolve_shape(to_problem p, const to_solver_opts* o, int B, double frac, int* G, int* gpb, int* grid, int* bps,
                     int* depth) {
  return resolve_shape(p, o, B, frac, G, gpb, grid, bps, depth);
}

int to_ensure_workspace(to_batch b, const to_solver_opts* o, bool want_traj) {
  int rc = ensure_options(b, o, false, false);
  if (rc) return rc;
  to_problem p = b->p;
  size_t dummy = 0;
  if (want_traj && !b->gX) TO_CK(grow(b->gX, (size_t)b->B_max * (p->T_max + 1) * p->n, dummy));
  if (want_traj && !b->gU) TO_CK(grow(b->gU, (size_t)b->B_max * p->T_max * p->m, dummy));
  return TO_OK;
}

int to_enqueue_gather(to_batch b, int B, const int* d_T, double* d_X, double* d_U, cudaStream_t s) {
  to_problem p = b->p;
  const int pi = b->prec == TO_FP64 ? 0 : 1;
  const int NS = std::min(b->G, kLsWidth) + 1;
  gather_kernel<<<1024, 256, 0, s>>>(B, p->T_max, p->n, p->m, p->ops->rs[pi], p->ops->gs[pi], NS, pi == 0 ? 8 : 4,
                                     b->toff, d_T, b->slot, b->traj, b->gains, nullptr, d_X, d_U, nullptr, nullptr,
                                     b->err);
  TO_CK(cudaGetLastError());
  return TO_OK;
}

int to_launch_core(to_batch b, int B, const double* d_x0, const int* d_T, const double* d_U, const int* d_forced,
                   const to_solver_opts* o, cudaStream_t s, const ServeArgs* serve) {
  return launch_solve(b, B, d_x0, d_T, d_U, d_forced, o, s, serve);
}

int tosolve_batch_device(to_batch b, int B, const double* d_x0, const int* d_T, const double* d_U_init,
                         const int* d_forced, const to_solver_opts* opts, void* cuda_stream) {
  if (!b) return fail(TO_ERR_ARG, "tosolve_batch_device: null batch");
  to_solver_opts def;
  to_default_opts(&def);
  if (!opts) opts = &def;
  int rc = check_opts(opts);
  if (rc) return rc;
  if (B < 0 || B > b->B_max) return fail(TO_ERR_BUDGET, "tosolve_batch_device: B exceeds the batch capacity");
  if (B > 0 && (!d_x0 || !d_T)) return fail(TO_ERR_ARG, "tosolve_batch_device: x0 and T are required");
  rc = ensure_options(b, opts, false, false);
  if (rc) return rc;
  if (B == 0) { b->B = 0; b->launches = 0; return TO_OK; }
  return launch_solve(b, B, d_x0, d_T, d_U_init, d_forced, opts, (cudaStream_t)cuda_stream);
}

int tosolve_systems(const to_batch* batches, const int* Bs, const double* const* d_x0, const int* const* d_T, int n,
                    const to_solver_opts* opts, void* cuda_stream) {
  if (!batches || !Bs || !d_x0 || !d_T || n < 1 || n > kMultiSystems)
    return fail(TO_ERR_ARG, "tosolve_systems: null argument or n outside [1, 3]");
  to_solver_opts def;
  to_default_opts(&def);
  if (!opts) opts = &def;
  int rc = check_opts(opts);
  if (rc) return rc;
  if (opts->forced_alpha || opts->want_vx || opts->profile_phases || opts->group_lanes || opts->groups_per_block)
    return fail(TO_ERR_UNSUPPORTED, "tosolve_systems: forced steps, want_vx, profiling and launch shapes are not available");
  const int prec = opts->prec == TO_FP64 ? PREC_FP64 : PREC_MIXED;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int cur_dev = -1;
  TO_CK(cudaGetDevice(&cur_dev));
  MultiArgs m{};
  int slot_of[kMultiSystems];
  for (int i = 0; i < n; ++i) {
    to_batch b = batches[i];
    if (!b) return fail(TO_ERR_ARG, "tosolve_systems: null batch");
    const int sys = b->p->sys;
    const int slot = sys == TO_SYS_ARM7 ? 0 : sys == TO_SYS_PLANAR3 ? 1 : sys == TO_SYS_POINTMASS2D ? 2 : -1;
    if (slot < 0) return fail(TO_ERR_UNSUPPORTED, "tosolve_systems: the fused launch covers the 7-DoF arm, the planar "
                                                  "arm and the point mass");
    if (m.present[slot]) return fail(TO_ERR_ARG, "tosolve_systems: one batch per system");
    if (b->p->device != cur_dev) return fail(TO_ERR_ARG, "tosolve_systems: a problem lives on another device");
    if (Bs[i] < 1 || Bs[i] > b->B_max || !d_x0[i] || !d_T[i])
      return fail(TO_ERR_ARG, "tosolve_systems: B outside [1, B_max] or missing inputs");
    rc = ensure_options(b, opts, false, false);
    if (rc) return rc;
    rc = fill_solve_args(b, Bs[i], d_x0[i], d_T[i], nullptr, nullptr, opts, m.a[slot]);
    if (rc) return rc;
    m.present[slot] = 1;
    slot_of[i] = slot;
  }
  size_t smem = 0;
  int bps = 0, sms = 0;
  TO_CK(multi_occupancy(prec, &smem, &bps));
  if (bps < 1) return fail(TO_ERR_ARG, "tosolve_systems: the fused kernel does not fit on an SM");
  TO_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cur_dev));
  for (int i = 0; i < n; ++i) {
    to_batch b = batches[i];
    prepare_kernel<<<1, 1024, 0, s>>>(Bs[i], d_T[i], b->p->T_max, b->knots_max, b->toff, b->order, b->hist, b->err,
                                      b->status, b->queue, b->J, b->iters);
    TO_CK(cudaGetLastError());
  }
  TO_CK(multi_launch(prec, bps * sms, s, m));
  for (int i = 0; i < n; ++i) {
    to_batch b = batches[i];
    b->B = Bs[i];
    b->max_iter = opts->max_iter;
    b->prec = opts->prec;
    b->want_vx = 0;
    b->stream = s;
    b->launches = i == 0 ? n + 1 : 0;     // n prepare kernels and the one fused solver launch
    b->G = multi_group_lanes(slot_of[i]);
    b->last_T = d_T[i];
  }
  return TO_OK;
}

int tosolve_batch(to_problem p, int B, const double* x0, const int* T, const double* U_init,
                  const to_solver_opts* opts, void* cuda_stream, to_batch* out) {
  if (!p || !out) return fail(TO_ERR_ARG, "tosolve_batch: null argument");
  to_solver_opts def;
  to_default_opts(&def);
  if (!opts) opts = &def;
  int rc = check_opts(opts);
  if (rc) return rc;
  if (B < 0 || (B > 0 && (!x0 || !T))) return fail(TO_ERR_ARG, "tosolve_batch: x0 and T are required");
  long long knots = 0;
  for (int i = 0; i < B; ++i) {
    if (T[i] < 1 || T[i] > p->T_max) return fail(TO_ERR_ARG, "tosolve_batch: horizon outside [1, T_max]");
    knots += (long long)T[i] + 1;
  }
  for (long long i = 0; i < (long long)B * p->n; ++i)
    if (!std::isfinite(x0[i])) { /* a non-finite x0 yields TO_ST_NONFINITE for that instance only */ }
  if (!*out) {
    rc = tocreate_batch(p, std::max(B, 1), std::max(knots, 2LL), opts, out);
    if (rc) return rc;
  }
  to_batch b = *out;
  if (b->p != p) return fail(TO_ERR_ARG, "tosolve_batch: batch belongs to another problem");
  if (B > b->B_max || knots > b->knots_max) return fail(TO_ERR_BUDGET, "tosolve_batch: batch capacity too small");
  rc = ensure_options(b, opts, U_init != nullptr, opts->forced_alpha != nullptr);
  if (rc) return rc;
  if (B == 0) { b->B = 0; b->launches = 0; return TO_OK; }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  TO_CK(cudaMemcpyAsync(b->x0, x0, sizeof(double) * B * p->n, cudaMemcpyHostToDevice, s));
  TO_CK(cudaMemcpyAsync(b->T, T, sizeof(int) * B, cudaMemcpyHostToDevice, s));
  if (U_init) TO_CK(cudaMemcpyAsync(b->U_init, U_init, sizeof(double) * B * p->T_max * p->m, cudaMemcpyHostToDevice, s));
  if (opts->forced_alpha)
    TO_CK(cudaMemcpyAsync(b->forced, opts->forced_alpha, sizeof(int) * B * opts->max_iter, cudaMemcpyHostToDevice, s));
  return launch_solve(b, B, b->x0, b->T, U_init ? b->U_init : nullptr, opts->forced_alpha ? b->forced : nullptr, opts, s);
}

int toget_device_results(to_batch b, const double** d_J, const int** d_iters, const int** d_status) {
  if (!b) return fail(TO_ERR_ARG, "toget_device_results: null batch");
  if (d_J) *d_J = b->J;
  if (d_iters) *d_iters = b->iters;
  if (d_status) *d_status = b->status;
  return TO_OK;
}

int tolast_launch_count(to_batch b) { return b ? b->launches : 0; }

int toget_phase_cycles(to_batch b, unsigned long long* out) {
  if (!b || !out) return fail(TO_ERR_ARG, "toget_phase_cycles: null argument");
  for (int i = 0; i < 8; ++i) out[i] = 0;
  if (!b->prof) return TO_OK;
  TO_CK(cudaStreamSynchronize(b->stream));
  TO_CK(cudaMemcpy(out, b->prof, 7 * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  for (int i = 0; i < 7; ++i) out[7] += out[i];
  return TO_OK;
}

int toget_trajectories(to_batch b, double* X, double* U, double* J, int* iters, int* status, double* Vx, double* K) {
  if (!b) return fail(TO_ERR_ARG, "toget_trajectories: null batch");
  to_problem p = b->p;
  const int B = b->B;
  TO_CK(cudaStreamSynchronize(b->stream));
  if (B == 0) return TO_OK;
  if ((Vx || K) && !b->want_vx) return fail(TO_ERR_ARG, "toget_trajectories: Vx / K need want_vx in the solve");
  const SysOps* o = p->ops;
  const int pi = b->elem_bytes == 8 && b->prec == TO_FP64 ? 0 : 1;
  const int rbytes = b->prec == TO_FP64 ? 8 : 4;
  const size_t nX = (size_t)B * (p->T_max + 1) * p->n, nU = (size_t)B * p->T_max * p->m;
  const size_t nK = (size_t)B * p->T_max * p->m * p->n;
  size_t dummy = 0;
  if (X && !b->gX) TO_CK(grow(b->gX, (size_t)b->B_max * (p->T_max + 1) * p->n, dummy));
  if (U && !b->gU) TO_CK(grow(b->gU, (size_t)b->B_max * p->T_max * p->m, dummy));
  if (Vx && !b->gV) TO_CK(grow(b->gV, (size_t)b->B_max * (p->T_max + 1) * p->n, dummy));
  if (K && !b->gK) TO_CK(grow(b->gK, (size_t)b->B_max * p->T_max * p->m * p->n, dummy));
  if (X || U || Vx || K) {
    const int rs = o->rs[rbytes == 8 ? 0 : 1], gs = o->gs[rbytes == 8 ? 0 : 1];
    (void)pi;
    const int NS = std::min(b->G, kLsWidth) + 1;
    gather_kernel<<<1024, 256, 0, b->stream>>>(B, p->T_max, p->n, p->m, rs, gs, NS, rbytes, b->toff, b->last_T, b->slot,
                                               b->traj,
                                               b->gains, b->vx, X ? b->gX : nullptr, U ? b->gU : nullptr,
                                               Vx ? b->gV : nullptr, K ? b->gK : nullptr, b->err);
    TO_CK(cudaGetLastError());
  }
  if (X) TO_CK(cudaMemcpyAsync(X, b->gX, nX * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  if (U) TO_CK(cudaMemcpyAsync(U, b->gU, nU * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  if (Vx) TO_CK(cudaMemcpyAsync(Vx, b->gV, nX * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  if (K) TO_CK(cudaMemcpyAsync(K, b->gK, nK * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  if (J) TO_CK(cudaMemcpyAsync(J, b->J, B * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  if (iters) TO_CK(cudaMemcpyAsync(iters, b->iters, B * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  if (status) TO_CK(cudaMemcpyAsync(status, b->status, B * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  TO_CK(cudaStreamSynchronize(b->stream));
  return TO_OK;
}

int toget_critic_targets(to_batch b, int K, double* Vbar) {
  if (!b || !Vbar || K < 1) return fail(TO_ERR_ARG, "toget_critic_targets: null batch / output or K < 1");
  to_problem p = b->p;
  const int B = b->B;
  TO_CK(cudaStreamSynchronize(b->stream));
  if (B == 0) return TO_OK;
  if (!b->last_T) return fail(TO_ERR_ARG, "toget_critic_targets: the batch holds no solve");
  const size_t cnt = (size_t)B * (p->T_max + 1);
  double* d = nullptr;
  TO_CK(cudaMalloc(&d, 2 * cnt * sizeof(double)));
  KnotCostArgs ka{};
  ka.B = B;
  ka.T_max = p->T_max;
  ka.NS = std::min(b->G, kLsWidth) + 1;
  ka.rbytes = b->prec == TO_FP64 ? 8 : 4;
  ka.RS = p->ops->rs[ka.rbytes == 8 ? 0 : 1];
  ka.toff = b->toff;
  ka.T = b->last_T;
  ka.slot = b->slot;
  ka.traj = b->traj;
  ka.params64 = p->d_params[0];
  ka.out = d;
  cudaError_t e = p->ops->knot_costs(ka, b->stream);
  if (e == cudaSuccess) {
    window_kernel<<<1024, 256, 0, b->stream>>>(B, p->T_max, K, b->last_T, d, d + cnt);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(Vbar, d + cnt, cnt * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  cudaFree(d);
  if (e != cudaSuccess) return fail(TO_ERR_CUDA, std::string("toget_critic_targets: ") + cudaGetErrorString(e));
  return TO_OK;
}

int toget_history(to_batch b, int* alpha_idx, double* J_hist) {
  if (!b) return fail(TO_ERR_ARG, "toget_history: null batch");
  const int B = b->B, mi = b->max_iter;
  TO_CK(cudaStreamSynchronize(b->stream));
  if (B == 0) return TO_OK;
  std::vector<int> it(B);
  TO_CK(cudaMemcpy(it.data(), b->iters, B * sizeof(int), cudaMemcpyDeviceToHost));
  if (alpha_idx && mi > 0) {
    TO_CK(cudaMemcpy(alpha_idx, b->ahist, sizeof(int) * B * mi, cudaMemcpyDeviceToHost));
    for (int i = 0; i < B; ++i)
      for (int k = std::max(0, it[i]); k < mi; ++k) alpha_idx[(size_t)i * mi + k] = -1;
  }
  if (J_hist) {
    TO_CK(cudaMemcpy(J_hist, b->Jhist, sizeof(double) * B * (mi + 1), cudaMemcpyDeviceToHost));
    for (int i = 0; i < B; ++i)
      for (int k = std::max(0, it[i]) + 1; k <= mi; ++k) J_hist[(size_t)i * (mi + 1) + k] = NAN;
  }
  return TO_OK;
}


// ===========================================================================
// Solve without any device allocation.
//
// For callers that must not allocate device memory while they run: a
// real-time control loop that has to keep its latency bounded, a process
// that works inside a fixed, pre-sized memory pool, or code that runs while
// other work is being captured into a CUDA graph.  The workspace (knot
// offsets, horizon order, trajectory slots, gains, per-iteration history)
// lives in one file-scope device array of TO_NOALLOC_SCRATCH_BYTES that every
// GPU loading this library keeps until the process exits.  Inputs and outputs
// are the caller's device buffers.
// ===========================================================================
namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[TO_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_base[kMaxDevices] = {};   // device address of the array, per device

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

int tosolve_batch_noalloc(to_problem p, int B, const double* d_x0, const int* d_T, const to_solver_opts* opts,
                          void* cuda_stream, double* d_J, int* d_iters, int* d_status, double* d_X, double* d_U) {
  if (!p) return fail(TO_ERR_ARG, "tosolve_batch_noalloc: null problem");
  to_solver_opts o;
  to_default_opts(&o);
  if (opts) o = *opts;
  if (o.forced_alpha || o.want_vx || o.profile_phases)
    return fail(TO_ERR_UNSUPPORTED, "tosolve_batch_noalloc: forced steps, want_vx and profiling are not available");
  int rc = check_opts(&o);
  if (rc) return rc;
  if (B < 0 || (B > 0 && (!d_x0 || !d_T || !d_J || !d_iters || !d_status)))
    return fail(TO_ERR_ARG, "tosolve_batch_noalloc: x0, T, J, iters and status are required");
  if (B == 0) return TO_OK;
  // the device address of the array: once per device, with that device current
  int dev = 0;
  TO_CK(cudaGetDevice(&dev));
  if (dev != p->device)
    return fail(TO_ERR_ARG, "tosolve_batch_noalloc: the current device is not the one the problem was created on");
  if (dev < 0 || dev >= kMaxDevices) return fail(TO_ERR_UNSUPPORTED, "tosolve_batch_noalloc: device index too large");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess)
        return fail(TO_ERR_CUDA, std::string("tosolve_batch_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_noalloc_base[dev] = ptr;
    }
    base = static_cast<unsigned char*>(g_noalloc_base[dev]);
  }
  // carve the workspace out of the array (horizons are bounded by T_max, so
  // B (T_max + 1) knot records always suffice)
  const SysOps* ops = p->ops;
  const int pi = o.prec == TO_FP64 ? 0 : 1;
  const int elem = o.prec == TO_FP64 ? 8 : 4;
  const long long knots = (long long)B * (p->T_max + 1);
  const int mi = std::max(o.max_iter, 1);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t at = off; off = align256(off + bytes); return at; };
  const size_t o_toff = take(sizeof(long long) * B), o_order = take(sizeof(int) * B),
               o_hist = take(sizeof(int) * (p->T_max + 2)), o_err = take(sizeof(int)), o_queue = take(sizeof(int)),
               o_slot = take(sizeof(int) * B), o_ahist = take(sizeof(int) * (size_t)B * mi),
               o_jhist = take(sizeof(double) * (size_t)B * (mi + 1)),
               o_traj = take((size_t)knots * kMaxSlots * ops->rs[pi] * elem),
               o_gains = take((size_t)knots * ops->gs[pi] * elem),
               o_dscr = take((size_t)knots * p->knot_scratch[pi] * elem);
  if (off > TO_NOALLOC_SCRATCH_BYTES)
    return fail(TO_ERR_BUDGET, "tosolve_batch_noalloc: needs " + std::to_string(off) + " bytes of workspace, more than "
                                   "the static " + std::to_string((size_t)TO_NOALLOC_SCRATCH_BYTES) + " bytes");
  to_batch_s w;
  w.p = p;
  w.B_max = B;
  w.knots_max = knots;
  w.elem_bytes = elem;
  w.toff = reinterpret_cast<long long*>(base + o_toff);
  w.order = reinterpret_cast<int*>(base + o_order);
  w.hist = reinterpret_cast<int*>(base + o_hist);
  w.err = reinterpret_cast<int*>(base + o_err);
  w.queue = reinterpret_cast<int*>(base + o_queue);
  w.slot = reinterpret_cast<int*>(base + o_slot);
  w.ahist = reinterpret_cast<int*>(base + o_ahist);
  w.Jhist = reinterpret_cast<double*>(base + o_jhist);
  w.traj = base + o_traj;
  w.gains = base + o_gains;
  w.dscr = p->knot_scratch[pi] ? base + o_dscr : nullptr;
  w.J = d_J;
  w.iters = d_iters;
  w.status = d_status;
  w.hist_iter_cap = mi;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the prepare kernel resets the queue, the error flag and the histogram;
  // every other region is written before it is read
  rc = launch_solve(&w, B, d_x0, d_T, nullptr, nullptr, &o, s);
  if (rc) return rc;
  if (d_X || d_U) {
    const int NS = std::min(w.G, kLsWidth) + 1;
    gather_kernel<<<1024, 256, 0, s>>>(B, p->T_max, p->n, p->m, ops->rs[pi], ops->gs[pi], NS, elem, w.toff, d_T,
                                       w.slot, w.traj, w.gains, nullptr, d_X, d_U, nullptr, nullptr, w.err);
    TO_CK(cudaGetLastError());
  }
  return TO_OK;
}
