// Kernel instantiation and launch glue shared by the per-system translation
// units.  Each system TU instantiates the solver for FP64 and mixed arithmetic
// and the group sizes it supports, and registers a SysOps table.
#pragma once
#include <algorithm>
#include <string>
#include <vector>

#include "ilqr.cuh"

namespace to {

// inputs of the per-knot cost pass over a batch's returned trajectories
struct KnotCostArgs {
  int B, T_max, NS, RS, rbytes;
  const long long* toff;
  const int* T;
  const int* slot;
  const void* traj;
  const void* params64;     // the system's parameter struct in float64
  double* out;              // B x (T_max + 1): l_k(x_k, u_k) for k < T, l_T(x_T) at k = T, 0 beyond
};

struct SysOps {
  int sys, n, m;
  int rs[2], gs[2];                 // knot / gain record lengths (elements) for FP64, mixed
  int n_groups;                     // supported group sizes
  int groups[6];
  int default_G, default_gpb[2];    // default launch shape (FP64, mixed)
  bool accepts_actor;
  // parse the flat parameter vector into the system's struct in float64 and float32
  int (*parse)(const double* p, size_t np, std::vector<unsigned char>& blob64, std::vector<unsigned char>& blob32,
               std::string& err);
  int max_depth;                    // largest staging depth (1 or 2) of its groups of more than one lane
  cudaError_t (*launch)(int prec, int G, int depth, int gpb, int grid, cudaStream_t s, const SolveArgs& a);
  cudaError_t (*occupancy)(int prec, int G, int depth, int gpb, size_t* smem, int* blocks_per_sm);
  // per-knot costs of the final trajectories in float64 (critic targets)
  cudaError_t (*knot_costs)(const KnotCostArgs& a, cudaStream_t s);
  // elements of per-knot derivative scratch (stored substep primals) for a
  // parameter vector and precision (0 FP64, 1 mixed); null: none
  size_t (*knot_scratch)(const double* p, size_t np, int prec);
};

const SysOps* sys_ops(int sys);

// One persistent launch over several systems (solve_multi.cu): slot 0 the
// 7-DoF arm, slot 1 the planar arm, slot 2 the point mass; a slot without a
// member is skipped.
constexpr int kMultiSystems = 3;
struct MultiArgs {
  SolveArgs a[kMultiSystems];
  int present[kMultiSystems];
};
cudaError_t multi_occupancy(int prec, size_t* smem, int* blocks_per_sm);
cudaError_t multi_launch(int prec, int grid, cudaStream_t s, const MultiArgs& m);
int multi_group_lanes(int slot);       // lanes per instance of the slot's solver

constexpr int kMaxCtaThreads = 256;

template <class Sys, class R, int G, int D>
__global__ void __launch_bounds__(kMaxCtaThreads, 1) ilqr_kernel(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Solver<Sys, R, G, D>::run(a, smem_raw);
}

template <class Sys, class R, int G, int D = 1>
inline size_t solver_smem(int gpb) {
  return ((sizeof(typename Sys::template ParamsT<R>) + 15) / 16) * 16 +
         (size_t)gpb * sizeof(typename Solver<Sys, R, G, D>::W);
}

template <class Sys, class R, int G, int D>
inline cudaError_t launch_one(int gpb, int grid, cudaStream_t s, const SolveArgs& a) {
  const int threads = G * gpb;
  const size_t smem = solver_smem<Sys, R, G, D>(gpb);
  auto k = ilqr_kernel<Sys, R, G, D>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <class Sys, class R, int G, int D>
inline cudaError_t occupancy_one(int gpb, size_t* smem, int* bps) {
  *smem = solver_smem<Sys, R, G, D>(gpb);
  auto k = ilqr_kernel<Sys, R, G, D>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, G * gpb, *smem);
}

// dispatch on (precision, group size) over a compile-time list of sizes, at
// one staging depth D
template <class Sys, int D, int... Gs>
struct Dispatch;

template <class Sys, int D>
struct Dispatch<Sys, D> {
  static cudaError_t launch(int, int, int, int, cudaStream_t, const SolveArgs&) { return cudaErrorInvalidValue; }
  static cudaError_t occupancy(int, int, int, size_t*, int*) { return cudaErrorInvalidValue; }
};

template <class Sys, int D, int G0, int... Gs>
struct Dispatch<Sys, D, G0, Gs...> {
  static cudaError_t launch(int prec, int G, int gpb, int grid, cudaStream_t s, const SolveArgs& a) {
    if (G == G0)
      return prec == PREC_FP64 ? launch_one<Sys, double, G0, D>(gpb, grid, s, a)
                               : launch_one<Sys, float, G0, D>(gpb, grid, s, a);
    return Dispatch<Sys, D, Gs...>::launch(prec, G, gpb, grid, s, a);
  }
  static cudaError_t occupancy(int prec, int G, int gpb, size_t* smem, int* bps) {
    if (G == G0)
      return prec == PREC_FP64 ? occupancy_one<Sys, double, G0, D>(gpb, smem, bps)
                               : occupancy_one<Sys, float, G0, D>(gpb, smem, bps);
    return Dispatch<Sys, D, Gs...>::occupancy(prec, G, gpb, smem, bps);
  }
};

constexpr int kDepth1 = 1, kDepth2 = 2;   // staging depths

// a system whose groups stage one knot ahead only (SysOps.max_depth = 1)
template <class Disp>
struct DepthOne {
  static cudaError_t launch(int prec, int G, int depth, int gpb, int grid, cudaStream_t s, const SolveArgs& a) {
    return depth == 1 ? Disp::launch(prec, G, gpb, grid, s, a) : cudaErrorInvalidValue;
  }
  static cudaError_t occupancy(int prec, int G, int depth, int gpb, size_t* smem, int* bps) {
    return depth == 1 ? Disp::occupancy(prec, G, gpb, smem, bps) : cudaErrorInvalidValue;
  }
};

// One thread per knot: the state is rebuilt in float64 from the record
// (float32 records add the low parts stored after u) and the system's own
// cost functions evaluate l_k or l_T in float64.
template <class Sys>
__global__ void knot_cost_kernel(KnotCostArgs a) {
  typedef typename Sys::template ParamsT<double> PD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  {
    const int words = (int)(sizeof(PD) / sizeof(int));
    for (int i = threadIdx.x; i < words; i += blockDim.x)
      reinterpret_cast<int*>(smem_raw)[i] = reinterpret_cast<const int*>(a.params64)[i];
  }
  __syncthreads();
  const PD& P = *reinterpret_cast<const PD*>(smem_raw);
  constexpr int n = Sys::n, m = Sys::m;
  const long long total = (long long)a.B * (a.T_max + 1);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / (a.T_max + 1)), k = (int)(t % (a.T_max + 1));
    const int Tb = a.T[b];
    if (k > Tb) {
      a.out[t] = 0.0;
      continue;
    }
    const long long r = ((a.toff[b] + k) * a.NS + a.slot[b]) * a.RS;
    double x[n], u[m];
    for (int i = 0; i < n; ++i)
      x[i] = a.rbytes == 8 ? reinterpret_cast<const double*>(a.traj)[r + i]
                           : (double)reinterpret_cast<const float*>(a.traj)[r + i] +
                                 (double)reinterpret_cast<const float*>(a.traj)[r + n + m + i];
    if (k < Tb) {
      for (int i = 0; i < m; ++i)
        u[i] = a.rbytes == 8 ? reinterpret_cast<const double*>(a.traj)[r + n + i]
                             : (double)reinterpret_cast<const float*>(a.traj)[r + n + i];
      a.out[t] = Sys::template running_cost<double>(P, x, u);
    } else {
      a.out[t] = Sys::template terminal_cost<double>(P, x);
    }
  }
}

template <class Sys>
inline cudaError_t knot_costs_one(const KnotCostArgs& a, cudaStream_t s) {
  const size_t smem = (sizeof(typename Sys::template ParamsT<double>) + 15) / 16 * 16;
  auto k = knot_cost_kernel<Sys>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long total = (long long)a.B * (a.T_max + 1);
  const int grid = (int)std::min<long long>((total + 255) / 256, 152 * 8);
  k<<<grid, 256, smem, s>>>(a);
  return cudaGetLastError();
}

template <class Sys>
inline void fill_layout(SysOps& o) {
  o.n = Sys::n;
  o.m = Sys::m;
  o.rs[0] = Layout<Sys, double>::RS;
  o.gs[0] = Layout<Sys, double>::GS;
  o.rs[1] = Layout<Sys, float>::RS;
  o.gs[1] = Layout<Sys, float>::GS;
}

// shared checks of the rigid-body parameter format (see include/to.h)
struct RigidBody {
  int parent, jtype;
  double off[3], mass, com[3], I[3];
};
struct RigidHeader {
  double dt, g[3];
  int N, a0, n_sub;
  std::vector<RigidBody> bodies;
  const double* cost;
  size_t n_cost;
};
inline bool parse_rigid(const double* p, size_t np, RigidHeader& h, std::string& err) {
  if (np < 8) { err = "params: rigid-body header needs 8 values"; return false; }
  h.dt = p[0];
  h.g[0] = p[1]; h.g[1] = p[2]; h.g[2] = p[3];
  h.N = (int)p[4];
  h.a0 = (int)p[5];
  h.n_sub = p[6] >= 1 ? (int)p[6] : 1;
  if (h.N <= 0 || h.N > 32 || h.a0 < 0 || h.a0 >= h.N || h.n_sub > 64) { err = "params: bad N / a0 / n_sub"; return false; }
  if (np < 8 + 16 * (size_t)h.N) { err = "params: body table truncated"; return false; }
  h.bodies.resize(h.N);
  for (int i = 0; i < h.N; ++i) {
    const double* r = p + 8 + 16 * i;
    RigidBody& b = h.bodies[i];
    b.parent = (int)r[0];
    b.jtype = (int)r[1];
    for (int k = 0; k < 3; ++k) { b.off[k] = r[2 + k]; b.com[k] = r[6 + k]; b.I[k] = r[9 + k]; }
    b.mass = r[5];
    if (b.parent >= i || b.parent < -1 || b.jtype < 0 || b.jtype > 5) { err = "params: bad body table"; return false; }
  }
  h.cost = p + 8 + 16 * h.N;
  h.n_cost = np - (8 + 16 * h.N);
  return true;
}

template <class P>
inline void to_blob(const P& prm, std::vector<unsigned char>& blob) {
  blob.assign(reinterpret_cast<const unsigned char*>(&prm), reinterpret_cast<const unsigned char*>(&prm) + sizeof(P));
  while (blob.size() % 4) blob.push_back(0);
}

// both precisions of a parsed parameter struct
template <template <class> class PT>
inline void to_blobs(const PT<double>& p64, std::vector<unsigned char>& blob64, std::vector<unsigned char>& blob32) {
  PT<float> p32;
  cast_params(p64, p32);
  to_blob(p64, blob64);
  to_blob(p32, blob32);
}

}  // namespace to
