// One persistent launch over several systems: the 7-DoF arm, the planar arm
// and the point mass (the serving mix's systems) in a single kernel.
//
// Every CTA serves the systems' queues in turn, the longest work first (7-DoF
// arm, then planar arm, then point mass): its groups claim instances of the
// first system until that queue is drained, then the CTA moves on to the
// next one.  A CTA that finishes early therefore takes work of the next
// system while others still solve the previous one, so uneven horizons,
// iteration counts and systems share one launch with no idle tail between
// systems.  The three solvers share one CTA shape (64 threads: 2 groups of 32
// lanes for the 7-DoF arm, 8 groups of 8 lanes for the others) and the
// shared memory of the largest workspace; each system's arithmetic is its own
// solver's, unchanged.
#include <algorithm>

#include "launch.cuh"
#include "sys_planar3.cuh"
#include "sys_pointmass.cuh"
#include "sys_rigid.cuh"

namespace to {

constexpr int kMultiThreads = 64;
constexpr int kMultiG[kMultiSystems] = {32, 8, 8};   // 7-DoF arm, planar arm, point mass

template <class R>
struct MultiSolvers {
  typedef Solver<SysArm7, R, 32> S0;
  typedef Solver<SysPlanar3, R, 8> S1;
  typedef Solver<SysPointMass, R, 8> S2;
  static size_t smem() {
    return std::max({solver_smem<SysArm7, R, 32>(kMultiThreads / 32), solver_smem<SysPlanar3, R, 8>(kMultiThreads / 8),
                     solver_smem<SysPointMass, R, 8>(kMultiThreads / 8)});
  }
};

template <class R>
__global__ void __launch_bounds__(kMultiThreads, 1) multi_kernel(MultiArgs m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typedef MultiSolvers<R> MS;
  if (m.present[0]) MS::S0::run(m.a[0], smem_raw);
  __syncthreads();
  if (m.present[1]) MS::S1::run(m.a[1], smem_raw);
  __syncthreads();
  if (m.present[2]) MS::S2::run(m.a[2], smem_raw);
}

template <class R>
static cudaError_t multi_shape(size_t* smem, int* bps) {
  *smem = MultiSolvers<R>::smem();
  auto k = multi_kernel<R>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, kMultiThreads, *smem);
}

cudaError_t multi_occupancy(int prec, size_t* smem, int* bps) {
  return prec == PREC_FP64 ? multi_shape<double>(smem, bps) : multi_shape<float>(smem, bps);
}

cudaError_t multi_launch(int prec, int grid, cudaStream_t s, const MultiArgs& m) {
  size_t smem = 0;
  int bps = 0;
  cudaError_t e = multi_occupancy(prec, &smem, &bps);
  if (e != cudaSuccess) return e;
  if (prec == PREC_FP64) multi_kernel<double><<<grid, kMultiThreads, smem, s>>>(m);
  else multi_kernel<float><<<grid, kMultiThreads, smem, s>>>(m);
  return cudaGetLastError();
}

int multi_group_lanes(int slot) { return kMultiG[slot]; }

}  // namespace to
