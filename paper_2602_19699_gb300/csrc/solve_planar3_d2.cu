// Planar 3-link arm: the solver instantiated at staging depth 2 (each group
// fetches its knot records, gains and stored derivative blocks two knots
// ahead of their use), for the group sizes of more than one lane.
#include "launch.cuh"
#include "sys_planar3.cuh"

namespace to {

typedef Dispatch<SysPlanar3, kDepth2, 4, 8, 16, 32> P3DispatchD2;

cudaError_t planar3_launch_d2(int prec, int G, int gpb, int grid, cudaStream_t s, const SolveArgs& a) {
  return P3DispatchD2::launch(prec, G, gpb, grid, s, a);
}

cudaError_t planar3_occupancy_d2(int prec, int G, int gpb, size_t* smem, int* bps) {
  return P3DispatchD2::occupancy(prec, G, gpb, smem, bps);
}

}  // namespace to
