// quad: placeholder until the system's device model lands.
#include "launch.cuh"

namespace to {

static int parse_quad(const double*, size_t, std::vector<unsigned char>&, std::vector<unsigned char>&,
                        std::string& err) {
  err = "quad: system not available in this build";
  return -1;
}

static cudaError_t launch_none(int, int, int, int, cudaStream_t, const SolveArgs&) { return cudaErrorNotSupported; }
static cudaError_t occ_none(int, int, int, size_t*, int*) { return cudaErrorNotSupported; }

const SysOps& quad_ops() {
  static SysOps o = [] {
    SysOps x{};
    x.parse = parse_quad;
    x.launch = launch_none;
    x.occupancy = occ_none;
    return x;
  }();
  return o;
}

}  // namespace to
