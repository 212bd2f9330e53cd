// Planar 3-link arm: parameter parsing and solver instantiation.
#include <cmath>

#include "launch.cuh"
#include "sys_planar3.cuh"

namespace to {

// The GPU model covers exactly the planar chain the format describes: three
// Rz joints in series, joint offsets and centres of mass along the parent's
// x axis, gravity in the xy plane, the end effector on the last link's x axis.
static int parse_planar3(const double* p, size_t np, std::vector<unsigned char>& blob64,
                           std::vector<unsigned char>& blob32, std::string& err) {
  RigidHeader h;
  if (!parse_rigid(p, np, h, err)) return -1;
  if (h.N != 3 || h.a0 != 0 || h.n_sub != 1) { err = "planar3 params: need N=3, a0=0, n_sub=1"; return -1; }
  if (h.g[2] != 0.0) { err = "planar3 params: gravity must lie in the xy plane"; return -1; }
  Planar3Params<double> P{};
  P.dt = h.dt; P.gx = h.g[0]; P.gy = h.g[1];
  for (int i = 0; i < 3; ++i) {
    const RigidBody& b = h.bodies[i];
    if (b.parent != i - 1 || b.jtype != 2) { err = "planar3 params: joints must be a chain of Rz"; return -1; }
    if (b.off[1] != 0 || b.off[2] != 0 || b.com[1] != 0 || b.com[2] != 0 || (i == 0 && b.off[0] != 0)) {
      err = "planar3 params: offsets and centres of mass must lie on the link's x axis";
      return -1;
    }
    if (i > 0) P.len[i - 1] = b.off[0];
    P.com[i] = b.com[0];
    P.mass[i] = b.mass;
    P.izz[i] = b.I[2];
  }
  if (h.n_cost < 16) { err = "planar3 params: cost block truncated"; return -1; }
  const double* c = h.cost;
  P.wtau = c[0]; P.bamp = c[1]; P.bsig = c[2]; P.nb = (int)c[3];
  if (P.nb < 0 || P.nb > 2 || !(P.bsig > 0)) { err = "planar3 params: bad bumps"; return -1; }
  for (int b = 0; b < P.nb; ++b) { P.bc[b][0] = c[4 + 2 * b]; P.bc[b][1] = c[5 + 2 * b]; }
  P.tgt[0] = c[8]; P.tgt[1] = c[9];
  P.wee = c[10]; P.wvT = c[11];
  if ((int)c[12] != 2 || c[14] != 0 || c[15] != 0) { err = "planar3 params: end effector must be on link 3's x axis"; return -1; }
  P.len[2] = c[13];
  to_blobs<Planar3Params>(P, blob64, blob32);
  return 0;
}

typedef Dispatch<SysPlanar3, kDepth1, 1, 4, 8, 16, 32> P3Dispatch;

// groups that stage two knots ahead (solve_planar3_d2.cu: its own translation
// unit, so the two kernel sets compile in parallel)
cudaError_t planar3_launch_d2(int prec, int G, int gpb, int grid, cudaStream_t s, const SolveArgs& a);
cudaError_t planar3_occupancy_d2(int prec, int G, int gpb, size_t* smem, int* bps);

static cudaError_t planar3_launch(int prec, int G, int depth, int gpb, int grid, cudaStream_t s, const SolveArgs& a) {
  if (depth == 2) return planar3_launch_d2(prec, G, gpb, grid, s, a);
  return depth == 1 ? P3Dispatch::launch(prec, G, gpb, grid, s, a) : cudaErrorInvalidValue;
}
static cudaError_t planar3_occupancy(int prec, int G, int depth, int gpb, size_t* smem, int* bps) {
  if (depth == 2) return planar3_occupancy_d2(prec, G, gpb, smem, bps);
  return depth == 1 ? P3Dispatch::occupancy(prec, G, gpb, smem, bps) : cudaErrorInvalidValue;
}

// every knot's stored derivative block (both precisions)
static size_t planar3_knot_scratch(const double*, size_t, int) { return SysPlanar3::kDerivStride; }

static SysOps make_ops() {
  SysOps o{};
  o.sys = 2;
  fill_layout<SysPlanar3>(o);
  o.n_groups = 5;
  o.groups[0] = 8; o.groups[1] = 16; o.groups[2] = 32; o.groups[3] = 1;   // 1: one thread per instance
  o.groups[4] = 4;   // stored derivatives need no lane per derivative role
  o.default_G = 8;
  o.default_gpb[0] = 8; o.default_gpb[1] = 8;
  o.accepts_actor = false;
  o.parse = parse_planar3;
  o.max_depth = 2;   // groups of 4 or more lanes
  o.launch = planar3_launch;
  o.occupancy = planar3_occupancy;
  o.knot_costs = knot_costs_one<SysPlanar3>;
  o.knot_scratch = planar3_knot_scratch;
  return o;
}

const SysOps& planar3_ops() {
  static SysOps o = make_ops();
  return o;
}

}  // namespace to
