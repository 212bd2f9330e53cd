// 7-DoF serial arm: parameter parsing and solver instantiation.
#include <algorithm>
#include <cmath>

#include "rigid_parse.cuh"

namespace to {

static int parse_arm7(const double* p, size_t np, std::vector<unsigned char>& blob64, std::vector<unsigned char>& blob32,
                      std::string& err) {
  RigidHeader h;
  if (!parse_rigid(p, np, h, err)) return -1;
  RigidParams<double, 7> P{};
  if (!fill_rigid<RK_ARM7, 7>(h, 0, P, err)) return -1;
  if (h.n_cost < 11) { err = "arm7 params: cost block truncated"; return -1; }
  const double* c = h.cost;
  P.wtau = c[0]; P.wv = c[1];
  P.tgt[0] = c[2]; P.tgt[1] = c[3]; P.tgt[2] = c[4];
  P.wee = c[5]; P.wvT = c[6];
  P.ee_body = (int)c[7];
  P.ee_pt[0] = c[8]; P.ee_pt[1] = c[9]; P.ee_pt[2] = c[10];
  if (P.ee_body != RigidTopo<RK_ARM7>::kEeBody) { err = "arm7 params: the end effector must be on body 6"; return -1; }
  P.nfeet = 0;
  to_blobs<RigidArm7P>(P, blob64, blob32);
  return 0;
}

typedef Dispatch<SysArm7, kDepth1, 32> A7Dispatch;

// the stored substep primals of one knot: n_sub of them (header [6], 0 means 1)
static size_t arm7_knot_scratch(const double* p, size_t np, int prec) {
  const int n_sub = np > 6 ? std::max(1, (int)p[6]) : 1;
  return (size_t)n_sub * (prec == 0 ? SysArm7::kPrimStride<double> : SysArm7::kPrimStride<float>);
}

static SysOps make_ops() {
  SysOps o{};
  o.sys = 3;
  fill_layout<SysArm7>(o);
  o.n_groups = 1;
  o.groups[0] = 32;
  o.default_G = 32;
  o.default_gpb[0] = 2; o.default_gpb[1] = 2;
  o.accepts_actor = false;
  o.parse = parse_arm7;
  o.max_depth = 1;
  o.launch = DepthOne<A7Dispatch>::launch;
  o.occupancy = DepthOne<A7Dispatch>::occupancy;
  o.knot_costs = knot_costs_one<SysArm7>;
  o.knot_scratch = arm7_knot_scratch;
  return o;
}

const SysOps& arm7_ops() {
  static SysOps o = make_ops();
  return o;
}

}  // namespace to
