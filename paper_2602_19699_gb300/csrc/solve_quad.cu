// Quadruped-shaped floating base: parameter parsing and solver instantiation.
#include <algorithm>
#include <cmath>

#include "rigid_parse.cuh"

namespace to {

static int parse_quad(const double* p, size_t np, std::vector<unsigned char>& blob64, std::vector<unsigned char>& blob32,
                      std::string& err) {
  RigidHeader h;
  if (!parse_rigid(p, np, h, err)) return -1;
  RigidParams<double, 18> P{};
  if (!fill_rigid<RK_QUAD, 18>(h, 6, P, err)) return -1;
  if (h.n_cost < 11) { err = "quad params: cost block truncated"; return -1; }
  const double* c = h.cost;
  P.wtau = c[0]; P.znom = c[1]; P.wz = c[2]; P.wrpy = c[3]; P.wvx = c[4]; P.vxt = c[5];
  P.tscale = c[6]; P.kc = c[7]; P.dc = c[8]; P.beta = c[9];
  P.nfeet = (int)c[10];
  if (P.nfeet != RigidTopo<RK_QUAD>::kFeet || h.n_cost < (size_t)(11 + 4 * P.nfeet) || !(P.beta > 0)) {
    err = "quad params: bad contact block (four feet)";
    return -1;
  }
  for (int f = 0; f < P.nfeet; ++f) {
    P.foot_body[f] = (int)c[11 + 4 * f];
    if (P.foot_body[f] != RigidTopo<RK_QUAD>::foot_body(f)) { err = "quad params: foot f must be on calf body 8 + 3 f"; return -1; }
    for (int k = 0; k < 3; ++k) P.foot_pt[f][k] = c[12 + 4 * f + k];
  }
  to_blobs<RigidQuadP>(P, blob64, blob32);
  return 0;
}

typedef Dispatch<SysQuad, kDepth1, 64, 32> QDispatch;

// the stored substep primals of one knot: n_sub of them (header [6], 0 means 1)
static size_t quad_knot_scratch(const double* p, size_t np, int prec) {
  const int n_sub = np > 6 ? std::max(1, (int)p[6]) : 1;
  return (size_t)n_sub * (prec == 0 ? SysQuad::kPrimStride<double> : SysQuad::kPrimStride<float>);
}

static SysOps make_ops() {
  SysOps o{};
  o.sys = 4;
  fill_layout<SysQuad>(o);
  o.n_groups = 2;
  o.groups[0] = 64;   // a candidate lane's partner on the other warp factors the mass matrix
  o.groups[1] = 32;   // one warp per instance: the partner is the candidate lane + 16
  o.default_G = 64;
  o.default_gpb[0] = 1; o.default_gpb[1] = 1;
  o.accepts_actor = true;
  o.parse = parse_quad;
  o.max_depth = 1;
  o.launch = DepthOne<QDispatch>::launch;
  o.occupancy = DepthOne<QDispatch>::occupancy;
  o.knot_costs = knot_costs_one<SysQuad>;
  o.knot_scratch = quad_knot_scratch;
  return o;
}

const SysOps& quad_ops() {
  static SysOps o = make_ops();
  return o;
}

}  // namespace to
