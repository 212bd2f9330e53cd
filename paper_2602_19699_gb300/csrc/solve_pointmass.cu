// Point-mass system: parameter parsing and solver instantiation.
#include <cmath>

#include "launch.cuh"
#include "sys_pointmass.cuh"

namespace to {

static int parse_pointmass(const double* p, size_t np, std::vector<unsigned char>& blob64,
                           std::vector<unsigned char>& blob32, std::string& err) {
  if (np < 5) { err = "pointmass params: need at least 5 values"; return -1; }
  PointMassParams<double> P{};
  P.dt = p[0]; P.wu = p[1]; P.bamp = p[2]; P.bsig = p[3];
  P.nb = (int)p[4];
  if (P.nb < 0 || P.nb > 8 || np < (size_t)(7 + 2 * P.nb)) { err = "pointmass params: bad bump count"; return -1; }
  if (!(P.bsig > 0)) { err = "pointmass params: bump sigma must be > 0"; return -1; }
  for (int b = 0; b < P.nb; ++b) { P.bc[b][0] = p[5 + 2 * b]; P.bc[b][1] = p[6 + 2 * b]; }
  P.wpT = p[5 + 2 * P.nb];
  P.wvT = p[6 + 2 * P.nb];
  to_blobs<PointMassParams>(P, blob64, blob32);
  return 0;
}

typedef Dispatch<SysPointMass, kDepth1, 1, 8, 16, 32> PMDispatch;

static SysOps make_ops() {
  SysOps o{};
  o.sys = 1;
  fill_layout<SysPointMass>(o);
  o.n_groups = 4;
  o.groups[0] = 8; o.groups[1] = 16; o.groups[2] = 32; o.groups[3] = 1;   // 1: one thread per instance
  o.default_G = 8;
  o.default_gpb[0] = 8; o.default_gpb[1] = 8;
  o.accepts_actor = false;
  o.parse = parse_pointmass;
  o.max_depth = 1;
  o.launch = DepthOne<PMDispatch>::launch;
  o.occupancy = DepthOne<PMDispatch>::occupancy;
  o.knot_costs = knot_costs_one<SysPointMass>;
  return o;
}

const SysOps& pointmass_ops() {
  static SysOps o = make_ops();
  return o;
}

}  // namespace to
