// Host-side parsing of the rigid-body parameter format (include/to.h) into
// the device model's parameter struct.
#pragma once
#include <string>
#include <vector>

#include "launch.cuh"
#include "sys_rigid.cuh"

namespace to {

// The device model is compiled for one joint tree per system (RigidTopo):
// the parameters must describe exactly that tree.
template <int KIND, int N>
inline bool fill_rigid(const RigidHeader& h, int a0, RigidParams<double, N>& P, std::string& err) {
  if (h.N != N || h.a0 != a0) {
    err = "rigid params: this system needs N=" + std::to_string(N) + ", a0=" + std::to_string(a0);
    return false;
  }
  typedef RigidTopo<KIND> Topo;
  for (int i = 0; i < N; ++i)
    if (h.bodies[i].parent != Topo::parent(i) || h.bodies[i].jtype != Topo::jtype(i)) {
      err = "rigid params: body " + std::to_string(i) + " must have parent " + std::to_string(Topo::parent(i)) +
            " and joint type " + std::to_string(Topo::jtype(i)) + " (the system's joint tree)";
      return false;
    }
  P.dt = h.dt;
  for (int k = 0; k < 3; ++k) P.g[k] = h.g[k];
  P.n_sub = h.n_sub;
  P.a0 = h.a0;
  for (int i = 0; i < N; ++i) {
    const RigidBody& b = h.bodies[i];
    P.parent[i] = b.parent;
    P.jtype[i] = b.jtype;
    P.mass[i] = b.mass;
    for (int k = 0; k < 3; ++k) { P.off[i][k] = b.off[k]; P.com[i][k] = b.com[k]; P.inertia[i][k] = b.I[k]; }
  }
  return true;
}

}  // namespace to
