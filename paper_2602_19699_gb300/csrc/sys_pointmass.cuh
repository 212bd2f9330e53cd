// Point-mass double integrator with Gaussian obstacle bumps (Sec. V-A systems;
// the synthetic workload's cost).  x = [px, py, vx, vy], u = [ax, ay],
// explicit Euler: p+ = p + dt v, v+ = v + dt u.
#pragma once
#include "common.cuh"

namespace to {

template <class R>
struct PointMassParams {
  R dt, wu, bamp, bsig, wpT, wvT;
  int nb;
  R bc[8][2];
};

template <class D, class S>
inline void cast_params(const PointMassParams<S>& s, PointMassParams<D>& d) {
  d.dt = (D)s.dt; d.wu = (D)s.wu; d.bamp = (D)s.bamp; d.bsig = (D)s.bsig; d.wpT = (D)s.wpT; d.wvT = (D)s.wvT;
  d.nb = s.nb;
  for (int b = 0; b < 8; ++b) { d.bc[b][0] = (D)s.bc[b][0]; d.bc[b][1] = (D)s.bc[b][1]; }
}

struct SysPointMass {
  static constexpr int n = 4, m = 2;
  static constexpr bool kActor = false;
  template <class R> using ParamsT = PointMassParams<R>;
  template <class R> struct Scratch { static constexpr int elems = 1; };
  template <int G> static constexpr bool kGroupStep = false;
  static constexpr bool kKnotParallel = false;
  static constexpr bool kStoredDerivs = false;


  template <class R>
  TO_DEV static R bumps(const ParamsT<R>& P, R px, R py) {
    R s = 0;
    const R inv = R(1) / (R(2) * P.bsig * P.bsig);
    for (int b = 0; b < P.nb; ++b) {
      R dx = px - P.bc[b][0], dy = py - P.bc[b][1];
      s += P.bamp * exp(-(dx * dx + dy * dy) * inv);
    }
    return s;
  }

  template <class R>
  TO_DEV static R running_cost(const ParamsT<R>& P, const R* x, const R* u) {
    return P.wu * (u[0] * u[0] + u[1] * u[1]) + bumps(P, x[0], x[1]);
  }

  // the same step on a state carried as (hi, lo) pairs, in place
  template <class R>
  TO_DEV static R cost_step2(const ParamsT<R>& P, R* xh, R* xl, const R* u) {
    const R l = running_cost(P, xh, u);
    const R dpx = P.dt * xh[2] + P.dt * xl[2], dpy = P.dt * xh[3] + P.dt * xl[3];
    acc2(xh[0], xl[0], dpx);
    acc2(xh[1], xl[1], dpy);
    acc2(xh[2], xl[2], P.dt * u[0]);
    acc2(xh[3], xl[3], P.dt * u[1]);
    return l;
  }

  template <class R>
  TO_DEV static R terminal_cost(const ParamsT<R>& P, const R* x) {
    return P.wpT * (x[0] * x[0] + x[1] * x[1]) + P.wvT * (x[2] * x[2] + x[3] * x[3]);
  }

  // Running-cost derivatives with the state and control Hessians clipped.
  // The bumps act on the position block only, so the clip of the full 4x4
  // state Hessian is the clip of the 2x2 position block with eps on the
  // velocity diagonal (the remaining eigenpairs are (0, e_i)).  One lane.
  template <class R>
  TO_DEV static void running_derivs(const ParamsT<R>& P, const R* x, const R* u, R eps, R* lxx, R* lx, R* luu,
                                    R* lu) {
    R gx = 0, gy = 0, hxx = 0, hxy = 0, hyy = 0;
    const R s2 = P.bsig * P.bsig;
    const R is2 = R(1) / s2;
    const R inv = R(0.5) * is2;
    for (int b = 0; b < P.nb; ++b) {
      R dx = x[0] - P.bc[b][0], dy = x[1] - P.bc[b][1];
      R e = P.bamp * exp(-(dx * dx + dy * dy) * inv);
      // d/dp e = -e d / s2 ;  d2/dp2 e = e (d d^T / s2^2 - I / s2)
      const R es = e * is2;
      gx -= es * dx;
      gy -= es * dy;
      hxx += es * (dx * dx * is2 - R(1));
      hyy += es * (dy * dy * is2 - R(1));
      hxy += es * dx * dy * is2;
    }
    eigclip_2x2(hxx, hxy, hyy, eps);
#pragma unroll
    for (int i = 0; i < n * n; ++i) lxx[i] = 0;
    lxx[0] = hxx; lxx[1] = hxy; lxx[4] = hxy; lxx[5] = hyy;
    lxx[10] = clip0(eps); lxx[15] = clip0(eps);
    lx[0] = gx; lx[1] = gy; lx[2] = 0; lx[3] = 0;
    const R w2 = R(2) * P.wu;
    const R d = w2 > eps ? w2 : eps;
    luu[0] = d; luu[1] = 0; luu[2] = 0; luu[3] = d;
    lu[0] = w2 * u[0]; lu[1] = w2 * u[1];
  }

  // A, B (row-major, constant) on every lane; the cost derivatives on the
  // last lane of the group
  template <class R, int G>
  TO_DEV static void derivs(const ParamsT<R>& P, const Group<G>& g, const R* x, const R* u, R eps, R* A, R* B,
                            R* lxx, R* lx, R* luu, R* lu, R*) {
    for (int e = g.lane; e < n * n + n * m; e += G) {
      if (e < n * n) {
        int i = e / n, j = e % n;
        A[e] = (i == j) ? R(1) : ((j == i + 2) ? P.dt : R(0));
      } else {
        int f = e - n * n, i = f / m, j = f % m;
        B[f] = (i == j + 2) ? P.dt : R(0);
      }
    }
    if (g.lane == G - 1) running_derivs(P, x, u, eps, lxx, lx, luu, lu);
  }

  // the same on one lane (single-lane groups)
  template <class R>
  TO_DEV static void derivs_lane(const ParamsT<R>& P, const R* x, const R* u, R eps, R* A, R* B, R* lxx, R* lx,
                                 R* luu, R* lu) {
#pragma unroll
    for (int i = 0; i < n; ++i)
#pragma unroll
      for (int j = 0; j < n; ++j) A[i * n + j] = (i == j) ? R(1) : ((j == i + 2) ? P.dt : R(0));
#pragma unroll
    for (int i = 0; i < n; ++i)
#pragma unroll
      for (int j = 0; j < m; ++j) B[i * m + j] = (i == j + 2) ? P.dt : R(0);
    running_derivs(P, x, u, eps, lxx, lx, luu, lu);
  }

  template <class R>
  TO_DEV static void terminal_derivs(const ParamsT<R>& P, const R* x, R eps, R* lxx, R* lx) {
    const R a = R(2) * P.wpT, b = R(2) * P.wvT;
#pragma unroll
    for (int i = 0; i < n * n; ++i) lxx[i] = 0;
    lxx[0] = a > eps ? a : eps; lxx[5] = lxx[0];
    lxx[10] = b > eps ? b : eps; lxx[15] = lxx[10];
    lx[0] = a * x[0]; lx[1] = a * x[1]; lx[2] = b * x[2]; lx[3] = b * x[3];
  }
};

}  // namespace to
