// Jerk-controlled Dubins car with Gaussian obstacle bumps (Sec. V-A's second
// system, with the time state dropped).  x = [px, py, theta, v, a],
// u = [omega, jerk], explicit Euler:
//   px+ = px + dt v cos(theta),  py+ = py + dt v sin(theta),
//   theta+ = theta + dt omega,   v+ = v + dt a,   a+ = a + dt jerk.
// Running cost w_u |u|^2 + bumps(p); terminal w_pT |p|^2 + w_vT v^2 + w_aT a^2.
#pragma once
#include "common.cuh"

namespace to {

template <class R>
struct DubinsParams {
  R dt, wu, bamp, bsig, wpT, wvT, waT;
  int nb;
  R bc[8][2];
};

template <class D, class S>
inline void cast_params(const DubinsParams<S>& s, DubinsParams<D>& d) {
  d.dt = (D)s.dt; d.wu = (D)s.wu; d.bamp = (D)s.bamp; d.bsig = (D)s.bsig;
  d.wpT = (D)s.wpT; d.wvT = (D)s.wvT; d.waT = (D)s.waT;
  d.nb = s.nb;
  for (int b = 0; b < 8; ++b) { d.bc[b][0] = (D)s.bc[b][0]; d.bc[b][1] = (D)s.bc[b][1]; }
}

struct SysDubins {
  static constexpr int n = 5, m = 2;
  static constexpr bool kActor = false;
  template <class R> using ParamsT = DubinsParams<R>;
  template <class R> struct Scratch { static constexpr int elems = 1; };
  template <int G> static constexpr bool kGroupStep = false;
  static constexpr bool kKnotParallel = false;
  static constexpr bool kStoredDerivs = false;


  template <class R>
  TO_DEV static R bumps(const ParamsT<R>& P, R px, R py) {
    R s = 0;
    const R inv = R(1) / (R(2) * P.bsig * P.bsig);
    for (int b = 0; b < P.nb; ++b) {
      const R dx = px - P.bc[b][0], dy = py - P.bc[b][1];
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
    R s, c;
    sincos(xh[2], &s, &c);
    const R v = xh[3] + xl[3];
    const R dpx = P.dt * (v * c), dpy = P.dt * (v * s), dv = P.dt * xh[4] + P.dt * xl[4];
    acc2(xh[0], xl[0], dpx);
    acc2(xh[1], xl[1], dpy);
    acc2(xh[2], xl[2], P.dt * u[0]);
    acc2(xh[3], xl[3], dv);
    acc2(xh[4], xl[4], P.dt * u[1]);
    return l;
  }

  template <class R>
  TO_DEV static R terminal_cost(const ParamsT<R>& P, const R* x) {
    return P.wpT * (x[0] * x[0] + x[1] * x[1]) + P.wvT * x[3] * x[3] + P.waT * x[4] * x[4];
  }

  // Running-cost derivatives: the bumps act on the position block only, so
  // the clipped 5x5 state Hessian is the clipped 2x2 position block with the
  // clip of 0 on the other diagonal entries.  One lane.
  template <class R>
  TO_DEV static void running_derivs(const ParamsT<R>& P, const R* x, const R* u, R eps, R* lxx, R* lx, R* luu,
                                    R* lu) {
    R gx = 0, gy = 0, hxx = 0, hxy = 0, hyy = 0;
    const R is2 = R(1) / (P.bsig * P.bsig);
    const R inv = R(0.5) * is2;
    for (int b = 0; b < P.nb; ++b) {
      const R dx = x[0] - P.bc[b][0], dy = x[1] - P.bc[b][1];
      const R es = P.bamp * exp(-(dx * dx + dy * dy) * inv) * is2;
      gx -= es * dx;
      gy -= es * dy;
      hxx += es * (dx * dx * is2 - R(1));
      hyy += es * (dy * dy * is2 - R(1));
      hxy += es * dx * dy * is2;
    }
    eigclip_2x2(hxx, hxy, hyy, eps);
#pragma unroll
    for (int i = 0; i < n * n; ++i) lxx[i] = 0;
    lxx[0] = hxx; lxx[1] = hxy; lxx[n] = hxy; lxx[n + 1] = hyy;
    lxx[2 * n + 2] = clip0(eps); lxx[3 * n + 3] = clip0(eps); lxx[4 * n + 4] = clip0(eps);
    lx[0] = gx; lx[1] = gy; lx[2] = 0; lx[3] = 0; lx[4] = 0;
    const R w2 = R(2) * P.wu;
    const R d = w2 > eps ? w2 : eps;
    luu[0] = d; luu[1] = 0; luu[2] = 0; luu[3] = d;
    lu[0] = w2 * u[0]; lu[1] = w2 * u[1];
  }

  // A = df/dx, B = df/du in closed form, entries spread over the lanes; the
  // cost derivatives on the last lane of the group
  template <class R, int G>
  TO_DEV static void derivs(const ParamsT<R>& P, const Group<G>& g, const R* x, const R* u, R eps, R* A, R* B,
                            R* lxx, R* lx, R* luu, R* lu, R*) {
    R s, c;
    sincos(x[2], &s, &c);
    for (int e = g.lane; e < n * n + n * m; e += G) {
      if (e < n * n) {
        const int i = e / n, j = e % n;
        R v = (i == j) ? R(1) : R(0);
        if (i == 0 && j == 2) v = -P.dt * x[3] * s;
        if (i == 0 && j == 3) v = P.dt * c;
        if (i == 1 && j == 2) v = P.dt * x[3] * c;
        if (i == 1 && j == 3) v = P.dt * s;
        if (i == 3 && j == 4) v = P.dt;
        A[e] = v;
      } else {
        const int f = e - n * n, i = f / m, j = f % m;
        B[f] = ((i == 2 && j == 0) || (i == 4 && j == 1)) ? P.dt : R(0);
      }
    }
    if (g.lane == G - 1) running_derivs(P, x, u, eps, lxx, lx, luu, lu);
  }

  // the same on one lane (single-lane groups)
  template <class R>
  TO_DEV static void derivs_lane(const ParamsT<R>& P, const R* x, const R* u, R eps, R* A, R* B, R* lxx, R* lx,
                                 R* luu, R* lu) {
    R s, c;
    sincos(x[2], &s, &c);
#pragma unroll
    for (int i = 0; i < n; ++i)
#pragma unroll
      for (int j = 0; j < n; ++j) A[i * n + j] = (i == j) ? R(1) : R(0);
    A[0 * n + 2] = -P.dt * x[3] * s;
    A[0 * n + 3] = P.dt * c;
    A[1 * n + 2] = P.dt * x[3] * c;
    A[1 * n + 3] = P.dt * s;
    A[3 * n + 4] = P.dt;
#pragma unroll
    for (int i = 0; i < n * m; ++i) B[i] = R(0);
    B[2 * m + 0] = P.dt;
    B[4 * m + 1] = P.dt;
    running_derivs(P, x, u, eps, lxx, lx, luu, lu);
  }

  template <class R>
  TO_DEV static void terminal_derivs(const ParamsT<R>& P, const R* x, R eps, R* lxx, R* lx) {
    const R a = R(2) * P.wpT, b = R(2) * P.wvT, c = R(2) * P.waT;
#pragma unroll
    for (int i = 0; i < n * n; ++i) lxx[i] = 0;
    lxx[0] = a > eps ? a : eps; lxx[n + 1] = lxx[0];
    lxx[2 * n + 2] = clip0(eps);
    lxx[3 * n + 3] = b > eps ? b : eps;
    lxx[4 * n + 4] = c > eps ? c : eps;
    lx[0] = a * x[0]; lx[1] = a * x[1]; lx[2] = 0; lx[3] = b * x[3]; lx[4] = c * x[4];
  }
};

}  // namespace to
