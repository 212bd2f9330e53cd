// Planar 3-link arm in a vertical plane (Sec. V-A's manipulator, the
// synthetic workload's parameters).  x = [q1..q3, qd1..qd3], u = joint torques.
//
// Dynamics: M(q) qdd + h(q, qd) = tau with
//   * h from a world-frame planar Newton-Euler recursion (gravity enters as a
//     base acceleration -g),
//   * M_ij = sum_{k >= max(i,j)} I_k + m_k (c_k - P_i).(c_k - P_j), the
//     composite-rigid-body form for revolute z joints (c_k: centre of mass of
//     link k, P_i: position of joint i),
//   * semi-implicit Euler  qd+ = qd + dt qdd,  q+ = q + dt qd+.
// Derivatives: d qdd / d(q, qd) = -M^{-1} d ID(q, qd, qdd) / d(q, qd) with the
// directional derivative of the Newton-Euler recursion written out by hand,
// d qdd / d tau = M^{-1}: all six directions and the columns of M^{-1} on one
// lane (derivs_lane), which the solver runs for every knot before the
// backward pass and stores (kStoredDerivs).
#pragma once
#include "common.cuh"

namespace to {

template <class R>
struct Planar3Params {
  R dt, gx, gy;
  R len[3];   // joint i -> joint i+1 (len[2]: joint 3 -> end effector)
  R com[3];   // centre of mass along the link
  R mass[3], izz[3];
  R wtau, bamp, bsig, wee, wvT;
  int nb;
  R bc[2][2];
  R tgt[2];
};

template <class D, class S>
inline void cast_params(const Planar3Params<S>& s, Planar3Params<D>& d) {
  d.dt = (D)s.dt; d.gx = (D)s.gx; d.gy = (D)s.gy;
  for (int i = 0; i < 3; ++i) {
    d.len[i] = (D)s.len[i]; d.com[i] = (D)s.com[i]; d.mass[i] = (D)s.mass[i]; d.izz[i] = (D)s.izz[i];
  }
  d.wtau = (D)s.wtau; d.bamp = (D)s.bamp; d.bsig = (D)s.bsig; d.wee = (D)s.wee; d.wvT = (D)s.wvT;
  d.nb = s.nb;
  for (int b = 0; b < 2; ++b) { d.bc[b][0] = (D)s.bc[b][0]; d.bc[b][1] = (D)s.bc[b][1]; }
  d.tgt[0] = (D)s.tgt[0]; d.tgt[1] = (D)s.tgt[1];
}

struct SysPlanar3 {
  static constexpr int n = 6, m = 3;
  static constexpr bool kActor = false;
  template <class R> using ParamsT = Planar3Params<R>;
  template <class R> struct Scratch { static constexpr int elems = 1; };
  template <int G> static constexpr bool kGroupStep = false;
  static constexpr bool kKnotParallel = false;
  // derivatives computed for every knot before the backward pass, one knot
  // per lane (derivs_lane), and stored: A, B, l_xx, l_x, l_uu, l_u
  static constexpr bool kStoredDerivs = true;
  static constexpr int kDerivStride = n * n + n * m + n * n + n + m * m + m;

  // absolute link angles, link and centre-of-mass vectors, joint positions
  template <class R>
  struct Kin {
    R cs[3], sn[3];     // cos, sin of absolute angles
    R r[3][2];          // joint i -> joint i+1 (r[2]: to the end effector)
    R rc[3][2];         // joint i -> centre of mass i
    R P[4][2];          // joint positions, P[3] = end effector
  };

  template <class R>
  TO_DEV static void kinematics(const Planar3Params<R>& P, const R* q, Kin<R>& k) {
    R phi = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      phi += q[i];
      sincos(phi, &k.sn[i], &k.cs[i]);
      k.r[i][0] = P.len[i] * k.cs[i];
      k.r[i][1] = P.len[i] * k.sn[i];
      k.rc[i][0] = P.com[i] * k.cs[i];
      k.rc[i][1] = P.com[i] * k.sn[i];
    }
    k.P[0][0] = 0; k.P[0][1] = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) { k.P[i + 1][0] = k.P[i][0] + k.r[i][0]; k.P[i + 1][1] = k.P[i][1] + k.r[i][1]; }
  }

  // mass matrix (symmetric, row-major 3x3)
  template <class R>
  TO_DEV static void mass_matrix(const Planar3Params<R>& P, const Kin<R>& k, R* M) {
    R c[3][2];
#pragma unroll
    for (int i = 0; i < 3; ++i) { c[i][0] = k.P[i][0] + k.rc[i][0]; c[i][1] = k.P[i][1] + k.rc[i][1]; }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        R s = 0;
#pragma unroll
        for (int b = j; b < 3; ++b) {
          R ax = c[b][0] - k.P[i][0], ay = c[b][1] - k.P[i][1];
          R bx = c[b][0] - k.P[j][0], by = c[b][1] - k.P[j][1];
          s += P.izz[b] + P.mass[b] * (ax * bx + ay * by);
        }
        M[i * 3 + j] = s;
        M[j * 3 + i] = s;
      }
  }

  // planar Newton-Euler inverse dynamics; if tangent directions dq, dqd are
  // given (qdd held fixed) also returns the directional derivative dtau
  template <class R, bool kTangent>
  TO_DEV static void rnea(const Planar3Params<R>& P, const Kin<R>& k, const R* qd, const R* qdd, R* tau, const R* dq,
                          const R* dqd, R* dtau) {
    R w[3], al[3], ac[3][2], aP[2];
    R dw[3], dphi[3], dr[3][2], drc[3][2], dac[3][2], daP[2];
    R ws = 0, as = 0, dws = 0, dps = 0;
    aP[0] = -P.gx; aP[1] = -P.gy;
    daP[0] = 0; daP[1] = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      ws += qd[i]; as += qdd[i];
      w[i] = ws; al[i] = as;
      // a_c = a_P + al x rc - w^2 rc ;  a_P(next) = a_P + al x r - w^2 r
      ac[i][0] = aP[0] - al[i] * k.rc[i][1] - w[i] * w[i] * k.rc[i][0];
      ac[i][1] = aP[1] + al[i] * k.rc[i][0] - w[i] * w[i] * k.rc[i][1];
      if (kTangent) {
        dws += dqd[i]; dps += dq[i];
        dw[i] = dws; dphi[i] = dps;
        // rotating a vector by dphi: d r = dphi (-r_y, r_x)
        dr[i][0] = -dphi[i] * k.r[i][1]; dr[i][1] = dphi[i] * k.r[i][0];
        drc[i][0] = -dphi[i] * k.rc[i][1]; drc[i][1] = dphi[i] * k.rc[i][0];
        const R ww = w[i] * w[i], w2d = R(2) * w[i] * dw[i];
        dac[i][0] = daP[0] - al[i] * drc[i][1] - w2d * k.rc[i][0] - ww * drc[i][0];
        dac[i][1] = daP[1] + al[i] * drc[i][0] - w2d * k.rc[i][1] - ww * drc[i][1];
        daP[0] = daP[0] - al[i] * dr[i][1] - w2d * k.r[i][0] - ww * dr[i][0];
        daP[1] = daP[1] + al[i] * dr[i][0] - w2d * k.r[i][1] - ww * dr[i][1];
      }
      R nx = aP[0] - al[i] * k.r[i][1] - w[i] * w[i] * k.r[i][0];
      R ny = aP[1] + al[i] * k.r[i][0] - w[i] * w[i] * k.r[i][1];
      aP[0] = nx; aP[1] = ny;
    }
    // backward: F_i force from link i-1 on link i, N_i moment about joint i
    R F[2] = {0, 0}, N = 0, dF[2] = {0, 0}, dN = 0;
#pragma unroll
    for (int i = 2; i >= 0; --i) {
      const R mx = P.mass[i] * ac[i][0], my = P.mass[i] * ac[i][1];
      // N_i = I al + rc x m a_c + r x F_{i+1} + N_{i+1}
      R Nn = P.izz[i] * al[i] + (k.rc[i][0] * my - k.rc[i][1] * mx) + (k.r[i][0] * F[1] - k.r[i][1] * F[0]) + N;
      if (kTangent) {
        const R dmx = P.mass[i] * dac[i][0], dmy = P.mass[i] * dac[i][1];
        R dNn = (k.rc[i][0] * dmy - k.rc[i][1] * dmx) + (drc[i][0] * my - drc[i][1] * mx) +
                (k.r[i][0] * dF[1] - k.r[i][1] * dF[0]) + (dr[i][0] * F[1] - dr[i][1] * F[0]) + dN;
        dF[0] += dmx; dF[1] += dmy;
        dN = dNn;
        dtau[i] = dNn;
      }
      F[0] += mx; F[1] += my;
      N = Nn;
      tau[i] = Nn;
    }
  }

  // M = L L^T with the reciprocal pivots stored on L's diagonal
  template <class R>
  TO_DEV static void chol3(const R* M, R* L) {
    L[0] = rsqrt_(M[0]);
    L[3] = M[3] * L[0];
    L[6] = M[6] * L[0];
    L[4] = rsqrt_(M[4] - L[3] * L[3]);
    L[7] = (M[7] - L[6] * L[3]) * L[4];
    L[8] = rsqrt_(M[8] - L[6] * L[6] - L[7] * L[7]);
  }
  template <class R>
  TO_DEV static void chol3_solve(const R* L, const R* b, R* x) {
    R y0 = b[0] * L[0];
    R y1 = (b[1] - L[3] * y0) * L[4];
    R y2 = (b[2] - L[6] * y0 - L[7] * y1) * L[8];
    x[2] = y2 * L[8];
    x[1] = (y1 - L[7] * x[2]) * L[4];
    x[0] = (y0 - L[3] * x[1] - L[6] * x[2]) * L[0];
  }

  template <class R>
  TO_DEV static void forward_dynamics(const Planar3Params<R>& P, const Kin<R>& k, const R* qd, const R* tau, R* qdd, R* L) {
    R M[9], h[3], z[3] = {0, 0, 0}, rhs[3];
    mass_matrix(P, k, M);
    chol3(M, L);
    rnea<R, false>(P, k, qd, z, h, nullptr, nullptr, nullptr);
#pragma unroll
    for (int i = 0; i < 3; ++i) rhs[i] = tau[i] - h[i];
    chol3_solve(L, rhs, qdd);
  }


  // Columns of [A | B] and the clipped running-cost derivatives on one lane:
  // the primal (kinematics, M's factor, qdd), then the tangent Newton-Euler
  // pass along each x_c, the three columns of M^{-1} for B, and the cost
  // terms.  The solver runs it for every knot before the backward pass (one
  // knot per lane, blocks stored) and inside single-lane groups.
  template <class R>
  TO_DEV static void derivs_lane(const Planar3Params<R>& P, const R* x, const R* u, R eps, R* A, R* B, R* lxx,
                                 R* lx, R* luu, R* lu) {
    const R dt = P.dt;
    Kin<R> k;
    kinematics(P, x, k);
    R qdd[3], L[9], d[3];
    forward_dynamics(P, k, x + 3, u, qdd, L);
#pragma unroll
    for (int c = 0; c < n; ++c) {
      R dq[3] = {0, 0, 0}, dqd[3] = {0, 0, 0}, tau[3], dtau[3];
      if (c < 3) dq[c] = 1; else dqd[c - 3] = 1;
      rnea<R, true>(P, k, x + 3, qdd, tau, dq, dqd, dtau);
      chol3_solve(L, dtau, d);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const R eq = (c == i) ? R(1) : R(0);
        const R ev = (c == 3 + i) ? R(1) : R(0);
        const R dv = ev - dt * d[i];
        A[(3 + i) * n + c] = dv;
        A[i * n + c] = eq + dt * dv;
      }
    }
#pragma unroll
    for (int c = 0; c < m; ++c) {
      R e[3] = {0, 0, 0};
      e[c] = 1;
      chol3_solve(L, e, d);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        B[(3 + i) * m + c] = dt * d[i];
        B[i * m + c] = dt * dt * d[i];
      }
    }
    running_derivs_k(P, k, u, eps, lxx, lx, luu, lu);
  }

  // running cost at (x, u) and the next state, sharing one kinematics pass

  // the same step on a state carried as (hi, lo) pairs, in place
  template <class R>
  TO_DEV static R cost_step2(const Planar3Params<R>& P, R* xh, R* xl, const R* u) {
    Kin<R> k;
    kinematics(P, xh, k);
    R l = P.wtau * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const R inv = R(0.5) / (P.bsig * P.bsig);
    for (int b = 0; b < P.nb; ++b) {
      R dx = k.P[3][0] - P.bc[b][0], dy = k.P[3][1] - P.bc[b][1];
      l += P.bamp * exp(-(dx * dx + dy * dy) * inv);
    }
    R qdd[3], L[9];
    forward_dynamics(P, k, xh + 3, u, qdd, L);
    semi_implicit2<R, 3>(xh, xl, xh + 3, xl + 3, qdd, P.dt);
    return l;
  }

  // end-effector Jacobian J (2x3) and the second-derivative structure:
  // d2 ee / dq_i dq_j = -(ee - P_max(i,j))
  template <class R>
  TO_DEV static void ee_derivs(const Kin<R>& k, R* ee, R J[2][3]) {
    ee[0] = k.P[3][0]; ee[1] = k.P[3][1];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      J[0][j] = -(ee[1] - k.P[j][1]);
      J[1][j] = ee[0] - k.P[j][0];
    }
  }

  // l_qq = J^T H_ee J + sum_d g_ee[d] d2ee_d/dq2, written to the 6x6 lxx with
  // the q-block clipped and eps on the qd diagonal
  template <class R>
  TO_DEV static void assemble_q_block(const Kin<R>& k, const R* ee, const R J[2][3], const R* gee, const R H[2][2],
                                      R eps, R* lxx, R* lx) {
    R Q[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int b = i > j ? i : j;
        R s = 0;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int c = 0; c < 2; ++c) s += J[a][i] * H[a][c] * J[c][j];
        s -= gee[0] * (ee[0] - k.P[b][0]) + gee[1] * (ee[1] - k.P[b][1]);
        Q[i * 3 + j] = s;
      }
    eigclip_small<R, 3>(Q, eps);
#pragma unroll
    for (int i = 0; i < n * n; ++i) lxx[i] = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) lxx[i * n + j] = Q[i * 3 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i) lx[i] = J[0][i] * gee[0] + J[1][i] * gee[1];
  }

  template <class R>
  TO_DEV static R running_cost(const Planar3Params<R>& P, const R* x, const R* u) {
    Kin<R> k;
    kinematics(P, x, k);
    R l = P.wtau * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const R inv = R(1) / (R(2) * P.bsig * P.bsig);
    for (int b = 0; b < P.nb; ++b) {
      R dx = k.P[3][0] - P.bc[b][0], dy = k.P[3][1] - P.bc[b][1];
      l += P.bamp * exp(-(dx * dx + dy * dy) * inv);
    }
    return l;
  }

  template <class R>
  TO_DEV static R terminal_cost(const Planar3Params<R>& P, const R* x) {
    Kin<R> k;
    kinematics(P, x, k);
    R dx = k.P[3][0] - P.tgt[0], dy = k.P[3][1] - P.tgt[1];
    return P.wee * (dx * dx + dy * dy) + P.wvT * (x[3] * x[3] + x[4] * x[4] + x[5] * x[5]);
  }

  template <class R>
  TO_DEV static void running_derivs_k(const Planar3Params<R>& P, const Kin<R>& k, const R* u, R eps, R* lxx, R* lx,
                                      R* luu, R* lu) {
    R ee[2], J[2][3];
    ee_derivs(k, ee, J);
    R gee[2] = {0, 0}, H[2][2] = {{0, 0}, {0, 0}};
    const R s2 = P.bsig * P.bsig;
    const R is2 = R(1) / s2, inv = R(0.5) * is2;
    for (int b = 0; b < P.nb; ++b) {
      const R d0 = ee[0] - P.bc[b][0], d1 = ee[1] - P.bc[b][1];
      const R e = P.bamp * exp(-(d0 * d0 + d1 * d1) * inv);
      const R g0 = d0 * is2, g1 = d1 * is2;     // gradient of the exponent / -1
      gee[0] -= e * g0;
      gee[1] -= e * g1;
      H[0][0] += e * (g0 * g0 - is2);
      H[1][1] += e * (g1 * g1 - is2);
      H[0][1] += e * g0 * g1;
    }
    H[1][0] = H[0][1];
    assemble_q_block(k, ee, J, gee, H, eps, lxx, lx);
#pragma unroll
    for (int i = 3; i < 6; ++i) { lxx[i * n + i] = clip0(eps); lx[i] = 0; }
    const R w2 = R(2) * P.wtau;
    const R d = w2 > eps ? w2 : eps;
#pragma unroll
    for (int i = 0; i < 9; ++i) luu[i] = 0;
    luu[0] = d; luu[4] = d; luu[8] = d;
#pragma unroll
    for (int i = 0; i < 3; ++i) lu[i] = w2 * u[i];
  }

  template <class R>
  TO_DEV static void terminal_derivs(const Planar3Params<R>& P, const R* x, R eps, R* lxx, R* lx) {
    Kin<R> k;
    kinematics(P, x, k);
    R ee[2], J[2][3];
    ee_derivs(k, ee, J);
    const R w2 = R(2) * P.wee;
    R gee[2] = {w2 * (ee[0] - P.tgt[0]), w2 * (ee[1] - P.tgt[1])};
    R H[2][2] = {{w2, 0}, {0, w2}};
    assemble_q_block(k, ee, J, gee, H, eps, lxx, lx);
    const R v2 = R(2) * P.wvT;
    const R d = v2 > eps ? v2 : eps;
#pragma unroll
    for (int i = 3; i < 6; ++i) { lxx[i * n + i] = d; lx[i] = v2 * x[i]; }
  }
};

}  // namespace to
