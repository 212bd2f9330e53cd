// Rigid-body trees for the 7-DoF arm and the quadruped-shaped floating base
// (Sec. V-A's manipulators, Sec. V-D's quadruped; the synthetic workloads'
// parameters).  x = [q; qd], u = torques of joints a0..N-1.
//
// Dynamics: M(q) qdd + h(q, qd) = [0; u] (+ soft ground contact at the feet
// for the quadruped), n_sub semi-implicit Euler substeps of h = dt / n_sub:
//   qd+ = qd + h qdd,  q+ = q + h qd+.
// * h(q, qd): body-frame spatial Newton-Euler (Featherstone 2008, ch. 5) with
//   gravity as a base acceleration and the contact forces as external forces;
// * M(q): composite-rigid-body algorithm (Featherstone 2008, Sec. 6.2),
//   Cholesky-factored.
// Derivatives: each lane propagates one tangent direction (a state
// coordinate, or a control) through the substeps:
//   dqdd = M^{-1} (dtau - d ID(q, qd, qdd) / d(q, qd) . (dq, dqd)),
// with the directional derivative of the inverse dynamics (qdd held fixed)
// from a hand-written tangent pass over per-body primal quantities (the
// product rule of the Newton-Euler recursion).  The primal quantities of
// every knot's substeps are computed before the backward pass, one knot per
// lane, and stored; the tangent lanes stage them into shared memory.  A
// dual-number pass of the same recursion serves the arm's nested terminal
// Hessian.
#pragma once
#include "common.cuh"

namespace to {

// ---------------------------------------------------------------------------
// a dual number: value and one directional derivative
// ---------------------------------------------------------------------------
template <class R>
struct Dl {
  R v, d;
  TO_DEV Dl() {}
  TO_DEV Dl(R a) : v(a), d(0) {}
  TO_DEV Dl(R a, R b) : v(a), d(b) {}
};
template <class R> TO_DEV Dl<R> operator+(Dl<R> a, Dl<R> b) { return Dl<R>(a.v + b.v, a.d + b.d); }
template <class R> TO_DEV Dl<R> operator-(Dl<R> a, Dl<R> b) { return Dl<R>(a.v - b.v, a.d - b.d); }
template <class R> TO_DEV Dl<R> operator-(Dl<R> a) { return Dl<R>(-a.v, -a.d); }
template <class R> TO_DEV Dl<R> operator*(Dl<R> a, Dl<R> b) { return Dl<R>(a.v * b.v, a.v * b.d + a.d * b.v); }
template <class R> TO_DEV Dl<R> operator*(R a, Dl<R> b) { return Dl<R>(a * b.v, a * b.d); }
template <class R> TO_DEV Dl<R> operator/(Dl<R> a, Dl<R> b) {
  const R iv = R(1) / b.v;
  return Dl<R>(a.v * iv, (a.d - a.v * iv * b.d) * iv);
}
template <class R> TO_DEV Dl<R>& operator+=(Dl<R>& a, Dl<R> b) { a = a + b; return a; }
template <class R> TO_DEV Dl<R>& operator-=(Dl<R>& a, Dl<R> b) { a = a - b; return a; }
TO_DEV float dexp(float a) { return expf(a); }
TO_DEV double dexp(double a) { return exp(a); }
TO_DEV float dlog1p(float a) { return log1pf(a); }
TO_DEV double dlog1p(double a) { return log1p(a); }
TO_DEV void dsincos(float a, float* s, float* c) { sincosf(a, s, c); }
TO_DEV void dsincos(double a, double* s, double* c) { sincos(a, s, c); }
TO_DEV float value_of(float a) { return a; }
TO_DEV double value_of(double a) { return a; }
template <class R> TO_DEV auto value_of(Dl<R> a) { return value_of(a.v); }
template <class R> TO_DEV Dl<R> dexp(Dl<R> a) { const R e = dexp(a.v); return Dl<R>(e, e * a.d); }
template <class R> TO_DEV Dl<R> dlog1p(Dl<R> a) { return Dl<R>(dlog1p(a.v), a.d / (R(1) + a.v)); }
template <class R> TO_DEV void dsincos(Dl<R> a, Dl<R>* s, Dl<R>* c) {
  R sv, cv;
  dsincos(a.v, &sv, &cv);
  *s = Dl<R>(sv, cv * a.d);
  *c = Dl<R>(cv, -(sv * a.d));
}

// ---------------------------------------------------------------------------
// parameters
// ---------------------------------------------------------------------------
enum { RK_ARM7 = 3, RK_QUAD = 4 };

template <class R, int N>
struct RigidParams {
  R dt, g[3];
  int n_sub, a0;
  int parent[N], jtype[N];
  R off[N][3], mass[N], com[N][3], inertia[N][3];
  // arm reaching cost
  R wtau, wv, tgt[3], wee, wvT, ee_pt[3];
  int ee_body;
  // quadruped cost and contact
  R znom, wz, wrpy, wvx, vxt, tscale, kc, dc, beta;
  int nfeet, foot_body[4];
  R foot_pt[4][3];
};

template <class D, class S, int N>
inline void cast_params(const RigidParams<S, N>& s, RigidParams<D, N>& d) {
  d.dt = (D)s.dt;
  for (int k = 0; k < 3; ++k) { d.g[k] = (D)s.g[k]; d.tgt[k] = (D)s.tgt[k]; d.ee_pt[k] = (D)s.ee_pt[k]; }
  d.n_sub = s.n_sub; d.a0 = s.a0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    d.parent[i] = s.parent[i]; d.jtype[i] = s.jtype[i]; d.mass[i] = (D)s.mass[i];
    for (int k = 0; k < 3; ++k) { d.off[i][k] = (D)s.off[i][k]; d.com[i][k] = (D)s.com[i][k]; d.inertia[i][k] = (D)s.inertia[i][k]; }
  }
  d.wtau = (D)s.wtau; d.wv = (D)s.wv; d.wee = (D)s.wee; d.wvT = (D)s.wvT; d.ee_body = s.ee_body;
  d.znom = (D)s.znom; d.wz = (D)s.wz; d.wrpy = (D)s.wrpy; d.wvx = (D)s.wvx; d.vxt = (D)s.vxt;
  d.tscale = (D)s.tscale; d.kc = (D)s.kc; d.dc = (D)s.dc; d.beta = (D)s.beta; d.nfeet = s.nfeet;
  for (int f = 0; f < 4; ++f) {
    d.foot_body[f] = s.foot_body[f];
    for (int k = 0; k < 3; ++k) d.foot_pt[f][k] = (D)s.foot_pt[f][k];
  }
}

// ---------------------------------------------------------------------------
// Joint trees, fixed at compile time: every loop over the bodies and over an
// ancestor chain has a compile-time trip count and unrolls, so the per-body
// arrays of the recursions are registers (or fixed stack slots) rather than
// dynamically indexed local memory.  parent(i) < i (parents first); depth(i)
// counts the ancestors of body i and anc(i, d) is its d-th ancestor
// (anc(i, 0) = i).  Joint types: 0..2 revolute about x, y, z; 3..5 prismatic
// along x, y, z.  The host parser accepts exactly these trees.
// ---------------------------------------------------------------------------
template <int KIND>
struct RigidTopo;

// 7-DoF arm: a chain of revolute joints about z, y, z, y, z, y, z; the end
// effector on the last body
template <>
struct RigidTopo<RK_ARM7> {
  static constexpr int kBodies = 7, kDepthMax = 6, kFeet = 0, kEeBody = 6;
  static constexpr int parent(int i) { return i - 1; }
  static constexpr int jtype(int i) { return (i & 1) ? 1 : 2; }
  static constexpr int depth(int i) { return i; }
  static constexpr int anc(int i, int d) { return i - d; }
  static constexpr int foot_body(int) { return -1; }
};

// quadruped: the floating base as the chain Px, Py, Pz, Rz, Ry, Rx (bodies
// 0..5, the base's mass on body 5), then four legs of hip (x), thigh (y) and
// calf (y) joints hanging from body 5; the feet on the calves
template <>
struct RigidTopo<RK_QUAD> {
  static constexpr int kBodies = 18, kDepthMax = 8, kFeet = 4, kEeBody = -1;
  static constexpr int parent(int i) { return i < 6 ? i - 1 : ((i - 6) % 3 == 0 ? 5 : i - 1); }
  static constexpr int jtype(int i) { return i < 3 ? 3 + i : (i < 6 ? 5 - i : ((i - 6) % 3 == 0 ? 0 : 1)); }
  static constexpr int depth(int i) { return i < 6 ? i : 6 + (i - 6) % 3; }
  static constexpr int anc(int i, int d) { return (i < 6 || d <= (i - 6) % 3) ? i - d : 6 + (i - 6) % 3 - d; }
  static constexpr int foot_body(int f) { return 8 + 3 * f; }
};

// ---------------------------------------------------------------------------
// the model
// ---------------------------------------------------------------------------
template <int N_, int A0, int KIND>
struct SysRigid {
  static constexpr int N = N_;
  static constexpr int n = 2 * N, m = N - A0;
  static constexpr bool kActor = (KIND == RK_QUAD);   // 36 -> 256 -> 256 -> 12 actor warm start
  template <class R> using ParamsT = RigidParams<R, N>;
  typedef RigidTopo<KIND> Topo;
  static_assert(Topo::kBodies == N, "joint tree size");
  static constexpr int kDepthMax = Topo::kDepthMax, kFeet = Topo::kFeet, kEeBody = Topo::kEeBody;
  static constexpr int parent(int i) { return Topo::parent(i); }
  static constexpr int jtype(int i) { return Topo::jtype(i); }
  static constexpr int depth(int i) { return Topo::depth(i); }
  static constexpr int anc(int i, int d) { return Topo::anc(i, d); }
  static constexpr int foot_body(int f) { return Topo::foot_body(f); }

  // 3-vectors
  template <class S> TO_DEV static void cross(const S* a, const S* b, S* c) {
    const S c0 = a[1] * b[2] - a[2] * b[1], c1 = a[2] * b[0] - a[0] * b[2], c2 = a[0] * b[1] - a[1] * b[0];
    c[0] = c0; c[1] = c1; c[2] = c2;
  }
  // y = E x and y = E^T x for a row-major 3x3 E
  template <class S> TO_DEV static void mv(const S* E, const S* x, S* y) {
    const S y0 = E[0] * x[0] + E[1] * x[1] + E[2] * x[2];
    const S y1 = E[3] * x[0] + E[4] * x[1] + E[5] * x[2];
    const S y2 = E[6] * x[0] + E[7] * x[1] + E[8] * x[2];
    y[0] = y0; y[1] = y1; y[2] = y2;
  }
  template <class S> TO_DEV static void mtv(const S* E, const S* x, S* y) {
    const S y0 = E[0] * x[0] + E[3] * x[1] + E[6] * x[2];
    const S y1 = E[1] * x[0] + E[4] * x[1] + E[7] * x[2];
    const S y2 = E[2] * x[0] + E[5] * x[1] + E[8] * x[2];
    y[0] = y0; y[1] = y1; y[2] = y2;
  }

  // y = E x and y = E^T x for a joint transform: a rotation about the joint's
  // coordinate axis (4 nonzeros besides the unit entry) or the identity
  // (prismatic).  The joint type is a compile-time constant at every call
  // (the body loops unroll), so the switch folds away.
  template <class S> TO_DEV static void jmv(int jt, const S* E, const S* x, S* y) {
    const S x0 = x[0], x1 = x[1], x2 = x[2];
    switch (jt) {
      case 0: { const S c = E[4], s = E[5]; y[0] = x0; y[1] = c * x1 + s * x2; y[2] = c * x2 - s * x1; break; }
      case 1: { const S c = E[0], s = E[6]; y[0] = c * x0 - s * x2; y[1] = x1; y[2] = c * x2 + s * x0; break; }
      case 2: { const S c = E[0], s = E[1]; y[0] = c * x0 + s * x1; y[1] = c * x1 - s * x0; y[2] = x2; break; }
      default: y[0] = x0; y[1] = x1; y[2] = x2;
    }
  }
  template <class S> TO_DEV static void jmtv(int jt, const S* E, const S* x, S* y) {
    const S x0 = x[0], x1 = x[1], x2 = x[2];
    switch (jt) {
      case 0: { const S c = E[4], s = E[5]; y[0] = x0; y[1] = c * x1 - s * x2; y[2] = c * x2 + s * x1; break; }
      case 1: { const S c = E[0], s = E[6]; y[0] = c * x0 + s * x2; y[1] = x1; y[2] = c * x2 - s * x0; break; }
      case 2: { const S c = E[0], s = E[1]; y[0] = c * x0 - s * x1; y[1] = c * x1 + s * x0; y[2] = x2; break; }
      default: y[0] = x0; y[1] = x1; y[2] = x2;
    }
  }

  // Plucker transform of joint i: E maps parent coordinates to body
  // coordinates (a rotation by q about the joint axis, or identity), r is the
  // body origin in parent coordinates
  template <class R, class S>
  TO_DEV static void joint_transform(const ParamsT<R>& P, int i, S q, S* E, S* r) {
    const int jt = jtype(i);
#pragma unroll
    for (int k = 0; k < 3; ++k) r[k] = S(P.off[i][k]);
#pragma unroll
    for (int k = 0; k < 9; ++k) E[k] = S(R(0));
    if (jt <= 2) {
      S s, c;
      dsincos(q, &s, &c);
      const int a = jt, b = (jt + 1) % 3, cc = (jt + 2) % 3;
      E[a * 3 + a] = S(R(1));
      E[b * 3 + b] = c; E[b * 3 + cc] = s;
      E[cc * 3 + b] = -s; E[cc * 3 + cc] = c;
    } else {
      E[0] = S(R(1)); E[4] = S(R(1)); E[8] = S(R(1));
      r[jt - 3] = r[jt - 3] + q;
    }
  }

  // world pose: E0 maps world to body coordinates, p0 is the body origin
  template <class R, class S>
  TO_DEV static void world_pose(const ParamsT<R>& P, const S* q, S (*E0)[9], S (*p0)[3]) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      S E[9], r[3];
      joint_transform(P, i, q[i], E, r);
      const int pa = parent(i);
      if (pa < 0) {
#pragma unroll
        for (int k = 0; k < 9; ++k) E0[i][k] = E[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) p0[i][k] = r[k];
      } else {
        // E0_i = E E0_p ;  p0_i = p0_p + E0_p^T r
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b)
            E0[i][a * 3 + b] = E[a * 3 + 0] * E0[pa][0 * 3 + b] + E[a * 3 + 1] * E0[pa][1 * 3 + b] + E[a * 3 + 2] * E0[pa][2 * 3 + b];
        S wr[3];
        mtv(E0[pa], r, wr);
#pragma unroll
        for (int k = 0; k < 3; ++k) p0[i][k] = p0[pa][k] + wr[k];
      }
    }
  }

  // spatial inertia times a motion vector (w, v): momentum about the body
  // origin, (I_c w + c x p, p) with p = m (v + w x c)
  template <class R, class S>
  TO_DEV static void inertia_mul(const ParamsT<R>& P, int i, const S* w, const S* v, S* n, S* f) {
    S c[3] = {S(P.com[i][0]), S(P.com[i][1]), S(P.com[i][2])};
    S wc[3];
    cross(w, c, wc);
    S p[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) p[k] = P.mass[i] * (v[k] + wc[k]);
    S cp[3];
    cross(c, p, cp);
#pragma unroll
    for (int k = 0; k < 3; ++k) { n[k] = P.inertia[i][k] * w[k] + cp[k]; f[k] = p[k]; }
  }

  // inverse dynamics: tau = ID(q, qd, qdd) with optional gravity and contact
  template <class R, class S>
  TO_DEV static void rnea(const ParamsT<R>& P, const S* q, const S* qd, const S* qdd, bool grav, bool contact,
                          S* tau) {
    S E[N][9], r[N][3], vw[N][3], vv[N][3], fn[N][3], ff[N][3];
    S aw[3], av[3];
    S E0[KIND == RK_QUAD ? N : 1][9], p0[KIND == RK_QUAD ? N : 1][3];
    S awb[N][3], avb[N][3];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      joint_transform(P, i, q[i], E[i], r[i]);
      const int pa = parent(i);
      S pw[3], pv[3], paw[3], pav[3];
      if (pa < 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          pw[k] = S(R(0)); pv[k] = S(R(0)); paw[k] = S(R(0));
          pav[k] = grav ? S(-P.g[k]) : S(R(0));
        }
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          pw[k] = vw[pa][k]; pv[k] = vv[pa][k]; paw[k] = awb[pa][k]; pav[k] = avb[pa][k];
        }
      }
      // X m = (E w, E (v - r x w))
      S t[3], rw[3];
      cross(r[i], pw, rw);
#pragma unroll
      for (int k = 0; k < 3; ++k) t[k] = pv[k] - rw[k];
      jmv(jtype(i), E[i], pw, vw[i]);
      jmv(jtype(i), E[i], t, vv[i]);
      cross(r[i], paw, rw);
#pragma unroll
      for (int k = 0; k < 3; ++k) t[k] = pav[k] - rw[k];
      jmv(jtype(i), E[i], paw, aw);
      jmv(jtype(i), E[i], t, av);
      // joint motion S qd, S qdd; velocity-product term v x (S qd)
      const int jt = jtype(i);
      S sw[3] = {S(R(0)), S(R(0)), S(R(0))}, sv[3] = {S(R(0)), S(R(0)), S(R(0))};
      if (jt <= 2) sw[jt] = qd[i]; else sv[jt - 3] = qd[i];
#pragma unroll
      for (int k = 0; k < 3; ++k) { vw[i][k] = vw[i][k] + sw[k]; vv[i][k] = vv[i][k] + sv[k]; }
      S c1[3], c2[3], c3[3];
      cross(vw[i], sw, c1);
      cross(vw[i], sv, c2);
      cross(vv[i], sw, c3);
#pragma unroll
      for (int k = 0; k < 3; ++k) { aw[k] = aw[k] + c1[k]; av[k] = av[k] + c2[k] + c3[k]; }
      if (jt <= 2) aw[jt] = aw[jt] + qdd[i]; else av[jt - 3] = av[jt - 3] + qdd[i];
#pragma unroll
      for (int k = 0; k < 3; ++k) { awb[i][k] = aw[k]; avb[i][k] = av[k]; }
      // f = I a + v x* (I v)
      S In[3], If[3], hn[3], hf[3];
      inertia_mul(P, i, aw, av, In, If);
      inertia_mul(P, i, vw[i], vv[i], hn, hf);
      S x1[3], x2[3], x3[3];
      cross(vw[i], hn, x1);
      cross(vv[i], hf, x2);
      cross(vw[i], hf, x3);
#pragma unroll
      for (int k = 0; k < 3; ++k) { fn[i][k] = In[k] + x1[k] + x2[k]; ff[i][k] = If[k] + x3[k]; }
      if (KIND == RK_QUAD) {
        if (pa < 0) {
#pragma unroll
          for (int k = 0; k < 9; ++k) E0[i][k] = E[i][k];
#pragma unroll
          for (int k = 0; k < 3; ++k) p0[i][k] = r[i][k];
        } else {
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
              E0[i][a * 3 + b] = E[i][a * 3 + 0] * E0[pa][b] + E[i][a * 3 + 1] * E0[pa][3 + b] + E[i][a * 3 + 2] * E0[pa][6 + b];
          S wr[3];
          mtv(E0[pa], r[i], wr);
#pragma unroll
          for (int k = 0; k < 3; ++k) p0[i][k] = p0[pa][k] + wr[k];
        }
      }
    }
    if (KIND == RK_QUAD && contact) {
#pragma unroll
      for (int ft = 0; ft < kFeet; ++ft) {
        const int bi = foot_body(ft);
        S pt[3] = {S(P.foot_pt[ft][0]), S(P.foot_pt[ft][1]), S(P.foot_pt[ft][2])};
        S wpt[3], Pw[3], wxp[3], vb[3], vwld[3];
        mtv(E0[bi], pt, wpt);
#pragma unroll
        for (int k = 0; k < 3; ++k) Pw[k] = p0[bi][k] + wpt[k];
        cross(vw[bi], pt, wxp);
#pragma unroll
        for (int k = 0; k < 3; ++k) vb[k] = vv[bi][k] + wxp[k];
        mtv(E0[bi], vb, vwld);
        // normal: k softplus_beta(-z) - d sigmoid(-beta z) zdot; tangential damper
        // softplus_beta(-z) = log(1 + exp(-beta z)) / beta and sigmoid(-beta z),
        // evaluated with exp of a non-positive argument only (no overflow)
        const S bz = P.beta * Pw[2];
        S sp, gate;
        if (value_of(bz) >= R(0)) {
          const S e = dexp(-bz);
          sp = (R(1) / P.beta) * dlog1p(e);
          gate = e / (S(R(1)) + e);
        } else {
          const S e = dexp(bz);
          sp = (R(1) / P.beta) * (dlog1p(e) - bz);
          gate = S(R(1)) / (S(R(1)) + e);
        }
        S F[3];
        F[0] = -(P.dc * (gate * vwld[0]));
        F[1] = -(P.dc * (gate * vwld[1]));
        F[2] = P.kc * sp - P.dc * (gate * vwld[2]);
        S mw[3], mb[3], fb[3];
        cross(wpt, F, mw);
        mv(E0[bi], mw, mb);
        mv(E0[bi], F, fb);
#pragma unroll
        for (int k = 0; k < 3; ++k) { fn[bi][k] = fn[bi][k] - mb[k]; ff[bi][k] = ff[bi][k] - fb[k]; }
      }
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
      const int jt = jtype(i);
      tau[i] = jt <= 2 ? fn[i][jt] : ff[i][jt - 3];
      const int pa = parent(i);
      if (pa >= 0) {
        // X^T f = (E^T n + r x E^T f, E^T f)
        S en[3], ef[3], rf[3];
        jmtv(jt, E[i], fn[i], en);
        jmtv(jt, E[i], ff[i], ef);
        cross(r[i], ef, rf);
#pragma unroll
        for (int k = 0; k < 3; ++k) { fn[pa][k] = fn[pa][k] + en[k] + rf[k]; ff[pa][k] = ff[pa][k] + ef[k]; }
      }
    }
  }

  // Joint-space mass matrix by the composite-rigid-body algorithm
  // (Featherstone 2008, Sec. 6.2), written into the lower triangle of L and
  // factored in place as M = L^T L along the tree (reciprocal pivots).  A subtree's composite
  // inertia is kept about its root body's origin, in that body's coordinates,
  // as (mass, first moment h = mass * com, rotational inertia about the
  // origin); moving it to the parent frame rotates it and applies the
  // parallel-axis shift.  Bodies are ordered parents first.
  template <class R>
  TO_DEV static void mass_chol(const ParamsT<R>& P, const R* q, R* L) {
    R E[N][9], r[N][3];
    R cm[N], ch[N][3], cI[N][6];   // cI: xx, yy, zz, xy, xz, yz
#pragma unroll
    for (int i = 0; i < N; ++i) {
      joint_transform(P, i, q[i], E[i], r[i]);
      const R mi = P.mass[i], c0 = P.com[i][0], c1 = P.com[i][1], c2 = P.com[i][2];
      cm[i] = mi;
      ch[i][0] = mi * c0; ch[i][1] = mi * c1; ch[i][2] = mi * c2;
      // I_origin = I_com + m (|c|^2 1 - c c^T)
      cI[i][0] = P.inertia[i][0] + mi * (c1 * c1 + c2 * c2);
      cI[i][1] = P.inertia[i][1] + mi * (c0 * c0 + c2 * c2);
      cI[i][2] = P.inertia[i][2] + mi * (c0 * c0 + c1 * c1);
      cI[i][3] = -mi * c0 * c1; cI[i][4] = -mi * c0 * c2; cI[i][5] = -mi * c1 * c2;
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
      const int pa = parent(i);
      if (pa < 0) continue;
      const R* e = E[i];
      const R* rr = r[i];
      const R mi = cm[i];
      // h_A = E^T h (parent coordinates, about the child origin)
      R hA[3];
      jmtv(jtype(i), e, ch[i], hA);
      // I_A = E^T I E
      const R I3[9] = {cI[i][0], cI[i][3], cI[i][4], cI[i][3], cI[i][1], cI[i][5], cI[i][4], cI[i][5], cI[i][2]};
      R T[9];   // I E
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) T[a * 3 + b] = I3[a * 3 + 0] * e[0 * 3 + b] + I3[a * 3 + 1] * e[1 * 3 + b] + I3[a * 3 + 2] * e[2 * 3 + b];
      R IA[6];
      const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int k = 0; k < 6; ++k)
        IA[k] = e[0 * 3 + ia[k]] * T[0 * 3 + ib[k]] + e[1 * 3 + ia[k]] * T[1 * 3 + ib[k]] + e[2 * 3 + ia[k]] * T[2 * 3 + ib[k]];
      // shift to the parent origin (child origin at r):
      // I_O = I_A + m (|r|^2 1 - r r^T) + 2 (r.h_A) 1 - (h_A r^T + r h_A^T)
      const R r2 = rr[0] * rr[0] + rr[1] * rr[1] + rr[2] * rr[2];
      const R rh = rr[0] * hA[0] + rr[1] * hA[1] + rr[2] * hA[2];
#pragma unroll
      for (int k = 0; k < 3; ++k) cI[pa][k] += IA[k] + mi * (r2 - rr[k] * rr[k]) + R(2) * (rh - hA[k] * rr[k]);
#pragma unroll
      for (int k = 3; k < 6; ++k) cI[pa][k] += IA[k] - mi * rr[ia[k]] * rr[ib[k]] - (hA[ia[k]] * rr[ib[k]] + rr[ia[k]] * hA[ib[k]]);
#pragma unroll
      for (int k = 0; k < 3; ++k) ch[pa][k] += hA[k] + mi * rr[k];
      cm[pa] += mi;
    }
    // only (body, ancestor) entries are formed and read: the others are zero
#pragma unroll
    for (int i = 0; i < N; ++i) {
      // F = Ic_i S_i: revolute about axis a: (I e_a, e_a x h); prismatic along a: (h x e_a, m e_a)
      R fn[3], ff[3];
      const int jt = jtype(i);
      const R* c6 = cI[i];
      if (jt <= 2) {
        const int a = jt;
        const int col[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
        fn[0] = c6[col[0][a]]; fn[1] = c6[col[1][a]]; fn[2] = c6[col[2][a]];
        R ea[3] = {R(0), R(0), R(0)};
        ea[a] = R(1);
        cross(ea, ch[i], ff);
      } else {
        const int a = jt - 3;
        R ea[3] = {R(0), R(0), R(0)};
        ea[a] = R(1);
        cross(ch[i], ea, fn);
        ff[0] = R(0); ff[1] = R(0); ff[2] = R(0);
        ff[a] = cm[i];
      }
      L[i * N + i] = jt <= 2 ? fn[jt] : ff[jt - 3];
#pragma unroll
      for (int d = 0; d < kDepthMax; ++d) {
        if (d >= depth(i)) continue;
        // force across joint j into its parent's frame: f_p = E^T f, n_p = E^T n + r x f_p
        const int j = anc(i, d), jp = anc(i, d + 1);
        R en[3], ef[3], rf[3];
        jmtv(jtype(j), E[j], fn, en);
        jmtv(jtype(j), E[j], ff, ef);
        cross(r[j], ef, rf);
#pragma unroll
        for (int k = 0; k < 3; ++k) { fn[k] = en[k] + rf[k]; ff[k] = ef[k]; }
        const int jj = jtype(jp);
        L[i * N + jp] = jj <= 2 ? fn[jj] : ff[jj - 3];
      }
    }
    // M = L^T L with L lower triangular and the tree's sparsity (Featherstone
    // 2008, Sec. 6.5): eliminating from the last body up touches only
    // (body, ancestor) pairs, so nothing fills in; 1 / L_kk on the diagonal
#pragma unroll
    for (int k = N - 1; k >= 0; --k) {
      const R rk = rsqrt_(L[k * N + k]);
      L[k * N + k] = rk;
#pragma unroll
      for (int d = 1; d <= kDepthMax; ++d)
        if (d <= depth(k)) L[k * N + anc(k, d)] *= rk;
#pragma unroll
      for (int d = 1; d <= kDepthMax; ++d) {
        if (d > depth(k)) continue;
        const int i = anc(k, d);
        const R lki = L[k * N + i];
#pragma unroll
        for (int e = 0; e <= kDepthMax; ++e)
          if (e <= depth(i)) L[i * N + anc(i, e)] -= lki * L[k * N + anc(i, e)];
      }
    }
  }
  // mass_chol of q held in (shared) memory into (shared) memory: q read once,
  // the factor formed in registers, then only its tree-sparse entries (the
  // diagonal and the (body, ancestor) pairs, all that chol_solve reads) stored
  template <class R>
  TO_DEV static void mass_chol_mem(const ParamsT<R>& P, const R* qm, R* Lm) {
    R q[N], L[N * N];
#pragma unroll
    for (int i = 0; i < N; ++i) q[i] = qm[i];
    mass_chol(P, q, L);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      Lm[k * N + k] = L[k * N + k];
#pragma unroll
      for (int d = 1; d <= kDepthMax; ++d)
        if (d <= depth(k)) Lm[k * N + anc(k, d)] = L[k * N + anc(k, d)];
    }
  }

  // x = M^{-1} b with M = L^T L from mass_chol: L^T y = b from the leaves up,
  // then L x = y from the root down, each along the ancestor chains
  template <class R>
  TO_DEV static void chol_solve(const ParamsT<R>& P, const R* L, const R* b, R* x) {
    R y[N];
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] = b[i];
#pragma unroll
    for (int k = N - 1; k >= 0; --k) {
      y[k] *= L[k * N + k];
#pragma unroll
      for (int d = 1; d <= kDepthMax; ++d)
        if (d <= depth(k)) y[anc(k, d)] -= L[k * N + anc(k, d)] * y[k];
    }
#pragma unroll
    for (int k = 0; k < N; ++k) {
      R t = y[k];
#pragma unroll
      for (int d = 1; d <= kDepthMax; ++d)
        if (d <= depth(k)) t -= L[k * N + anc(k, d)] * x[anc(k, d)];
      x[k] = t * L[k * N + k];
    }
  }

  // one substep's acceleration: qdd = M^{-1} (tau - h); also returns L
  template <class R>
  TO_DEV static void accel(const ParamsT<R>& P, const R* q, const R* qd, const R* tau, R* qdd, R* L) {
    R z[N], h[N], rhs[N];
#pragma unroll
    for (int i = 0; i < N; ++i) z[i] = R(0);
    rnea<R, R>(P, q, qd, z, true, KIND == RK_QUAD, h);
    mass_chol(P, q, L);
#pragma unroll
    for (int i = 0; i < N; ++i) rhs[i] = tau[i] - h[i];
    chol_solve(P, L, rhs, qdd);
  }


  // ---- costs ----
  template <class R, class S>
  TO_DEV static void ee_world(const ParamsT<R>& P, const S* q, S* ee) {
    S E0[N][9], p0[N][3];
    world_pose(P, q, E0, p0);
    const int b = kEeBody < 0 ? 0 : kEeBody;   // the arm's end-effector body (unused for the quadruped)
    S pt[3] = {S(P.ee_pt[0]), S(P.ee_pt[1]), S(P.ee_pt[2])}, w[3];
    mtv(E0[b], pt, w);
#pragma unroll
    for (int k = 0; k < 3; ++k) ee[k] = p0[b][k] + w[k];
  }

  template <class R>
  TO_DEV static R running_cost(const ParamsT<R>& P, const R* x, const R* u) {
    R l = 0;
    for (int j = 0; j < m; ++j) l += P.wtau * u[j] * u[j];
    if (KIND == RK_ARM7) {
#pragma unroll
      for (int j = 0; j < N; ++j) l += P.wv * x[N + j] * x[N + j];
    } else {
      const R dz = x[2] - P.znom, dv = x[N] - P.vxt;
      l += P.wz * dz * dz + P.wrpy * (x[3] * x[3] + x[4] * x[4] + x[5] * x[5]) + P.wvx * dv * dv;
    }
    return l;
  }
  // the same step on a state carried as (hi, lo) pairs, in place
  template <class R>
  TO_DEV static R cost_step2(const ParamsT<R>& P, R* xh, R* xl, const R* u) {
    const R l = running_cost(P, xh, u);
    R tau[N], qdd[N], L[N * N];
#pragma unroll
    for (int i = 0; i < N; ++i) tau[i] = i < A0 ? R(0) : u[i - A0];
    const R h = P.dt / (R)P.n_sub;
    for (int s = 0; s < P.n_sub; ++s) {
      accel(P, xh, xh + N, tau, qdd, L);
      semi_implicit2<R, N>(xh, xl, xh + N, xl + N, qdd, h);
    }
    return l;
  }
  // cost_step2 shared by a candidate lane and its partner (kGroupStep): every
  // lane of the group calls it, mine on the candidate lanes (all < kStepSlots);
  // returns the running cost on those.  Two group barriers per substep.
  template <class R, int G>
  TO_DEV static R cost_step_group(const ParamsT<R>& P, const Group<G>& g, bool mine, R* xh, R* xl, const R* u,
                                  R* scratch) {
    static_assert(kGroupStep<G>, "a partner lane in the group's other half");
    constexpr int H = G / 2;                  // candidate c's partner is lane c + H
    static_assert(H >= kStepSlots, "a partner for every candidate slot");
    const int c = g.lane;
    const int slot = c < H ? c : c - H;
    R* sq = scratch + slot * kStepSlot;       // q of the candidate's substep
    R* sL = sq + N;                           // the factor of M(q)
    R* flag = scratch + kStepSlots * kStepSlot;
    R l = R(0), tau[N];
    if (mine) {
      l = running_cost(P, xh, u);
#pragma unroll
      for (int i = 0; i < N; ++i) tau[i] = i < A0 ? R(0) : u[i - A0];
    }
    if (c < kStepSlots) flag[c] = mine ? R(1) : R(0);
    const R h = P.dt / (R)P.n_sub;
    for (int s = 0; s < P.n_sub; ++s) {
      if (mine)
#pragma unroll
        for (int i = 0; i < N; ++i) sq[i] = xh[i];
      g.sync();
      R hb[N];
      if (mine) {
        R z[N];
#pragma unroll
        for (int i = 0; i < N; ++i) z[i] = R(0);
        rnea<R, R>(P, xh, xh + N, z, true, KIND == RK_QUAD, hb);
      } else if (c >= H && slot < kStepSlots && flag[slot] != R(0)) {
        mass_chol_mem(P, sq, sL);
      }
      g.sync();
      if (mine) {
        R rhs[N], qdd[N];
#pragma unroll
        for (int i = 0; i < N; ++i) rhs[i] = tau[i] - hb[i];
        chol_solve(P, sL, rhs, qdd);
        semi_implicit2<R, N>(xh, xl, xh + N, xl + N, qdd, h);
      }
    }
    return l;
  }

  template <class R>
  TO_DEV static R terminal_cost(const ParamsT<R>& P, const R* x) {
    R l = 0;
    if (KIND == RK_ARM7) {
      R ee[3];
      ee_world(P, x, ee);
      for (int k = 0; k < 3; ++k) { const R d = ee[k] - P.tgt[k]; l += P.wee * d * d; }
#pragma unroll
      for (int j = 0; j < N; ++j) l += P.wvT * x[N + j] * x[N + j];
    } else {
      const R dz = x[2] - P.znom, dv = x[N] - P.vxt;
      l = P.tscale * (P.wz * dz * dz + P.wrpy * (x[3] * x[3] + x[4] * x[4] + x[5] * x[5]) + P.wvx * dv * dv);
    }
    return l;
  }

  // separable running costs: the clipped Hessians are diagonal, max(d, eps)
  template <class R>
  TO_DEV static void running_derivs(const ParamsT<R>& P, const R* x, const R* u, R eps, R* lxx, R* lx, R* luu,
                                    R* lu) {
    for (int i = 0; i < n * n; ++i) lxx[i] = 0;
    for (int i = 0; i < m * m; ++i) luu[i] = 0;
    for (int i = 0; i < n; ++i) lx[i] = 0;
    const R w2 = R(2) * P.wtau;
    for (int j = 0; j < m; ++j) { lu[j] = w2 * u[j]; luu[j * m + j] = w2 > eps ? w2 : eps; }
    R dq[N];   // diagonal of the q-block and qd-block
    for (int i = 0; i < n; ++i) lxx[i * n + i] = clip0(eps);
    if (KIND == RK_ARM7) {
      const R v2 = R(2) * P.wv;
#pragma unroll
      for (int j = 0; j < N; ++j) { lx[N + j] = v2 * x[N + j]; lxx[(N + j) * n + N + j] = v2 > eps ? v2 : eps; }
    } else {
      const R z2 = R(2) * P.wz, r2 = R(2) * P.wrpy, x2 = R(2) * P.wvx;
      lx[2] = z2 * (x[2] - P.znom); lxx[2 * n + 2] = z2 > eps ? z2 : eps;
      for (int k = 3; k < 6; ++k) { lx[k] = r2 * x[k]; lxx[k * n + k] = r2 > eps ? r2 : eps; }
      lx[N] = x2 * (x[N] - P.vxt); lxx[N * n + N] = x2 > eps ? x2 : eps;
    }
    (void)dq;
  }

  // terminal-cost derivatives; the arm's end-effector term through forward
  // kinematics: gradient and exact Hessian by nested dual numbers (one lane),
  // then the q-block is eigen-clipped
  template <class R>
  TO_DEV static void terminal_derivs(const ParamsT<R>& P, const R* x, R eps, R* lxx, R* lx) {
    for (int i = 0; i < n * n; ++i) lxx[i] = 0;
    for (int i = 0; i < n; ++i) lx[i] = 0;
    if (KIND == RK_ARM7) {
      typedef Dl<Dl<R>> H;
      R Q[N * N];
      for (int a = 0; a < N; ++a)
        for (int b = a; b < N; ++b) {
          H q[N];
#pragma unroll
          for (int k = 0; k < N; ++k) q[k] = H(Dl<R>(x[k], k == a ? R(1) : R(0)), Dl<R>(k == b ? R(1) : R(0), R(0)));
          H ee[3];
          ee_world(P, q, ee);
          H l(Dl<R>(R(0)));
          const H wee(Dl<R>(P.wee));
          for (int k = 0; k < 3; ++k) {
            const H d = ee[k] - H(Dl<R>(P.tgt[k]));
            l = l + wee * (d * d);
          }
          Q[a * N + b] = l.d.d;
          Q[b * N + a] = l.d.d;
          if (a == b) lx[a] = l.v.d;
        }
      eigclip_jacobi<R, N>(Q, eps);
      for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) lxx[a * n + b] = Q[a * N + b];
      const R v2 = R(2) * P.wvT;
#pragma unroll
      for (int j = 0; j < N; ++j) { lx[N + j] = v2 * x[N + j]; lxx[(N + j) * n + N + j] = v2 > eps ? v2 : eps; }
    } else {
      const R s = P.tscale;
      const R z2 = R(2) * P.wz * s, r2 = R(2) * P.wrpy * s, x2 = R(2) * P.wvx * s;
      for (int i = 0; i < n; ++i) lxx[i * n + i] = clip0(eps);
      lx[2] = z2 * (x[2] - P.znom); lxx[2 * n + 2] = z2 > eps ? z2 : eps;
      for (int k = 3; k < 6; ++k) { lx[k] = r2 * x[k]; lxx[k * n + k] = r2 > eps ? r2 : eps; }
      lx[N] = x2 * (x[N] - P.vxt); lxx[N * n + N] = x2 > eps ? x2 : eps;
    }
  }

  // ---- group-shared primal of one substep and the per-lane tangent pass ----
  static constexpr int NF = (KIND == RK_QUAD) ? 4 : 1;
  // Per-body quantities of the Newton-Euler pass at (q, qd, qdd), the mass
  // matrix factor and the contact terms: computed once per substep by one
  // lane into shared memory, read by every tangent lane.
  template <class R>
  struct Prim {
    R q[N], qd[N], qdd[N], tau[N], tin[N];
    R L[N * N];
    R E[N][9], r[N][3];
    R vw[N][3], vv[N][3];       // body velocity
    R Epw[N][3], Ept[N][3];     // E pw and E (pv - r x pw): the parent's velocity in body coordinates
    R Epa[N][3], Epb[N][3];     // E paw and E (pav - r x paw): the same for the acceleration
    R aw[N][3];                 // body angular acceleration
    R hn[N][3], hf[N][3];       // I v
    R fn[N][3], ff[N][3];       // body force as sent to the parent (children and contact included)
    R E0[KIND == RK_QUAD ? N : 1][9], p0[KIND == RK_QUAD ? N : 1][3];
    R wpt[NF][3], F[NF][3], vb[NF][3], vwld[NF][3], gate[NF];
  };
  // Knot-parallel derivatives (both trees): before each backward pass every
  // lane runs the substep primal chains of its own knots (primal_knot) and
  // stores each substep's Prim in a per-knot global scratch; inside the
  // backward pass the group stages those Prims into shared memory
  // (cp.async, one substep ahead) and every direction lane runs its tangent
  // pass at once (derivs_staged).  No lane waits for a primal.
  static constexpr bool kKnotParallel = true;
  static constexpr bool kStoredDerivs = false;
  // elements per stored substep primal (a whole number of 16-byte chunks)
  template <class R> static constexpr int kPrimStride = (int)(((sizeof(Prim<R>) + 15) / 16 * 16) / sizeof(R));

  // Line search of the quadruped's groups: candidate lane c < kStepSlots
  // steps its rollout with lane c + G/2 as its partner (the other warp of a
  // 64-lane group, the other half-warp of a 32-lane one), which forms and
  // factors the mass matrix while lane c runs the bias Newton-Euler pass.
  // Per candidate the scratch holds its substep's q and the factor.  The
  // 7-DoF arm's candidates step alone: its 7-body mass matrix is cheap, and
  // the partner split measured 2 % slower there in mixed mode.
  template <int G> static constexpr bool kGroupStep = (KIND == RK_QUAD) && G >= 32;
  static constexpr int kStepSlots = 16, kStepSlot = N + N * N;
  // the group's shared-memory scratch (the solver reserves it in its work
  // area): the derivative primal, or the line search's per-candidate slots
  template <class R>
  struct Scratch {
    static constexpr int prim = 2 * kPrimStride<R>;   // the staged substep primals, double-buffered
    static constexpr int step = KIND == RK_QUAD ? kStepSlots * kStepSlot + kStepSlots : 0;
    static constexpr int elems = prim > step ? prim : step;
  };

  // y += a x b
  template <class S> TO_DEV static void cross_acc(const S* a, const S* b, S* y) {
    y[0] += a[1] * b[2] - a[2] * b[1];
    y[1] += a[2] * b[0] - a[0] * b[2];
    y[2] += a[0] * b[1] - a[1] * b[0];
  }
  // y -= s (e_ax x z): the change of E x under dq about joint axis ax
  template <class S> TO_DEV static void rot_tangent(int ax, S s, const S* z, S* y) {
    if (ax == 0) { y[1] += s * z[2]; y[2] -= s * z[1]; }
    else if (ax == 1) { y[0] -= s * z[2]; y[2] += s * z[0]; }
    else { y[0] += s * z[1]; y[1] -= s * z[0]; }
  }
  // e_ax x z
  template <class S> TO_DEV static void axis_cross(int ax, const S* z, S* y) {
    if (ax == 0) { y[0] = S(0); y[1] = -z[2]; y[2] = z[1]; }
    else if (ax == 1) { y[0] = z[2]; y[1] = S(0); y[2] = -z[0]; }
    else { y[0] = -z[1]; y[1] = z[0]; y[2] = S(0); }
  }

  // A substep's primal for the derivative lanes comes in two halves around
  // the solve for qdd, so that the joint transforms, the velocities, the
  // world poses and the contact forces are evaluated once (the tangent pass
  // reads them all from pr):
  // bias_store (one lane): those quantities, I v, and the inverse dynamics at
  // qdd = 0 (gravity, velocity products, contact), i.e. the bias torques h.
  template <class R>
  TO_DEV static void bias_store(const ParamsT<R>& P, Prim<R>& pr, const R* q, const R* qd, R* h) {
    R aw[N][3], av[N][3], fn[N][3], ff[N][3];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int pa = parent(i), jt = jtype(i);
      R E[9], r[3];
      joint_transform(P, i, q[i], E, r);
#pragma unroll
      for (int k = 0; k < 9; ++k) pr.E[i][k] = E[k];
#pragma unroll
      for (int k = 0; k < 3; ++k) pr.r[i][k] = r[k];
      R pw[3], pv[3], paw[3], pav[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        pw[k] = pa < 0 ? R(0) : pr.vw[pa][k];
        pv[k] = pa < 0 ? R(0) : pr.vv[pa][k];
        paw[k] = pa < 0 ? R(0) : aw[pa][k];
        pav[k] = pa < 0 ? -P.g[k] : av[pa][k];
      }
      R t[3], rw[3], Epw[3], Ept[3];
      cross(r, pw, rw);
#pragma unroll
      for (int k = 0; k < 3; ++k) t[k] = pv[k] - rw[k];
      jmv(jt, E, pw, Epw);
      jmv(jt, E, t, Ept);
      R sw[3] = {R(0), R(0), R(0)}, sv[3] = {R(0), R(0), R(0)};
      if (jt <= 2) sw[jt] = qd[i]; else sv[jt - 3] = qd[i];
      R vw[3], vv[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        vw[k] = Epw[k] + sw[k];
        vv[k] = Ept[k] + sv[k];
        pr.Epw[i][k] = Epw[k]; pr.Ept[i][k] = Ept[k];
        pr.vw[i][k] = vw[k]; pr.vv[i][k] = vv[k];
      }
      // the acceleration at qdd = 0 and the body force it needs
      cross(r, paw, rw);
#pragma unroll
      for (int k = 0; k < 3; ++k) t[k] = pav[k] - rw[k];
      jmv(jt, E, paw, aw[i]);
      jmv(jt, E, t, av[i]);
      cross_acc(vw, sw, aw[i]);
      cross_acc(vw, sv, av[i]);
      cross_acc(vv, sw, av[i]);
      R In[3], If[3], hn[3], hf[3];
      inertia_mul(P, i, aw[i], av[i], In, If);
      inertia_mul(P, i, vw, vv, hn, hf);
#pragma unroll
      for (int k = 0; k < 3; ++k) { pr.hn[i][k] = hn[k]; pr.hf[i][k] = hf[k]; fn[i][k] = In[k]; ff[i][k] = If[k]; }
      cross_acc(vw, hn, fn[i]);
      cross_acc(vv, hf, fn[i]);
      cross_acc(vw, hf, ff[i]);
      if (KIND == RK_QUAD) {
        if (pa < 0) {
#pragma unroll
          for (int k = 0; k < 9; ++k) pr.E0[i][k] = E[k];
#pragma unroll
          for (int k = 0; k < 3; ++k) pr.p0[i][k] = r[k];
        } else {
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
              pr.E0[i][a * 3 + b] = E[a * 3 + 0] * pr.E0[pa][b] + E[a * 3 + 1] * pr.E0[pa][3 + b] + E[a * 3 + 2] * pr.E0[pa][6 + b];
          R wr[3];
          mtv(pr.E0[pa], r, wr);
#pragma unroll
          for (int k = 0; k < 3; ++k) pr.p0[i][k] = pr.p0[pa][k] + wr[k];
        }
      }
    }
    if (KIND == RK_QUAD) {
#pragma unroll
      for (int ft = 0; ft < kFeet; ++ft) {
        const int bi = foot_body(ft);
        const R pt[3] = {P.foot_pt[ft][0], P.foot_pt[ft][1], P.foot_pt[ft][2]};
        R wpt[3], vb[3], vwld[3], wxp[3];
        mtv(pr.E0[bi], pt, wpt);
        cross(pr.vw[bi], pt, wxp);
#pragma unroll
        for (int k = 0; k < 3; ++k) vb[k] = pr.vv[bi][k] + wxp[k];
        mtv(pr.E0[bi], vb, vwld);
        const R bz = P.beta * (pr.p0[bi][2] + wpt[2]);
        R sp, gate;
        if (bz >= R(0)) {
          const R e = dexp(-bz);
          sp = (R(1) / P.beta) * dlog1p(e);
          gate = e / (R(1) + e);
        } else {
          const R e = dexp(bz);
          sp = (R(1) / P.beta) * (dlog1p(e) - bz);
          gate = R(1) / (R(1) + e);
        }
        R F[3];
        F[0] = -(P.dc * (gate * vwld[0]));
        F[1] = -(P.dc * (gate * vwld[1]));
        F[2] = P.kc * sp - P.dc * (gate * vwld[2]);
        pr.gate[ft] = gate;
#pragma unroll
        for (int k = 0; k < 3; ++k) { pr.wpt[ft][k] = wpt[k]; pr.vb[ft][k] = vb[k]; pr.vwld[ft][k] = vwld[k]; pr.F[ft][k] = F[k]; }
        R mw[3], mb[3], fb[3];
        cross(wpt, F, mw);
        mv(pr.E0[bi], mw, mb);
        mv(pr.E0[bi], F, fb);
#pragma unroll
        for (int k = 0; k < 3; ++k) { fn[bi][k] -= mb[k]; ff[bi][k] -= fb[k]; }
      }
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
      const int jt = jtype(i);
      h[i] = jt <= 2 ? fn[i][jt] : ff[i][jt - 3];
      const int pa = parent(i);
      if (pa >= 0) {
        R en[3], ef[3], rf[3];
        jmtv(jt, pr.E[i], fn[i], en);
        jmtv(jt, pr.E[i], ff[i], ef);
        cross(pr.r[i], ef, rf);
#pragma unroll
        for (int k = 0; k < 3; ++k) { fn[pa][k] += en[k] + rf[k]; ff[pa][k] += ef[k]; }
      }
    }
  }

  // accel_store (one lane, after the solve put qdd in pr): the accelerations
  // with qdd, the parents' acceleration transforms, and the body forces as
  // sent to the parent (children and contact included), from the stored
  // transforms, velocities, I v and contact forces.
  template <class R>
  TO_DEV static void accel_store(const ParamsT<R>& P, Prim<R>& pr) {
    R av[N][3], fn[N][3], ff[N][3];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int pa = parent(i), jt = jtype(i);
      R paw[3], pav[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        paw[k] = pa < 0 ? R(0) : pr.aw[pa][k];
        pav[k] = pa < 0 ? -P.g[k] : av[pa][k];
      }
      const R* E = pr.E[i];
      R t[3], rw[3], Epa[3], Epb[3], vw[3], vv[3], hn[3], hf[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) { vw[k] = pr.vw[i][k]; vv[k] = pr.vv[i][k]; hn[k] = pr.hn[i][k]; hf[k] = pr.hf[i][k]; }
      cross(pr.r[i], paw, rw);
#pragma unroll
      for (int k = 0; k < 3; ++k) t[k] = pav[k] - rw[k];
      jmv(jt, E, paw, Epa);
      jmv(jt, E, t, Epb);
      R sw[3] = {R(0), R(0), R(0)}, sv[3] = {R(0), R(0), R(0)};
      if (jt <= 2) sw[jt] = pr.qd[i]; else sv[jt - 3] = pr.qd[i];
      R aw[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) { pr.Epa[i][k] = Epa[k]; pr.Epb[i][k] = Epb[k]; aw[k] = Epa[k]; av[i][k] = Epb[k]; }
      cross_acc(vw, sw, aw);
      cross_acc(vw, sv, av[i]);
      cross_acc(vv, sw, av[i]);
      if (jt <= 2) aw[jt] += pr.qdd[i]; else av[i][jt - 3] += pr.qdd[i];
#pragma unroll
      for (int k = 0; k < 3; ++k) pr.aw[i][k] = aw[k];
      R In[3], If[3];
      inertia_mul(P, i, aw, av[i], In, If);
#pragma unroll
      for (int k = 0; k < 3; ++k) { fn[i][k] = In[k]; ff[i][k] = If[k]; }
      cross_acc(vw, hn, fn[i]);
      cross_acc(vv, hf, fn[i]);
      cross_acc(vw, hf, ff[i]);
    }
    if (KIND == RK_QUAD) {
#pragma unroll
      for (int ft = 0; ft < kFeet; ++ft) {
        const int bi = foot_body(ft);
        R mw[3], mb[3], fb[3];
        cross(pr.wpt[ft], pr.F[ft], mw);
        mv(pr.E0[bi], mw, mb);
        mv(pr.E0[bi], pr.F[ft], fb);
#pragma unroll
        for (int k = 0; k < 3; ++k) { fn[bi][k] -= mb[k]; ff[bi][k] -= fb[k]; }
      }
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
      const int jt = jtype(i);
      pr.tau[i] = jt <= 2 ? fn[i][jt] : ff[i][jt - 3];
#pragma unroll
      for (int k = 0; k < 3; ++k) { pr.fn[i][k] = fn[i][k]; pr.ff[i][k] = ff[i][k]; }
      const int pa = parent(i);
      if (pa >= 0) {
        R en[3], ef[3], rf[3];
        jmtv(jt, pr.E[i], fn[i], en);
        jmtv(jt, pr.E[i], ff[i], ef);
        cross(pr.r[i], ef, rf);
#pragma unroll
        for (int k = 0; k < 3; ++k) { fn[pa][k] += en[k] + rf[k]; ff[pa][k] += ef[k]; }
      }
    }
  }

  // Directional derivative of the inverse dynamics along (dq, dqd) at the
  // stored substep (qdd held fixed): the product rule through the forward
  // recursion (velocities, accelerations, body forces, world poses and
  // contact) and the backward force recursion.  Only the tangents live in
  // the lane's own arrays.
  template <class R>
  TO_DEV static void rnea_tangent(const ParamsT<R>& P, const Prim<R>& pr, const R* dq, const R* dqd, R* dtau) {
    R dvw[N][3], dvv[N][3], daw[N][3], dav[N][3], dfn[N][3], dff[N][3];
    R dE0[KIND == RK_QUAD ? N : 1][9], dp0[KIND == RK_QUAD ? N : 1][3];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int pa = parent(i);
      const int jt = jtype(i);
      const bool rev = jt <= 2;
      const int ax = rev ? jt : jt - 3;
      const R sq = rev ? dq[i] : R(0);          // rotation tangent
      R dr[3] = {R(0), R(0), R(0)};
      if (!rev) dr[ax] = dq[i];
      const R* E = pr.E[i];
      const R* r = pr.r[i];
      R dpw[3], dpv[3], dpaw[3], dpav[3], pw[3], paw[3];
      for (int k = 0; k < 3; ++k) {
        dpw[k] = pa < 0 ? R(0) : dvw[pa][k];
        dpv[k] = pa < 0 ? R(0) : dvv[pa][k];
        dpaw[k] = pa < 0 ? R(0) : daw[pa][k];
        dpav[k] = pa < 0 ? R(0) : dav[pa][k];
        pw[k] = pa < 0 ? R(0) : pr.vw[pa][k];
        paw[k] = pa < 0 ? R(0) : pr.aw[pa][k];
      }
      // velocity
      R t[3], u3[3];
      jmv(jt, E, dpw, dvw[i]);
      rot_tangent(ax, rev ? sq : R(0), pr.Epw[i], dvw[i]);
      for (int k = 0; k < 3; ++k) t[k] = dpv[k];
      cross(r, dpw, u3);
      for (int k = 0; k < 3; ++k) t[k] -= u3[k];
      cross(dr, pw, u3);
      for (int k = 0; k < 3; ++k) t[k] -= u3[k];
      jmv(jt, E, t, dvv[i]);
      rot_tangent(ax, rev ? sq : R(0), pr.Ept[i], dvv[i]);
      R sw[3] = {R(0), R(0), R(0)}, sv[3] = {R(0), R(0), R(0)}, dsw[3] = {R(0), R(0), R(0)}, dsv[3] = {R(0), R(0), R(0)};
      if (rev) { sw[ax] = pr.qd[i]; dsw[ax] = dqd[i]; } else { sv[ax] = pr.qd[i]; dsv[ax] = dqd[i]; }
      for (int k = 0; k < 3; ++k) { dvw[i][k] += dsw[k]; dvv[i][k] += dsv[k]; }
      // acceleration (qdd fixed)
      jmv(jt, E, dpaw, daw[i]);
      rot_tangent(ax, rev ? sq : R(0), pr.Epa[i], daw[i]);
      for (int k = 0; k < 3; ++k) t[k] = dpav[k];
      cross(r, dpaw, u3);
      for (int k = 0; k < 3; ++k) t[k] -= u3[k];
      cross(dr, paw, u3);
      for (int k = 0; k < 3; ++k) t[k] -= u3[k];
      jmv(jt, E, t, dav[i]);
      rot_tangent(ax, rev ? sq : R(0), pr.Epb[i], dav[i]);
      cross_acc(dvw[i], sw, daw[i]);
      cross_acc(pr.vw[i], dsw, daw[i]);
      cross_acc(dvw[i], sv, dav[i]);
      cross_acc(pr.vw[i], dsv, dav[i]);
      cross_acc(dvv[i], sw, dav[i]);
      cross_acc(pr.vv[i], dsw, dav[i]);
      // body force
      R dIn[3], dIf[3], dhn[3], dhf[3];
      inertia_mul(P, i, daw[i], dav[i], dIn, dIf);
      inertia_mul(P, i, dvw[i], dvv[i], dhn, dhf);
      for (int k = 0; k < 3; ++k) { dfn[i][k] = dIn[k]; dff[i][k] = dIf[k]; }
      cross_acc(dvw[i], pr.hn[i], dfn[i]);
      cross_acc(pr.vw[i], dhn, dfn[i]);
      cross_acc(dvv[i], pr.hf[i], dfn[i]);
      cross_acc(pr.vv[i], dhf, dfn[i]);
      cross_acc(dvw[i], pr.hf[i], dff[i]);
      cross_acc(pr.vw[i], dhf, dff[i]);
      if (KIND == RK_QUAD) {
        // world pose: dE0_i = dE_i E0_p + E_i dE0_p, dp0_i = dp0_p + dE0_p^T r + E0_p^T dr
        const R* E0 = pr.E0[i];
        if (pa < 0) {
          for (int k = 0; k < 9; ++k) dE0[i][k] = R(0);
          for (int k = 0; k < 3; ++k) dp0[i][k] = dr[k];
        } else {
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
              dE0[i][a * 3 + b] = E[a * 3 + 0] * dE0[pa][b] + E[a * 3 + 1] * dE0[pa][3 + b] + E[a * 3 + 2] * dE0[pa][6 + b];
          R w1[3], w2[3];
          mtv(dE0[pa], r, w1);
          mtv(pr.E0[pa], dr, w2);
          for (int k = 0; k < 3; ++k) dp0[i][k] = dp0[pa][k] + w1[k] + w2[k];
        }
        if (rev) {
          // column b of E0_i turns with the joint: -dq (e_ax x column)
          for (int b = 0; b < 3; ++b) {
            const R col[3] = {E0[0 * 3 + b], E0[1 * 3 + b], E0[2 * 3 + b]};
            R y[3] = {R(0), R(0), R(0)};
            rot_tangent(ax, sq, col, y);
            for (int a = 0; a < 3; ++a) dE0[i][a * 3 + b] += y[a];
          }
        }
      }
    }
    if (KIND == RK_QUAD) {
#pragma unroll
      for (int ft = 0; ft < kFeet; ++ft) {
        const int bi = foot_body(ft);
        const R pt[3] = {P.foot_pt[ft][0], P.foot_pt[ft][1], P.foot_pt[ft][2]};
        const R* E0 = pr.E0[bi];
        R dwpt[3], dvb[3], dvwld[3], w1[3];
        mtv(dE0[bi], pt, dwpt);
        const R dz = dp0[bi][2] + dwpt[2];
        cross(dvw[bi], pt, w1);
        for (int k = 0; k < 3; ++k) dvb[k] = dvv[bi][k] + w1[k];
        mtv(dE0[bi], pr.vb[ft], dvwld);
        mtv(E0, dvb, w1);
        for (int k = 0; k < 3; ++k) dvwld[k] += w1[k];
        const R gate = pr.gate[ft];
        const R dgate = -P.beta * gate * (R(1) - gate) * dz;
        const R dsp = -gate * dz;
        R dF[3];
        dF[0] = -P.dc * (dgate * pr.vwld[ft][0] + gate * dvwld[0]);
        dF[1] = -P.dc * (dgate * pr.vwld[ft][1] + gate * dvwld[1]);
        dF[2] = P.kc * dsp - P.dc * (dgate * pr.vwld[ft][2] + gate * dvwld[2]);
        R mw[3], dmw[3] = {R(0), R(0), R(0)}, dmb[3], dfb[3];
        cross(pr.wpt[ft], pr.F[ft], mw);
        cross_acc(dwpt, pr.F[ft], dmw);
        cross_acc(pr.wpt[ft], dF, dmw);
        mv(dE0[bi], mw, dmb);
        mv(E0, dmw, w1);
        for (int k = 0; k < 3; ++k) dmb[k] += w1[k];
        mv(dE0[bi], pr.F[ft], dfb);
        mv(E0, dF, w1);
        for (int k = 0; k < 3; ++k) dfb[k] += w1[k];
        for (int k = 0; k < 3; ++k) { dfn[bi][k] -= dmb[k]; dff[bi][k] -= dfb[k]; }
      }
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
      const int jt = jtype(i);
      const bool rev = jt <= 2;
      const int ax = rev ? jt : jt - 3;
      dtau[i] = rev ? dfn[i][ax] : dff[i][ax];
      const int pa = parent(i);
      if (pa >= 0) {
        // d(E^T y) = E^T dy + dq E^T (e_ax x y) for a revolute joint
        const R* E = pr.E[i];
        R yn[3], yf[3], den[3], def[3], w1[3];
        for (int k = 0; k < 3; ++k) { yn[k] = dfn[i][k]; yf[k] = dff[i][k]; }
        if (rev) {
          axis_cross(ax, pr.fn[i], w1);
          for (int k = 0; k < 3; ++k) yn[k] += dq[i] * w1[k];
          axis_cross(ax, pr.ff[i], w1);
          for (int k = 0; k < 3; ++k) yf[k] += dq[i] * w1[k];
        }
        jmtv(jt, E, yn, den);
        jmtv(jt, E, yf, def);
        R ef[3], dr[3] = {R(0), R(0), R(0)};
        if (!rev) dr[ax] = dq[i];
        jmtv(jt, E, pr.ff[i], ef);
        cross_acc(dr, ef, den);
        cross_acc(pr.r[i], def, den);
        for (int k = 0; k < 3; ++k) { dfn[pa][k] += den[k]; dff[pa][k] += def[k]; }
      }
    }
  }

  // The substep primal chain of one knot on one lane, every substep's Prim
  // stored at out + s kPrimStride (global memory): the same arithmetic as
  // derivs' primal lane, with the mass matrix factored on this lane.
  template <class R>
  TO_DEV static void primal_knot(const ParamsT<R>& P, const R* x, const R* u, R* out) {
    R q[N], qd[N], tin[N];
#pragma unroll
    for (int i = 0; i < N; ++i) { q[i] = x[i]; qd[i] = x[N + i]; tin[i] = i < A0 ? R(0) : u[i - A0]; }
    const R h = P.dt / (R)P.n_sub;
    for (int s = 0; s < P.n_sub; ++s) {
      Prim<R>& pr = *reinterpret_cast<Prim<R>*>(out + (size_t)s * kPrimStride<R>);
      R hb[N], L[N * N], rhs[N], qdd[N];
      bias_store(P, pr, q, qd, hb);
      mass_chol(P, q, L);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        pr.L[k * N + k] = L[k * N + k];
#pragma unroll
        for (int d = 1; d <= kDepthMax; ++d)
          if (d <= depth(k)) pr.L[k * N + anc(k, d)] = L[k * N + anc(k, d)];
      }
#pragma unroll
      for (int i = 0; i < N; ++i) rhs[i] = tin[i] - hb[i];
      chol_solve(P, L, rhs, qdd);
#pragma unroll
      for (int i = 0; i < N; ++i) { pr.q[i] = q[i]; pr.qd[i] = qd[i]; pr.tin[i] = tin[i]; pr.qdd[i] = qdd[i]; }
      accel_store(P, pr);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        qd[i] = qd[i] + h * qdd[i];
        q[i] = q[i] + h * qd[i];
      }
    }
  }

  // group copy of one stored Prim into shared memory, 16 bytes per cp.async
  template <class R, int G>
  TO_DEV static void stage_prim(const Group<G>& g, const R* src, R* dst) {
    constexpr int chunks = kPrimStride<R> * (int)sizeof(R) / 16;
    const char* s = reinterpret_cast<const char*>(src);
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    for (int c = g.lane; c < chunks; c += G)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d + 16u * c), "l"(s + 16 * c) : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }

  // Columns of [A | B] from the knot's stored substep primals (prims, global):
  // each substep's Prim is staged into shared memory one substep ahead while
  // the direction lanes run the tangent pass of the current one.  A group
  // narrower than the n + m directions takes them in passes of G (the
  // substeps are staged again for each pass).
  template <class R, int G>
  TO_DEV static void derivs_staged(const ParamsT<R>& P, const Group<G>& g, const R* x, const R* u, R eps, R* A, R* B,
                                   R* lxx, R* lx, R* luu, R* lu, R* scratch, const R* prims) {
    for (int pass = 0; pass < (n + m + G - 1) / G; ++pass) {
    if (pass > 0) g.sync();   // every lane done with the staging buffers of the previous pass
    const int c = pass * G + g.lane;
    const bool dir = c < n + m;
    R dq[N], dqd[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      dq[i] = (c == i) ? R(1) : R(0);
      dqd[i] = (c == N + i) ? R(1) : R(0);
    }
    const R h = P.dt / (R)P.n_sub;
    stage_prim<R, G>(g, prims, scratch);
    for (int s = 0; s < P.n_sub; ++s) {
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      g.sync();   // substep s staged by every lane; every lane done with the other buffer
      if (s + 1 < P.n_sub)
        stage_prim<R, G>(g, prims + (size_t)(s + 1) * kPrimStride<R>, scratch + ((s + 1) & 1) * kPrimStride<R>);
      const Prim<R>& pr = *reinterpret_cast<const Prim<R>*>(scratch + (s & 1) * kPrimStride<R>);
      if (dir) {
        R dtau[N], rhs[N], dqdd[N];
        rnea_tangent(P, pr, dq, dqd, dtau);
#pragma unroll
        for (int i = 0; i < N; ++i) rhs[i] = ((c >= n && i == A0 + (c - n)) ? R(1) : R(0)) - dtau[i];
        chol_solve(P, pr.L, rhs, dqdd);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          dqd[i] = dqd[i] + h * dqdd[i];
          dq[i] = dq[i] + h * dqd[i];
        }
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (dir) {
      if (c < n) {
#pragma unroll
        for (int i = 0; i < N; ++i) { A[i * n + c] = dq[i]; A[(N + i) * n + c] = dqd[i]; }
      } else {
#pragma unroll
        for (int i = 0; i < N; ++i) { B[i * m + (c - n)] = dq[i]; B[(N + i) * m + (c - n)] = dqd[i]; }
      }
    }
    }
    if (g.lane == G - 1) running_derivs(P, x, u, eps, lxx, lx, luu, lu);
  }

};

typedef SysRigid<7, 0, RK_ARM7> SysArm7;
typedef SysRigid<18, 6, RK_QUAD> SysQuad;

}  // namespace to

namespace to {
template <class R> using RigidArm7P = RigidParams<R, 7>;
template <class R> using RigidQuadP = RigidParams<R, 18>;
}  // namespace to
