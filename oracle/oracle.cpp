// Plain FP64 CPU oracle of the batched iLQR trajectory-optimisation path.
//
// TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
// CPU-baseline leg are the only code allowed to load this library.  It shares
// no code, header or table with the CUDA library: it reads the same flat
// parameter vectors (the documented input format) and implements every step
// on its own, slowly and plainly.
//
// What it computes (paper section / equation in brackets):
//   * the finite-horizon discrete OCP  min sum_k l_k(x_k,u_k) + l_T(x_T)
//     s.t. x_{k+1} = f_k(x_k,u_k), x_0 = x_init           [Sec. II, Eq. 1]
//     (|u| <= u_max is not active in any workload: u_max = +inf)
//   * iLQR (DDP backward pass without second-order dynamics terms) whose
//     backward pass also yields the value gradient V_x     [Sec. II; Sec. IV-C]
//   * eigenvalue-clipping regularisation of the state- and control-cost
//     Hessians, S' = max(S, eps), Q+ = W diag(S') W^T, Q_psd = (Q+ + Q+^T)/2
//                                                          [Sec. IV-B]
//   * the LM term Q_uu + mu I, used only as a guard when the Cholesky
//     pivot test fails                                      [Sec. IV-B]
//   * a fixed iteration budget per instance                 [Sec. IV-A]
//   * the actor-policy warm start (MLP rolled out through the dynamics)
//                                                          [Sec. II, Sec. III-D]
// Derivatives are exact: forward-mode dual numbers (first derivatives of the
// dynamics) and nested duals (second derivatives of the costs).  Rigid-body
// dynamics are textbook spatial-vector recursive Newton-Euler with the mass
// matrix taken column by column from unit accelerations and a Cholesky solve
// (Featherstone, Rigid Body Dynamics Algorithms, 2008, ch. 2 and 5).
//
// Parity status: every function here is pinned by tests (closed forms,
// Lagrangian identities, finite differences, dense KKT / QP solves); see the
// test files that load this library.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace orc {
using std::sin; using std::cos; using std::exp; using std::log; using std::sqrt; using std::tanh;

// ----------------------------------------------------------------------------
// dual numbers: D<double> carries one directional derivative, D<D<double>>
// carries two directions and their mixed second derivative.
// ----------------------------------------------------------------------------
template <class B>
struct D {
  B v, d;
  D() : v(0.0), d(0.0) {}
  D(double c) : v(c), d(0.0) {}
  D(const B& a, const B& b) : v(a), d(b) {}
};

template <class B> D<B> operator+(const D<B>& a, const D<B>& b) { return D<B>(a.v + b.v, a.d + b.d); }
template <class B> D<B> operator-(const D<B>& a, const D<B>& b) { return D<B>(a.v - b.v, a.d - b.d); }
template <class B> D<B> operator*(const D<B>& a, const D<B>& b) { return D<B>(a.v * b.v, a.v * b.d + a.d * b.v); }
template <class B> D<B> operator/(const D<B>& a, const D<B>& b) {
  return D<B>(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
template <class B> D<B> operator-(const D<B>& a) { return D<B>(-a.v, -a.d); }
template <class B> D<B> operator+(const D<B>& a, double b) { return D<B>(a.v + b, a.d); }
template <class B> D<B> operator+(double a, const D<B>& b) { return D<B>(a + b.v, b.d); }
template <class B> D<B> operator-(const D<B>& a, double b) { return D<B>(a.v - b, a.d); }
template <class B> D<B> operator-(double a, const D<B>& b) { return D<B>(a - b.v, -b.d); }
template <class B> D<B> operator*(const D<B>& a, double b) { return D<B>(a.v * b, a.d * b); }
template <class B> D<B> operator*(double a, const D<B>& b) { return D<B>(a * b.v, a * b.d); }
template <class B> D<B> operator/(const D<B>& a, double b) { return D<B>(a.v / b, a.d / b); }
template <class B> D<B> operator/(double a, const D<B>& b) { return D<B>(a / b.v, -a * b.d / (b.v * b.v)); }
template <class B> D<B>& operator+=(D<B>& a, const D<B>& b) { a = a + b; return a; }
template <class B> D<B>& operator-=(D<B>& a, const D<B>& b) { a = a - b; return a; }
template <class B> D<B>& operator*=(D<B>& a, const D<B>& b) { a = a * b; return a; }

template <class B> D<B> sin(const D<B>& a) { using std::sin; using std::cos; return D<B>(sin(a.v), cos(a.v) * a.d); }
template <class B> D<B> cos(const D<B>& a) { using std::sin; using std::cos; return D<B>(cos(a.v), -sin(a.v) * a.d); }
template <class B> D<B> exp(const D<B>& a) { using std::exp; B e = exp(a.v); return D<B>(e, e * a.d); }
template <class B> D<B> log(const D<B>& a) { using std::log; return D<B>(log(a.v), a.d / a.v); }
template <class B> D<B> sqrt(const D<B>& a) { using std::sqrt; B s = sqrt(a.v); return D<B>(s, a.d / (2.0 * s)); }
template <class B> D<B> tanh(const D<B>& a) { using std::tanh; B t = tanh(a.v); return D<B>(t, (1.0 - t * t) * a.d); }

inline double val(double x) { return x; }
template <class B> double val(const D<B>& x) { return val(x.v); }

// ----------------------------------------------------------------------------
// problem description, parsed from the flat parameter vector
// ----------------------------------------------------------------------------
enum { SYS_PM = 1, SYS_PLANAR3 = 2, SYS_ARM7 = 3, SYS_QUAD = 4, SYS_DUBINS = 5 };
enum { J_RX = 0, J_RY, J_RZ, J_PX, J_PY, J_PZ };

struct Body {
  int parent, jtype;
  double off[3], mass, com[3], I[3];
};

struct Model {
  int sys = 0, n = 0, m = 0;
  double dt = 0;
  // point mass, Dubins car
  double wu = 0, wpT = 0, wvT = 0, waT = 0;
  // bumps (point mass, planar arm)
  double bamp = 0, bsig = 1;
  int nb = 0;
  double bc[8][2] = {};
  // rigid-body tree
  int N = 0, a0 = 0, n_sub = 1;
  double g[3] = {0, 0, 0};
  Body b[32];
  // arm costs
  double wtau = 0, wv = 0, wee = 0, tgt[3] = {0, 0, 0};
  int ee_body = 0;
  double ee_pt[3] = {0, 0, 0};
  // quadruped cost and contact
  double znom = 0, wz = 0, wrpy = 0, wvx = 0, vxt = 0, tscale = 1, kc = 0, dc = 0, beta = 1;
  int nfeet = 0, foot_body[4] = {0, 0, 0, 0};
  double foot_pt[4][3] = {};
};

static bool parse(int sys, const double* p, int np, Model& md) {
  md.sys = sys;
  if (sys == SYS_PM) {
    if (np < 5) return false;
    md.n = 4; md.m = 2;
    md.dt = p[0]; md.wu = p[1]; md.bamp = p[2]; md.bsig = p[3]; md.nb = (int)p[4];
    if (md.nb < 0 || md.nb > 8 || np < 7 + 2 * md.nb) return false;
    for (int i = 0; i < md.nb; ++i) { md.bc[i][0] = p[5 + 2 * i]; md.bc[i][1] = p[6 + 2 * i]; }
    md.wpT = p[5 + 2 * md.nb]; md.wvT = p[6 + 2 * md.nb];
    return true;
  }
  if (sys == SYS_DUBINS) {
    if (np < 5) return false;
    md.n = 5; md.m = 2;
    md.dt = p[0]; md.wu = p[1]; md.bamp = p[2]; md.bsig = p[3]; md.nb = (int)p[4];
    if (md.nb < 0 || md.nb > 8 || np < 8 + 2 * md.nb) return false;
    for (int i = 0; i < md.nb; ++i) { md.bc[i][0] = p[5 + 2 * i]; md.bc[i][1] = p[6 + 2 * i]; }
    md.wpT = p[5 + 2 * md.nb]; md.wvT = p[6 + 2 * md.nb]; md.waT = p[7 + 2 * md.nb];
    return true;
  }
  if (sys < SYS_PLANAR3 || sys > SYS_QUAD || np < 8) return false;
  md.dt = p[0];
  md.g[0] = p[1]; md.g[1] = p[2]; md.g[2] = p[3];
  md.N = (int)p[4]; md.a0 = (int)p[5]; md.n_sub = p[6] >= 1 ? (int)p[6] : 1;
  if (md.N <= 0 || md.N > 32 || md.a0 < 0 || md.a0 >= md.N || md.n_sub > 64) return false;
  if (np < 8 + 16 * md.N) return false;
  for (int i = 0; i < md.N; ++i) {
    const double* r = p + 8 + 16 * i;
    Body& bd = md.b[i];
    bd.parent = (int)r[0]; bd.jtype = (int)r[1];
    if (bd.parent >= i || bd.parent < -1 || bd.jtype < 0 || bd.jtype > 5) return false;
    for (int k = 0; k < 3; ++k) { bd.off[k] = r[2 + k]; bd.com[k] = r[6 + k]; bd.I[k] = r[9 + k]; }
    bd.mass = r[5];
  }
  md.n = 2 * md.N; md.m = md.N - md.a0;
  const double* c = p + 8 + 16 * md.N;
  int nc = np - (8 + 16 * md.N);
  if (sys == SYS_PLANAR3) {
    if (nc < 16) return false;
    md.wtau = c[0]; md.bamp = c[1]; md.bsig = c[2]; md.nb = (int)c[3];
    if (md.nb < 0 || md.nb > 2) return false;
    for (int i = 0; i < md.nb; ++i) { md.bc[i][0] = c[4 + 2 * i]; md.bc[i][1] = c[5 + 2 * i]; }
    md.tgt[0] = c[8]; md.tgt[1] = c[9]; md.wee = c[10]; md.wvT = c[11];
    md.ee_body = (int)c[12]; md.ee_pt[0] = c[13]; md.ee_pt[1] = c[14]; md.ee_pt[2] = c[15];
  } else if (sys == SYS_ARM7) {
    if (nc < 11) return false;
    md.wtau = c[0]; md.wv = c[1];
    md.tgt[0] = c[2]; md.tgt[1] = c[3]; md.tgt[2] = c[4];
    md.wee = c[5]; md.wvT = c[6];
    md.ee_body = (int)c[7]; md.ee_pt[0] = c[8]; md.ee_pt[1] = c[9]; md.ee_pt[2] = c[10];
  } else {
    if (nc < 11) return false;
    md.wtau = c[0]; md.znom = c[1]; md.wz = c[2]; md.wrpy = c[3]; md.wvx = c[4]; md.vxt = c[5];
    md.tscale = c[6]; md.kc = c[7]; md.dc = c[8]; md.beta = c[9]; md.nfeet = (int)c[10];
    if (md.nfeet < 0 || md.nfeet > 4 || nc < 11 + 4 * md.nfeet) return false;
    for (int f = 0; f < md.nfeet; ++f) {
      md.foot_body[f] = (int)c[11 + 4 * f];
      for (int k = 0; k < 3; ++k) md.foot_pt[f][k] = c[12 + 4 * f + k];
    }
  }
  if (md.ee_body < 0 || md.ee_body >= md.N) return false;
  return true;
}

// ----------------------------------------------------------------------------
// spatial vector algebra (Featherstone 2008, ch. 2): motion m = (w, v),
// force f = (n, f); a Plucker transform X = (E, r) maps parent coordinates
// to child coordinates, r = child origin in parent coordinates.
// ----------------------------------------------------------------------------
template <class S> struct V3 { S x[3]; };
template <class S> struct M3 { S a[3][3]; };
template <class S> struct SV { S w[3], v[3]; };

template <class S> static void cross(const S* a, const S* b, S* c) {
  S c0 = a[1] * b[2] - a[2] * b[1];
  S c1 = a[2] * b[0] - a[0] * b[2];
  S c2 = a[0] * b[1] - a[1] * b[0];
  c[0] = c0; c[1] = c1; c[2] = c2;
}
template <class S> static void matvec(const M3<S>& E, const S* x, S* y) {
  S t[3];
  for (int i = 0; i < 3; ++i) t[i] = E.a[i][0] * x[0] + E.a[i][1] * x[1] + E.a[i][2] * x[2];
  for (int i = 0; i < 3; ++i) y[i] = t[i];
}
template <class S> static void matTvec(const M3<S>& E, const S* x, S* y) {
  S t[3];
  for (int i = 0; i < 3; ++i) t[i] = E.a[0][i] * x[0] + E.a[1][i] * x[1] + E.a[2][i] * x[2];
  for (int i = 0; i < 3; ++i) y[i] = t[i];
}
template <class S> static M3<S> matmul(const M3<S>& A, const M3<S>& B) {
  M3<S> C;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C.a[i][j] = A.a[i][0] * B.a[0][j] + A.a[i][1] * B.a[1][j] + A.a[i][2] * B.a[2][j];
  return C;
}
template <class S> static M3<S> eye3() {
  M3<S> E;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) E.a[i][j] = (i == j) ? S(1.0) : S(0.0);
  return E;
}
// coordinate transform parent -> child for a rotation by angle th about axis ax
template <class S> static M3<S> rot(int ax, const S& th) {
  S c = cos(th), s = sin(th);
  M3<S> E = eye3<S>();
  int i = (ax + 1) % 3, j = (ax + 2) % 3;
  E.a[i][i] = c; E.a[i][j] = s;
  E.a[j][i] = -s; E.a[j][j] = c;
  return E;
}
// X m
template <class S> static SV<S> xmot(const M3<S>& E, const S* r, const SV<S>& m) {
  SV<S> o;
  S t[3], rw[3];
  cross(r, m.w, rw);
  for (int k = 0; k < 3; ++k) t[k] = m.v[k] - rw[k];
  matvec(E, m.w, o.w);
  matvec(E, t, o.v);
  return o;
}
// X^T f  (force from child coordinates to parent coordinates)
template <class S> static SV<S> xtforce(const M3<S>& E, const S* r, const SV<S>& f) {
  SV<S> o;
  S ef[3], rf[3];
  matTvec(E, f.w, o.w);
  matTvec(E, f.v, ef);
  cross(r, ef, rf);
  for (int k = 0; k < 3; ++k) { o.w[k] = o.w[k] + rf[k]; o.v[k] = ef[k]; }
  return o;
}
// motion cross product  v x m
template <class S> static SV<S> crm(const SV<S>& v, const SV<S>& m) {
  SV<S> o;
  S a[3], b[3];
  cross(v.w, m.w, o.w);
  cross(v.w, m.v, a);
  cross(v.v, m.w, b);
  for (int k = 0; k < 3; ++k) o.v[k] = a[k] + b[k];
  return o;
}
// force cross product  v x* f
template <class S> static SV<S> crf(const SV<S>& v, const SV<S>& f) {
  SV<S> o;
  S a[3], b[3];
  cross(v.w, f.w, a);
  cross(v.v, f.v, b);
  for (int k = 0; k < 3; ++k) o.w[k] = a[k] + b[k];
  cross(v.w, f.v, o.v);
  return o;
}
// spatial inertia of a body (mass m, centre of mass c, rotational inertia
// diag(I) about c in body axes) times a motion vector: momentum about the
// body origin, h = (I_c w + c x p, p) with p = m (v + w x c)
template <class S> static SV<S> inertia_mul(const Body& bd, const SV<S>& m) {
  SV<S> o;
  S c[3] = {S(bd.com[0]), S(bd.com[1]), S(bd.com[2])};
  S wc[3], p[3], cp[3];
  cross(m.w, c, wc);
  for (int k = 0; k < 3; ++k) p[k] = bd.mass * (m.v[k] + wc[k]);
  cross(c, p, cp);
  for (int k = 0; k < 3; ++k) { o.w[k] = bd.I[k] * m.w[k] + cp[k]; o.v[k] = p[k]; }
  return o;
}

template <class S> static void joint_transform(const Body& bd, const S& q, M3<S>& E, S* r) {
  for (int k = 0; k < 3; ++k) r[k] = S(bd.off[k]);
  if (bd.jtype <= J_RZ) {
    E = rot<S>(bd.jtype, q);
  } else {
    E = eye3<S>();
    r[bd.jtype - J_PX] = r[bd.jtype - J_PX] + q;
  }
}
template <class S> static SV<S> motion_subspace(const Body& bd, const S& s) {
  SV<S> o;
  for (int k = 0; k < 3; ++k) { o.w[k] = S(0.0); o.v[k] = S(0.0); }
  if (bd.jtype <= J_RZ) o.w[bd.jtype] = s; else o.v[bd.jtype - J_PX] = s;
  return o;
}
template <class S> static S subspace_dot(const Body& bd, const SV<S>& f) {
  return bd.jtype <= J_RZ ? f.w[bd.jtype] : f.v[bd.jtype - J_PX];
}

// world pose of every body: E0[i] maps world coordinates to body coordinates,
// p0[i] is the body origin in world coordinates
template <class S> static void forward_kinematics(const Model& md, const S* q, std::vector<M3<S>>& E0,
                                                  std::vector<V3<S>>& p0) {
  E0.resize(md.N); p0.resize(md.N);
  for (int i = 0; i < md.N; ++i) {
    M3<S> E; S r[3];
    joint_transform(md.b[i], q[i], E, r);
    int pa = md.b[i].parent;
    if (pa < 0) {
      E0[i] = E;
      for (int k = 0; k < 3; ++k) p0[i].x[k] = r[k];
    } else {
      E0[i] = matmul(E, E0[pa]);
      S wr[3];
      matTvec(E0[pa], r, wr);
      for (int k = 0; k < 3; ++k) p0[i].x[k] = p0[pa].x[k] + wr[k];
    }
  }
}

template <class S> static void point_world(const Model& md, const S* q, int body, const double* pt, S* out) {
  std::vector<M3<S>> E0; std::vector<V3<S>> p0;
  forward_kinematics(md, q, E0, p0);
  S lp[3] = {S(pt[0]), S(pt[1]), S(pt[2])}, w[3];
  matTvec(E0[body], lp, w);
  for (int k = 0; k < 3; ++k) out[k] = p0[body].x[k] + w[k];
}

// recursive Newton-Euler inverse dynamics, optionally with gravity and the
// soft ground contact forces applied at the feet
template <class S> static void rnea(const Model& md, const S* q, const S* qd, const S* qdd, bool grav,
                                    bool contact, S* tau) {
  const int N = md.N;
  std::vector<M3<S>> E(N), E0(N);
  std::vector<V3<S>> r(N), p0(N);
  std::vector<SV<S>> v(N), a(N), f(N);
  for (int i = 0; i < N; ++i) {
    joint_transform(md.b[i], q[i], E[i], r[i].x);
    int pa = md.b[i].parent;
    SV<S> vJ = motion_subspace(md.b[i], qd[i]);
    SV<S> aJ = motion_subspace(md.b[i], qdd[i]);
    SV<S> vp, ap;
    if (pa < 0) {
      for (int k = 0; k < 3; ++k) {
        vp.w[k] = S(0.0); vp.v[k] = S(0.0); ap.w[k] = S(0.0);
        ap.v[k] = grav ? S(-md.g[k]) : S(0.0);   // base acceleration -g
      }
      E0[i] = E[i];
      for (int k = 0; k < 3; ++k) p0[i].x[k] = r[i].x[k];
    } else {
      vp = v[pa]; ap = a[pa];
      E0[i] = matmul(E[i], E0[pa]);
      S wr[3];
      matTvec(E0[pa], r[i].x, wr);
      for (int k = 0; k < 3; ++k) p0[i].x[k] = p0[pa].x[k] + wr[k];
    }
    SV<S> xv = xmot(E[i], r[i].x, vp), xa = xmot(E[i], r[i].x, ap);
    for (int k = 0; k < 3; ++k) { v[i].w[k] = xv.w[k] + vJ.w[k]; v[i].v[k] = xv.v[k] + vJ.v[k]; }
    SV<S> c = crm(v[i], vJ);
    for (int k = 0; k < 3; ++k) { a[i].w[k] = xa.w[k] + aJ.w[k] + c.w[k]; a[i].v[k] = xa.v[k] + aJ.v[k] + c.v[k]; }
    SV<S> Ia = inertia_mul(md.b[i], a[i]), Iv = inertia_mul(md.b[i], v[i]);
    SV<S> vIv = crf(v[i], Iv);
    for (int k = 0; k < 3; ++k) { f[i].w[k] = Ia.w[k] + vIv.w[k]; f[i].v[k] = Ia.v[k] + vIv.v[k]; }
  }
  if (contact) {
    for (int ft = 0; ft < md.nfeet; ++ft) {
      int bi = md.foot_body[ft];
      S pt[3] = {S(md.foot_pt[ft][0]), S(md.foot_pt[ft][1]), S(md.foot_pt[ft][2])};
      // foot position and velocity in world coordinates
      S wpt[3], P[3], wxp[3], vb[3], vw[3];
      matTvec(E0[bi], pt, wpt);
      for (int k = 0; k < 3; ++k) P[k] = p0[bi].x[k] + wpt[k];
      cross(v[bi].w, pt, wxp);
      for (int k = 0; k < 3; ++k) vb[k] = v[bi].v[k] + wxp[k];
      matTvec(E0[bi], vb, vw);
      // penalty contact: normal k*softplus_beta(-z) - d*sigmoid(-beta z)*zdot,
      // tangential damper -d*sigmoid(-beta z)*v_xy
      S z = P[2];
      S ez = exp(md.beta * z);
      S sp = log(1.0 + 1.0 / ez) / md.beta;
      S gate = 1.0 / (1.0 + ez);
      S F[3];
      F[0] = -md.dc * gate * vw[0];
      F[1] = -md.dc * gate * vw[1];
      F[2] = md.kc * sp - md.dc * gate * vw[2];
      // as a spatial force on the body about its origin, in body coordinates
      S mw[3], mb[3], fb[3];
      cross(wpt, F, mw);
      matvec(E0[bi], mw, mb);
      matvec(E0[bi], F, fb);
      for (int k = 0; k < 3; ++k) { f[bi].w[k] = f[bi].w[k] - mb[k]; f[bi].v[k] = f[bi].v[k] - fb[k]; }
    }
  }
  for (int i = N - 1; i >= 0; --i) {
    tau[i] = subspace_dot(md.b[i], f[i]);
    int pa = md.b[i].parent;
    if (pa >= 0) {
      SV<S> fp = xtforce(E[i], r[i].x, f[i]);
      for (int k = 0; k < 3; ++k) { f[pa].w[k] = f[pa].w[k] + fp.w[k]; f[pa].v[k] = f[pa].v[k] + fp.v[k]; }
    }
  }
}

// joint-space mass matrix, column j = inverse dynamics at unit acceleration e_j
// with zero velocity, no gravity and no contact
template <class S> static void mass_matrix(const Model& md, const S* q, S* M) {
  const int N = md.N;
  std::vector<S> z(N, S(0.0)), e(N, S(0.0)), col(N);
  for (int j = 0; j < N; ++j) {
    for (int i = 0; i < N; ++i) e[i] = S(i == j ? 1.0 : 0.0);
    rnea(md, q, z.data(), e.data(), false, false, col.data());
    for (int i = 0; i < N; ++i) M[i * N + j] = col[i];
  }
}

// dense Cholesky factorisation A = L L^T and solve; no pivoting
template <class S> static void chol_solve(int n, std::vector<S> A, const S* b, S* x) {
  for (int j = 0; j < n; ++j) {
    S s = A[j * n + j];
    for (int k = 0; k < j; ++k) s = s - A[j * n + k] * A[j * n + k];
    A[j * n + j] = sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      S t = A[i * n + j];
      for (int k = 0; k < j; ++k) t = t - A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / A[j * n + j];
    }
  }
  std::vector<S> y(n);
  for (int i = 0; i < n; ++i) {
    S t = b[i];
    for (int k = 0; k < i; ++k) t = t - A[i * n + k] * y[k];
    y[i] = t / A[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    S t = y[i];
    for (int k = i + 1; k < n; ++k) t = t - A[k * n + i] * x[k];
    x[i] = t / A[i * n + i];
  }
}

// forward dynamics  qdd = M(q)^{-1} (tau - h(q, qd))
template <class S> static void forward_dynamics(const Model& md, const S* q, const S* qd, const S* tau, S* qdd) {
  const int N = md.N;
  std::vector<S> z(N, S(0.0)), h(N), M(N * N), rhs(N);
  rnea(md, q, qd, z.data(), true, md.sys == SYS_QUAD, h.data());
  mass_matrix(md, q, M.data());
  for (int i = 0; i < N; ++i) rhs[i] = tau[i] - h[i];
  chol_solve(N, M, rhs.data(), qdd);
}

// ----------------------------------------------------------------------------
// the discrete dynamics x_{k+1} = f(x_k, u_k)                  [Sec. II, Eq. 1]
// point mass: explicit Euler; rigid bodies: n_sub semi-implicit Euler substeps
// of dt / n_sub, each  v+ = v + h qdd(q, v, tau),  q+ = q + h v+
// ----------------------------------------------------------------------------
template <class S> static void step(const Model& md, const S* x, const S* u, S* xn) {
  if (md.sys == SYS_PM) {
    xn[0] = x[0] + md.dt * x[2];
    xn[1] = x[1] + md.dt * x[3];
    xn[2] = x[2] + md.dt * u[0];
    xn[3] = x[3] + md.dt * u[1];
    return;
  }
  if (md.sys == SYS_DUBINS) {
    // jerk-controlled Dubins car: (px, py, theta, v, a), u = (omega, jerk)
    xn[0] = x[0] + md.dt * x[3] * cos(x[2]);
    xn[1] = x[1] + md.dt * x[3] * sin(x[2]);
    xn[2] = x[2] + md.dt * u[0];
    xn[3] = x[3] + md.dt * x[4];
    xn[4] = x[4] + md.dt * u[1];
    return;
  }
  const int N = md.N;
  const double h = md.dt / md.n_sub;
  std::vector<S> tau(N, S(0.0)), qdd(N), cur(x, x + 2 * N);
  for (int j = 0; j < md.m; ++j) tau[md.a0 + j] = u[j];
  for (int s = 0; s < md.n_sub; ++s) {
    forward_dynamics(md, cur.data(), cur.data() + N, tau.data(), qdd.data());
    for (int i = 0; i < N; ++i) {
      cur[N + i] = cur[N + i] + h * qdd[i];
      cur[i] = cur[i] + h * cur[N + i];
    }
  }
  for (int i = 0; i < 2 * N; ++i) xn[i] = cur[i];
}

// ----------------------------------------------------------------------------
// running and terminal costs l_k(x,u), l_T(x)                 [Sec. II, Eq. 1]
// ----------------------------------------------------------------------------
template <class S> static S bump(const Model& md, const S& px, const S& py) {
  S s = S(0.0);
  for (int i = 0; i < md.nb; ++i) {
    S dx = px - md.bc[i][0], dy = py - md.bc[i][1];
    s = s + md.bamp * exp(-(dx * dx + dy * dy) / (2.0 * md.bsig * md.bsig));
  }
  return s;
}

template <class S> static S running_cost(const Model& md, const S* x, const S* u) {
  S l = S(0.0);
  if (md.sys == SYS_PM || md.sys == SYS_DUBINS) {
    l = md.wu * (u[0] * u[0] + u[1] * u[1]) + bump(md, x[0], x[1]);
  } else if (md.sys == SYS_PLANAR3) {
    S ee[3];
    point_world(md, x, md.ee_body, md.ee_pt, ee);
    for (int j = 0; j < md.m; ++j) l = l + md.wtau * u[j] * u[j];
    l = l + bump(md, ee[0], ee[1]);
  } else if (md.sys == SYS_ARM7) {
    for (int j = 0; j < md.m; ++j) l = l + md.wtau * u[j] * u[j];
    for (int j = 0; j < md.N; ++j) l = l + md.wv * x[md.N + j] * x[md.N + j];
  } else {
    S dz = x[2] - md.znom, dv = x[md.N] - md.vxt;
    l = md.wz * dz * dz + md.wrpy * (x[3] * x[3] + x[4] * x[4] + x[5] * x[5]) + md.wvx * dv * dv;
    for (int j = 0; j < md.m; ++j) l = l + md.wtau * u[j] * u[j];
  }
  return l;
}

template <class S> static S terminal_cost(const Model& md, const S* x) {
  S l = S(0.0);
  if (md.sys == SYS_PM) {
    l = md.wpT * (x[0] * x[0] + x[1] * x[1]) + md.wvT * (x[2] * x[2] + x[3] * x[3]);
  } else if (md.sys == SYS_DUBINS) {
    l = md.wpT * (x[0] * x[0] + x[1] * x[1]) + md.wvT * x[3] * x[3] + md.waT * x[4] * x[4];
  } else if (md.sys == SYS_PLANAR3 || md.sys == SYS_ARM7) {
    S ee[3];
    point_world(md, x, md.ee_body, md.ee_pt, ee);
    int dims = md.sys == SYS_PLANAR3 ? 2 : 3;
    for (int k = 0; k < dims; ++k) { S d = ee[k] - md.tgt[k]; l = l + md.wee * d * d; }
    for (int j = 0; j < md.N; ++j) l = l + md.wvT * x[md.N + j] * x[md.N + j];
  } else {
    S dz = x[2] - md.znom, dv = x[md.N] - md.vxt;
    l = md.tscale * (md.wz * dz * dz + md.wrpy * (x[3] * x[3] + x[4] * x[4] + x[5] * x[5]) + md.wvx * dv * dv);
  }
  return l;
}

// ----------------------------------------------------------------------------
// exact derivatives by dual numbers
// ----------------------------------------------------------------------------
typedef D<double> D1;
typedef D<D1> D2;

// A = df/dx (n x n), B = df/du (n x m), row-major
static void linearize(const Model& md, const double* x, const double* u, double* A, double* Bm) {
  const int n = md.n, m = md.m;
  std::vector<D1> xd(n), ud(m), xn(n);
  for (int dir = 0; dir < n + m; ++dir) {
    for (int i = 0; i < n; ++i) xd[i] = D1(x[i], dir == i ? 1.0 : 0.0);
    for (int j = 0; j < m; ++j) ud[j] = D1(u[j], dir == n + j ? 1.0 : 0.0);
    step(md, xd.data(), ud.data(), xn.data());
    for (int i = 0; i < n; ++i) {
      if (dir < n) A[i * n + dir] = xn[i].d; else Bm[i * m + (dir - n)] = xn[i].d;
    }
  }
}

// gradient and Hessian of l(z), z = [x; u] (terminal: z = x), by nested duals
static void cost_derivs(const Model& md, const double* x, const double* u, bool terminal, double* l, double* g,
                        double* H) {
  const int n = md.n, m = terminal ? 0 : md.m, nz = n + m;
  std::vector<D2> z(nz);
  for (int i = 0; i < nz; ++i) {
    for (int j = i; j < nz; ++j) {
      for (int k = 0; k < nz; ++k) {
        double zk = k < n ? x[k] : u[k - n];
        z[k] = D2(D1(zk, k == i ? 1.0 : 0.0), D1(k == j ? 1.0 : 0.0, 0.0));
      }
      D2 r = terminal ? terminal_cost(md, z.data()) : running_cost(md, z.data(), z.data() + n);
      H[i * nz + j] = r.d.d;
      H[j * nz + i] = r.d.d;
      if (j == i) g[i] = r.v.d;
      if (i == 0 && j == 0) *l = r.v.v;
    }
  }
}

// ----------------------------------------------------------------------------
// eigenvalue clipping (cyclic Jacobi, Golub & Van Loan sec. 8.5)  [Sec. IV-B]
// ----------------------------------------------------------------------------
static void jacobi_eig(int n, const double* Ain, double* S, double* W) {
  std::vector<double> A(Ain, Ain + n * n);
  for (int i = 0; i < n * n; ++i) W[i] = 0.0;
  for (int i = 0; i < n; ++i) W[i * n + i] = 1.0;
  double fro = 0;
  for (int i = 0; i < n * n; ++i) fro += A[i] * A[i];
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += 2 * A[p * n + q] * A[p * n + q];
    if (off <= 1e-30 * fro || off == 0.0) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double tau = (A[q * n + q] - A[p * n + p]) / (2 * apq);
        double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1 + tau * tau));
        double c = 1 / std::sqrt(1 + t * t), s = t * c;
        // A <- J^T A J with J the rotation in the (p, q) plane
        for (int k = 0; k < n; ++k) {
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double wkp = W[k * n + p], wkq = W[k * n + q];
          W[k * n + p] = c * wkp - s * wkq;
          W[k * n + q] = s * wkp + c * wkq;
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) S[i] = A[i * n + i];
}

static void eigclip(int n, const double* Q, double eps, double* out) {
  std::vector<double> S(n), W(n * n), P(n * n, 0.0);
  jacobi_eig(n, Q, S.data(), W.data());
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0;
      for (int k = 0; k < n; ++k) s += W[i * n + k] * std::max(S[k], eps) * W[j * n + k];
      P[i * n + j] = s;
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) out[i * n + j] = 0.5 * (P[i * n + j] + P[j * n + i]);
}

// ----------------------------------------------------------------------------
// Cholesky of Q_uu with the pivot test; mu I added (x10 per retry) only when
// the test fails                                                 [Sec. IV-B]
// ----------------------------------------------------------------------------
static bool chol_factor(int m, const double* A, double delta, double* L) {
  for (int i = 0; i < m * m; ++i) L[i] = 0;
  for (int j = 0; j < m; ++j) {
    double s = A[j * m + j];
    for (int k = 0; k < j; ++k) s -= L[j * m + k] * L[j * m + k];
    if (!(s > delta)) return false;
    L[j * m + j] = std::sqrt(s);
    for (int i = j + 1; i < m; ++i) {
      double t = A[i * m + j];
      for (int k = 0; k < j; ++k) t -= L[i * m + k] * L[j * m + k];
      L[i * m + j] = t / L[j * m + j];
    }
  }
  return true;
}

// returns 0 ok, 1 regularised, -1 failed
static int chol_guarded(int m, const double* Quu, double* L) {
  double mx = 0;
  for (int i = 0; i < m; ++i) mx = std::max(mx, std::fabs(Quu[i * m + i]));
  if (!(mx > 0) || !std::isfinite(mx)) return -1;
  if (chol_factor(m, Quu, 1e-12 * mx, L)) return 0;
  std::vector<double> R(Quu, Quu + m * m);
  double mu = 1e-6 * mx;
  for (int tries = 0; tries < 40; ++tries) {
    for (int i = 0; i < m * m; ++i) R[i] = Quu[i];
    for (int i = 0; i < m; ++i) R[i * m + i] += mu;
    if (chol_factor(m, R.data(), 1e-12 * mx, L)) return 1;
    mu *= 10;
  }
  return -1;
}

// Levenberg-Marquardt variant (Sec. IV-B's standard regularisation): factor
// Q_uu + mu I under the pivot test d_j > 1e-12 (max|diag Q_uu| + mu); 0 ok,
// -3 when mu must grow (a non-finite Q_uu included: the backward pass failed)
static int chol_shifted(int m, const double* Quu, double mu, double* L) {
  double mx = 0;
  for (int i = 0; i < m; ++i) mx = std::max(mx, std::fabs(Quu[i * m + i]));
  if (!std::isfinite(mx)) return -3;
  std::vector<double> R(Quu, Quu + m * m);
  for (int i = 0; i < m; ++i) R[i * m + i] += mu;
  return chol_factor(m, R.data(), 1e-12 * (mx + mu), L) ? 0 : -3;
}

static void chol_apply_inv(int m, const double* L, const double* b, double* x) {
  std::vector<double> y(m);
  for (int i = 0; i < m; ++i) {
    double t = b[i];
    for (int k = 0; k < i; ++k) t -= L[i * m + k] * y[k];
    y[i] = t / L[i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double t = y[i];
    for (int k = i + 1; k < m; ++k) t -= L[k * m + i] * x[k];
    x[i] = t / L[i * m + i];
  }
}

// ----------------------------------------------------------------------------
// actor policy  u = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3        [Sec. II]
// ----------------------------------------------------------------------------
static void actor(const float* w, int nin, int nh1, int nh2, int nout, const double* x, double* u) {
  const float* W1 = w;
  const float* b1 = W1 + nh1 * nin;
  const float* W2 = b1 + nh1;
  const float* b2 = W2 + nh2 * nh1;
  const float* W3 = b2 + nh2;
  const float* b3 = W3 + nout * nh2;
  std::vector<double> h1(nh1), h2(nh2);
  for (int i = 0; i < nh1; ++i) {
    double s = b1[i];
    for (int k = 0; k < nin; ++k) s += (double)W1[i * nin + k] * x[k];
    h1[i] = std::tanh(s);
  }
  for (int i = 0; i < nh2; ++i) {
    double s = b2[i];
    for (int k = 0; k < nh1; ++k) s += (double)W2[i * nh1 + k] * h1[k];
    h2[i] = std::tanh(s);
  }
  for (int i = 0; i < nout; ++i) {
    double s = b3[i];
    for (int k = 0; k < nh2; ++k) s += (double)W3[i * nh2 + k] * h2[k];
    u[i] = s;
  }
}

// ----------------------------------------------------------------------------
// iLQR                                                   [Sec. II; Sec. IV]
// ----------------------------------------------------------------------------
enum { ST_CONVERGED = 1, ST_MAX_ITER = 2, ST_LS_FAIL = 3, ST_NONFINITE = 4, ST_FLAG_REG = 16 };

struct Opts {
  int max_iter;
  double tol, eps;
  int n_alpha;
  double alpha_decay;
  const int* forced;   // [max_iter], -1 ends the run; NULL: line search decides
  int lm;              // 1: Levenberg-Marquardt variant (no clipping, mu retry loop)
};

// the Levenberg-Marquardt variant's mu schedule
static const double kMu0 = 1e-6, kMuMin = 1e-8, kMuMax = 1e10, kMuFactor = 10.0;

static double rollout_cost(const Model& md, int T, const double* x0, const double* U, double* X) {
  const int n = md.n, m = md.m;
  for (int i = 0; i < n; ++i) X[i] = x0[i];
  double J = 0;
  for (int k = 0; k < T; ++k) {
    J += running_cost(md, X + k * n, U + k * m);
    step(md, X + k * n, U + k * m, X + (k + 1) * n);
  }
  return J + terminal_cost(md, X + T * n);
}

// backward pass at (X, U): gains K (T x m x n), k (T x m), value gradient Vx
// ((T+1) x n). Returns 0, or ST_FLAG_REG if a Cholesky needed mu, or -1.
// lm = 1: the cost Hessians are used as they are and every Q_uu gets + mu I;
// returns -3 when some Q_uu + mu I fails the pivot test.
static int backward(const Model& md, int T, const double* X, const double* U, double eps, double* K,
                    double* kff, double* Vx_out, int lm = 0, double mu = 0.0) {
  const int n = md.n, m = md.m;
  std::vector<double> Vx(n), Vxx(n * n), lg(n + m), lH((n + m) * (n + m)), lxx(n * n), luu(m * m),
      A(n * n), Bm(n * m), Qx(n), Qu(m), Qxx(n * n), Quu(m * m), Qux(m * n), VA(n * n), VB(n * m),
      L(m * m), col(m), sol(m), tmp(n * n);
  double l;
  cost_derivs(md, X + T * n, nullptr, true, &l, lg.data(), lH.data());
  for (int i = 0; i < n; ++i) Vx[i] = lg[i];
  if (lm) std::memcpy(Vxx.data(), lH.data(), sizeof(double) * n * n);
  else eigclip(n, lH.data(), eps, Vxx.data());
  if (Vx_out) for (int i = 0; i < n; ++i) Vx_out[T * n + i] = Vx[i];
  int flag = 0;
  for (int k = T - 1; k >= 0; --k) {
    const double* x = X + k * n;
    const double* u = U + k * m;
    linearize(md, x, u, A.data(), Bm.data());
    cost_derivs(md, x, u, false, &l, lg.data(), lH.data());
    const int nz = n + m;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) tmp[i * n + j] = lH[i * nz + j];
    if (lm) std::memcpy(lxx.data(), tmp.data(), sizeof(double) * n * n);
    else eigclip(n, tmp.data(), eps, lxx.data());
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) tmp[i * m + j] = lH[(n + i) * nz + n + j];
    if (lm) std::memcpy(luu.data(), tmp.data(), sizeof(double) * m * m);
    else eigclip(m, tmp.data(), eps, luu.data());
    // Q terms
    for (int i = 0; i < n; ++i) {
      double s = lg[i];
      for (int r = 0; r < n; ++r) s += A[r * n + i] * Vx[r];
      Qx[i] = s;
    }
    for (int i = 0; i < m; ++i) {
      double s = lg[n + i];
      for (int r = 0; r < n; ++r) s += Bm[r * m + i] * Vx[r];
      Qu[i] = s;
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double s = 0;
        for (int r = 0; r < n; ++r) s += Vxx[i * n + r] * A[r * n + j];
        VA[i * n + j] = s;
      }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < m; ++j) {
        double s = 0;
        for (int r = 0; r < n; ++r) s += Vxx[i * n + r] * Bm[r * m + j];
        VB[i * m + j] = s;
      }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double s = lxx[i * n + j];
        for (int r = 0; r < n; ++r) s += A[r * n + i] * VA[r * n + j];
        Qxx[i * n + j] = s;
      }
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        double s = luu[i * m + j];
        for (int r = 0; r < n; ++r) s += Bm[r * m + i] * VB[r * m + j];
        Quu[i * m + j] = s;
      }
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < n; ++j) {
        double s = lH[(n + i) * nz + j];   // l_ux
        for (int r = 0; r < n; ++r) s += Bm[r * m + i] * VA[r * n + j];
        Qux[i * n + j] = s;
      }
    int rc = lm ? chol_shifted(m, Quu.data(), mu, L.data()) : chol_guarded(m, Quu.data(), L.data());
    if (rc == -3) return -3;
    if (rc < 0) return -1;
    if (rc == 1) flag = ST_FLAG_REG;
    // K = -Quu^{-1} Qux, k = -Quu^{-1} Qu
    double* Kk = K + (size_t)k * m * n;
    double* kk = kff + (size_t)k * m;
    for (int j = 0; j < n; ++j) {
      for (int i = 0; i < m; ++i) col[i] = -Qux[i * n + j];
      chol_apply_inv(m, L.data(), col.data(), sol.data());
      for (int i = 0; i < m; ++i) Kk[i * n + j] = sol[i];
    }
    for (int i = 0; i < m; ++i) col[i] = -Qu[i];
    chol_apply_inv(m, L.data(), col.data(), sol.data());
    for (int i = 0; i < m; ++i) kk[i] = sol[i];
    // V_x = Q_x + Q_ux^T k ; V_xx = sym(Q_xx + Q_ux^T K)
    for (int i = 0; i < n; ++i) {
      double s = Qx[i];
      for (int r = 0; r < m; ++r) s += Qux[r * n + i] * kk[r];
      Vx[i] = s;
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double s = Qxx[i * n + j];
        for (int r = 0; r < m; ++r) s += Qux[r * n + i] * Kk[r * n + j];
        tmp[i * n + j] = s;
      }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) Vxx[i * n + j] = 0.5 * (tmp[i * n + j] + tmp[j * n + i]);
    if (Vx_out) for (int i = 0; i < n; ++i) Vx_out[k * n + i] = Vx[i];
  }
  return flag;
}

// forward pass with step alpha: u^ = u + alpha k + K (x^ - x)
static double forward_pass(const Model& md, int T, const double* X, const double* U, const double* K,
                           const double* kff, double alpha, double* Xn, double* Un) {
  const int n = md.n, m = md.m;
  for (int i = 0; i < n; ++i) Xn[i] = X[i];
  double J = 0;
  for (int k = 0; k < T; ++k) {
    const double* Kk = K + (size_t)k * m * n;
    for (int i = 0; i < m; ++i) {
      double s = U[k * m + i] + alpha * kff[k * m + i];
      for (int j = 0; j < n; ++j) s += Kk[i * n + j] * (Xn[k * n + j] - X[k * n + j]);
      Un[k * m + i] = s;
    }
    J += running_cost(md, Xn + k * n, Un + k * m);
    step(md, Xn + k * n, Un + k * m, Xn + (k + 1) * n);
  }
  return J + terminal_cost(md, Xn + T * n);
}

struct Result {
  double J;
  int iters, status;
};

static Result ilqr(const Model& md, int T, const double* x0, const double* U0, const float* actor_w,
                   const Opts& o, double* X, double* U, double* Vx, double* K_out, double* k_out,
                   int* alpha_hist, double* J_hist) {
  const int n = md.n, m = md.m;
  Result res{0, 0, 0};
  // initial guess: given controls, the actor rolled out, or zero controls
  if (U0) {
    for (int i = 0; i < T * m; ++i) U[i] = U0[i];
  } else if (actor_w) {
    for (int i = 0; i < n; ++i) X[i] = x0[i];
    for (int k = 0; k < T; ++k) {
      actor(actor_w, n, 256, 256, m, X + k * n, U + k * m);
      step(md, X + k * n, U + k * m, X + (k + 1) * n);
    }
  } else {
    for (int i = 0; i < T * m; ++i) U[i] = 0.0;
  }
  double J = rollout_cost(md, T, x0, U, X);
  if (J_hist) J_hist[0] = J;
  if (!std::isfinite(J)) { res.J = J; res.status = ST_NONFINITE; return res; }
  std::vector<double> K((size_t)T * m * n), kff((size_t)T * m), Xn((size_t)(T + 1) * n), Un((size_t)T * m);
  int flags = 0, status = ST_MAX_ITER, it = 0;
  double mu = kMu0;
  while (it < o.max_iter) {
    if (o.forced && o.forced[it] < 0) break;
    int rc = backward(md, T, X, U, o.eps, K.data(), kff.data(), nullptr, o.lm, mu);
    if (rc == -3) {
      // Levenberg-Marquardt: grow mu and redo the backward pass
      mu *= kMuFactor;
      if (mu > kMuMax) { status = ST_LS_FAIL; break; }
      continue;
    }
    if (rc < 0) { status = ST_NONFINITE; break; }
    flags |= rc;
    int acc = -1;
    double Jn = 0;
    if (o.forced) {
      acc = o.forced[it];
      Jn = forward_pass(md, T, X, U, K.data(), kff.data(), std::pow(o.alpha_decay, acc), Xn.data(), Un.data());
    } else {
      for (int j = 0; j < o.n_alpha; ++j) {
        double Jj = forward_pass(md, T, X, U, K.data(), kff.data(), std::pow(o.alpha_decay, j), Xn.data(),
                                 Un.data());
        if (Jj < J) { acc = j; Jn = Jj; break; }   // smallest j with strict decrease
      }
    }
    if (acc < 0 && o.lm) {
      mu *= kMuFactor;
      if (mu > kMuMax) { status = ST_LS_FAIL; break; }
      continue;
    }
    if (acc < 0) { status = ST_LS_FAIL; break; }
    if (o.lm) mu = std::max(mu / kMuFactor, kMuMin);
    std::memcpy(X, Xn.data(), sizeof(double) * (T + 1) * n);
    std::memcpy(U, Un.data(), sizeof(double) * T * m);
    if (alpha_hist) alpha_hist[it] = acc;
    ++it;
    if (J_hist) J_hist[it] = Jn;
    if (!std::isfinite(Jn)) { J = Jn; status = ST_NONFINITE; break; }
    double rel = (J - Jn) / std::max(std::fabs(J), 1e-300);
    J = Jn;
    if (!o.forced && rel < o.tol) { status = ST_CONVERGED; break; }
  }
  if ((Vx || K_out || k_out) && std::isfinite(J)) {
    std::vector<double> vx((size_t)(T + 1) * n);
    int rc = backward(md, T, X, U, o.eps, K.data(), kff.data(), vx.data(), o.lm, mu);
    if (rc > 0) flags |= rc;
    if (Vx) std::memcpy(Vx, vx.data(), sizeof(double) * (T + 1) * n);
    if (K_out) std::memcpy(K_out, K.data(), sizeof(double) * T * m * n);
    if (k_out) std::memcpy(k_out, kff.data(), sizeof(double) * T * m);
  }
  res.J = J;
  res.iters = it;
  res.status = status | flags;
  return res;
}

}  // namespace orc

// ============================================================================
// C interface (ctypes)
// ============================================================================
using namespace orc;

extern "C" {

int oracle_dims(int sys, const double* p, int np, int* n, int* m) {
  Model md;
  if (!parse(sys, p, np, md)) return -1;
  *n = md.n; *m = md.m;
  return 0;
}

int oracle_step(int sys, const double* p, int np, const double* x, const double* u, double* xn) {
  Model md;
  if (!parse(sys, p, np, md)) return -1;
  step(md, x, u, xn);
  return 0;
}

int oracle_linearize(int sys, const double* p, int np, const double* x, const double* u, double* A, double* B) {
  Model md;
  if (!parse(sys, p, np, md)) return -1;
  linearize(md, x, u, A, B);
  return 0;
}

// gradient g and Hessian H over z = [x; u] (terminal: z = x)
int oracle_cost(int sys, const double* p, int np, const double* x, const double* u, int terminal, double* l,
                double* g, double* H) {
  Model md;
  if (!parse(sys, p, np, md)) return -1;
  cost_derivs(md, x, u, terminal != 0, l, g, H);
  return 0;
}

int oracle_cost_value(int sys, const double* p, int np, const double* x, const double* u, int terminal, double* l) {
  Model md;
  if (!parse(sys, p, np, md)) return -1;
  *l = terminal ? terminal_cost(md, x) : running_cost(md, x, u);
  return 0;
}

int oracle_rnea(int sys, const double* p, int np, const double* q, const double* qd, const double* qdd, int grav,
                int contact, double* tau) {
  Model md;
  if (!parse(sys, p, np, md) || sys == SYS_PM || sys == SYS_DUBINS) return -1;
  rnea(md, q, qd, qdd, grav != 0, contact != 0, tau);
  return 0;
}

int oracle_mass_matrix(int sys, const double* p, int np, const double* q, double* M) {
  Model md;
  if (!parse(sys, p, np, md) || sys == SYS_PM || sys == SYS_DUBINS) return -1;
  mass_matrix(md, q, M);
  return 0;
}

int oracle_forward_dynamics(int sys, const double* p, int np, const double* q, const double* qd, const double* tau,
                            double* qdd) {
  Model md;
  if (!parse(sys, p, np, md) || sys == SYS_PM || sys == SYS_DUBINS) return -1;
  forward_dynamics(md, q, qd, tau, qdd);
  return 0;
}

// world position of a point fixed in a body, and the body's world rotation
// (E0 maps world coordinates to body coordinates, row-major 3x3)
int oracle_point_world(int sys, const double* p, int np, const double* q, int body, const double* pt, double* out,
                       double* E0out) {
  Model md;
  if (!parse(sys, p, np, md) || sys == SYS_PM || sys == SYS_DUBINS || body < 0 || body >= md.N) return -1;
  point_world(md, q, body, pt, out);
  if (E0out) {
    std::vector<M3<double>> E0; std::vector<V3<double>> p0;
    forward_kinematics(md, q, E0, p0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) E0out[i * 3 + j] = E0[body].a[i][j];
  }
  return 0;
}

int oracle_eigclip(int n, const double* Q, double eps, double* out) {
  if (n <= 0) return -1;
  eigclip(n, Q, eps, out);
  return 0;
}

int oracle_eig(int n, const double* Q, double* S, double* W) {
  if (n <= 0) return -1;
  jacobi_eig(n, Q, S, W);
  return 0;
}

// guarded Cholesky solve: x = Quu^{-1} b; returns 0, 1 (regularised) or -1
int oracle_chol_solve(int m, const double* Quu, const double* b, double* x) {
  std::vector<double> L(m * m);
  int rc = chol_guarded(m, Quu, L.data());
  if (rc < 0) return -1;
  chol_apply_inv(m, L.data(), b, x);
  return rc;
}

int oracle_actor(const float* w, int nin, int nh1, int nh2, int nout, const double* x, double* u) {
  actor(w, nin, nh1, nh2, nout, x, u);
  return 0;
}

int oracle_rollout(int sys, const double* p, int np, int T, const double* x0, const double* U, double* X,
                   double* J) {
  Model md;
  if (!parse(sys, p, np, md)) return -1;
  *J = rollout_cost(md, T, x0, U, X);
  return 0;
}

// critic targets of one trajectory (Sec. II): the partial K-step cost-to-go
// Vbar_k = sum_{j=k}^{min(k+K,T)-1} l_j(x_j, u_j) + [k + K >= T] l_T(x_T),
// k = 0..T, summed in order from the definition
int oracle_critic_targets(int sys, const double* p, int np, int T, int K, const double* X, const double* U,
                          double* Vbar) {
  Model md;
  if (!parse(sys, p, np, md) || K < 1) return -1;
  const int n = md.n, m = md.m;
  for (int k = 0; k <= T; ++k) {
    double s = 0.0;
    for (int j = k; j < std::min(k + K, T); ++j) s += running_cost(md, X + (size_t)j * n, U + (size_t)j * m);
    if (k + K >= T) s += terminal_cost(md, X + (size_t)T * n);
    Vbar[k] = s;
  }
  return 0;
}

// one backward pass at (X, U)
int oracle_backward(int sys, const double* p, int np, int T, const double* X, const double* U, double eps,
                    double* K, double* kff, double* Vx) {
  Model md;
  if (!parse(sys, p, np, md)) return -1;
  return backward(md, T, X, U, eps, K, kff, Vx);
}

int oracle_forward_pass(int sys, const double* p, int np, int T, const double* X, const double* U, const double* K,
                        const double* kff, double alpha, double* Xn, double* Un, double* J) {
  Model md;
  if (!parse(sys, p, np, md)) return -1;
  *J = forward_pass(md, T, X, U, K, kff, alpha, Xn, Un);
  return 0;
}

// Solve B instances (x0: B x n, T: B horizons).  Per-instance outputs are
// packed with stride T_max: X (B x (T_max+1) x n), U (B x T_max x m),
// Vx like X (or NULL), K (B x T_max x m x n, or NULL), alpha_hist and J_hist
// (B x max_iter and B x (max_iter+1), or NULL).  forced: B x max_iter or NULL.
// Padding: U beyond T is 0; X beyond T repeats x_T.  Threads: 0 = all cores.
int oracle_solve_batch(int sys, const double* p, int np, const float* actor_w, int B, int T_max, const double* x0,
                       const int* T, const double* U_init, int max_iter, double tol, double eps, int n_alpha,
                       double alpha_decay, const int* forced, int n_threads, double* X, double* U, double* J,
                       int* iters, int* status, double* Vx, double* K, int* alpha_hist, double* J_hist, int lm) {
  Model md;
  if (!parse(sys, p, np, md)) return -1;
  const int n = md.n, m = md.m;
  for (int b = 0; b < B; ++b)
    if (T[b] < 1 || T[b] > T_max) return -2;
  if (n_threads <= 0) n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
  n_threads = std::min(n_threads, std::max(B, 1));
  auto work = [&](int t0) {
    for (int b = t0; b < B; b += n_threads) {
      const int Tb = T[b];
      Opts o{max_iter, tol, eps, n_alpha, alpha_decay, forced ? forced + (size_t)b * max_iter : nullptr, lm};
      std::vector<double> Xb((size_t)(Tb + 1) * n), Ub((size_t)Tb * m), vx, kk;
      std::vector<double> Kb;
      if (Vx) vx.resize((size_t)(Tb + 1) * n);
      if (K) Kb.resize((size_t)Tb * m * n);
      Result r = ilqr(md, Tb, x0 + (size_t)b * n, U_init ? U_init + (size_t)b * T_max * m : nullptr, actor_w, o,
                      Xb.data(), Ub.data(), Vx ? vx.data() : nullptr, K ? Kb.data() : nullptr, nullptr,
                      alpha_hist ? alpha_hist + (size_t)b * max_iter : nullptr,
                      J_hist ? J_hist + (size_t)b * (max_iter + 1) : nullptr);
      J[b] = r.J; iters[b] = r.iters; status[b] = r.status;
      double* Xo = X + (size_t)b * (T_max + 1) * n;
      double* Uo = U + (size_t)b * T_max * m;
      for (int k = 0; k <= T_max; ++k)
        for (int i = 0; i < n; ++i) Xo[k * n + i] = Xb[(size_t)std::min(k, Tb) * n + i];
      for (int k = 0; k < T_max; ++k)
        for (int i = 0; i < m; ++i) Uo[k * m + i] = k < Tb ? Ub[(size_t)k * m + i] : 0.0;
      if (Vx) {
        double* Vo = Vx + (size_t)b * (T_max + 1) * n;
        for (int k = 0; k <= T_max; ++k)
          for (int i = 0; i < n; ++i) Vo[k * n + i] = k <= Tb ? vx[(size_t)k * n + i] : 0.0;
      }
      if (K) {
        double* Ko = K + (size_t)b * T_max * m * n;
        for (size_t i = 0; i < (size_t)T_max * m * n; ++i) Ko[i] = i < Kb.size() ? Kb[i] : 0.0;
      }
    }
  };
  if (n_threads == 1) {
    work(0);
  } else {
    std::vector<std::thread> th;
    for (int t = 0; t < n_threads; ++t) th.emplace_back(work, t);
    for (auto& t : th) t.join();
  }
  return 0;
}

}  // extern "C"
