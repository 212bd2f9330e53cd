// Batched iLQR solver kernel, generic over the system and the arithmetic.
//
// One group of G threads owns one OCP instance (Sec. II, Eq. 1) and runs the
// whole iteration for it:
//   backward pass  (Sec. II: DDP backward pass without second-order dynamics
//                   terms; Sec. IV-B: eigenvalue-clipped cost Hessians and the
//                   Cholesky of Q_uu with mu I only when the pivot test fails)
//   line search    (step sizes alpha_j = decay^j evaluated LW at a time, one
//                   per lane, each rolled out into its own trajectory slot; the
//                   smallest j with J(alpha_j) < J_old is accepted and its slot
//                   becomes the current iterate, so nothing is rolled out
//                   twice; a further round of LW runs only if no step in the
//                   round decreased the cost)
//   bookkeeping    (fixed iteration budget per instance, Sec. IV-A; relative
//                   cost-decrease test)
// The grid is persistent: a group that finishes an instance takes the next
// one from a queue ordered by horizon (longest first), so instances with
// uneven horizons and iteration counts share one launch.  Groups that share a
// warp run warp-uniform control flow; per-group work is predicated.  Every
// phase prefetches the next knot record into registers while the current
// knot computes.  Systems may move derivative work off the backward
// recursion: the planar arm stores every knot's derivative block, the rigid
// trees every knot's substep primals, computed before the pass one knot per
// lane (per-knot scratch, a.dscr).  G = 1 (single-lane groups) keeps the
// whole backward knot in registers (backward_lane).
//
// Arithmetic: R = double (FP64 mode) or float (mixed mode).  In mixed mode
// rollouts, derivatives and Riccati products are float32; the Q_uu Cholesky
// and its pivot test are float64; the residual of the one-step refinement of
// the gain solve is float-float (refine = 1, about 48 significant bits) or
// float64 (refine = 2); the cost is accumulated as a compensated float32 pair
// (about 48 significant bits) and compared in float64.
#pragma once
#include <cfloat>
#include <type_traits>

#include "common.cuh"

namespace to {

constexpr int kMaxAlpha = 32;
constexpr int kLsWidth = 16;                 // most step sizes tried at once
constexpr int kMaxSlots = kLsWidth + 1;      // trajectory slots per knot for the widest groups

// A serving request as published by the host in pinned, mapped memory.
constexpr int kServeMaxN = 36;
struct ServeDesc {
  int seat;            // workspace seat (instance index) of the request
  int T;               // horizon
  unsigned seq;        // ring index + 1
  int pad;
  double x0[kServeMaxN];
};

// Serving mode: instead of a fixed batch, groups claim requests from a ring
// that the host fills while the kernel runs (null ring = batch mode).
struct ServeArgs {
  const volatile ServeDesc* ring;   // host-mapped descriptor ring
  int ring_size;
  const volatile unsigned* tail;    // host-mapped: number of published requests
  unsigned* head;                   // device: number of claimed requests
  volatile unsigned* done;          // host-mapped, per seat: ring index + 1 when solved
  const volatile int* stop;         // host-mapped: leave as soon as every group is idle
  int* seat_T;                      // device, per seat: horizon of its last request
  int* ctl;                         // device, per launch: [0] groups solving, [1] closing latch
  volatile int* closing;            // host-mapped mirror of the latch (the host then launches anew)
  int idle_polls;                   // polls (2 us apart) with no group solving before the kernel closes
  double grid_frac;                 // host side: the kernel's share of the resident CTAs
};

struct SolveArgs {
  ServeArgs serve;
  int B, T_max, max_iter, n_alpha, refine, want_vx;
  int lm;                  // 1: Levenberg-Marquardt variant (no clip, mu retry loop)
  double tol, eps;
  double alpha_d[kMaxAlpha];   // alpha_j = decay^j
  float alpha_f[kMaxAlpha];
  const double* x0;         // B x n
  const int* T;             // B
  const double* U_init;     // B x T_max x m or null
  const int* forced;        // B x max_iter or null
  const long long* toff;    // B: first knot record of each instance
  const int* order;         // B: instance indices, longest horizon first
  int* queue;               // work counter
  void* traj;               // knot records [x | u | pad] (R), (LW + 1) slots per knot
  void* gains;              // gain records [K (m x n) | k (m) | pad] (R)
  double* vx;               // knots x n, or null
  double* J_out;
  int* iters_out;
  int* status_out;
  int* slot_out;            // B: trajectory slot holding the returned iterate
  int* ahist;               // B x max_iter
  double* Jhist;            // B x (max_iter + 1)
  const void* params;       // the system's parameter struct in the kernel's precision
  const float* actor_w;     // actor weights or null
  void* dscr;               // per-knot derivative scratch (stored substep primals) or null
  long long kscr;           // its elements per knot
  const int* err;           // set by the prepare kernel on malformed input
  unsigned long long* prof; // 8 per-phase cycle counters, or null (tracing off)
  long long knots_cap;      // knot records the buffers hold (traj, gains, vx, dscr)
  unsigned long long* chk;  // bounds-check report (checked build), or null
};

// Bounds checks of the checked build (compiled with TO_CHECKED).  An index
// outside [0, lim) is recorded in a.chk -- [0] the number of violations,
// [1] the first one's site, [2] its index, [3] its limit -- and replaced by
// 0, so the access lands on the buffer's first element instead of outside
// the buffer.  In the release build both helpers compile to nothing.
#ifdef TO_CHECKED
TO_DEV bool ck_ok(const SolveArgs& a, long long i, long long lim, int site) {
  if (i >= 0 && i < lim) return true;
  if (a.chk && atomicAdd(a.chk, 1ull) == 0ull) {
    a.chk[1] = (unsigned long long)site;
    a.chk[2] = (unsigned long long)i;
    a.chk[3] = (unsigned long long)lim;
  }
  return false;
}
#else
TO_DEV constexpr bool ck_ok(const SolveArgs&, long long, long long, int) { return true; }
#endif
TO_DEV long long ck(const SolveArgs& a, long long i, long long lim, int site) {
  return ck_ok(a, i, lim, site) ? i : 0;
}
// check sites (the report's [1])
enum {
  CK_ORDER = 1, CK_SEAT, CK_HORIZON, CK_RECORD, CK_SLOT, CK_GAINS, CK_VX, CK_DSCR, CK_FORCED, CK_UINIT,
  CK_HIST
};

// per-phase clock64 accounting (tracing); one timer thread per warp / CTA
#define TO_TICK(ph)                                                                  \
  if (a.prof) {                                                                      \
    const long long t_ = clock64();                                                  \
    if (timer) atomicAdd(a.prof + (ph), (unsigned long long)(t_ - tlast));           \
    tlast = t_;                                                                      \
  }

// knot record [x | u | x_lo | pad]: in float32 the state's low parts ride
// along (the rollouts carry the state as (hi, lo) pairs, acc2); gain record
// [K | k | pad]; both padded to 16 bytes
template <class Sys, class R>
struct Layout {
  static constexpr int n = Sys::n, m = Sys::m;
  static constexpr int kVec = 16 / (int)sizeof(R);
  static constexpr int kLo = sizeof(R) == 4 ? n : 0;
  static constexpr int RS = (n + m + kLo + kVec - 1) / kVec * kVec;
  static constexpr int GS = (m * (n + 1) + kVec - 1) / kVec * kVec;
};

// cost accumulator: plain float64, or a compensated float32 pair (two-sum)
template <class R> struct Acc;
template <> struct Acc<double> {
  double s = 0;
  TO_DEV void add(double v) { s += v; }
  TO_DEV double value() const { return s; }
};
template <> struct Acc<float> {
  float hi = 0.f, lo = 0.f;
  TO_DEV void add(float v) {
    const float t = hi + v;
    const float bv = t - hi;
    lo += (hi - (t - bv)) + (v - bv);
    hi = t;
  }
  TO_DEV double value() const { return (double)hi + (double)lo; }
};

// per-group shared-memory workspace
template <class Sys, class R>
struct Work {
  static constexpr int n = Sys::n, m = Sys::m;
  double Quu[m * m];
  double L[m * m];       // float64 Cholesky factor of Q_uu (+ mu I)
  double mu;
  double red;
  R Lf[m * m];           // the factor rounded to R, unit diagonal scaled: Lf[jj] = 1 / L_jj
  R Quf[m * m];          // Q_uu as formed in R (float-float refinement residual)
  R V[n * n];            // V_xx, then Q_xx, then the new V_xx (in place)
  R v[n];                // V_x
  R A[n * n];
  R Bm[n * m];
  R VA[n * n];           // V A; scratch of the derivatives
  R VB[n * m];
  R lxx[n * n];
  R Qux[m * n];
  R Qx[n];
  R Qu[m];
  R lx[n];
  R lu[m];
  R luu[m * m];
  R xk[n];               // staged knot record: x_k, u_k (adjacent)
  R uk[m];
  R xl[n];               // low parts of x_k (float32 rollouts)
  R K[m * n];            // gains K_k, k_k (adjacent)
  R kf[m];
  alignas(16) R sx[Sys::template Scratch<R>::elems];   // the system's derivative scratch (rigid trees: per-substep primal)
  int flag;              // Cholesky: 0 ok, 1 regularised, 2 failed
  int sel;
  int wslot;             // slot of the accepted line-search candidate
};

// Element loop of a group whose loads should be in flight together: the
// trips unroll (predicated), element e = lane + s G.
template <int NE, int G, class F>
TO_DEV void for_each_lane(const Group<G>& g, F&& f) {
#pragma unroll
  for (int s = 0; s < (NE + G - 1) / G; ++s) {
    const int e = g.lane + s * G;
    if (e < NE) f(e);
  }
}

// per-lane workspace of single-lane groups: every matrix lives in registers
struct WorkLane {
  double red;
  int flag;
  int sel;
  int wslot;
};

enum { M_IDLE = 0, M_NEW, M_RUN, M_FINAL, M_DRAINED };

// Levenberg-Marquardt variant: mu starts at kMu0, is multiplied by kMuFactor
// when Q_uu + mu I fails the pivot test or the line search finds no decrease
// (and the backward pass is redone), divided by it after an accepted step
// (not below kMuMin); beyond kMuMax the instance stops with LS_FAIL
constexpr double kMu0 = 1e-6, kMuMin = 1e-8, kMuMax = 1e10, kMuFactor = 10.0;

// D is the staging depth: a group fetches the records it will read D knots
// ahead of the knot that reads them (the backward pass's knot record or
// stored derivative block, the forward pass's knot record and gains), into a
// ring of D register sets per lane.  1 or 2; the autotuner picks it.
template <class Sys, class R, int G, int D = 1>
struct Solver {
  static_assert(D == 1 || D == 2, "staging depth 1 or 2");
  static_assert(G > 1 || D == 1, "a single-lane group stages one knot ahead");
  static constexpr int n = Sys::n, m = Sys::m;
  static constexpr int RS = Layout<Sys, R>::RS, GS = Layout<Sys, R>::GS;
  static constexpr int kLo = Layout<Sys, R>::kLo;
  static constexpr int NF = n + m + m * (n + 1) + kLo;    // forward record: x, u, K, k, x_lo
  static constexpr int PF = (NF + G - 1) / G;             // prefetch registers per lane (forward)
  // prefetch registers per lane (backward): the knot record x_k, u_k, or,
  // for systems that store a derivative block per knot, that block
  template <class S> static constexpr int bwd_prefetch_elems() {
    if constexpr (S::kStoredDerivs) return S::kDerivStride;
    else return S::n + S::m;
  }
  static constexpr int PB = (bwd_prefetch_elems<Sys>() + G - 1) / G;
  static constexpr int LW = G < kLsWidth ? G : kLsWidth;   // step sizes per line-search round
  static constexpr int NS = LW + 1;                        // trajectory slots per knot
  static constexpr int kRounds = (kMaxAlpha + LW - 1) / LW; // most line-search rounds
  // a system whose rollout step is shared by partner lanes has a slot for
  // every line-search lane
  template <class S> static constexpr bool step_slots_fit() {
    if constexpr (S::template kGroupStep<G>) return LW <= S::kStepSlots;
    else return true;
  }
  static_assert(step_slots_fit<Sys>(), "line-search lanes exceed the system's step slots");
  static_assert(!Sys::kKnotParallel || G >= 32, "knot-parallel derivatives need groups of whole warps");
  typedef typename Sys::template ParamsT<R> Params;
  static constexpr bool kLane = (G == 1);                  // one thread per instance, matrices in registers
  // lanes of a warp that are not a group's first lane (sub-warp groups)
  static constexpr unsigned non_leaders() {
    unsigned mk = 0xffffffffu;
    for (int i = 0; i < 32; i += (G < 32 ? G : 32)) mk &= ~(1u << i);
    return mk;
  }
  static constexpr unsigned kNonLeaders = non_leaders();
  typedef std::conditional_t<kLane, WorkLane, Work<Sys, R>> W;
  static_assert(!(kLane && Sys::kActor), "the actor warm start needs a lane group");

  // ------------------------------------------------------------------------
  // Cholesky of Q_uu in float64 with the pivot test  d_j > 1e-12 max|diag|;
  // on failure mu I is added, mu = 1e-6 max|diag| growing x10 (Sec. IV-B's
  // Levenberg-Marquardt term, used only as this guard).  One thread; the
  // reciprocal pivots come from rsqrt, so there is no float64 division.
  // ------------------------------------------------------------------------
  template <bool kShift>
  TO_DEV static bool chol(const double* A, double shift, double delta, double* L) {
#pragma unroll
    for (int j = 0; j < m; ++j) {
      double s = A[j * m + j];
      if (kShift) s += shift;
      for (int k = 0; k < j; ++k) s -= L[j * m + k] * L[j * m + k];
      if (!(s > delta)) return false;
      const double r = rsqrt(s);
      L[j * m + j] = r;                      // stores 1 / L_jj
#pragma unroll
      for (int i = j + 1; i < m; ++i) {
        double t = A[i * m + j];
#pragma unroll
        for (int k = 0; k < j; ++k) t -= L[i * m + k] * L[j * m + k];
        L[i * m + j] = t * r;
      }
    }
    return true;
  }
  // The float64 factor of Q_uu with the pivot test.  lm = 0: the guard
  // above (flag 0 plain, 1 regularised with mu, 2 failed).  lm = 1: the
  // Levenberg-Marquardt variant (Sec. IV-B's standard regularisation), the
  // factor of Q_uu + mu I with the instance's mu (flag 0, or 3: a larger mu
  // is needed).  Q is Q_uu in float64 and Qr the same entries in R (the
  // largest diagonal magnitude is exact in either).  On success the factor's
  // lower triangle is also rounded to R in Lf.
  TO_DEV static int factor(const double* Q, const R* Qr, bool lm, double mu_lm, double* L, R* Lf, double& mu) {
    R mxr = R(0);
#pragma unroll
    for (int i = 0; i < m; ++i) mxr = max_abs(mxr, Qr[i * m + i]);
    const double mx = (double)mxr;
    int flag;
    if (lm) {
      mu = mu_lm;
      flag = 3;
      if (isfinite(mx) && chol<true>(Q, mu, 1e-12 * (mx + mu), L)) flag = 0;
    } else {
      mu = 0;
      flag = 2;
      if (mx > 0 && isfinite(mx)) {
        const double delta = 1e-12 * mx;
        if (chol<false>(Q, 0.0, delta, L)) {
          flag = 0;
        } else {
          double mt = 1e-6 * mx;
          for (int t = 0; t < 40; ++t) {
            if (chol<true>(Q, mt, delta, L)) { flag = 1; mu = mt; break; }
            mt *= 10.0;
          }
        }
      }
    }
    if (flag < 2)
#pragma unroll
      for (int i = 0; i < m; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) Lf[i * m + j] = (R)L[i * m + j];
    return flag;
  }
  // ------------------------------------------------------------------------
  // The float64 factor of Q_uu spread over the 32 lanes of a warp (groups of
  // whole warps).  Lane l holds the lower-triangle entries t = l + 32 e
  // (row-major, diagonal included) in registers; step k of the right-looking
  // elimination takes the pivot from its owner by a shuffle, scales column k
  // (the diagonal keeps 1 / L_kk), publishes it in Lm (shared) and
  // subtracts l_ik l_jk from every entry (i, j) with j > k.  Each entry thus
  // takes exactly the operations of chol()'s sums, in the same order
  // k = 0, 1, ..., so the factor is the one-lane factor's; the difference is
  // that the m^3/3 multiply-adds of a step issue as one warp instruction per
  // register slot.  kSeeded (mixed mode, where the factor is rounded to
  // float32 for the solves): reciprocal roots from rsqrt_newton for pivots
  // in the normal float32 range, else rsqrt.  Returns whether every pivot
  // passed d > delta (the same on every lane).
  // ------------------------------------------------------------------------
  static constexpr int kTri = m * (m + 1) / 2, kTriSlots = (kTri + 31) / 32;
  template <bool kSeeded>
  TO_DEV static bool chol_warp_try(const double* Q, double* Lm, double shift, double delta, const int (&ri)[kTriSlots],
                                   const int (&ci)[kTriSlots]) {
    double a[kTriSlots];
#pragma unroll
    for (int e = 0; e < kTriSlots; ++e) {
      a[e] = ri[e] >= 0 ? Q[ri[e] * m + ci[e]] : 0.0;
      if (ri[e] >= 0 && ri[e] == ci[e]) a[e] += shift;
    }
    bool ok = true;
#pragma unroll
    for (int k = 0; k < m; ++k) {
      const int tkk = k * (k + 1) / 2 + k;                  // compile-time once the loop unrolls
      const double d = __shfl_sync(0xffffffffu, a[tkk / 32], tkk % 32);
      ok = ok & dgt_nonneg(d, delta);
      double r;
      if (kSeeded) {
        const long long bits = __double_as_longlong(d);
        if (bits >= 0x3810000000000000LL && bits <= 0x47efffffe0000000LL) r = rsqrt_newton(d);   // FLT_MIN .. FLT_MAX
        else r = rsqrt(d);
      } else {
        r = rsqrt(d);
      }
#pragma unroll
      for (int e = 0; e < kTriSlots; ++e)
        if (ci[e] == k) {
          const double v = ri[e] == k ? r : a[e] * r;
          a[e] = v;
          Lm[ri[e] * m + k] = v;
        }
      __syncwarp();
#pragma unroll
      for (int e = 0; e < kTriSlots; ++e)
        if (ci[e] > k) a[e] -= Lm[ri[e] * m + k] * Lm[ci[e] * m + k];
    }
    return ok;
  }
  // factor() with chol_warp_try, run by the 32 lanes of the group's first
  // warp; the flags, mu schedule and float rounding of the factor are
  // factor()'s.  Writes w.L, w.Lf, w.flag and w.mu.
  TO_DEV static void chol_warp(W& w, bool lm, double mu_lm, int lane) {
    constexpr bool kSeed = sizeof(R) == 4;
    int ri[kTriSlots], ci[kTriSlots];
#pragma unroll
    for (int e = 0; e < kTriSlots; ++e) {
      const int t = lane + 32 * e;
      int i = 0;
      while ((i + 1) * (i + 2) / 2 <= t) ++i;               // row of entry t (t < kTri: i < m)
      ri[e] = t < kTri ? i : -1;
      ci[e] = t < kTri ? t - i * (i + 1) / 2 : -1;
    }
    R mxr = R(0);
#pragma unroll
    for (int i = 0; i < m; ++i) mxr = max_abs(mxr, w.Quf[i * m + i]);
    const double mx = (double)mxr;
    int flag;
    double mu;
    if (lm) {
      mu = mu_lm;
      flag = 3;
      if (isfinite(mx) && chol_warp_try<kSeed>(w.Quu, w.L, mu, 1e-12 * (mx + mu), ri, ci)) flag = 0;
    } else {
      mu = 0;
      flag = 2;
      if (mx > 0 && isfinite(mx)) {
        const double delta = 1e-12 * mx;
        if (chol_warp_try<kSeed>(w.Quu, w.L, 0.0, delta, ri, ci)) {
          flag = 0;
        } else {
          double mt = 1e-6 * mx;
          for (int t = 0; t < 40; ++t) {
            if (chol_warp_try<kSeed>(w.Quu, w.L, mt, delta, ri, ci)) { flag = 1; mu = mt; break; }
            mt *= 10.0;
          }
        }
      }
    }
    if (flag < 2)
#pragma unroll
      for (int e = 0; e < kTriSlots; ++e)
        if (ri[e] >= 0) w.Lf[ri[e] * m + ci[e]] = (R)w.L[ri[e] * m + ci[e]];
    if (lane == 0) {
      w.flag = flag;
      w.mu = mu;
    }
  }

  // x = (L L^T)^{-1} b with L's diagonal stored as reciprocals
  template <class T, class LT>
  TO_DEV static void chol_apply(const LT* L, const T* b, T* x) {
    T y[m];
#pragma unroll
    for (int i = 0; i < m; ++i) {
      T t = b[i];
#pragma unroll
      for (int k = 0; k < i; ++k) t -= (T)L[i * m + k] * y[k];
      y[i] = t * (T)L[i * m + i];
    }
#pragma unroll
    for (int i = m - 1; i >= 0; --i) {
      T t = y[i];
#pragma unroll
      for (int k = i + 1; k < m; ++k) t -= (T)L[k * m + i] * x[k];
      x[i] = t * (T)L[i * m + i];
    }
  }

  // gain column c (c < n: K[:, c] from -Q_ux[:, c]; c == n: k from -Q_u)
  TO_DEV static void gain_col(int c, int refine, const R* Qux, const R* Qu, const double* Quu, const R* Quf,
                              const double* L, const R* Lf, double mu, R* K, R* kf) {
    R out[m];
    if (sizeof(R) == sizeof(double)) {
      double b[m], x[m];
#pragma unroll
      for (int i = 0; i < m; ++i) b[i] = -(double)(c < n ? Qux[i * n + c] : Qu[i]);
      chol_apply<double, double>(L, b, x);
#pragma unroll
      for (int i = 0; i < m; ++i) out[i] = (R)x[i];
    } else {
      // float32 triangular solves with the rounded factor, then one
      // refinement step on the residual b - (Q_uu + mu I) x.  refine = 1
      // forms it in float-float: Q_uu's entries and x are float32, so every
      // product is exact as a (p, e) pair from one FMA and the sum is
      // compensated (about 48 significant bits, float32 pipe only);
      // refine = 2 forms it in native float64.
      float b[m], x[m];
#pragma unroll
      for (int i = 0; i < m; ++i) b[i] = -(float)(c < n ? Qux[i * n + c] : Qu[i]);
      chol_apply<float, R>(Lf, b, x);
      if (refine) {
        float r[m], d[m];
        if (refine == 2) {
#pragma unroll
          for (int i = 0; i < m; ++i) {
            double t = (double)b[i] - mu * (double)x[i];
#pragma unroll
            for (int k = 0; k < m; ++k) t = fma(-Quu[i * m + k], (double)x[k], t);
            r[i] = (float)t;
          }
        } else {
          const float muf = (float)mu;
#pragma unroll
          for (int i = 0; i < m; ++i) {
            Acc<float> t;
            t.add(b[i]);
            if (muf != 0.f) {
              const float p = muf * x[i];
              t.add(-p);
              t.add(-fmaf(muf, x[i], -p));
            }
#pragma unroll
            for (int k = 0; k < m; ++k) {
              const float q = (float)Quf[i * m + k];
              const float p = q * x[k];
              t.add(-p);
              t.add(-fmaf(q, x[k], -p));
            }
            r[i] = t.hi + t.lo;
          }
        }
        chol_apply<float, R>(Lf, r, d);
#pragma unroll
        for (int i = 0; i < m; ++i) x[i] += d[i];
      }
#pragma unroll
      for (int i = 0; i < m; ++i) out[i] = (R)x[i];
    }
    if (c < n) {
#pragma unroll
      for (int i = 0; i < m; ++i) K[i * n + c] = out[i];
    } else {
#pragma unroll
      for (int i = 0; i < m; ++i) kf[i] = out[i];
    }
  }

  TO_DEV static void gain_column(W& w, int c, int refine) {
    gain_col(c, refine, w.Qux, w.Qu, w.Quu, w.Quf, w.L, w.Lf, w.mu, w.K, w.kf);
  }

  // e-th entry (row-major) of the upper triangle of an n x n matrix -> (i, j)
  TO_DEV static void unrank_upper(int e, int& i, int& j) {
    constexpr int NT = n * (n + 1) / 2;
    const int eb = NT - 1 - e;                                   // index counted from the end
    const int rb = (int)((__fsqrt_rn((float)(8 * eb + 1)) - 1.0f) * 0.5f);   // row counted from the bottom
    i = n - 1 - rb;
    j = n - 1 - (eb - rb * (rb + 1) / 2);
  }

  // the same for small n on the integer pipe: walk the rows (no square root)
  TO_DEV static void unrank_upper_small(int e, int& i, int& j) {
    int r = e, row = 0;
#pragma unroll
    for (int t = 0; t < n - 1; ++t) {
      const bool next = r >= n - row;
      r = next ? r - (n - row) : r;
      row = next ? row + 1 : row;
    }
    i = row;
    j = row + r;
  }

  // ------------------------------------------------------------------------
  // float64 Cholesky of Q (+ shift I when kShift) under the pivot test
  // d_j > delta, with every branch folded: each lane of a group runs it on the
  // group's Q_uu (a float64 warp instruction occupies the FP64 pipe for the
  // same time whatever lanes are active, so the copies cost nothing extra and
  // no lane diverges), and the caller can interleave it with float32 work.
  // Returns true when every pivot passed the test and, with kSeeded (the
  // reciprocal pivot roots from rsqrt_newton), lies in the normal float32
  // range; otherwise the caller redoes the factor on the guarded path, which
  // decides exactly as before.  The diagonal of L holds 1 / L_jj.
  // ------------------------------------------------------------------------
  template <bool kSeeded, bool kShift>
  TO_DEV static bool chol_nb(const double (&Q)[m * m], double shift, double delta, double (&L)[m * m]) {
    bool ok = true;
#pragma unroll
    for (int j = 0; j < m; ++j) {
      double s = Q[j * m + j];
      if (kShift) s += shift;
#pragma unroll
      for (int k = 0; k < j; ++k) s -= L[j * m + k] * L[j * m + k];
      ok = ok & dgt_nonneg(s, delta);
      if (kSeeded) ok = ok & (__double_as_longlong(s) >= 0x3810000000000000LL);   // s >= FLT_MIN
      const double r = kSeeded ? rsqrt_newton(s) : rsqrt(s);
      L[j * m + j] = r;
#pragma unroll
      for (int i = j + 1; i < m; ++i) {
        double t = Q[i * m + j];
#pragma unroll
        for (int k = 0; k < j; ++k) t -= L[i * m + k] * L[j * m + k];
        L[i * m + j] = t * r;
      }
    }
    return ok;
  }

  // The factor of Q_uu in float32 (reciprocal pivots on the diagonal), from
  // the float32 Q_uu; true when every pivot exceeds 2^-10 of the largest
  // diagonal magnitude (and FLT_MIN).  The float32 pivots are those of Q_uu
  // + dQ with |dQ| <= (m + 1) 2^-24 max|diag| entrywise (Higham 2002,
  // Thm. 10.3), so a pivot at the threshold is ~2^14 / (m + 1) times that
  // perturbation, and nine orders of magnitude above the float64 test's
  // 1e-12; a NaN or infinite entry reaches a pivot and fails the test.
  TO_DEV static bool chol_f32(const R* Q, R mxr, float (&L)[m * m]) {
    const float tau = fmaxf(0x1p-10f * (float)mxr, FLT_MIN);
    bool ok = true;
#pragma unroll
    for (int j = 0; j < m; ++j) {
      float s = (float)Q[j * m + j];
#pragma unroll
      for (int k = 0; k < j; ++k) s -= L[j * m + k] * L[j * m + k];
      ok = ok & (s > tau);
      const float r = rsqrtf(s);
      L[j * m + j] = r;
#pragma unroll
      for (int i = j + 1; i < m; ++i) {
        float t = (float)Q[i * m + j];
#pragma unroll
        for (int k = 0; k < j; ++k) t -= L[i * m + k] * L[j * m + k];
        L[i * m + j] = t * r;
      }
    }
    return ok;
  }

  // ------------------------------------------------------------------------
  // One backward knot for sub-warp groups (2 <= G < 32), split by columns.
  //   1. Q_uu and Q_u: lane c forms column c of V B in registers, then
  //      column c of Q_uu = l_uu + B^T (V B).
  //   2. Every lane factors the group's Q_uu (in float32 when its pivots
  //      clear chol_f32's test, else in float64: chol_nb) while lane
  //      j forms column j of V A in registers and from it column j of Q_xx,
  //      of Q_ux and Q_x[j]: no barrier between the products, no branch, and
  //      no lane waits for a leader's float64 chain.  Q_xx goes to the V A
  //      buffer, so V stays readable by every lane meanwhile.
  //   3. Gain columns from each lane's own copy of the factor.
  //   4. V_xx <- sym(Q_xx + Q_ux^T K), V_x <- Q_x + Q_ux^T k, gains to memory.
  // The arithmetic (and its summation order) is that of the single-pass
  // form; lanes past the last column recompute the last one and store
  // nothing, so the code of each phase is straight-line.
  // ------------------------------------------------------------------------
  TO_DEV static int backward_cols(const Group<G>& g, W& w, bool act, const SolveArgs& a, R* grec, double* vxrec,
                                  double mu_lm, bool timer, long long& tlast) {
    static_assert(G >= 2 && G < 32, "sub-warp groups");
    constexpr int NT = n * (n + 1) / 2;
    R* QX = w.VA;                                         // Q_xx, full (mirrored)
    // the float64 copy of Q_uu is read only by the float64 factors (FP64
    // mode, the Levenberg-Marquardt variant) and by the native float64
    // refinement residual; the fallback of the float32 factor converts Q_uu
    // itself
    const bool q64 = sizeof(R) == 8 || a.lm || a.refine == 2;
    // 1. Q_uu (R copy, and the float64 copy when q64) and Q_u
#pragma unroll
    for (int s = 0; s < (m + G - 1) / G; ++s) {
      const int c0 = g.lane + s * G;
      const bool st = act && c0 < m;
      const int c = c0 < m ? c0 : m - 1;
      R vb[n];
#pragma unroll
      for (int i = 0; i < n; ++i) {
        R t = 0;
#pragma unroll
        for (int r = 0; r < n; ++r) t += w.V[i * n + r] * w.Bm[r * m + c];
        vb[i] = t;
      }
#pragma unroll
      for (int i = 0; i < m; ++i) {
        R t = w.luu[i * m + c];
#pragma unroll
        for (int r = 0; r < n; ++r) t += w.Bm[r * m + i] * vb[r];
        if (st) {
          if (q64) w.Quu[i * m + c] = (double)t;
          w.Quf[i * m + c] = t;
        }
      }
      R t = w.lu[c];
#pragma unroll
      for (int r = 0; r < n; ++r) t += w.Bm[r * m + c] * w.v[r];
      if (st) w.Qu[c] = t;
    }
    g.sync();
    TO_TICK(2);
    // 2. the factor on every lane, interleaved with the column products
    double Lr[m * m];
    float L32[m * m];
    double mu = 0;
    bool ok;
    bool f32 = false;            // the float32 factor L32 was accepted
    constexpr bool kSeed = sizeof(R) == 4;
    {
      double Q[m * m];
      R mxr = R(0);
#pragma unroll
      for (int i = 0; i < m; ++i) mxr = max_abs(mxr, w.Quf[i * m + i]);
      auto load_q64 = [&]() {
#pragma unroll
        for (int i = 0; i < m; ++i)
#pragma unroll
          for (int j = 0; j <= i; ++j) Q[i * m + j] = w.Quu[i * m + j];
      };
      auto cols = [&]() {
#pragma unroll
        for (int s = 0; s < (n + G - 1) / G; ++s) {
          const int j0 = g.lane + s * G;
          const bool st = act && j0 < n;
          const int j = j0 < n ? j0 : n - 1;
          R va[n];
#pragma unroll
          for (int i = 0; i < n; ++i) {
            R t = 0;
#pragma unroll
            for (int r = 0; r < n; ++r) t += w.V[i * n + r] * w.A[r * n + j];
            va[i] = t;
          }
#pragma unroll
          for (int i = 0; i < n; ++i) {
            R t = w.lxx[i * n + j];
#pragma unroll
            for (int r = 0; r < n; ++r) t += w.A[r * n + i] * va[r];
            if (st) QX[i * n + j] = t;                    // the whole column: Q_xx as the oracle forms it
          }
#pragma unroll
          for (int i = 0; i < m; ++i) {
            R t = 0;
#pragma unroll
            for (int r = 0; r < n; ++r) t += w.Bm[r * m + i] * va[r];
            if (st) w.Qux[i * n + j] = t;                 // Q_ux (l_ux = 0)
          }
          R t = w.lx[j];
#pragma unroll
          for (int r = 0; r < n; ++r) t += w.A[r * n + j] * w.v[r];
          if (st) w.Qx[j] = t;
        }
      };
      if (a.lm) {
        load_q64();
        const double mx = (double)mxr;
        mu = mu_lm;
        ok = chol_nb<kSeed, true>(Q, mu, 1e-12 * (mx + mu), Lr);
        cols();
        ok = ok & (mxr == mxr) & (mxr <= R(3.0e38));
      } else if constexpr (sizeof(R) == 4) {
        // mixed, clipped Hessians: float32 when every pivot is well clear of
        // zero; any other Q_uu goes to the float64 factor and its guard below
        ok = chol_f32(w.Quf, mxr, L32);
        cols();
        ok = ok & (mxr > R(0)) & (mxr <= R(3.0e38));
        f32 = true;
      } else {
        load_q64();
        const double mx = (double)mxr;
        ok = chol_nb<kSeed, false>(Q, 0.0, 1e-12 * mx, Lr);
        cols();
        ok = ok & (mxr > R(0)) & (mxr <= R(3.0e38));
      }
    }
    // the guarded path (a failed pivot test, a pivot outside the seed's
    // range, or a float32 factor not accepted): the float64 factor with the
    // shift schedule, as in factor()
    R Lf[m * m];
    int flag = 0;
    if (!ok && act) {          // (an idle group's stale Q_uu takes no guarded retries)
      double Qd[m * m];
#pragma unroll
      for (int i = 0; i < m * m; ++i) Qd[i] = q64 ? w.Quu[i] : (double)w.Quf[i];
      flag = factor(Qd, w.Quf, a.lm, mu_lm, Lr, Lf, mu);
    } else if (f32) {
#pragma unroll
      for (int i = 0; i < m; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) Lf[i * m + j] = (R)L32[i * m + j];
    } else {
#pragma unroll
      for (int i = 0; i < m; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) Lf[i * m + j] = (R)Lr[i * m + j];
    }
    g.sync();
    // 3. gain columns (c < n: K[:, c]; c == n: k)
    if (act && flag < 2)
      for (int c = g.lane; c <= n; c += G) gain_col(c, a.refine, w.Qux, w.Qu, w.Quu, w.Quf, Lr, Lf, mu, w.K, w.kf);
    g.sync();
    TO_TICK(3);
    // 4. lane j: column j of V_xx <- sym(Q_xx + Q_ux^T K) and V_x[j] <-
    //    Q_x[j] + Q_ux[:, j]^T k (Q_xx is read from its own buffer, so V is
    //    written in place without a barrier); entry (i, j) and entry (j, i)
    //    take the same operations in the same order, so V stays exactly
    //    symmetric.  The gain record goes to memory in 16-byte vectors.
#pragma unroll
    for (int s = 0; s < (n + G - 1) / G; ++s) {
      const int j0 = g.lane + s * G;
      const bool st = act && j0 < n;
      const int j = j0 < n ? j0 : n - 1;
#pragma unroll
      for (int i = 0; i < n; ++i) {
        R sij = QX[i * n + j], sji = QX[j * n + i];
#pragma unroll
        for (int r = 0; r < m; ++r) {
          sij += w.Qux[r * n + i] * w.K[r * n + j];
          sji += w.Qux[r * n + j] * w.K[r * n + i];
        }
        const R t = R(0.5) * (sij + sji);                  // a + b == b + a: (j, i) gets the same bits
        if (st) w.V[i * n + j] = t;
      }
      R t = w.Qx[j];
#pragma unroll
      for (int r = 0; r < m; ++r) t += w.Qux[r * n + j] * w.kf[r];
      if (st) {
        w.v[j] = t;
        if (vxrec) vxrec[j] = (double)t;
      }
    }
    {
      constexpr int kV = 16 / (int)sizeof(R), NV = GS / kV;   // K then k, adjacent in W and in memory; then padding
      static_assert(GS % kV == 0, "gain record in whole vectors");
#pragma unroll
      for (int s = 0; s < (NV + G - 1) / G; ++s) {
        const int v = g.lane + s * G;
        if (act && v < NV) {
          R o[kV];
#pragma unroll
          for (int q = 0; q < kV; ++q) {
            const int f = v * kV + q;
            o[q] = f < m * (n + 1) ? w.K[f] : R(0);
          }
          st16(grec + v * kV, o);
        }
      }
    }
    g.sync();
    TO_TICK(4);
    return act ? flag : 0;
  }

  // ------------------------------------------------------------------------
  // one knot of the backward pass (all syncs unconditional, work predicated).
  // The knot's record is in pb (prefetched); the record of the knot D
  // earlier (trec_next; stored blocks: kprim) is fetched into pb while this
  // one computes (act_next: that knot exists).  Returns the Cholesky flag.
  // ------------------------------------------------------------------------
  TO_DEV static int backward_knot(const Params& P, const Group<G>& g, W& w, bool act, bool act_next,
                                  const SolveArgs& a, R (&pb)[PB], const R* trec_next, R* grec, double* vxrec,
                                  double mu_lm, bool timer, long long& tlast, const R* kprim) {
    const R eps = (R)a.eps;
    if constexpr (!Sys::kStoredDerivs) {   // x_k, u_k feed the derivative step (stored blocks need neither)
      if (act) {
#pragma unroll
        for (int s = 0; s < PB; ++s) {
          const int e = g.lane + s * G;
          if (e < n + m) w.xk[e] = pb[s];
        }
      }
      g.sync();
      if (act_next) {
#pragma unroll
        for (int s = 0; s < PB; ++s) {
          const int e = g.lane + s * G;
          if (e < n + m) pb[s] = trec_next[e];
        }
      }
    }
    // dynamics Jacobians and clipped running-cost derivatives
    // (a system whose derivative step holds group barriers has groups of a
    // whole warp or CTA, so act is uniform over every barrier's scope)
    if constexpr (Sys::kStoredDerivs) {
      // the knot's stored block (A, B, l_xx, l_x, l_uu, l_u), prefetched into
      // pb D knots earlier; then the block of the knot D further on is
      // fetched into pb (kprim: that block)
      constexpr int DS = Sys::kDerivStride;
      if (act) {
#pragma unroll
        for (int s = 0; s < PB; ++s) {
          const int e = g.lane + s * G;
          const R v = pb[s];
          if (e >= DS) continue;
          if (e < n * n) w.A[e] = v;
          else if (e < n * n + n * m) w.Bm[e - n * n] = v;
          else if (e < 2 * n * n + n * m) w.lxx[e - n * n - n * m] = v;
          else if (e < 2 * n * n + n * m + n) w.lx[e - 2 * n * n - n * m] = v;
          else if (e < 2 * n * n + n * m + n + m * m) w.luu[e - 2 * n * n - n * m - n] = v;
          else w.lu[e - 2 * n * n - n * m - n - m * m] = v;
        }
      }
      if (act_next) {
#pragma unroll
        for (int s = 0; s < PB; ++s) {
          const int e = g.lane + s * G;
          if (e < DS) pb[s] = kprim[e];
        }
      }
    } else if (act) {
      if constexpr (Sys::kKnotParallel)
        Sys::template derivs_staged<R, G>(P, g, w.xk, w.uk, eps, w.A, w.Bm, w.lxx, w.lx, w.luu, w.lu, w.sx, kprim);
      else
        Sys::template derivs<R, G>(P, g, w.xk, w.uk, eps, w.A, w.Bm, w.lxx, w.lx, w.luu, w.lu, w.sx);
    }
    g.sync();
    TO_TICK(1);
    if constexpr (G >= 2 && G < 32) {
      return backward_cols(g, w, act, a, grec, vxrec, mu_lm, timer, tlast);
    } else {
    constexpr int NT = n * (n + 1) / 2;
      // V A and V B
      if (act)
        for (int e = g.lane; e < n * n + n * m; e += G) {
          if (e < n * n) {
            const int i = e / n, j = e % n;
            R s = 0;
#pragma unroll 6
            for (int r = 0; r < n; ++r) s += w.V[i * n + r] * w.A[r * n + j];
            w.VA[e] = s;
          } else {
            const int f = e - n * n, i = f / m, j = f % m;
            R s = 0;
#pragma unroll 6
            for (int r = 0; r < n; ++r) s += w.V[i * n + r] * w.Bm[r * m + j];
            w.VB[f] = s;
          }
        }
      g.sync();
      // Q terms; Q_xx (upper triangle, mirrored) overwrites V
      if (act)
        for (int e = g.lane; e < NT + m * n + m * m + n + m; e += G) {
          if (e < NT) {
            // unrank e -> (i, j), i <= j, row-major over the upper triangle
            int i, j;
            unrank_upper(e, i, j);
            R s = w.lxx[i * n + j];
#pragma unroll 6
            for (int r = 0; r < n; ++r) s += w.A[r * n + i] * w.VA[r * n + j];
            w.V[i * n + j] = s;
            w.V[j * n + i] = s;
          } else if (e < NT + m * n) {
            const int f = e - NT, i = f / n, j = f % n;
            R s = 0;
#pragma unroll 6
            for (int r = 0; r < n; ++r) s += w.Bm[r * m + i] * w.VA[r * n + j];
            w.Qux[f] = s;                                 // Q_ux (l_ux = 0)
          } else if (e < NT + m * n + m * m) {
            const int f = e - NT - m * n, i = f / m, j = f % m;
            R s = w.luu[f];
#pragma unroll 6
            for (int r = 0; r < n; ++r) s += w.Bm[r * m + i] * w.VB[r * m + j];
            w.Quu[f] = (double)s;                         // Q_uu
            w.Quf[f] = s;
          } else if (e < NT + m * n + m * m + n) {
            const int i = e - NT - m * n - m * m;
            R s = w.lx[i];
#pragma unroll 6
            for (int r = 0; r < n; ++r) s += w.A[r * n + i] * w.v[r];
            w.Qx[i] = s;
          } else {
            const int i = e - NT - m * n - m * m - n;
            R s = w.lu[i];
#pragma unroll 6
            for (int r = 0; r < n; ++r) s += w.Bm[r * m + i] * w.v[r];
            w.Qu[i] = s;
          }
        }
      g.sync();
      TO_TICK(2);
      if (act && g.lane < 32) chol_warp(w, a.lm, mu_lm, g.lane);   // act is uniform over the group
      g.sync();
    const int flag = act ? w.flag : 0;
    if (act && flag < 2)
      for (int c = g.lane; c <= n; c += G) gain_column(w, c, a.refine);
    g.sync();
    TO_TICK(3);
    // V_xx <- sym(Q_xx + Q_ux^T K) in place (one lane per unordered pair),
    // V_x <- Q_x + Q_ux^T k, gains to memory
    if (act)
      for (int e = g.lane; e < NT + n + GS; e += G) {
        if (e < NT) {
          int i, j;
          unrank_upper(e, i, j);
          R sij = w.V[i * n + j], sji = w.V[j * n + i];
#pragma unroll
          for (int r = 0; r < m; ++r) {
            sij += w.Qux[r * n + i] * w.K[r * n + j];
            sji += w.Qux[r * n + j] * w.K[r * n + i];
          }
          const R s = R(0.5) * (sij + sji);
          w.V[i * n + j] = s;
          w.V[j * n + i] = s;
        } else if (e < NT + n) {
          const int i = e - NT;
          R s = w.Qx[i];
#pragma unroll
          for (int r = 0; r < m; ++r) s += w.Qux[r * n + i] * w.kf[r];
          w.v[i] = s;
          if (vxrec) vxrec[i] = (double)s;
        } else {
          const int f = e - NT - n;     // K then k, adjacent in W and in memory; then the padding
          grec[f] = f < m * (n + 1) ? w.K[f] : R(0);
        }
      }
    g.sync();
    TO_TICK(4);
    return flag;
    }
  }

  // ------------------------------------------------------------------------
  // The backward pass of a single-lane group (G == 1).  One thread owns the
  // instance and every per-knot matrix stays in registers (each loop over the
  // compile-time dimensions unrolls), so there is no barrier and no
  // shared-memory traffic, and each float64 instruction of the Q_uu Cholesky
  // serves the 32 instances of the warp.  Same steps and summation order as
  // backward_knot; the pass stops at the first knot whose factor fails (the
  // instance is then released, or redone with a larger mu).
  // ------------------------------------------------------------------------
  TO_DEV static void backward_lane(const Params& P, const SolveArgs& a, R* traj, R* gains, long long base, int T,
                                   int cur, double mu_lm, int& flags, bool& bad, bool& need_mu, bool timer,
                                   long long& tlast) {
    const R eps = (R)a.eps;
    double* vx = (a.vx && a.want_vx) ? a.vx : nullptr;
    R V[n * n], v[n], nx[RS];
    ld_vec<RS>(rec(a, traj, base, T, cur), nx);
    Sys::terminal_derivs(P, nx, eps, V, v);
    if (vx)
#pragma unroll
      for (int i = 0; i < n; ++i) vx_at(a, vx, base + T)[i] = (double)v[i];
    ld_vec<RS>(rec(a, traj, base, T - 1, cur), nx);
    for (int k = T - 1; k >= 0; --k) {
      R x[n], u[m];
#pragma unroll
      for (int i = 0; i < n; ++i) x[i] = nx[i];
#pragma unroll
      for (int i = 0; i < m; ++i) u[i] = nx[n + i];
      if (k >= 1) ld_vec<RS>(rec(a, traj, base, k - 1, cur), nx);
      R A[n * n], Bm[n * m], lxx[n * n], lx[n], luu[m * m], lu[m];
      Sys::derivs_lane(P, x, u, eps, A, Bm, lxx, lx, luu, lu);
      TO_TICK(1);
      // Q_xx (upper triangle, mirrored) and Q_ux from the columns of V A,
      // Q_uu from the columns of V B
      R Qxx[n * n], Qux[m * n], Quf[m * m], Qx[n], Qu[m];
#pragma unroll
      for (int j = 0; j < n; ++j) {
        R c[n];
#pragma unroll
        for (int i = 0; i < n; ++i) {
          R t = 0;
#pragma unroll
          for (int r = 0; r < n; ++r) t += V[i * n + r] * A[r * n + j];
          c[i] = t;
        }
#pragma unroll
        for (int i = 0; i <= j; ++i) {
          R t = lxx[i * n + j];
#pragma unroll
          for (int r = 0; r < n; ++r) t += A[r * n + i] * c[r];
          Qxx[i * n + j] = t;
          Qxx[j * n + i] = t;
        }
#pragma unroll
        for (int i = 0; i < m; ++i) {
          R t = 0;
#pragma unroll
          for (int r = 0; r < n; ++r) t += Bm[r * m + i] * c[r];
          Qux[i * n + j] = t;                     // Q_ux (l_ux = 0)
        }
      }
#pragma unroll
      for (int j = 0; j < m; ++j) {
        R c[n];
#pragma unroll
        for (int i = 0; i < n; ++i) {
          R t = 0;
#pragma unroll
          for (int r = 0; r < n; ++r) t += V[i * n + r] * Bm[r * m + j];
          c[i] = t;
        }
#pragma unroll
        for (int i = 0; i < m; ++i) {
          R t = luu[i * m + j];
#pragma unroll
          for (int r = 0; r < n; ++r) t += Bm[r * m + i] * c[r];
          Quf[i * m + j] = t;
        }
      }
#pragma unroll
      for (int i = 0; i < n; ++i) {
        R t = lx[i];
#pragma unroll
        for (int r = 0; r < n; ++r) t += A[r * n + i] * v[r];
        Qx[i] = t;
      }
#pragma unroll
      for (int i = 0; i < m; ++i) {
        R t = lu[i];
#pragma unroll
        for (int r = 0; r < n; ++r) t += Bm[r * m + i] * v[r];
        Qu[i] = t;
      }
      TO_TICK(2);
      double Q[m * m], L[m * m], mu;
      R Lf[m * m];
#pragma unroll
      for (int i = 0; i < m * m; ++i) Q[i] = (double)Quf[i];
      const int f = factor(Q, Quf, a.lm, mu_lm, L, Lf, mu);
      if (f == 1) flags |= ST_FLAG_REG;
      if (a.lm) {
        if (f >= 2) { need_mu = true; break; }
      } else if (f == 2) {
        bad = true;
        break;
      }
      R g[GS];                                    // gain record: K, k, padding
#pragma unroll
      for (int c = 0; c <= n; ++c) gain_col(c, a.refine, Qux, Qu, Q, Quf, L, Lf, mu, g, g + m * n);
#pragma unroll
      for (int i = m * (n + 1); i < GS; ++i) g[i] = R(0);
      TO_TICK(3);
      // V_xx <- sym(Q_xx + Q_ux^T K), V_x <- Q_x + Q_ux^T k, gains to memory
#pragma unroll
      for (int i = 0; i < n; ++i)
#pragma unroll
        for (int j = i; j < n; ++j) {
          R sij = Qxx[i * n + j], sji = Qxx[j * n + i];
#pragma unroll
          for (int r = 0; r < m; ++r) {
            sij += Qux[r * n + i] * g[r * n + j];
            sji += Qux[r * n + j] * g[r * n + i];
          }
          const R t = R(0.5) * (sij + sji);
          V[i * n + j] = t;
          V[j * n + i] = t;
        }
#pragma unroll
      for (int i = 0; i < n; ++i) {
        R t = Qx[i];
#pragma unroll
        for (int r = 0; r < m; ++r) t += Qux[r * n + i] * g[m * n + r];
        v[i] = t;
        if (vx) vx_at(a, vx, base + k)[i] = (double)t;
      }
      st_vec<GS>(grec_at(a, gains, base + k), g);
      TO_TICK(4);
    }
  }

  // forward record (x_k, u_k, K_k, k_k, x_lo) element e of the lane's prefetch slot
  TO_DEV static R load_fwd(const R* trec, const R* grec, int e) {
    constexpr int NG = m * (n + 1);
    return e < n + m ? trec[e] : (e < n + m + NG ? grec[e - (n + m)] : trec[e - NG]);
  }
  TO_DEV static void prefetch_fwd(const Group<G>& g, R (&pf)[PF], const R* trec, const R* grec) {
#pragma unroll
    for (int s = 0; s < PF; ++s) {
      const int e = g.lane + s * G;
      if (e < NF) pf[s] = load_fwd(trec, grec, e);
    }
  }
  TO_DEV static void store_fwd(const Group<G>& g, W& w, const R (&pf)[PF]) {
#pragma unroll
    for (int s = 0; s < PF; ++s) {
      const int e = g.lane + s * G;
      if (e < n + m) w.xk[e] = pf[s];
      else if (e < n + m + m * (n + 1)) w.K[e - (n + m)] = pf[s];
      else if (e < NF) w.xl[e - (n + m + m * (n + 1))] = pf[s];
    }
  }

  // u^ = u + alpha k + K (x^ - x), the difference taken on (hi, lo) pairs
  TO_DEV static void policy(const W& w, R alpha, const R* xh, const R* xlo, R* uh) {
    R dx[n];
#pragma unroll
    for (int j = 0; j < n; ++j) dx[j] = kLo ? (xh[j] - w.xk[j]) + (xlo[j] - w.xl[j]) : xh[j] - w.xk[j];
#pragma unroll
    for (int i = 0; i < m; ++i) {
      R s = w.uk[i] + alpha * w.kf[i];
#pragma unroll
      for (int j = 0; j < n; ++j) s += w.K[i * n + j] * dx[j];
      uh[i] = s;
    }
  }

  // the same from a record and gain record held in registers (single lane)
  TO_DEV static void policy_regs(const R* cr, const R* cg, R alpha, const R* xh, const R* xlo, R* uh) {
    R dx[n];
#pragma unroll
    for (int j = 0; j < n; ++j) dx[j] = kLo ? (xh[j] - cr[j]) + (xlo[j] - cr[n + m + j]) : xh[j] - cr[j];
#pragma unroll
    for (int i = 0; i < m; ++i) {
      R s = cr[n + i] + alpha * cg[m * n + i];
#pragma unroll
      for (int j = 0; j < n; ++j) s += cg[i * n + j] * dx[j];
      uh[i] = s;
    }
  }

  // knot record [x | u | x_lo | 0...] written with 16-byte stores
  TO_DEV static void put_record(R* r, const R* xh, const R* uh, const R* xlo) {
    R o[RS];
#pragma unroll
    for (int i = 0; i < n; ++i) o[i] = xh[i];
#pragma unroll
    for (int i = 0; i < m; ++i) o[n + i] = uh[i];
#pragma unroll
    for (int i = 0; i < kLo; ++i) o[n + m + i] = xlo[i];
#pragma unroll
    for (int i = n + m + kLo; i < RS; ++i) o[i] = R(0);
    st_vec<RS>(r, o);
  }

  // actor policy u = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3 (Sec. II: the
  // actor's rollout is the TO warm start), x in w.xk, u to w.uk.  The host
  // stores every weight matrix transposed (input-major), so lanes reading
  // consecutive outputs of one input read consecutive words.  The hidden
  // activations use the V A buffer, free during forward rounds.
  static constexpr int kHidden = 256;
  TO_DEV static void actor_mlp(const Group<G>& g, W& w, bool act, const float* aw) {
    static_assert(!Sys::kActor || n * n >= 2 * kHidden, "hidden activations must fit the scratch buffer");
    R* h1 = w.VA;
    R* h2 = w.VA + kHidden;
    const float* W1 = aw;
    const float* b1 = W1 + n * kHidden;
    const float* W2 = b1 + kHidden;
    const float* b2 = W2 + kHidden * kHidden;
    const float* W3 = b2 + kHidden;
    const float* b3 = W3 + kHidden * m;
    if (act)
      for (int j = g.lane; j < kHidden; j += G) {
        R s = (R)b1[j];
        for (int i = 0; i < n; ++i) s += (R)W1[i * kHidden + j] * w.xk[i];
        h1[j] = tanh(s);
      }
    g.sync();
    if (act)
      for (int j = g.lane; j < kHidden; j += G) {
        R s = (R)b2[j];
#pragma unroll 8
        for (int i = 0; i < kHidden; ++i) s += (R)W2[i * kHidden + j] * h1[i];
        h2[j] = tanh(s);
      }
    g.sync();
    if (act)
      for (int j = g.lane; j < m; j += G) {
        R s = (R)b3[j];
#pragma unroll 8
        for (int i = 0; i < kHidden; ++i) s += (R)W3[i * m + j] * h2[i];
        w.uk[j] = s;
      }
    g.sync();
  }

  TO_DEV static R alpha_of(const SolveArgs& a, int j) {
    return sizeof(R) == sizeof(double) ? (R)a.alpha_d[j] : (R)a.alpha_f[j];
  }

  // knot record k of trajectory slot s of the instance whose first record is base
  TO_DEV static R* rec(const SolveArgs& a, R* traj, long long base, int k, int s) {
    const long long kn = ck(a, base + k, a.knots_cap, CK_RECORD);
    return traj + (kn * NS + ck(a, s, NS, CK_SLOT)) * RS;
  }
  // the gain record of knot kn, the V_x row of knot kn, the derivative scratch of knot kn
  TO_DEV static R* grec_at(const SolveArgs& a, R* gains, long long kn) {
    return gains + ck(a, kn, a.knots_cap, CK_GAINS) * GS;
  }
  TO_DEV static double* vx_at(const SolveArgs& a, double* vx, long long kn) {
    return vx + ck(a, kn, a.knots_cap, CK_VX) * n;
  }
  TO_DEV static R* dscr_at(const SolveArgs& a, long long kn) {
    return reinterpret_cast<R*>(a.dscr) + ck(a, kn, a.knots_cap, CK_DSCR) * a.kscr;
  }

  // ------------------------------------------------------------------------
  // the kernel body
  // ------------------------------------------------------------------------
  TO_DEV static void run(const SolveArgs& a, unsigned char* smem) {
    const Params& P = *reinterpret_cast<const Params*>(smem);
    {
      const int words = (int)(sizeof(Params) / sizeof(int));
      for (int i = threadIdx.x; i < words; i += blockDim.x)
        reinterpret_cast<int*>(smem)[i] = reinterpret_cast<const int*>(a.params)[i];
    }
    __syncthreads();
    if (*a.err) return;
    const Group<G> g;
    W* works = reinterpret_cast<W*>(smem + ((sizeof(Params) + 15) / 16) * 16);
    W& w = works[g.index];
    R* traj = reinterpret_cast<R*>(a.traj);
    R* gains = reinterpret_cast<R*>(a.gains);
    const bool forced_mode = a.forced != nullptr;
    const bool timer = (G <= 32) ? ((threadIdx.x & 31) == 0) : (threadIdx.x == 0);
    long long tlast = a.prof ? clock64() : 0;

    // per-group state (identical in the group's lanes); cur is the slot that
    // holds the current iterate
    int mode = M_IDLE, inst = 0, T = 0, iter = 0, status = 0, flags = 0, cur = 0;
    double J = 0;
    long long base = 0;
    int sq = 0;          // serving: ring index of the request being solved
    double mu_lm = kMu0;  // Levenberg-Marquardt variant: the instance's mu
    int idle = 0;        // serving: consecutive polls with every group idle

    while (true) {
      // ---- refill idle groups: the batch's queue, or the serving ring
      {
        const bool need = (mode == M_IDLE);
        int q = -1;
        if (need && g.lane == 0) {
          if (a.serve.ring) {
            // claim the next published request, if any (never waits here)
            // a closing launch claims nothing more; the host has launched its successor
            if (!*reinterpret_cast<volatile int*>(a.serve.ctl + 1)) {
              const unsigned h = *reinterpret_cast<volatile unsigned*>(a.serve.head);
              const unsigned t = *a.serve.tail;
              if (h < t && atomicCAS(a.serve.head, h, h + 1) == h) {
                q = (int)h;
                atomicAdd(a.serve.ctl, 1);
              }
            }
          } else {
            const int qq = atomicAdd(a.queue, 1);
            q = qq < a.B ? qq : -2;
          }
        }
        q = g.bcast(q, &w.sel);
        if (need) {
          if (q >= 0 && a.serve.ring) {
            __threadfence_system();
            const volatile ServeDesc& d = a.serve.ring[q % a.serve.ring_size];
            inst = (int)ck(a, d.seat, a.B, CK_SEAT);
            T = d.T;
            if (!ck_ok(a, T - 1, a.T_max, CK_HORIZON)) T = 1;
            base = (long long)inst * (a.T_max + 1);
            sq = q;
            if (g.lane == 0) a.serve.seat_T[inst] = T;
            mode = M_NEW; iter = 0; status = 0; flags = 0; J = 0; cur = 0; mu_lm = kMu0;
          } else if (q >= 0) {
            inst = (int)ck(a, a.order[q], a.B, CK_ORDER);
            T = a.T[inst];
            if (!ck_ok(a, T - 1, a.T_max, CK_HORIZON)) T = 1;
            base = a.toff[inst];
            mode = M_NEW; iter = 0; status = 0; flags = 0; J = 0; cur = 0; mu_lm = kMu0;
          } else if (q == -2) {
            mode = M_DRAINED;
          }
        }
      }
      if (a.serve.ring) {
        // every group of this warp (CTA) idle: poll again after a pause.  The
        // launch closes once no group anywhere in it has been solving for
        // idle_polls polls: the latch stops every claim, so the whole launch
        // drains at once and never lingers with a few warps holding it open
        // (the host launches a successor as soon as it sees the latch)
        if (g.uniform_all(mode == M_IDLE)) {
          ++idle;
          int leave = 0;
          if (g.unit_leader()) {
            leave = (*a.serve.stop || *reinterpret_cast<volatile int*>(a.serve.ctl + 1)) ? 1 : 0;
            if (!leave && idle >= a.serve.idle_polls && *reinterpret_cast<volatile int*>(a.serve.ctl) == 0) {
              atomicExch(a.serve.ctl + 1, 1);
              *a.serve.closing = 1;
              leave = 1;
            }
          }
          if (g.unit_bcast(leave, &w.sel)) break;
          __nanosleep(2000);
          continue;
        }
        idle = 0;
      } else if (g.uniform_all(mode == M_DRAINED)) {
        break;
      }
      TO_TICK(0);
      bool release = false;
      bool retry = false;   // Levenberg-Marquardt: redo the backward pass with a larger mu
      // ---- a forced sequence ends with -1
      if (mode == M_RUN && forced_mode && a.forced[(size_t)inst * a.max_iter + ck(a, iter, a.max_iter, CK_FORCED)] < 0) {
        status = ST_MAX_ITER;
        if (a.want_vx) mode = M_FINAL; else release = true;
      }

      // ---- phase A: backward pass along slot cur
      {
        const bool bw = (mode == M_RUN || mode == M_FINAL) && !release;
        bool bad = false, need_mu = false;
        if constexpr (kLane) {
          if (bw) backward_lane(P, a, traj, gains, base, T, cur, mu_lm, flags, bad, need_mu, timer, tlast);
        } else {
        const int kmax = g.uniform_max(bw ? T : 0, &w.sel);
        if (kmax > 0) {
          // the staging ring: knot k's record (or block) sits in slot
          // (kmax - 1 - k) % D, so the knot loop below indexes it statically
          R pb[D][PB];
          auto ring = [&](int k, auto&& f) {
            const int sl = (kmax - 1 - k) % D;
#pragma unroll
            for (int d = 0; d < D; ++d)
              if (d == sl) f(pb[d]);
          };
          if (bw) {
            if (g.lane == 0) {
              const R* r = rec(a, traj, base, T, cur);
              R xT[n];
#pragma unroll
              for (int i = 0; i < n; ++i) xT[i] = r[i];
              Sys::terminal_derivs(P, xT, (R)a.eps, w.V, w.v);
              if (a.vx && a.want_vx)
                for (int i = 0; i < n; ++i) vx_at(a, a.vx, base + T)[i] = (double)w.v[i];
            }
            if constexpr (!Sys::kStoredDerivs) {
#pragma unroll
              for (int i = 0; i < D; ++i) {
                if (T - 1 - i < 0) break;
                const R* r = rec(a, traj, base, T - 1 - i, cur);
                ring(T - 1 - i, [&](R (&b)[PB]) {
#pragma unroll
                  for (int s = 0; s < PB; ++s) {
                    const int e = g.lane + s * G;
                    if (e < n + m) b[s] = r[e];
                  }
                });
              }
            }
          }
          if constexpr (Sys::kStoredDerivs) {
            // every lane: the whole derivative block of its knots, stored
            // (no barrier inside: the groups of a warp may run different T)
            if (bw) {
              const R eps = (R)a.eps;
              // the next knot's record is loaded (16-byte vectors) while this one computes
              R nr[RS];
              if (g.lane < T) ld_vec<RS>(rec(a, traj, base, g.lane, cur), nr);
              for (int k = g.lane; k < T; k += G) {
                R x[n], u[m];
#pragma unroll
                for (int i = 0; i < n; ++i) x[i] = nr[i];
#pragma unroll
                for (int i = 0; i < m; ++i) u[i] = nr[n + i];
                if (k + G < T) ld_vec<RS>(rec(a, traj, base, k + G, cur), nr);
                R d[Sys::kDerivStride];
                Sys::derivs_lane(P, x, u, eps, d, d + n * n, d + n * n + n * m, d + 2 * n * n + n * m,
                                 d + 2 * n * n + n * m + n, d + 2 * n * n + n * m + n + m * m);
                st_vec<Sys::kDerivStride>(dscr_at(a, base + k), d);
              }
            }
          }
          if constexpr (Sys::kKnotParallel) {
            // every lane: the substep primal chains of its knots (bw is uniform over a group of whole warps)
            if (bw)
              for (int k = g.lane; k < T; k += G) {
                const R* r = rec(a, traj, base, k, cur);
                R x[n], u[m];
#pragma unroll
                for (int i = 0; i < n; ++i) x[i] = r[i];
#pragma unroll
                for (int i = 0; i < m; ++i) u[i] = r[n + i];
                Sys::primal_knot(P, x, u, dscr_at(a, base + k));
              }
          }
          g.sync();
          if constexpr (Sys::kStoredDerivs) {
            // the last D knots' stored blocks (written above by the group's lanes)
            if (bw)
#pragma unroll
              for (int i = 0; i < D; ++i) {
                if (T - 1 - i < 0) break;
                const R* d = dscr_at(a, base + T - 1 - i);
                ring(T - 1 - i, [&](R (&b)[PB]) {
#pragma unroll
                  for (int s = 0; s < PB; ++s) {
                    const int e = g.lane + s * G;
                    if (e < Sys::kDerivStride) b[s] = d[e];
                  }
                });
              }
          }
          TO_TICK(1);
          for (int k0 = kmax - 1; k0 >= 0; k0 -= D) {
#pragma unroll
            for (int d = 0; d < D; ++d) {      // knot k0 - d reads ring slot d
              const int k = k0 - d;
              if (k < 0) break;
              const bool act = bw && k < T;
              const bool act_next = bw && k >= D && k - D < T;   // the knot whose record this slot takes next
              const long long kk = base + (act ? k : 0);
              const R* rn = rec(a, traj, base, act_next ? k - D : 0, cur);
              // rigid trees: the knot's stored substep primals; planar arm: the
              // stored derivative block of the knot D earlier (this knot's is in pb)
              const long long kd = Sys::kStoredDerivs ? base + (act_next ? k - D : 0) : kk;
              const R* kprim = (Sys::kKnotParallel || Sys::kStoredDerivs) ? dscr_at(a, kd) : nullptr;
              const int f = backward_knot(P, g, w, act, act_next, a, pb[d], rn, grec_at(a, gains, kk),
                                          (a.vx && a.want_vx && act) ? vx_at(a, a.vx, kk) : nullptr, mu_lm, timer,
                                          tlast, kprim);
              if (f == 1) flags |= ST_FLAG_REG;
              // Levenberg-Marquardt: any failed factor (pivot test, or a
              // non-finite Q_uu once an earlier knot's gains were skipped)
              // asks for a larger mu; the rest of this pass is discarded
              if (a.lm) { if (f >= 2) need_mu = true; }
              else if (f == 2) bad = true;
            }
          }
        }
        }
        if (bw && bad) {
          status = ST_NONFINITE;
          release = true;
        } else if (bw && need_mu) {
          // Levenberg-Marquardt: Q_uu + mu I was not positive definite at some
          // knot; grow mu and redo the backward pass (no iteration counted)
          mu_lm *= kMuFactor;
          if (mu_lm > kMuMax) { status = ST_LS_FAIL; release = true; }
          else retry = true;
        }
      }
      if (mode == M_FINAL && !release) release = true;   // V_x pass done

      // ---- phase B: forward rounds.  Line search: LW step sizes per round,
      // one per lane, each rolled out into its own candidate slot (never the
      // current one).  Forced replay: lane 0 rolls out the forced step.  New
      // instance: lane 0 rolls out the warm start into slot 0.
      int jstar = -1, newslot = cur;
      double Jnew = 0;
      {
        const bool fwd = (mode == M_NEW) || (mode == M_RUN && !release && !retry);
        const bool single = (mode == M_NEW) || forced_mode;
        // the actor warm start runs when the problem has actor weights and no
        // caller-given controls (uniform over the warp / CTA: it holds barriers)
        const bool actor_rnd = Sys::kActor && a.actor_w != nullptr && a.U_init == nullptr &&
                               !g.uniform_all(mode != M_NEW);
        const int nr = single ? 1 : (a.n_alpha + LW - 1) / LW;
        const int jforced = (mode == M_RUN && forced_mode && fwd) ? a.forced[(size_t)inst * a.max_iter + ck(a, iter, a.max_iter, CK_FORCED)] : 0;
        // the trip count is the same for every group of the warp / CTA (each
        // round holds barriers); groups that need fewer rounds idle through
        for (int round = 0; round < kRounds; ++round) {
          const bool need = fwd && jstar < 0 && round < nr;
          if (g.uniform_all(!need)) break;
          const int j = single ? (mode == M_NEW ? 0 : jforced) : round * LW + g.lane;
          const bool mine = need && (single ? g.lane == 0 : (g.lane < LW && j < a.n_alpha));
          const int slot = (mode == M_NEW) ? 0 : (g.lane < cur ? g.lane : g.lane + 1);
          const R alpha = alpha_of(a, (j >= 0 && j < kMaxAlpha) ? j : 0);
          const bool nominal = need && mode != M_NEW;   // needs the current iterate and gains
          R xh[n], xlo[n];   // the candidate's state as (hi, lo) pairs (lo = 0 in float64)
          Acc<R> Jc;
          R pf[D][kLane ? 1 : PF];   // staging ring: knot k's record and gains in slot k % D
          R pr[kLane ? RS : 1], pg[kLane ? GS : 1];   // single lane: next knot's record and gains
          if (mine) {
            if (mode == M_NEW) {
#pragma unroll
              for (int i = 0; i < n; ++i) {
                const double x0 = a.serve.ring ? a.serve.ring[sq % a.serve.ring_size].x0[i] : a.x0[(size_t)inst * n + i];
                xh[i] = (R)x0;
                xlo[i] = kLo ? (R)(x0 - (double)xh[i]) : R(0);
              }
            } else {
              const R* r = rec(a, traj, base, 0, cur);
#pragma unroll
              for (int i = 0; i < n; ++i) {
                xh[i] = r[i];
                xlo[i] = kLo ? r[n + m + i] : R(0);
              }
            }
          }
          if (nominal) {
            if constexpr (kLane) {
              ld_vec<RS>(rec(a, traj, base, 0, cur), pr);
              ld_vec<GS>(grec_at(a, gains, base), pg);
            } else {
#pragma unroll
              for (int d = 0; d < D; ++d)
                if (d < T) prefetch_fwd(g, pf[d], rec(a, traj, base, d, cur), grec_at(a, gains, base + d));
            }
          }
          const int kr = g.uniform_max(need ? T : 0, &w.sel);
          for (int k0 = 0; k0 < kr; k0 += D) {
#pragma unroll
          for (int d = 0; d < D; ++d) {        // knot k0 + d reads ring slot d
            const int k = k0 + d;
            if (k >= kr) break;
            const bool act = need && k < T;
            R cr[kLane ? RS : 1], cg[kLane ? GS : 1];
            if constexpr (kLane) {
              if (act && nominal) {
#pragma unroll
                for (int i = 0; i < RS; ++i) cr[i] = pr[i];
#pragma unroll
                for (int i = 0; i < GS; ++i) cg[i] = pg[i];
                if (k + 1 < T) {
                  ld_vec<RS>(rec(a, traj, base, k + 1, cur), pr);
                  ld_vec<GS>(grec_at(a, gains, base + k + 1), pg);
                }
              }
            } else {
              if (act && nominal) store_fwd(g, w, pf[d]);
              g.sync();
              if (act && nominal && k + D < T)
                prefetch_fwd(g, pf[d], rec(a, traj, base, k + D, cur), grec_at(a, gains, base + k + D));
            }
            if constexpr (Sys::kActor) {
              // warm start from the actor policy u_k = pi(x_k): the group
              // evaluates the MLP, lane 0 then steps the dynamics
              if (actor_rnd) {
                const bool run = act && mode == M_NEW;
                if (run && g.lane == 0)
#pragma unroll
                  for (int i = 0; i < n; ++i) w.xk[i] = xh[i];
                g.sync();
                actor_mlp(g, w, run, a.actor_w);
              }
            }
            R uh[m];
            if (act && mine) {
              if (mode == M_NEW) {
                bool from_actor = false;
                if constexpr (Sys::kActor) {
                  from_actor = actor_rnd;
                  if (from_actor)
#pragma unroll
                    for (int i = 0; i < m; ++i) uh[i] = w.uk[i];
                }
                if (!from_actor)
#pragma unroll
                  for (int i = 0; i < m; ++i)
                    uh[i] = a.U_init ? (R)a.U_init[((size_t)inst * a.T_max + ck(a, k, a.T_max, CK_UINIT)) * m + i] : R(0);
              } else {
                if constexpr (kLane) policy_regs(cr, cg, alpha, xh, xlo, uh);
                else policy(w, alpha, xh, xlo, uh);
              }
              // the padding too: whole 32-byte sectors reach L2 without a read
              put_record(rec(a, traj, base, k, slot), xh, uh, xlo);
              if constexpr (!Sys::template kGroupStep<G>) Jc.add(Sys::cost_step2(P, xh, xlo, uh));
            }
            if constexpr (Sys::template kGroupStep<G>) {
              // the system's step is shared by partner lanes (group barriers inside;
              // act is uniform over the group)
              const R l = Sys::template cost_step_group<R, G>(P, g, act && mine, xh, xlo, uh, w.sx);
              if (act && mine) Jc.add(l);
            }
            if constexpr (!kLane) g.sync();
          }
          }
          double Jt = 0;
          int best = 0x7fffffff;
          if (mine) {
            const R u0[m] = {};                                 // no control at the terminal knot
            put_record(rec(a, traj, base, T, slot), xh, u0, xlo);
            Jc.add(Sys::terminal_cost(P, xh));
            Jt = Jc.value();
            if (single || Jt < J) best = single ? 0 : j;   // strict decrease, compared in float64
          }
          best = g.min_int(best, &w.sel);
          if (mine && best == (single ? 0 : j)) {       // the accepted lane publishes its cost and slot
            w.red = Jt;
            w.wslot = slot;
          }
          g.sync();
          if (need && best != 0x7fffffff) {
            jstar = single ? (mode == M_NEW ? 0 : jforced) : best;
            Jnew = w.red;
            newslot = w.wslot;
          }
          g.sync();
        }
      }
      TO_TICK(5);
      if (mode == M_RUN && !release && !retry && jstar < 0) {
        if (a.lm) {
          // no step size decreased the cost: grow mu and redo the backward pass
          mu_lm *= kMuFactor;
          if (mu_lm > kMuMax) { status = ST_LS_FAIL; release = true; }
          else retry = true;
        } else {
          status = ST_LS_FAIL;
          release = true;
        }
      }

      // ---- phase D: bookkeeping
      if (mode == M_NEW) {
        J = Jnew;
        cur = 0;
        if (g.lane == 0) a.Jhist[(size_t)inst * (a.max_iter + 1)] = J;
        if (!isfinite(J)) { status = ST_NONFINITE; release = true; }
        else if (a.max_iter == 0) { status = ST_MAX_ITER; release = true; }
        else mode = M_RUN;
      } else if (mode == M_RUN && !release && !retry) {
        ++iter;
        cur = newslot;
        mu_lm = fmax(mu_lm / kMuFactor, kMuMin);
        if (g.lane == 0) {
          a.ahist[(size_t)inst * a.max_iter + ck(a, iter - 1, a.max_iter, CK_HIST)] = jstar;
          a.Jhist[(size_t)inst * (a.max_iter + 1) + ck(a, iter, a.max_iter + 1, CK_HIST)] = Jnew;
        }
        const double rel = (J - Jnew) / fmax(fabs(J), 1e-300);
        J = Jnew;
        bool done = false;
        if (!isfinite(Jnew)) { status = ST_NONFINITE; done = true; release = true; }
        else if (!forced_mode && rel < a.tol) { status = ST_CONVERGED; done = true; }
        else if (iter >= a.max_iter) { status = ST_MAX_ITER; done = true; }
        if (done && !release) {
          if (a.want_vx) mode = M_FINAL; else release = true;
        }
      }
      if (release) {
        if (g.lane == 0) {
          a.J_out[inst] = J;
          a.iters_out[inst] = iter;
          a.status_out[inst] = status | flags;
          a.slot_out[inst] = cur;
          if (a.serve.ring) {
            // results first, then the completion flag the host polls
            __threadfence_system();
            a.serve.done[inst] = (unsigned)sq + 1u;
            atomicSub(a.serve.ctl, 1);
          }
        }
        mode = M_IDLE;
      }
      TO_TICK(0);
    }
  }
};

// Counting sort of the instances by horizon (longest first), prefix sums of
// the knot offsets, validation.  One CTA.
__global__ void prepare_kernel(int B, const int* __restrict__ T, int T_max, long long knots_max,
                               long long* __restrict__ toff, int* __restrict__ order, int* __restrict__ hist,
                               int* __restrict__ err, int* __restrict__ status_out, int* __restrict__ queue,
                               double* __restrict__ J_out, int* __restrict__ iters_out);

__global__ void gather_kernel(int B, int T_max, int n, int m, int RS, int GS, int NS, int rbytes,
                              const long long* __restrict__ toff, const int* __restrict__ T,
                              const int* __restrict__ slot,
                              const void* __restrict__ traj, const void* __restrict__ gains,
                              const double* __restrict__ vx, double* __restrict__ X, double* __restrict__ U,
                              double* __restrict__ Vx, double* __restrict__ K, const int* __restrict__ err);

}  // namespace to
