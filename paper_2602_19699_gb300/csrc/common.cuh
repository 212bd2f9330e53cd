// Device-side building blocks shared by every system and solver kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define TO_DEV __device__ __forceinline__

namespace to {

enum { ST_CONVERGED = 1, ST_MAX_ITER = 2, ST_LS_FAIL = 3, ST_NONFINITE = 4, ST_TIMEOUT = 5, ST_FLAG_REG = 16 };
enum { PREC_FP64 = 0, PREC_MIXED = 1 };

// A group of G threads owns one instance.  G <= 32: 32/G groups share a warp
// and every warp runs warp-uniform control flow (work is predicated per group),
// so a group barrier is a warp barrier.  G > 32: one group per CTA.  G = 1:
// one thread per instance (32 instances per warp).
template <int G>
struct Group {
  static_assert(G == 1 || G == 4 || G == 8 || G == 16 || G == 32 || G == 64 || G == 128 || G == 256, "group size");
  static constexpr bool kSubWarp = G <= 32;
  int lane;    // 0..G-1
  int index;   // group index within the CTA
  TO_DEV Group() : lane(threadIdx.x % G), index(threadIdx.x / G) {}
  TO_DEV void sync() const {
    if (kSubWarp) __syncwarp(); else __syncthreads();
  }
  // first lane of this group inside its warp (G <= 32)
  TO_DEV int leader_in_warp() const { return (threadIdx.x & 31) & ~(G - 1); }
  // value of lane 0 of the group
  template <class T> TO_DEV T bcast(T v, T* smem_slot) const {
    if (kSubWarp) return __shfl_sync(0xffffffffu, v, leader_in_warp());
    if (lane == 0) *smem_slot = v;
    __syncthreads();
    T r = *smem_slot;
    __syncthreads();
    return r;
  }
  // minimum over the group's lanes
  TO_DEV int min_int(int v, int* smem_slot) const {
    if (kSubWarp) {
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o, G));
      return v;
    }
    if (lane == 0) *smem_slot = 0x7fffffff;
    __syncthreads();
    atomicMin(smem_slot, v);
    __syncthreads();
    int r = *smem_slot;
    __syncthreads();
    return r;
  }
  // maximum over every group sharing the warp (sub-warp) or the CTA
  TO_DEV int uniform_max(int v, int* smem_slot) const {
    if (kSubWarp) return __reduce_max_sync(0xffffffffu, v);
    return v;   // one group per CTA: already uniform
  }
  TO_DEV bool uniform_all(bool v) const {
    if (kSubWarp) return __all_sync(0xffffffffu, v);
    return v;
  }
  // the unit that shares control flow: the warp (sub-warp groups) or the CTA
  TO_DEV bool unit_leader() const { return kSubWarp ? (threadIdx.x & 31) == 0 : lane == 0; }
  template <class T> TO_DEV T unit_bcast(T v, T* smem_slot) const {
    if (kSubWarp) return __shfl_sync(0xffffffffu, v, 0);
    return bcast(v, smem_slot);
  }
};

// State accumulation (hi, lo) += d.  In float32 the pair carries the state
// to about 48 bits (two-sum, then renormalised so |lo| <= ulp(hi) / 2), so a
// long rollout loses no more than the increments' own rounding; in float64
// it is the plain sum (lo stays 0).
template <class R>
TO_DEV void acc2(R& hi, R& lo, R d) {
  if constexpr (sizeof(R) == 4) {
    const R s = hi + d;
    const R bv = s - hi;
    const R e = (hi - (s - bv)) + (d - bv);
    const R l = lo + e;
    hi = s + l;
    lo = l - (hi - s);
  } else {
    hi += d;
  }
}

// one semi-implicit Euler step of (q, v) carried as (hi, lo) pairs:
// v+ = v + h a,  q+ = q + h v+
template <class R, int N>
TO_DEV void semi_implicit2(R* qh, R* ql, R* vh, R* vl, const R* a, R h) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    acc2(vh[i], vl[i], h * a[i]);
    acc2(qh[i], ql[i], h * vh[i] + h * vl[i]);
  }
}

// clip of a zero eigenvalue, max(0, eps): the value a Hessian's entries
// outside a cost's support take (0 when clipping is off, eps < 0)
template <class R> TO_DEV R clip0(R eps) { return eps > R(0) ? eps : R(0); }

// max(a, |x|) ignoring a NaN x, in the operands' own precision
TO_DEV float max_abs(float a, float x) { return fmaxf(a, fabsf(x)); }
TO_DEV double max_abs(double a, double x) { return fmax(a, fabs(x)); }

// 16-byte vector moves of a record (the record and its address 16-byte aligned)
TO_DEV void ld16(const float* p, float* d) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  d[0] = t.x; d[1] = t.y; d[2] = t.z; d[3] = t.w;
}
TO_DEV void ld16(const double* p, double* d) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  d[0] = t.x; d[1] = t.y;
}
TO_DEV void st16(float* p, const float* s) { *reinterpret_cast<float4*>(p) = make_float4(s[0], s[1], s[2], s[3]); }
TO_DEV void st16(double* p, const double* s) { *reinterpret_cast<double2*>(p) = make_double2(s[0], s[1]); }
template <int NE, class R>
TO_DEV void ld_vec(const R* p, R* d) {
  constexpr int V = 16 / (int)sizeof(R);
  static_assert(NE % V == 0, "whole 16-byte vectors");
#pragma unroll
  for (int i = 0; i < NE; i += V) ld16(p + i, d + i);
}
template <int NE, class R>
TO_DEV void st_vec(R* p, const R* s) {
  constexpr int V = 16 / (int)sizeof(R);
  static_assert(NE % V == 0, "whole 16-byte vectors");
#pragma unroll
  for (int i = 0; i < NE; i += V) st16(p + i, s + i);
}

template <class R> TO_DEV R rsqrt_(R x);
template <> TO_DEV float rsqrt_(float x) { return rsqrtf(x); }
template <> TO_DEV double rsqrt_(double x) { return rsqrt(x); }

TO_DEV bool finite_d(double x) { return isfinite(x); }

// 1 / sqrt(s) for a float64 s in the normal float32 range: the float32
// hardware estimate y0 (relative error e0 <= 2^-22) refined by one
// Newton-Raphson step for f(y) = 1/y^2 - s, y1 = y0 (1 + (1 - s y0^2) / 2),
// in float64; the relative error is about 1.5 e0^2 <= 1e-13 (measured: at
// most 3.8e-14 against 1 / sqrt over 2.7e8 inputs).  Three float64
// arithmetic instructions instead of the full-precision sequence; used
// where the float64 factor is rounded to float32 afterwards.  Outside that
// range the result is meaningless and the caller must not use it.
TO_DEV double rsqrt_newton(double s) {
  const float yf = rsqrtf((float)s);
  const double y = (double)yf;
  const double e = fma(-s * y, y, 1.0);
  return fma((double)(0.5f * yf), e, y);
}

// s > t for float64 s and a finite t >= 0, exactly, on the integer pipe: for
// non-negative doubles the bit patterns order like the values.  Infinities
// and NaNs compare false.
TO_DEV bool dgt_nonneg(double s, double t) {
  const long long a = __double_as_longlong(s), b = __double_as_longlong(t);
  return a > b && a < 0x7ff0000000000000LL;
}

// Unit eigenvector of the symmetric 3x3 A for the eigenvalue lam: the largest
// cross product of two rows of A - lam I (they span the orthogonal complement
// when lam is simple).
template <class R>
TO_DEV void eigvec_sym3(const R* A, R lam, R* w) {
  const R r0[3] = {A[0] - lam, A[1], A[2]}, r1[3] = {A[3], A[4] - lam, A[5]}, r2[3] = {A[6], A[7], A[8] - lam};
  R c[3][3];
  const R* ra[3] = {r0, r0, r1};
  const R* rb[3] = {r1, r2, r2};
  R best = R(-1);
  int bi = 0;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    c[t][0] = ra[t][1] * rb[t][2] - ra[t][2] * rb[t][1];
    c[t][1] = ra[t][2] * rb[t][0] - ra[t][0] * rb[t][2];
    c[t][2] = ra[t][0] * rb[t][1] - ra[t][1] * rb[t][0];
    const R nn = c[t][0] * c[t][0] + c[t][1] * c[t][1] + c[t][2] * c[t][2];
    if (nn > best) { best = nn; bi = t; }
  }
  const R inv = best > R(0) ? rsqrt_(best) : R(0);
  w[0] = c[bi][0] * inv; w[1] = c[bi][1] * inv; w[2] = c[bi][2] * inv;
}

// Clip of a symmetric 2x2 [a b; b c]: one Jacobi rotation diagonalises it
// exactly (Golub & Van Loan sec. 8.5.2); the rotation is scale-free, so tiny
// entries (far from a bump, in float32) cannot underflow into 0/0.
template <class R>
TO_DEV void eigclip_2x2(R& a, R& b, R& c, R eps) {
  if (b == R(0)) {
    a = a > eps ? a : eps;
    c = c > eps ? c : eps;
    return;
  }
  const R tau = (c - a) / (R(2) * b);
  const R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
  const R cs = rsqrt_(R(1) + t * t), sn = t * cs;
  R d1 = a - t * b, d2 = c + t * b;     // eigenvalues
  d1 = d1 > eps ? d1 : eps;
  d2 = d2 > eps ? d2 : eps;
  // [a b; b c] = J diag(d1, d2) J^T with J = [cs sn; -sn cs]
  a = cs * cs * d1 + sn * sn * d2;
  c = sn * sn * d1 + cs * cs * d2;
  b = cs * sn * (d2 - d1);
}

// Eigenvalue clip of a symmetric 3x3 without iteration.  The eigenvalue that
// is farthest from the other two comes from the characteristic cubic in
// trigonometric form (Smith, CACM 4(4), 1961) -- the largest when the cubic's
// angle puts the close pair below, else the smallest; unlike the close pair
// it is well conditioned there -- and its eigenvector from a cross product
// of two rows of Q - lam I.  The rest is the exact 2x2 problem on the
// orthogonal complement (one Jacobi rotation).  Q' = max(lam, eps) w w^T
// + U clip(U^T Q U) U^T.
template <class R>
TO_DEV void eigclip_sym3(R* Qio, R eps_in) {
  // work on Q / max|Q_ij| (the clip commutes with positive scaling), so that
  // products of tiny entries cannot underflow
  R mx = R(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) mx = fabs(Qio[i]) > mx ? fabs(Qio[i]) : mx;
  if (!(mx > R(0))) {
#pragma unroll
    for (int i = 0; i < 9; ++i) Qio[i] = (i % 4 == 0) ? (eps_in > R(0) ? eps_in : R(0)) : R(0);
    return;
  }
  const R sc = R(1) / mx;
  R Q[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) Q[i] = Qio[i] * sc;
  const R eps = eps_in * sc;
  const R a00 = Q[0], a11 = Q[4], a22 = Q[8], a01 = Q[1], a02 = Q[2], a12 = Q[5];
  const R p1 = a01 * a01 + a02 * a02 + a12 * a12;
  if (p1 == R(0)) {
    Qio[0] = (a00 > eps ? a00 : eps) * mx;
    Qio[4] = (a11 > eps ? a11 : eps) * mx;
    Qio[8] = (a22 > eps ? a22 : eps) * mx;
    return;
  }
  const R q = (a00 + a11 + a22) * R(1.0 / 3.0);
  const R b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
  const R p = sqrt((b00 * b00 + b11 * b11 + b22 * b22 + R(2) * p1) * R(1.0 / 6.0));
  const R ip = R(1) / p;
  const R c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip, c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
  R r = R(0.5) * (c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02));
  r = r < R(-1) ? R(-1) : (r > R(1) ? R(1) : r);
  const R phi = acos(r) * R(1.0 / 3.0);
  const R lam = r >= R(0) ? q + R(2) * p * cos(phi) : q + R(2) * p * cos(phi + R(2.0943951023931954923));
  R w[3];
  eigvec_sym3(Q, lam, w);
  // orthonormal basis (u1, u2) of the complement of w
  const R aw0 = fabs(w[0]), aw1 = fabs(w[1]), aw2 = fabs(w[2]);
  const int k = (aw0 <= aw1 && aw0 <= aw2) ? 0 : (aw1 <= aw2 ? 1 : 2);
  R u1[3];   // w x e_k
  u1[0] = k == 0 ? R(0) : (k == 1 ? -w[2] : w[1]);
  u1[1] = k == 0 ? w[2] : (k == 1 ? R(0) : -w[0]);
  u1[2] = k == 0 ? -w[1] : (k == 1 ? w[0] : R(0));
  const R n1 = rsqrt_(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
  u1[0] *= n1; u1[1] *= n1; u1[2] *= n1;
  const R u2[3] = {w[1] * u1[2] - w[2] * u1[1], w[2] * u1[0] - w[0] * u1[2], w[0] * u1[1] - w[1] * u1[0]};
  R Qu1[3], Qu2[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Qu1[i] = Q[i * 3] * u1[0] + Q[i * 3 + 1] * u1[1] + Q[i * 3 + 2] * u1[2];
    Qu2[i] = Q[i * 3] * u2[0] + Q[i * 3 + 1] * u2[1] + Q[i * 3 + 2] * u2[2];
  }
  const R e11 = u1[0] * Qu1[0] + u1[1] * Qu1[1] + u1[2] * Qu1[2];
  const R e12 = u1[0] * Qu2[0] + u1[1] * Qu2[1] + u1[2] * Qu2[2];
  const R e22 = u2[0] * Qu2[0] + u2[1] * Qu2[1] + u2[2] * Qu2[2];
  // the clip as a correction to Q (exact zero where nothing is clipped):
  // dl along w, and the 2x2 block's eigen-corrections rotated back
  const R dl = lam < eps ? eps - lam : R(0);
  R f11, f12, f22;
  if (e12 == R(0)) {
    f11 = e11 < eps ? eps - e11 : R(0);
    f22 = e22 < eps ? eps - e22 : R(0);
    f12 = R(0);
  } else {
    const R tau = (e22 - e11) / (R(2) * e12);
    const R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
    const R cs = rsqrt_(R(1) + t * t), sn = t * cs;
    const R d1 = e11 - t * e12, d2 = e22 + t * e12;
    const R g1 = d1 < eps ? eps - d1 : R(0), g2 = d2 < eps ? eps - d2 : R(0);
    f11 = cs * cs * g1 + sn * sn * g2;
    f22 = sn * sn * g1 + cs * cs * g2;
    f12 = cs * sn * (g2 - g1);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const R v = Qio[i * 3 + j] + (dl * w[i] * w[j] + f11 * u1[i] * u1[j] + f12 * (u1[i] * u2[j] + u2[i] * u1[j]) +
                                    f22 * u2[i] * u2[j]) * mx;
      Qio[i * 3 + j] = v;
      Qio[j * 3 + i] = v;
    }
}

// Eigenvalue clipping of a small symmetric matrix (Sec. IV-B),
//   S' = max(S, eps),  Q_psd = sym(W diag(S') W^T),
// after two exact shortcuts; 3x3 blocks then take the closed form above,
// larger ones an in-place cyclic Jacobi eigen-decomposition (Golub & Van
// Loan sec. 8.5).  One thread; P is row-major P x P.
template <class R, int P>
TO_DEV void eigclip_small(R* Q, R eps) {
  // Two exact shortcuts before the iteration:
  //  * Gershgorin: if every eigenvalue is <= eps the clip is eps I;
  //  * if Q - eps I has a Cholesky factor (positive pivots) every eigenvalue
  //    is > eps and the clip is the identity map.
  {
    R gmax = -R(1e30);
#pragma unroll
    for (int i = 0; i < P; ++i) {
      R s = Q[i * P + i];
#pragma unroll
      for (int j = 0; j < P; ++j)
        if (j != i) s += fabs(Q[i * P + j]);
      gmax = s > gmax ? s : gmax;
    }
    if (gmax <= eps) {
#pragma unroll
      for (int i = 0; i < P; ++i)
#pragma unroll
        for (int j = 0; j < P; ++j) Q[i * P + j] = (i == j) ? eps : R(0);
      return;
    }
    R C[P][P];
    bool pd = true;
#pragma unroll
    for (int j = 0; j < P; ++j) {
      R s = Q[j * P + j] - eps;
#pragma unroll
      for (int k = 0; k < j; ++k) s -= C[j][k] * C[j][k];
      pd = pd && (s > R(0));
      const R r = rsqrt_(s > R(0) ? s : R(1));
#pragma unroll
      for (int i = j + 1; i < P; ++i) {
        R t = Q[i * P + j];
#pragma unroll
        for (int k = 0; k < j; ++k) t -= C[i][k] * C[j][k];
        C[i][j] = t * r;
      }
      C[j][j] = s * r;
    }
    if (pd) return;
  }
  if constexpr (P == 3) {
    eigclip_sym3(Q, eps);
    return;
  }
  R A[P][P], W[P][P];
#pragma unroll
  for (int i = 0; i < P; ++i)
#pragma unroll
    for (int j = 0; j < P; ++j) { A[i][j] = Q[i * P + j]; W[i][j] = (i == j) ? R(1) : R(0); }
  for (int sweep = 0; sweep < 12; ++sweep) {
    R off = 0, tot = 0;
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
      for (int q = 0; q < P; ++q) {
        tot += A[p][q] * A[p][q];
        if (p != q) off += A[p][q] * A[p][q];
      }
    if (!(off > R(sizeof(R) == 4 ? 1e-14 : 1e-30) * tot)) break;   // off-diagonal below (unit roundoff)^2
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
      for (int q = p + 1; q < P; ++q) {
        R apq = A[p][q];
        if (apq != R(0)) {
          R tau = (A[q][q] - A[p][p]) / (R(2) * apq);
          R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
          R c = rsqrt_(R(1) + t * t), s = t * c;
#pragma unroll
          for (int k = 0; k < P; ++k) {
            R akp = A[k][p], akq = A[k][q];
            A[k][p] = c * akp - s * akq;
            A[k][q] = s * akp + c * akq;
          }
#pragma unroll
          for (int k = 0; k < P; ++k) {
            R apk = A[p][k], aqk = A[q][k];
            A[p][k] = c * apk - s * aqk;
            A[q][k] = s * apk + c * aqk;
          }
#pragma unroll
          for (int k = 0; k < P; ++k) {
            R wkp = W[k][p], wkq = W[k][q];
            W[k][p] = c * wkp - s * wkq;
            W[k][q] = s * wkp + c * wkq;
          }
        }
      }
  }
  R S[P];
#pragma unroll
  for (int i = 0; i < P; ++i) S[i] = A[i][i] > eps ? A[i][i] : eps;
#pragma unroll
  for (int i = 0; i < P; ++i)
#pragma unroll
    for (int j = i; j < P; ++j) {
      R s = 0;
#pragma unroll
      for (int k = 0; k < P; ++k) s += W[i][k] * S[k] * W[j][k];
      Q[i * P + j] = s;
      Q[j * P + i] = s;
    }
}

// The same clip for larger blocks with runtime loops (small code; the
// matrices live in local memory).  One thread.
template <class R, int P>
TO_DEV void eigclip_jacobi(R* Q, R eps) {
  R gmax = -R(1e30);
  for (int i = 0; i < P; ++i) {
    R s = Q[i * P + i];
    for (int j = 0; j < P; ++j)
      if (j != i) s += fabs(Q[i * P + j]);
    gmax = s > gmax ? s : gmax;
  }
  if (gmax <= eps) {
    for (int i = 0; i < P * P; ++i) Q[i] = (i % (P + 1) == 0) ? eps : R(0);
    return;
  }
  R A[P * P], W[P * P];
  {
    bool pd = true;
    for (int j = 0; j < P && pd; ++j) {
      R s = Q[j * P + j] - eps;
      for (int k = 0; k < j; ++k) s -= A[j * P + k] * A[j * P + k];
      if (!(s > R(0))) { pd = false; break; }
      const R r = rsqrt_(s);
      A[j * P + j] = s * r;
      for (int i = j + 1; i < P; ++i) {
        R t = Q[i * P + j];
        for (int k = 0; k < j; ++k) t -= A[i * P + k] * A[j * P + k];
        A[i * P + j] = t * r;
      }
    }
    if (pd) return;
  }
  for (int i = 0; i < P * P; ++i) { A[i] = Q[i]; W[i] = (i % (P + 1) == 0) ? R(1) : R(0); }
  for (int sweep = 0; sweep < 30; ++sweep) {
    R off = 0, tot = 0;
    for (int p = 0; p < P; ++p)
      for (int q = 0; q < P; ++q) {
        tot += A[p * P + q] * A[p * P + q];
        if (p != q) off += A[p * P + q] * A[p * P + q];
      }
    if (!(off > R(sizeof(R) == 4 ? 1e-14 : 1e-30) * tot)) break;
    for (int p = 0; p < P; ++p)
      for (int q = p + 1; q < P; ++q) {
        const R apq = A[p * P + q];
        if (apq == R(0)) continue;
        const R tau = (A[q * P + q] - A[p * P + p]) / (R(2) * apq);
        const R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
        const R c = rsqrt_(R(1) + t * t), s = t * c;
        for (int k = 0; k < P; ++k) {
          const R akp = A[k * P + p], akq = A[k * P + q];
          A[k * P + p] = c * akp - s * akq;
          A[k * P + q] = s * akp + c * akq;
        }
        for (int k = 0; k < P; ++k) {
          const R apk = A[p * P + k], aqk = A[q * P + k];
          A[p * P + k] = c * apk - s * aqk;
          A[q * P + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < P; ++k) {
          const R wkp = W[k * P + p], wkq = W[k * P + q];
          W[k * P + p] = c * wkp - s * wkq;
          W[k * P + q] = s * wkp + c * wkq;
        }
      }
  }
  for (int i = 0; i < P; ++i)
    for (int j = i; j < P; ++j) {
      R s = 0;
      for (int k = 0; k < P; ++k) {
        const R d = A[k * P + k] > eps ? A[k * P + k] : eps;
        s += W[i * P + k] * d * W[j * P + k];
      }
      Q[i * P + j] = s;
      Q[j * P + i] = s;
    }
}

}  // namespace to
