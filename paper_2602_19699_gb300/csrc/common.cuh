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
// so a group barrier is a warp barrier.  G > 32: one group per CTA.
template <int G>
struct Group {
  static_assert(G == 4 || G == 8 || G == 16 || G == 32 || G == 64 || G == 128 || G == 256, "group size");
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

template <class R> TO_DEV R rsqrt_(R x);
template <> TO_DEV float rsqrt_(float x) { return rsqrtf(x); }
template <> TO_DEV double rsqrt_(double x) { return rsqrt(x); }

TO_DEV bool finite_d(double x) { return isfinite(x); }

// In-place cyclic Jacobi eigen-decomposition of a small symmetric matrix
// (Golub & Van Loan sec. 8.5) followed by eigenvalue clipping
//   S' = max(S, eps),  Q_psd = sym(W diag(S') W^T)        (Sec. IV-B)
// One thread; P is row-major P x P.
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

}  // namespace to
