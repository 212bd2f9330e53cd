// Biased-initial-condition ranking (Sec. III-C/D): the std-critic network
// scores 10N candidate initial states and the N with the largest predicted
// critic standard deviation start the next TO batch (include/to.h:
// toranker_create, torank_candidates).
//
// Network: x (n_in) -> 256 tanh -> 256 tanh -> 1 softplus (a positive std).
// One CTA scores 64 candidates: 256 threads, one hidden unit each, the
// candidates' activations in shared memory (read as broadcasts), every
// weight matrix stored input-major so the threads of a warp read
// consecutive words.  Selection: a 4-pass radix select of the scores'
// bit patterns (positive floats order like their bits) finds the N-th
// largest, then one CTA compacts the winners in index order (ties at the
// threshold go to the lowest indices).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "handles.h"

namespace {

constexpr int kH = 256;        // hidden width
constexpr int kTC = 64;        // candidates per CTA
constexpr int kMaxIn = 64;     // largest input width

__device__ __forceinline__ float softplus_(float z) { return z > 0.f ? z + log1pf(expf(-z)) : log1pf(expf(z)); }

__global__ void __launch_bounds__(kH) std_critic_kernel(int C, int n_in, const double* __restrict__ x,
                                                          const float* __restrict__ w, float* __restrict__ score,
                                                          unsigned* __restrict__ key) {
  extern __shared__ __align__(16) float sm[];
  float* xs = sm;                      // [kTC][n_in]
  float* h = sm + kTC * kMaxIn;        // [kH][kTC]
  const float* W1 = w;                 // [n_in][kH]
  const float* b1 = W1 + n_in * kH;
  const float* W2 = b1 + kH;           // [kH][kH] input-major
  const float* b2 = W2 + kH * kH;
  const float* W3 = b2 + kH;           // [kH]
  const float* b3 = W3 + kH;
  const int c0 = blockIdx.x * kTC;
  const int j = threadIdx.x;
  for (int e = j; e < kTC * n_in; e += kH) {
    const int c = e / n_in, i = e - c * n_in;
    xs[c * n_in + i] = c0 + c < C ? (float)x[(size_t)(c0 + c) * n_in + i] : 0.f;
  }
  __syncthreads();
  float acc[kTC];
  // layer 1
#pragma unroll
  for (int c = 0; c < kTC; ++c) acc[c] = b1[j];
  for (int i = 0; i < n_in; ++i) {
    const float wi = W1[i * kH + j];
#pragma unroll
    for (int c = 0; c < kTC; ++c) acc[c] += wi * xs[c * n_in + i];
  }
#pragma unroll
  for (int c = 0; c < kTC; ++c) h[j * kTC + c] = tanhf(acc[c]);
  __syncthreads();
  // layer 2
#pragma unroll
  for (int c = 0; c < kTC; ++c) acc[c] = b2[j];
  for (int i = 0; i < kH; ++i) {
    const float wi = W2[i * kH + j];
    const float4* hr = reinterpret_cast<const float4*>(h + i * kTC);
#pragma unroll
    for (int c4 = 0; c4 < kTC / 4; ++c4) {
      const float4 v = hr[c4];
      acc[4 * c4 + 0] += wi * v.x;
      acc[4 * c4 + 1] += wi * v.y;
      acc[4 * c4 + 2] += wi * v.z;
      acc[4 * c4 + 3] += wi * v.w;
    }
  }
  __syncthreads();   // every thread has read layer 1's activations
#pragma unroll
  for (int c = 0; c < kTC; ++c) h[j * kTC + c] = tanhf(acc[c]);
  __syncthreads();
  // output
  if (j < kTC && c0 + j < C) {
    float s = b3[0];
    for (int i = 0; i < kH; ++i) s += W3[i] * h[i * kTC + j];
    const float sd = softplus_(s);
    score[c0 + j] = sd;
    // positive floats order like their bit patterns; a non-finite score ranks last
    key[c0 + j] = (isfinite(sd) && sd > 0.f) ? __float_as_uint(sd) : 0u;
  }
}

// Radix select of the N largest keys and their compaction in index order.
// One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) select_kernel(int C, int N, const unsigned* __restrict__ key,
                                                      int* __restrict__ out) {
  __shared__ unsigned hist[256];
  __shared__ unsigned s_prefix, s_mask;
  __shared__ int s_remaining;
  __shared__ int scan[1024];
  const int t = threadIdx.x;
  if (t == 0) { s_prefix = 0u; s_mask = 0u; s_remaining = N; }
  __syncthreads();
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int d = t; d < 256; d += 1024) hist[d] = 0u;
    __syncthreads();
    const unsigned prefix = s_prefix, mask = s_mask;
    for (int i = t; i < C; i += 1024) {
      const unsigned k = key[i];
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (t == 0) {
      int rem = s_remaining;
      unsigned above = 0;
      int d = 255;
      for (; d > 0; --d) {
        if ((int)(above + hist[d]) >= rem) break;
        above += hist[d];
      }
      s_remaining = rem - (int)above;
      s_prefix = prefix | ((unsigned)d << shift);
      s_mask = mask | (255u << shift);
    }
    __syncthreads();
  }
  const unsigned thr = s_prefix;      // the N-th largest key
  const int need_eq = s_remaining;    // how many keys equal to it are taken
  // contiguous chunks per thread keep index order
  const int chunk = (C + 1023) / 1024;
  const int lo = min(C, t * chunk), hi = min(C, lo + chunk);
  int gt = 0, eq = 0;
  for (int i = lo; i < hi; ++i) {
    const unsigned k = key[i];
    gt += k > thr;
    eq += k == thr;
  }
  // exclusive scan of eq, then of the selected counts
  scan[t] = eq;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v = t >= off ? scan[t - off] : 0;
    __syncthreads();
    scan[t] += v;
    __syncthreads();
  }
  const int eq_before = scan[t] - eq;
  const int take_eq = max(0, min(eq, need_eq - eq_before));
  const int sel = gt + take_eq;
  __syncthreads();
  scan[t] = sel;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v = t >= off ? scan[t - off] : 0;
    __syncthreads();
    scan[t] += v;
    __syncthreads();
  }
  int pos = scan[t] - sel;
  int taken_eq = 0;
  for (int i = lo; i < hi; ++i) {
    const unsigned k = key[i];
    if (k > thr || (k == thr && taken_eq < take_eq)) {
      if (k == thr) ++taken_eq;
      if (pos < N) out[pos] = i;
      ++pos;
    }
  }
}

}  // namespace

struct to_ranker_s {
  int n_in = 0;
  float* d_w = nullptr;
  double* d_x = nullptr;
  float* d_score = nullptr;
  unsigned* d_key = nullptr;
  int* d_out = nullptr;
  int cap_c = 0, cap_n = 0;
  int launches = 0;
};

#define RK_CK(x)                                                                                \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) return to_fail(TO_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int toranker_create(int n_in, const float* weights, size_t n_weights, to_ranker* out) {
  if (!out || !weights || n_in < 1 || n_in > kMaxIn) return to_fail(TO_ERR_ARG, "toranker_create: bad arguments (1 <= n_in <= 64)");
  *out = nullptr;
  const size_t expect = (size_t)kH * n_in + kH + (size_t)kH * kH + kH + kH + 1;
  if (n_weights != expect) return to_fail(TO_ERR_ARG, "toranker_create: weights must be W1[256 x n_in] b1 W2[256 x 256] b2 W3[1 x 256] b3");
  // every W (out x in, row-major) stored transposed (input-major)
  std::vector<float> t(expect);
  size_t o = 0;
  auto transpose = [&](int rows, int cols) {
    for (int i = 0; i < cols; ++i)
      for (int r = 0; r < rows; ++r) t[o + (size_t)i * rows + r] = weights[o + (size_t)r * cols + i];
    o += (size_t)rows * cols;
  };
  auto copy = [&](int k) {
    std::memcpy(t.data() + o, weights + o, sizeof(float) * k);
    o += k;
  };
  transpose(kH, n_in); copy(kH); transpose(kH, kH); copy(kH); copy(kH); copy(1);
  to_ranker r = new to_ranker_s();
  r->n_in = n_in;
  cudaError_t e = cudaMalloc(&r->d_w, expect * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(r->d_w, t.data(), expect * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    toranker_destroy(r);
    return to_fail(TO_ERR_CUDA, std::string("toranker_create: ") + cudaGetErrorString(e));
  }
  *out = r;
  return TO_OK;
}

void toranker_destroy(to_ranker r) {
  if (!r) return;
  void* p[] = {r->d_w, r->d_x, r->d_score, r->d_key, r->d_out};
  for (void* q : p)
    if (q) cudaFree(q);
  delete r;
}

int torank_candidates(to_ranker r, int C, const double* x, int N, int* top_idx, float* scores, void* cuda_stream) {
  if (!r || !x || !top_idx || C < 1 || N < 1 || N > C) return to_fail(TO_ERR_ARG, "torank_candidates: bad arguments (1 <= N <= C)");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (C > r->cap_c) {
    for (void* q : {(void*)r->d_x, (void*)r->d_score, (void*)r->d_key})
      if (q) cudaFree(q);
    r->d_x = nullptr; r->d_score = nullptr; r->d_key = nullptr;
    RK_CK(cudaMalloc(&r->d_x, sizeof(double) * (size_t)C * r->n_in));
    RK_CK(cudaMalloc(&r->d_score, sizeof(float) * C));
    RK_CK(cudaMalloc(&r->d_key, sizeof(unsigned) * C));
    r->cap_c = C;
  }
  if (N > r->cap_n) {
    if (r->d_out) cudaFree(r->d_out);
    r->d_out = nullptr;
    RK_CK(cudaMalloc(&r->d_out, sizeof(int) * N));
    r->cap_n = N;
  }
  RK_CK(cudaMemcpyAsync(r->d_x, x, sizeof(double) * (size_t)C * r->n_in, cudaMemcpyHostToDevice, s));
  const size_t smem = sizeof(float) * ((size_t)kTC * kMaxIn + (size_t)kH * kTC);
  RK_CK(cudaFuncSetAttribute(std_critic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  std_critic_kernel<<<(C + kTC - 1) / kTC, kH, smem, s>>>(C, r->n_in, r->d_x, r->d_w, r->d_score, r->d_key);
  RK_CK(cudaGetLastError());
  select_kernel<<<1, 1024, 0, s>>>(C, N, r->d_key, r->d_out);
  RK_CK(cudaGetLastError());
  r->launches = 2;
  RK_CK(cudaMemcpyAsync(top_idx, r->d_out, sizeof(int) * N, cudaMemcpyDeviceToHost, s));
  if (scores) RK_CK(cudaMemcpyAsync(scores, r->d_score, sizeof(float) * C, cudaMemcpyDeviceToHost, s));
  RK_CK(cudaStreamSynchronize(s));
  return TO_OK;
}
