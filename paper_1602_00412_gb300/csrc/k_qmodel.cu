// Learned power count q for SimultaneousIteration (Alg. 1 inside Alg. 3; Sec.
// 3.2 fixes q only up to a constant and Alg. 4 verifies every result).
//
//  - Buffer features (16 floats) from the CSR/CSC copies of A' and the Gram
//    S0 of the first product A'G. Every cross-block combination is an integer
//    sum or a maximum, so the features do not depend on scheduling.
//  - A 16 -> 64 -> 64 -> 1 ReLU network: forward (one thread per sample),
//    loss gradient (one CTA, fixed summation order) and Adam, hand-written.
//
// Parameter layout (float32, kQParams): W1 [16][64] (input-major), b1[64],
// W2 [64][64] (input-major), b2[64], w3[64], b3.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "sfd_internal.cuh"

namespace sfd {
namespace {

constexpr int kQB = 304;  // blocks of the feature passes
constexpr int oW1 = 0, ob1 = oW1 + kQF * kQH, oW2 = ob1 + kQH, ob2 = oW2 + kQH * kQH,
              ow3 = ob2 + kQH, ob3 = ow3 + kQH;
static_assert(ob3 + 1 == kQParams, "parameter layout");

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- features
// acc: [0] max row norm^2 (float bits), [1] max column count, [2] nonempty
// columns (32-bit); acc64: [0] sum of row counts^2, [1] sum of column counts^2.
__global__ void k_qf_rows(const int* __restrict__ ptr, const float* __restrict__ val, int m,
                          unsigned* __restrict__ acc, unsigned long long* __restrict__ acc64) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  float mx = 0.f;
  unsigned long long r2 = 0;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < m; r += warps) {
    const int b = ptr[r], e = ptr[r + 1];
    float s = 0.f;
    for (int p = b + lane; p < e; p += 32) s = fmaf(val[p], val[p], s);
    s = wsum(s);
    mx = fmaxf(mx, s);
    if (lane == 0) r2 += (unsigned long long)(e - b) * (unsigned long long)(e - b);
  }
  if (lane == 0) {
    atomicMax(&acc[0], __float_as_uint(mx));  // non-negative floats order as integers
    atomicAdd(&acc64[0], r2);
  }
}

__global__ void k_qf_cols(const int* __restrict__ colptr, int d, unsigned* __restrict__ acc,
                          unsigned long long* __restrict__ acc64) {
  unsigned mx = 0, ne = 0;
  unsigned long long c2 = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x) {
    const unsigned c = (unsigned)(colptr[j + 1] - colptr[j]);
    mx = max(mx, c);
    ne += c > 0;
    c2 += (unsigned long long)c * c;
  }
  atomicMax(&acc[1], mx);
  atomicAdd(&acc[2], ne);
  atomicAdd(&acc64[1], c2);
}

// One CTA of 256 threads: trace, squared Frobenius norm and largest diagonal
// entry of S0 (fixed-order reductions), then the 16 features.
__global__ void k_qf_final(const unsigned* __restrict__ acc, const unsigned long long* __restrict__ acc64,
                           const double* __restrict__ fro2_ptr, const float* __restrict__ S0, int ell,
                           int m, long long N, int d, int q_fixed, float* __restrict__ feat) {
  __shared__ double red[3][8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double tr = 0.0, f2 = 0.0, dmax = 0.0;
  for (int e = tid; e < ell * ell; e += blockDim.x) {
    const double v = S0[e];
    f2 += v * v;
    if (e / ell == e % ell) {
      tr += v;
      dmax = fmax(dmax, v);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    f2 += __shfl_xor_sync(0xffffffffu, f2, o);
    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  }
  if (lane == 0) {
    red[0][warp] = tr;
    red[1][warp] = f2;
    red[2][warp] = dmax;
  }
  __syncthreads();
  if (tid != 0) return;
  tr = f2 = dmax = 0.0;
  for (int w = 0; w < 8; ++w) {
    tr += red[0][w];
    f2 += red[1][w];
    dmax = fmax(dmax, red[2][w]);
  }
  const double fro2 = *fro2_ptr;
  const double dN = (double)N;
  double f[kQF] = {};
  f[0] = 1.0;
  f[1] = m > 0 ? log((double)m) / 10.0 : 0.0;
  f[2] = N > 0 ? log(dN) / 20.0 : 0.0;
  f[3] = log((double)d) / 15.0;
  f[4] = ell / 256.0;
  if (N > 0) {
    f[5] = log(dN / m) / 5.0;
    f[6] = fro2 > 0.0 ? log(fro2 / dN) / 10.0 : 0.0;
    f[7] = fro2 > 0.0 ? (double)__uint_as_float(acc[0]) / fro2 : 0.0;
    f[8] = (double)acc[1] / dN;
    f[9] = (double)acc64[1] / (dN * dN);
    f[10] = (double)m * (double)acc64[0] / (dN * dN) - 1.0;
    f[14] = log(1.0 + dN / ((double)m * ell));
    f[15] = 1.0 - (double)acc[2] / d;
  } else {
    f[15] = 1.0;
  }
  f[11] = log((double)q_fixed) / 3.0;
  if (tr > 0.0) {
    f[12] = f2 / (tr * tr);
    f[13] = dmax / tr;
  }
  for (int i = 0; i < kQF; ++i) feat[i] = (float)f[i];
}

// ------------------------------------------------------------------ network
// y[s] = network(X[s]) for n samples, one thread each; the first hidden layer
// sits in shared memory.
constexpr int kFwdThreads = 64;

__global__ void __launch_bounds__(kFwdThreads)
    k_mlp_forward(const float* __restrict__ P, const float* __restrict__ X, int n,
                  float* __restrict__ y) {
  __shared__ float h1s[kQH][kFwdThreads];
  const int t = threadIdx.x;
  const int s = blockIdx.x * kFwdThreads + t;
  const bool live = s < n;
  float x[kQF];
#pragma unroll
  for (int i = 0; i < kQF; ++i) x[i] = live ? X[(int64_t)s * kQF + i] : 0.f;
  for (int j = 0; j < kQH; ++j) {
    float z = P[ob1 + j];
#pragma unroll
    for (int i = 0; i < kQF; ++i) z = fmaf(x[i], P[oW1 + i * kQH + j], z);
    h1s[j][t] = fmaxf(z, 0.f);
  }
  float out = P[ob3];
  for (int j = 0; j < kQH; ++j) {
    float z = P[ob2 + j];
    for (int i = 0; i < kQH; ++i) z = fmaf(h1s[i][t], P[oW2 + i * kQH + j], z);
    out = fmaf(fmaxf(z, 0.f), P[ow3 + j], out);
  }
  if (live) y[s] = out;
}

// Loss L = (1/2n) sum (y - t)^2 and its gradient over n samples, one CTA of
// 256 threads, samples in chunks of kGB with activations in shared memory.
// Each parameter's gradient is summed by one thread in sample order.
constexpr int kGThreads = 256;
constexpr int kGB = 128;

__global__ void __launch_bounds__(kGThreads)
    k_mlp_grad(const float* __restrict__ P, const float* __restrict__ X,
               const float* __restrict__ T, int n, float* __restrict__ grad,
               float* __restrict__ loss) {
  extern __shared__ float sm[];
  float* xs = sm;                  // kGB x 16
  float* z1 = xs + kGB * kQF;      // kGB x 64: z1, then dz1
  float* z2 = z1 + kGB * kQH;      // kGB x 64: z2, then dz2
  float* dy = z2 + kGB * kQH;      // kGB
  const int tid = threadIdx.x;
  for (int e = tid; e < kQParams; e += kGThreads) grad[e] = 0.f;
  float lsum = 0.f;  // thread 0's running loss (sample order)
  const float inv_n = 1.f / (float)n;
  for (int s0 = 0; s0 < n; s0 += kGB) {
    const int B = min(kGB, n - s0);
    __syncthreads();
    for (int e = tid; e < B * kQF; e += kGThreads) xs[e] = X[(int64_t)s0 * kQF + e];
    __syncthreads();
    for (int e = tid; e < B * kQH; e += kGThreads) {
      const int b = e / kQH, j = e % kQH;
      float z = P[ob1 + j];
#pragma unroll
      for (int i = 0; i < kQF; ++i) z = fmaf(xs[b * kQF + i], P[oW1 + i * kQH + j], z);
      z1[e] = z;
    }
    __syncthreads();
    for (int e = tid; e < B * kQH; e += kGThreads) {
      const int b = e / kQH, j = e % kQH;
      float z = P[ob2 + j];
      for (int i = 0; i < kQH; ++i) z = fmaf(fmaxf(z1[b * kQH + i], 0.f), P[oW2 + i * kQH + j], z);
      z2[e] = z;
    }
    __syncthreads();
    // output and dL/dy: one warp per sample, lanes over the 64 hidden units
    for (int b = tid >> 5; b < B; b += kGThreads / 32) {
      const int lane = tid & 31;
      float v = fmaxf(z2[b * kQH + lane], 0.f) * P[ow3 + lane] +
                fmaxf(z2[b * kQH + lane + 32], 0.f) * P[ow3 + lane + 32];
      v = wsum(v);
      if (lane == 0) dy[b] = (v + P[ob3] - T[s0 + b]) * inv_n;
    }
    __syncthreads();
    if (tid == 0)
      for (int b = 0; b < B; ++b) lsum += 0.5f * (dy[b] / inv_n) * (dy[b] / inv_n);
    // gradients of w3, b3 (they need z2 before it becomes dz2)
    for (int j = tid; j < kQH; j += kGThreads) {
      float g = 0.f;
      for (int b = 0; b < B; ++b) g = fmaf(fmaxf(z2[b * kQH + j], 0.f), dy[b], g);
      grad[ow3 + j] += g;
    }
    if (tid == kQH) {
      float g = 0.f;
      for (int b = 0; b < B; ++b) g += dy[b];
      grad[ob3] += g;
    }
    __syncthreads();
    for (int e = tid; e < B * kQH; e += kGThreads) {  // dz2 in place
      const int b = e / kQH, j = e % kQH;
      z2[e] = z2[e] > 0.f ? dy[b] * P[ow3 + j] : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < kQH * kQH; e += kGThreads) {  // W2: h1^T dz2
      const int i = e / kQH, j = e % kQH;
      float g = 0.f;
      for (int b = 0; b < B; ++b) g = fmaf(fmaxf(z1[b * kQH + i], 0.f), z2[b * kQH + j], g);
      grad[oW2 + e] += g;
    }
    for (int j = tid; j < kQH; j += kGThreads) {
      float g = 0.f;
      for (int b = 0; b < B; ++b) g += z2[b * kQH + j];
      grad[ob2 + j] += g;
    }
    __syncthreads();
    for (int e = tid; e < B * kQH; e += kGThreads) {  // dz1 in place (own entry only)
      const int b = e / kQH, i = e % kQH;
      float g = 0.f;
      for (int j = 0; j < kQH; ++j) g = fmaf(z2[b * kQH + j], P[oW2 + i * kQH + j], g);
      z1[e] = z1[e] > 0.f ? g : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < kQF * kQH; e += kGThreads) {  // W1: X^T dz1
      const int i = e / kQH, j = e % kQH;
      float g = 0.f;
      for (int b = 0; b < B; ++b) g = fmaf(xs[b * kQF + i], z1[b * kQH + j], g);
      grad[oW1 + e] += g;
    }
    for (int j = tid; j < kQH; j += kGThreads) {
      float g = 0.f;
      for (int b = 0; b < B; ++b) g += z1[b * kQH + j];
      grad[ob1 + j] += g;
    }
  }
  if (tid == 0 && loss) *loss = lsum * inv_n;
}

// Adam (Kingma & Ba 2015, Algorithm 1) with bias correction, step >= 1.
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, int n, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = 0.9f * m1[i] + 0.1f * gi;
  const float b = 0.999f * m2[i] + 0.001f * gi * gi;
  m1[i] = a;
  m2[i] = b;
  P[i] -= lr * (a / c1) / (sqrtf(b / c2) + 1e-8f);
}

// q = ceil(y + margin) clamped to [1, q_fixed]
__global__ void k_q_from_pred(const float* __restrict__ y, float margin, int q_fixed,
                              int* __restrict__ q_out) {
  const float v = ceilf(y[0] + margin);
  *q_out = (int)fminf((float)q_fixed, fmaxf(1.f, isfinite(v) ? v : (float)q_fixed));
}

}  // namespace

void q_features(const Csr& csr, const Csr& csc, int64_t d, int ell, int q_fixed,
                const double* fro2, const float* S0, float* feat, unsigned* acc_dev,
                cudaStream_t s) {
  // acc_dev: 3 unsigned, padding, then 2 unsigned long long (16-byte offset)
  unsigned long long* acc64 = reinterpret_cast<unsigned long long*>(acc_dev + 4);
  SFD_CUDA(cudaMemsetAsync(acc_dev, 0, 4 * sizeof(unsigned) + 2 * sizeof(unsigned long long), s));
  if (csr.nseg > 0) {
    k_qf_rows<<<kQB, 256, 0, s>>>(csr.ptr, csr.val, csr.nseg, acc_dev, acc64);
    SFD_LAUNCH_CHECK();
  }
  k_qf_cols<<<kQB, 256, 0, s>>>(csc.ptr, (int)d, acc_dev, acc64);
  SFD_LAUNCH_CHECK();
  k_qf_final<<<1, 256, 0, s>>>(acc_dev, acc64, fro2, S0, ell, csr.nseg, (long long)csr.nnz, (int)d,
                               q_fixed, feat);
  SFD_LAUNCH_CHECK();
}

void mlp_forward(const float* P, const float* X, int n, float* y, cudaStream_t s) {
  if (n <= 0) return;
  k_mlp_forward<<<(n + kFwdThreads - 1) / kFwdThreads, kFwdThreads, 0, s>>>(P, X, n, y);
  SFD_LAUNCH_CHECK();
}

void predict_q(const float* P, const float* feat, float margin, int q_fixed, float* y_tmp,
               int* q_out, cudaStream_t s) {
  mlp_forward(P, feat, 1, y_tmp, s);
  k_q_from_pred<<<1, 1, 0, s>>>(y_tmp, margin, q_fixed, q_out);
  SFD_LAUNCH_CHECK();
}

size_t mlp_grad_smem_bytes() {
  return (size_t)(kGB * kQF + 2 * kGB * kQH + kGB) * sizeof(float);
}

void mlp_grad(const float* P, const float* X, const float* T, int n, float* grad, float* loss,
              cudaStream_t s) {
  static std::atomic<unsigned> attr{0};
  int dev = 0;
  SFD_CUDA(cudaGetDevice(&dev));
  if (dev < 32 && !(attr.load() & (1u << dev))) {
    SFD_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)mlp_grad_smem_bytes()));
    attr.fetch_or(1u << dev);
  }
  k_mlp_grad<<<1, kGThreads, mlp_grad_smem_bytes(), s>>>(P, X, T, n, grad, loss);
  SFD_LAUNCH_CHECK();
}

void adam_update(float* P, const float* grad, float* m1, float* m2, int step, float lr,
                 cudaStream_t s) {
  const float c1 = 1.f - powf(0.9f, (float)step);
  const float c2 = 1.f - powf(0.999f, (float)step);
  k_adam<<<(kQParams + 255) / 256, 256, 0, s>>>(P, grad, m1, m2, kQParams, lr, c1, c2);
  SFD_LAUNCH_CHECK();
}

}  // namespace sfd
