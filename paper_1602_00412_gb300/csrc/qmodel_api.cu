// C ABI of the learned power count's network (include/sfd.h): prediction,
// loss gradient and Adam training on the GPU. Host arrays in and out; each
// call allocates its device buffers and runs synchronously.
#include <string.h>

#include <cmath>
#include <cstdint>
#include <random>
#include <vector>

#include "engine.cuh"

using namespace sfd;

namespace {

int code_of(const CudaError& e) {
  return e.err == cudaErrorMemoryAllocation ? SFD_ENOMEM : SFD_ECUDA;
}

bool all_finite(const float* p, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Device copies of a call's arrays, freed together.
struct Buffers {
  DevArena A;
  cudaStream_t s = nullptr;
  Buffers() { SFD_CUDA(cudaStreamCreate(&s)); }
  ~Buffers() {
    if (s) cudaStreamSynchronize(s);
    A.release();
    if (s) cudaStreamDestroy(s);
  }
  float* upload(const float* h, int64_t n) {
    float* d = A.alloc<float>((size_t)std::max<int64_t>(n, 1));
    if (n > 0) SFD_CUDA(cudaMemcpyAsync(d, h, n * sizeof(float), cudaMemcpyHostToDevice, s));
    return d;
  }
};

}  // namespace

extern "C" {

int sfd_q_predict(int64_t n, const float* features, const float* params, float* y_out) {
  if (n < 0 || n > INT32_MAX || !params || (n > 0 && (!features || !y_out))) return SFD_EINVAL;
  if (n == 0) return SFD_OK;
  try {
    Buffers B;
    float* P = B.upload(params, kQParams);
    float* X = B.upload(features, n * kQF);
    float* y = B.A.alloc<float>(n);
    mlp_forward(P, X, (int)n, y, B.s);
    SFD_CUDA(cudaMemcpyAsync(y_out, y, n * sizeof(float), cudaMemcpyDeviceToHost, B.s));
    SFD_CUDA(cudaStreamSynchronize(B.s));
    return SFD_OK;
  } catch (const CudaError& e) {
    return code_of(e);
  }
}

int sfd_q_grad(int64_t n, const float* features, const float* targets, const float* params,
               float* grad_out, float* loss_out) {
  if (n < 1 || n > INT32_MAX || !features || !targets || !params || !grad_out) return SFD_EINVAL;
  try {
    Buffers B;
    float* P = B.upload(params, kQParams);
    float* X = B.upload(features, n * kQF);
    float* T = B.upload(targets, n);
    float* g = B.A.alloc<float>(kQParams);
    float* l = B.A.alloc<float>(1);
    mlp_grad(P, X, T, (int)n, g, l, B.s);
    SFD_CUDA(cudaMemcpyAsync(grad_out, g, kQParams * sizeof(float), cudaMemcpyDeviceToHost, B.s));
    float loss = 0.f;
    SFD_CUDA(cudaMemcpyAsync(&loss, l, sizeof(float), cudaMemcpyDeviceToHost, B.s));
    SFD_CUDA(cudaStreamSynchronize(B.s));
    if (loss_out) *loss_out = loss;
    return SFD_OK;
  } catch (const CudaError& e) {
    return code_of(e);
  }
}

int sfd_q_train(int64_t n, const float* features, const float* targets, int32_t epochs,
                int32_t batch, float lr, uint64_t seed, float* params, float* loss_out) {
  if (n < 1 || n > INT32_MAX || !features || !targets || !params || epochs < 0 || batch < 1 ||
      !(lr > 0.f) || !std::isfinite(lr))
    return SFD_EINVAL;
  if (!all_finite(features, n * kQF) || !all_finite(targets, n) || !all_finite(params, kQParams))
    return SFD_EINVAL;
  try {
    Buffers B;
    float* P = B.upload(params, kQParams);
    float* g = B.A.alloc<float>(kQParams);
    float* m1 = B.A.alloc<float>(kQParams);
    float* m2 = B.A.alloc<float>(kQParams);
    float* l = B.A.alloc<float>(1);
    SFD_CUDA(cudaMemsetAsync(m1, 0, kQParams * sizeof(float), B.s));
    SFD_CUDA(cudaMemsetAsync(m2, 0, kQParams * sizeof(float), B.s));
    float* X = B.A.alloc<float>((size_t)n * kQF);
    float* T = B.A.alloc<float>((size_t)n);
    // epoch order: Fisher-Yates over a 64-bit Mersenne Twister (both fully
    // specified, so the order is the same on every platform)
    std::mt19937_64 rng(seed);
    std::vector<int64_t> perm(n);
    std::vector<float> hx((size_t)n * kQF), ht(n);
    int step = 0;
    for (int ep = 0; ep < epochs; ++ep) {
      for (int64_t i = 0; i < n; ++i) perm[i] = i;
      for (int64_t i = n - 1; i > 0; --i) {
        const int64_t j = (int64_t)(rng() % (uint64_t)(i + 1));
        std::swap(perm[i], perm[j]);
      }
      SFD_CUDA(cudaStreamSynchronize(B.s));  // the previous epoch has read hx / ht
      for (int64_t i = 0; i < n; ++i) {
        memcpy(&hx[i * kQF], features + perm[i] * kQF, kQF * sizeof(float));
        ht[i] = targets[perm[i]];
      }
      SFD_CUDA(cudaMemcpyAsync(X, hx.data(), hx.size() * sizeof(float), cudaMemcpyHostToDevice, B.s));
      SFD_CUDA(cudaMemcpyAsync(T, ht.data(), ht.size() * sizeof(float), cudaMemcpyHostToDevice, B.s));
      for (int64_t s0 = 0; s0 < n; s0 += batch) {
        const int bn = (int)std::min<int64_t>(batch, n - s0);
        mlp_grad(P, X + s0 * kQF, T + s0, bn, g, nullptr, B.s);
        adam_update(P, g, m1, m2, ++step, lr, B.s);
      }
    }
    // loss of the trained network on the whole set (original order)
    SFD_CUDA(cudaMemcpyAsync(X, features, (size_t)n * kQF * sizeof(float), cudaMemcpyHostToDevice, B.s));
    SFD_CUDA(cudaMemcpyAsync(T, targets, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, B.s));
    mlp_grad(P, X, T, (int)n, g, l, B.s);
    float loss = 0.f;
    SFD_CUDA(cudaMemcpyAsync(params, P, kQParams * sizeof(float), cudaMemcpyDeviceToHost, B.s));
    SFD_CUDA(cudaMemcpyAsync(&loss, l, sizeof(float), cudaMemcpyDeviceToHost, B.s));
    SFD_CUDA(cudaStreamSynchronize(B.s));
    if (loss_out) *loss_out = loss;
    return SFD_OK;
  } catch (const CudaError& e) {
    return code_of(e);
  }
}

}  // extern "C"
