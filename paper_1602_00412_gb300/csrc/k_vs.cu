// VerifySpectral (Alg. 6, Sec. 4.1) on C = (A'^T A' - B'^T B') / (Delta / 2)
// as BoostedSparseShrink (Alg. 4) calls it. x is a Philox Gaussian vector
// normalised to the unit sphere; p power steps keep x normalised and add
// log ||C x_t|| to a running sum, so ||C^p x|| never overflows. Accept iff the
// sum is <= 0 (the host compares).
//
// One step: u = A' x (CSR), w = B' x (reduction over the d rows of B'^T),
// v = A'^T u (CSC) - B'^T w, ||v||, x <- v / ||v|| (the division is applied
// where x is read, and B' x is formed while v is written, so B'^T is read
// once per step). Every reduction runs in a fixed order (deterministic).
#include <math.h>

#include <algorithm>

#include "sfd_internal.cuh"

namespace sfd {

namespace {

// fixed grids, so every reduction has a fixed order; three blocks of
// k_v_update per SM (its register budget) make one wave on 152 SMs
constexpr int kVsBlocks = 3 * 152;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial[b] = sum over rows of block b's stripe of x_j^2 (fp32 in-block, fixed grid)
__global__ void k_norm2_partial(const float* __restrict__ x, int64_t n, float* __restrict__ part) {
  float a = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a = fmaf(x[i], x[i], a);
  __shared__ float red[32];
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    t = warp_sum(t);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

// scal[0] logsum, scal[1] inverse norm of the current x, scal[2] 1 if some C x_t was 0.
// mode 0: initial normalisation (no log term); mode 1: a power step with factor *scale.
// Run by one block of 256 threads (sh: 256 doubles of shared memory).
__device__ void norm_finalize_block(const float* part, int nb, const double* scale_ptr, int mode,
                                    double* scal, double* sh) {
  double a = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) a += (double)__ldcg(&part[i]);
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double n2 = sh[0];
    if (mode == 0) scal[0] = 0.0;
    if (n2 > 0.0) {
      if (mode == 1) scal[0] += log(*scale_ptr) + 0.5 * log(n2);
      scal[1] = 1.0 / sqrt(n2);
    } else {
      scal[1] = 0.0;
      if (mode == 1) scal[2] = 1.0;
    }
  }
}

__global__ void __launch_bounds__(256)
    k_norm_finalize(const float* __restrict__ part, int nb, const double* __restrict__ scale_ptr,
                    int mode, double* __restrict__ scal) {
  __shared__ double sh[256];
  norm_finalize_block(part, nb, scale_ptr, mode, scal, sh);
}

// wpart[b][c] = sum over the rows j of stripe b of Bt[j][c] * x[j]. A warp
// reads a row of B'^T as float4 lanes (ld % 4 == 0); the 8 warps of a block
// take rows j = warp, warp + 8, ... of the stripe, four at a time, and their
// partial sums are added in warp order (fixed).
__global__ void __launch_bounds__(256)
    k_btx_partial(const float* __restrict__ Bt, int ld, int ell, int64_t d,
                  const float* __restrict__ x, const double* __restrict__ xscale,
                  float* __restrict__ wpart) {
  __shared__ float4 red[8][kMaxEll / 4];
  // x is read as x * xs (its pending normalisation; 1 when xscale is null)
  const float xs = xscale ? (float)xscale[1] : 1.f;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int nvec = (ell + 3) >> 2;
  const int64_t rows = (d + gridDim.x - 1) / gridDim.x;
  const int64_t j0 = blockIdx.x * rows, j1 = min(d, j0 + rows);
  const float4* B4 = reinterpret_cast<const float4*>(Bt);
  const int ld4 = ld >> 2;
  for (int c4 = lane; c4 < (kMaxEll / 4); c4 += 32) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c4 < nvec) {
      int64_t j = j0 + wp;
      for (; j + 24 < j1; j += 32) {  // four rows of this warp in flight
        const float4 b0 = B4[(j + 0) * ld4 + c4], b1 = B4[(j + 8) * ld4 + c4];
        const float4 b2 = B4[(j + 16) * ld4 + c4], b3 = B4[(j + 24) * ld4 + c4];
        const float x0 = x[j] * xs, x1 = x[j + 8] * xs, x2 = x[j + 16] * xs, x3 = x[j + 24] * xs;
        a.x = fmaf(b0.x, x0, a.x); a.y = fmaf(b0.y, x0, a.y); a.z = fmaf(b0.z, x0, a.z); a.w = fmaf(b0.w, x0, a.w);
        a.x = fmaf(b1.x, x1, a.x); a.y = fmaf(b1.y, x1, a.y); a.z = fmaf(b1.z, x1, a.z); a.w = fmaf(b1.w, x1, a.w);
        a.x = fmaf(b2.x, x2, a.x); a.y = fmaf(b2.y, x2, a.y); a.z = fmaf(b2.z, x2, a.z); a.w = fmaf(b2.w, x2, a.w);
        a.x = fmaf(b3.x, x3, a.x); a.y = fmaf(b3.y, x3, a.y); a.z = fmaf(b3.z, x3, a.z); a.w = fmaf(b3.w, x3, a.w);
      }
      for (; j < j1; j += 8) {
        const float4 b0 = B4[j * ld4 + c4];
        const float x0 = x[j] * xs;
        a.x = fmaf(b0.x, x0, a.x); a.y = fmaf(b0.y, x0, a.y); a.z = fmaf(b0.z, x0, a.z); a.w = fmaf(b0.w, x0, a.w);
      }
    }
    red[wp][c4] = a;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ell; c += blockDim.x) {
    float t = 0.f;
    for (int w = 0; w < 8; ++w) t += reinterpret_cast<const float*>(&red[w][0])[c];
    wpart[blockIdx.x * ell + c] = t;
  }
}

// w[c] = s * sum_b wpart[b][c] (s = (float)scal[1], the pending normalisation
// of the x the partials were formed from): one block per column c,
// fixed-order tree
__global__ void __launch_bounds__(256)
    k_btx_reduce(const float* __restrict__ wpart, int nb, int ell, const double* __restrict__ scal,
                 float* __restrict__ w) {
  const int c = blockIdx.x;
  float a = 0.f;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) a += wpart[b * ell + c];
  __shared__ float red[8];
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    w[c] = t * (float)scal[1];
  }
}

// v[j] -= sum_c Bt[j][c] w[c]; part[block] = sum of v[j]^2 of the block
// (fixed grid). A warp takes four rows at a time: their float4 row pieces and
// the four v entries are loaded before any arithmetic, so the loads overlap;
// lane 0 keeps the block's squares in row order. With the rows of B'^T in
// registers, the warps also form the next step's B' v partials
// (wpart[block][c] = sum over the block's rows of Bt[j][c] v[j], v not yet
// normalised: k_btx_reduce applies the norm), so B'^T is read once per
// step. The last block to finish (a ticket on *counter, reset after use)
// adds the parts up and updates the log-sum and the inverse norm of v
// (norm_finalize_block, mode 1), so the step needs no separate reduction
// launch.
// WIDE: l > 128 (a row of B'^T takes two float4 per lane); otherwise one,
// which leaves the registers to hold the next four rows while the current
// four are reduced (the loads of iteration i + 1 are in flight during the
// shuffles of iteration i).
template <bool WIDE>
__global__ void __launch_bounds__(256, 3)
    k_v_update(float* __restrict__ v, const float* __restrict__ Bt, int ld, int ell, int64_t d,
               const float* __restrict__ w, float* __restrict__ part, float* __restrict__ wpart,
               const double* __restrict__ scale_ptr, double* __restrict__ scal,
               unsigned* __restrict__ counter) {
  __shared__ float4 ws[kMaxEll / 4];
  __shared__ float4 red4[8][kMaxEll / 4];
  __shared__ float red[8];
  __shared__ double sh[256];
  __shared__ bool last;
  const int nvec = (ell + 3) >> 2;  // <= 64
  for (int c = threadIdx.x; c < kMaxEll / 4; c += blockDim.x) {
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    if (4 * c + 0 < ell) t.x = w[4 * c + 0];
    if (4 * c + 1 < ell) t.y = w[4 * c + 1];
    if (4 * c + 2 < ell) t.z = w[4 * c + 2];
    if (4 * c + 3 < ell) t.w = w[4 * c + 3];
    ws[c] = t;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const float4* B4 = reinterpret_cast<const float4*>(Bt);
  const int ld4 = ld >> 2;
  const int64_t stride = (int64_t)gridDim.x * 8 * 4;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 q0 = lane < nvec ? ws[lane] : z4;
  const float4 q1 = WIDE && lane + 32 < nvec ? ws[lane + 32] : z4;
  float acc2 = 0.f;
  float4 wa0 = z4, wa1 = z4;  // next step's B' v partials, columns lane and lane + 32
  int64_t j = ((int64_t)blockIdx.x * 8 + wp) * 4;
  float4 b0[4], b1[4];
  float vv[4];
  auto load = [&](int64_t jj, float4 (&c0)[4], float4 (&c1)[4], float (&cv)[4]) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const bool row = jj + r < d;
      c0[r] = row && lane < nvec ? B4[(jj + r) * ld4 + lane] : z4;
      c1[r] = WIDE && row && lane + 32 < nvec ? B4[(jj + r) * ld4 + lane + 32] : z4;
      cv[r] = row && lane == 0 ? v[jj + r] : 0.f;
    }
  };
  // prefetch only where the registers allow it (one float4 per lane and row)
  constexpr bool kPrefetch = !WIDE;
  if (kPrefetch && j < d) load(j, b0, b1, vv);
  for (; j < d; j += stride) {
    float4 n0[4], n1[4];
    float nvv[4];
    if (!kPrefetch) load(j, b0, b1, vv);
    else if (j + stride < d) load(j + stride, n0, n1, nvv);
    float s[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float t = b0[r].x * q0.x;
      t = fmaf(b0[r].y, q0.y, t);
      t = fmaf(b0[r].z, q0.z, t);
      t = fmaf(b0[r].w, q0.w, t);
      if (WIDE) {
        t = fmaf(b1[r].x, q1.x, t);
        t = fmaf(b1[r].y, q1.y, t);
        t = fmaf(b1[r].z, q1.z, t);
        t = fmaf(b1[r].w, q1.w, t);
      }
      s[r] = warp_sum(t);
    }
    float nv[4];  // the new v (lane 0; 0 past d)
#pragma unroll
    for (int r = 0; r < 4; ++r) nv[r] = j + r < d ? vv[r] - s[r] : 0.f;
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (j + r < d) {
          v[j + r] = nv[r];
          acc2 = fmaf(nv[r], nv[r], acc2);
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float y = __shfl_sync(0xffffffffu, nv[r], 0);
      wa0.x = fmaf(b0[r].x, y, wa0.x); wa0.y = fmaf(b0[r].y, y, wa0.y);
      wa0.z = fmaf(b0[r].z, y, wa0.z); wa0.w = fmaf(b0[r].w, y, wa0.w);
      if (WIDE) {
        wa1.x = fmaf(b1[r].x, y, wa1.x); wa1.y = fmaf(b1[r].y, y, wa1.y);
        wa1.z = fmaf(b1[r].z, y, wa1.z); wa1.w = fmaf(b1[r].w, y, wa1.w);
      }
    }
    if (kPrefetch && j + stride < d) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        b0[r] = n0[r];
        if (WIDE) b1[r] = n1[r];
        vv[r] = nvv[r];
      }
    }
  }
  red4[wp][lane] = wa0;
  red4[wp][lane + 32] = wa1;
  if (lane == 0) red[wp] = acc2;
  __syncthreads();
  for (int c = threadIdx.x; c < ell; c += blockDim.x) {
    float t = 0.f;
    for (int i = 0; i < 8; ++i) t += reinterpret_cast<const float*>(&red4[i][0])[c];
    wpart[blockIdx.x * ell + c] = t;
  }
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < 8; ++i) t += red[i];
    part[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    norm_finalize_block(part, gridDim.x, scale_ptr, 1, scal, sh);
    if (threadIdx.x == 0) *counter = 0u;
  }
}

__global__ void k_delta(const double* __restrict__ fro2a, double* __restrict__ scal, int ell) {
  const double a = *fro2a, b = scal[kSfro2b];
  const double delta = (a - b) / ((double)(6.0 / 41.0) * ell);
  scal[kSdelta] = delta;
  scal[kSscale] = delta > 0.0 ? 2.0 / delta : 0.0;
  // Delta/2 at the resolution of the fp32 check: accept (64 * 2^-24 * ||A'||_F^2)
  scal[kSsmall] = (delta / 2.0 <= 64.0 * 5.9604644775390625e-8 * a) ? 1.0 : 0.0;
}

__global__ void k_verdict(const double* __restrict__ fro2a, const double* __restrict__ scal,
                          const int* __restrict__ flags, const float* __restrict__ evals, int ell,
                          int verify, Verdict* __restrict__ out) {
  Verdict v;
  v.fro2a = *fro2a;
  v.fro2b = scal[kSfro2b];
  v.delta = scal[kSdelta];
  v.small = scal[kSsmall] != 0.0;
  v.zero = scal[kSzero] != 0.0;
  v.logsum = v.small || v.zero ? -INFINITY : scal[kSlogsum];
  v.ok = !verify || v.small || v.zero || v.logsum <= 0.0;
  v.timeout = flags[2];
  double c = 0.0;
  for (int i = 0; i < ell; ++i) c += (double)evals[i];
  v.captured = c;
  *out = v;
}

}  // namespace

void launch_delta(const double* fro2a, double* scal, int ell, cudaStream_t s) {
  k_delta<<<1, 1, 0, s>>>(fro2a, scal, ell);
  SFD_LAUNCH_CHECK();
}

void launch_verdict(const double* fro2a, const double* scal, const int* flags,
                    const float* evals, int ell, int verify, Verdict* out, cudaStream_t s) {
  k_verdict<<<1, 1, 0, s>>>(fro2a, scal, flags, evals, ell, verify, out);
  SFD_LAUNCH_CHECK();
}

namespace {

// One power step x -> v (u = A'x, w = B'x, v = A'^T u - B'^T w, log ||v||,
// v /= ||v||); the caller swaps x and v.
// x is held unnormalised: its consumers (A' x, B' x) read x * scal[1], the
// value a separate scaling pass would have stored, and k_v_update's last
// block sets scal[1] for the new v.
// ws.wpart holds the B' x partials of the unnormalised x on entry (from the
// preamble or the previous step's k_v_update) and those of the new v on exit.
void vs_step(const VsArgs& a, Workspace& ws, float* x, float* u, float* v, float* w, float* part,
             double* scal, unsigned* counter, cudaStream_t s) {
  spmv(*a.csr, x, u, ws.partial_rows, s, scal);
  k_btx_reduce<<<a.ell, 256, 0, s>>>(ws.wpart, kVsBlocks, a.ell, scal, w);
  SFD_LAUNCH_CHECK();
  spmv(*a.csc, u, v, ws.partial_rows, s);
  if (a.ell > 128)
    k_v_update<true><<<kVsBlocks, 256, 0, s>>>(v, a.Bt, a.ld, a.ell, a.d, w, part, ws.wpart,
                                               a.scale_dev, scal, counter);
  else
    k_v_update<false><<<kVsBlocks, 256, 0, s>>>(v, a.Bt, a.ld, a.ell, a.d, w, part, ws.wpart,
                                                a.scale_dev, scal, counter);
  SFD_LAUNCH_CHECK();
}

// Capture `steps` power steps; *nodes = the kernels in the graph. The launches
// made while capturing are taken off the launch counter again: the kernels
// run when the graph is replayed, and each replay is counted then.
cudaGraphExec_t capture(cudaStream_t s, int steps, const VsArgs& a, Workspace& ws, float* x,
                        float* u, float* v, float* w, float* part, double* scal, unsigned* counter,
                        size_t* nodes) {
  SFD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  for (int t = 0; t < steps; ++t) {
    vs_step(a, ws, x, u, v, w, part, scal, counter, s);
    std::swap(x, v);
  }
  cudaGraph_t g = nullptr;
  SFD_CUDA(cudaStreamEndCapture(s, &g));
  *nodes = 0;
  cudaGraphGetNodes(g, nullptr, nodes);
  __atomic_sub_fetch(&g_kernel_launches, (unsigned long long)*nodes, __ATOMIC_RELAXED);
  cudaGraphExec_t e = nullptr;
  const cudaError_t rc = cudaGraphInstantiate(&e, g, 0);
  cudaGraphDestroy(g);
  if (rc != cudaSuccess) throw CudaError{rc, "cudaGraphInstantiate"};
  return e;
}

}  // namespace

void verify_spectral(const VsArgs& a, Workspace& ws, cudaStream_t s, VsGraphs* graphs) {
  float* x = ws.vec0;   // d
  float* u = ws.vec1;   // m
  float* v = ws.vec2;   // d
  float* w = ws.wpart + kVsBlocks * kMaxEll;  // ell
  float* part = ws.wpart + kVsBlocks * kMaxEll + kMaxEll;  // kVsBlocks
  double* scal = ws.scalars + kSlogsum;
  unsigned* counter = reinterpret_cast<unsigned*>(ws.flags + 8);  // k_v_update's tickets
  SFD_CUDA(cudaMemsetAsync(scal, 0, 4 * sizeof(double), s));
  SFD_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
  launch_gauss_fill(x, a.d, 1, 1, a.seed, a.b, a.r, 2 /* tag of Alg. 6's x */, s);
  k_norm2_partial<<<kVsBlocks, 256, 0, s>>>(x, a.d, part);
  SFD_LAUNCH_CHECK();
  k_norm_finalize<<<1, 256, 0, s>>>(part, kVsBlocks, nullptr, 0, scal);  // x stays unscaled
  SFD_LAUNCH_CHECK();
  k_btx_partial<<<kVsBlocks, 256, 0, s>>>(a.Bt, a.ld, a.ell, a.d, x, nullptr, ws.wpart);
  SFD_LAUNCH_CHECK();
  if (!graphs) {
    for (int t = 0; t < a.p; ++t) {
      vs_step(a, ws, x, u, v, w, part, scal, counter, s);
      std::swap(x, v);
    }
    return;
  }
  if (!graphs->one) {
    size_t n1 = 0, n2 = 0;
    graphs->one = capture(s, 1, a, ws, x, u, v, w, part, scal, counter, &n1);
    graphs->two = capture(s, 2, a, ws, x, u, v, w, part, scal, counter, &n2);
    graphs->kernels_per_step = (int)n1;
  }
  // x starts in vec0 and is back there after every two steps
  for (int t = 0; t + 1 < a.p; t += 2) SFD_CUDA(cudaGraphLaunch(graphs->two, s));
  if (a.p & 1) SFD_CUDA(cudaGraphLaunch(graphs->one, s));
  __atomic_add_fetch(&g_kernel_launches, (unsigned long long)graphs->kernels_per_step * a.p,
                     __ATOMIC_RELAXED);
}

}  // namespace sfd
