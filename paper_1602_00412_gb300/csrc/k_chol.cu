// Cholesky factor and its inverse for CholeskyQR (the GramSchmidt step of
// Alg. 1): G + shift I = L L^T and Rinv = L^-T, for k <= 128, one CTA.
//
// Blocked right-looking factorisation with 16-wide panels. For each panel:
//   1. one warp factors the 16 x 16 diagonal block in registers (lane i holds
//      row i; L[t][j] is broadcast with shuffles) and inverts it by forward
//      substitution (lane c solves column c);
//   2. the panel below is L21 = A21 L11^-T (a 16-term product per entry);
//   3. the trailing lower triangle is updated, A22 -= L21 L21^T, in 4 x 4
//      register tiles.
// Then the off-diagonal blocks of L^-1 follow block diagonal by block
// diagonal: X_ij = -X_ii sum_{t=j}^{i-1} L_it X_tj. That is 3 barriers per
// panel and 2 per block diagonal, instead of one per column.
#include <atomic>

#include "sfd_internal.cuh"

namespace sfd {
namespace {

constexpr int kCB = 16;         // panel width
constexpr int kCThreads = 256;
constexpr unsigned kFull = 0xffffffffu;
constexpr size_t kCholBlkSmemMax = 220 * 1024;  // dynamic shared memory of the fp64 form

// scalar helpers: the fp32 instantiation keeps the fp32 intrinsics
__device__ __forceinline__ float b_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double b_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float b_rsqrt(float x) { return rsqrtf(x); }  // hardware estimate
__device__ __forceinline__ double b_rsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float b_ldexp(float x, int e) { return ldexpf(x, e); }
__device__ __forceinline__ double b_ldexp(double x, int e) { return ldexp(x, e); }

// T: float, or double for the FP64 factor of the accurate CholeskyQR passes
// (G is read and Rinv written as fp32 either way).
template <typename T>
__global__ void __launch_bounds__(kCThreads)
    k_chol_inv_blk(const float* __restrict__ G, int k, float* __restrict__ Rinv,
                   int* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  const int KP = (k + kCB - 1) / kCB * kCB;  // padded with the identity
  const int LD = KP + 1;
  const int NB = KP / kCB;
  T* A = sm;             // KP x LD, lower triangle becomes L
  T* Li = A + KP * LD;   // KP x LD, lower triangle becomes L^-1
  T* S = Li + KP * LD;   // NB x 256 scratch
  __shared__ T red[kCThreads / 32];
  __shared__ T shift_sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // G's entries arrive by cp.async in fp32 (all in flight at once), by
  // converting loads in fp64; padding is the identity
  for (int i = warp; i < KP; i += kCThreads / 32)
    for (int j = lane; j < KP; j += 32) {
      if (i < k && j < k) {
        if constexpr (sizeof(T) == sizeof(float)) {
          const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&A[i * LD + j]);
          asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst),
                       "l"(G + (int64_t)i * k + j));
        } else {
          A[i * LD + j] = (T)G[(int64_t)i * k + j];
        }
      } else {
        A[i * LD + j] = (i == j) ? (T)1 : (T)0;
      }
    }
  asm volatile("cp.async.commit_group;" ::);
  asm volatile("cp.async.wait_group 0;" ::);
  __syncthreads();
  T tr = 0;
  for (int i = tid; i < k; i += kCThreads) tr += A[i * LD + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(kFull, tr, o);
  if (lane == 0) red[warp] = tr;
  __syncthreads();
  if (tid == 0) {
    T t = 0;
    for (int w = 0; w < kCThreads / 32; ++w) t += red[w];
    shift_sh = t > (T)0 ? b_ldexp(t / (T)k, -20) : (T)1e-30f;
  }
  __syncthreads();
  const T shift = shift_sh;
  for (int i = tid; i < k; i += kCThreads) A[i * LD + i] += shift;
  __syncthreads();

  for (int p = 0; p < NB; ++p) {
    const int j0 = p * kCB;
    // ---- 1. diagonal block: factor and invert in registers (warp 0)
    if (warp == 0) {
      const int i = lane & 15;  // lanes 16..31 repeat lanes 0..15
      T d[kCB];
#pragma unroll
      for (int t = 0; t < kCB; ++t) d[t] = A[(j0 + i) * LD + j0 + t];
      int clamped = 0;
      T rdiag[kCB];  // 1 / L[j][j], the same in every lane
#pragma unroll
      for (int j = 0; j < kCB; ++j) {
        T piv = __shfl_sync(kFull, d[j], j);
        clamped += !(piv > (T)0);
        piv = piv > (T)0 ? piv : shift;
        const T inv = b_rsqrt(piv);  // fp32: the hardware reciprocal square root
        rdiag[j] = inv;
        const T lij = i > j ? d[j] * inv : (i == j ? piv * inv : (T)0);
        d[j] = lij;
#pragma unroll
        for (int t = 0; t < kCB; ++t) {
          if (t > j) {
            const T ltj = __shfl_sync(kFull, lij, t);
            if (t <= i) d[t] = b_fma(-lij, ltj, d[t]);
          }
        }
      }
      if (lane == 0 && clamped) atomicAdd(&flags[1], clamped);
      // column c = i of the inverse of the block
      T x[kCB];
#pragma unroll
      for (int r = 0; r < kCB; ++r) {
        T s = r == i ? (T)1 : (T)0;
#pragma unroll
        for (int t = 0; t < r; ++t) s = b_fma(-__shfl_sync(kFull, d[t], r), x[t], s);
        x[r] = r >= i ? s * rdiag[r] : (T)0;
      }
      if (lane < kCB) {
#pragma unroll
        for (int t = 0; t < kCB; ++t) {
          if (t <= i) A[(j0 + i) * LD + j0 + t] = d[t];
          Li[(j0 + t) * LD + j0 + i] = x[t];  // column i; zero above the diagonal
        }
      }
    }
    __syncthreads();
    const int below = KP - j0 - kCB;
    if (below == 0) break;
    // ---- 2. panel below: L21[r][c] = sum_{t<=c} A21[r][t] Linv11[c][t]
    //         (one thread per row: it reads the whole row before writing it)
    if (tid < below) {
      const int r = j0 + kCB + tid;
      const T* X = Li + j0 * LD + j0;
      T a[kCB];
#pragma unroll
      for (int t = 0; t < kCB; ++t) a[t] = A[r * LD + j0 + t];
#pragma unroll
      for (int c = 0; c < kCB; ++c) {
        T s = 0;
#pragma unroll
        for (int t = 0; t <= c; ++t) s = b_fma(a[t], X[c * LD + t], s);
        A[r * LD + j0 + c] = s;
      }
    }
    __syncthreads();
    // ---- 3. trailing update of the lower triangle in 4 x 4 tiles
    {
      const int nb4 = below >> 2;
      const int ntile = nb4 * (nb4 + 1) / 2;
      const int base = j0 + kCB;
      for (int e = tid; e < ntile; e += kCThreads) {
        int bi = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
        while (bi * (bi + 1) / 2 > e) --bi;
        while ((bi + 1) * (bi + 2) / 2 <= e) ++bi;
        const int bj = e - bi * (bi + 1) / 2;
        const int r0 = base + bi * 4, c0 = base + bj * 4;
        T acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = 0;
#pragma unroll 4
        for (int t = 0; t < kCB; ++t) {
          T xr[4], yc[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            xr[u] = A[(r0 + u) * LD + j0 + t];
            yc[u] = A[(c0 + u) * LD + j0 + t];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = b_fma(xr[u], yc[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (c0 + v <= r0 + u) A[(r0 + u) * LD + c0 + v] -= acc[u][v];
      }
      __syncthreads();
    }
  }

  // ---- off-diagonal blocks of L^-1, one block diagonal at a time
  for (int dl = 1; dl < NB; ++dl) {
    const int nout = (NB - dl) * kCB * kCB;
    for (int e = tid; e < nout; e += kCThreads) {
      const int jb = e >> 8, rr = (e >> 4) & 15, cc = e & 15;
      const int ib = jb + dl;
      const int row = ib * kCB + rr, col = jb * kCB + cc;
      // t over blocks jb .. ib-1 (Li[t][col] is 0 above the diagonal of block jb)
      T s0 = 0, s1 = 0;
      for (int t0 = jb * kCB; t0 < ib * kCB; t0 += kCB) {
#pragma unroll
        for (int t = 0; t < kCB; t += 2) {
          s0 = b_fma(A[row * LD + t0 + t], Li[(t0 + t) * LD + col], s0);
          s1 = b_fma(A[row * LD + t0 + t + 1], Li[(t0 + t + 1) * LD + col], s1);
        }
      }
      S[e] = s0 + s1;
    }
    __syncthreads();
    for (int e = tid; e < nout; e += kCThreads) {
      const int jb = e >> 8, rr = (e >> 4) & 15, cc = e & 15;
      const int ib = jb + dl;
      const int row = ib * kCB + rr, col = jb * kCB + cc;
      T s = 0;
#pragma unroll
      for (int u = 0; u < kCB; ++u)  // Li[row][ib*16 + u] is 0 for u > rr
        s = b_fma(Li[row * LD + ib * kCB + u], S[(jb << 8) + (u << 4) + cc], s);
      Li[row * LD + col] = -s;
    }
    __syncthreads();
  }
  // Rinv = (L^-1)^T, upper triangular
  for (int c = warp; c < k; c += kCThreads / 32)
    for (int i = lane; i < k; i += 32) Rinv[c * k + i] = c <= i ? (float)Li[i * LD + c] : 0.f;
}

}  // namespace

size_t chol_blk_smem_bytes(int k, bool fp64) {
  const int KP = (k + kCB - 1) / kCB * kCB;
  return ((size_t)2 * KP * (KP + 1) + (size_t)(KP / kCB) * kCB * kCB) *
         (fp64 ? sizeof(double) : sizeof(float));
}

bool chol_blk_supported(int k, bool fp64) {
  return k >= 1 && k <= 128 && chol_blk_smem_bytes(k, fp64) <= kCholBlkSmemMax;
}

void chol_inv_blk(const float* G, int k, float* Rinv, int* flags, cudaStream_t s, bool fp64) {
  static std::atomic<unsigned> attr{0};
  int dev = 0;
  SFD_CUDA(cudaGetDevice(&dev));
  if (dev < 32 && !(attr.load() & (1u << dev))) {
    SFD_CUDA(cudaFuncSetAttribute(k_chol_inv_blk<float>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)chol_blk_smem_bytes(128, false)));
    SFD_CUDA(cudaFuncSetAttribute(k_chol_inv_blk<double>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kCholBlkSmemMax));
    attr.fetch_or(1u << dev);
  }
  if (fp64)
    k_chol_inv_blk<double><<<1, kCThreads, chol_blk_smem_bytes(k, true), s>>>(G, k, Rinv, flags);
  else
    k_chol_inv_blk<float><<<1, kCThreads, chol_blk_smem_bytes(k, false), s>>>(G, k, Rinv, flags);
  SFD_LAUNCH_CHECK();
}

}  // namespace sfd
