// Dense kernels of the SparseShrink / DenseShrink path:
//  - Philox4x64-10 Gaussian draws (G of Alg. 1, x of Alg. 6)
//  - Gram X^T X of tall-skinny blocks (CholeskyQR of Alg. 1's GramSchmidt,
//    P P^T of Alg. 3, [B; B'][B; B']^T of Alg. 5)
//  - tall-skinny products X * T (apply R^-1, H diag(s), U_l diag(s))
//  - Cholesky of a shifted Gram and the inverse of its factor (one CTA)
//  - shrink weights sqrt(1 - lambda_l^2 / lambda_i^2) (Alg. 3 / Alg. 5)
// All arithmetic is fp32; the small k x k factorisations live in one CTA.
#include <algorithm>
#include <atomic>

#include "sfd_internal.cuh"

namespace sfd {

namespace {

// ---------------------------------------------------------------- Philox
// Philox4x64-10 (Salmon et al., SC'11): 64x64->128 multiplies with the two
// published multipliers, key bumped by the two Weyl constants each round.
__device__ __forceinline__ void philox_round(uint64_t& x0, uint64_t& x1, uint64_t& x2, uint64_t& x3,
                                             uint64_t k0, uint64_t k1) {
  const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
  uint64_t p0_lo = m0 * x0, p0_hi = __umul64hi(m0, x0);
  uint64_t p1_lo = m1 * x2, p1_hi = __umul64hi(m1, x2);
  uint64_t n0 = p1_hi ^ x1 ^ k0;
  uint64_t n2 = p0_hi ^ x3 ^ k1;
  x0 = n0; x1 = p1_lo; x2 = n2; x3 = p0_lo;
}

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t key0, uint64_t key1) {
  uint64_t k0 = key0, k1 = key1;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    philox_round(c[0], c[1], c[2], c[3], k0, k1);
    k0 += 0x9E3779B97F4A7C15ull;
    k1 += 0xBB67AE8584CAA73Bull;
  }
}

__device__ __forceinline__ float u24(uint64_t w) {
  return ((float)(uint32_t)(w >> 40) + 0.5f) * 5.9604644775390625e-8f;  // 2^-24
}

__global__ void k_gauss_fill(float* __restrict__ out, int64_t rows, int cols, int ld, uint64_t seed,
                             uint64_t b, uint64_t r, uint64_t tag) {
  int64_t blk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t count = rows * (int64_t)cols;
  if (blk * 4 >= count) return;
  uint64_t c[4] = {(uint64_t)blk, b, r, tag};
  philox4x64_10(c, seed, 0ull);
  float z[4];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float ua = u24(c[2 * h]), ub = u24(c[2 * h + 1]);
    float rad = sqrtf(-2.f * logf(ua));
    float sn, cs;
    sincospif(2.f * ub, &sn, &cs);
    z[2 * h] = rad * cs;
    z[2 * h + 1] = rad * sn;
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    int64_t e = blk * 4 + t;
    if (e < count) {
      int64_t row = e / cols;
      int col = (int)(e - row * cols);
      out[row * ld + col] = z[t];
    }
  }
}

// ------------------------------------------------------------------ Gram
// 128 x 128 output tiles, 16 x 16 threads with 8 x 8 register micro-tiles:
// per staged row each thread does 64 FMAs for 4 float4 shared loads.
constexpr int kT = 128;  // output tile
constexpr int kR = 16;   // rows (Gram) / inner dimension (GEMM) per stage
constexpr int kGramBlocks = 304;  // split-K blocks per Gram, ~2 per SM

__device__ __forceinline__ void fma8x8(float (&acc)[8][8], const float4& a0, const float4& a1,
                                       const float4& b0, const float4& b1) {
  const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
  const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
}

__global__ void __launch_bounds__(256, 2)
    k_gram_tiles(const float* __restrict__ X, int ldx, ColMap map, int64_t rows,
                 int64_t rows_per_chunk, int ntiles, int npairs, float* __restrict__ partial) {
  __shared__ __align__(16) float As[kR][kT];
  __shared__ __align__(16) float Bs[kR][kT];
  const int tp = blockIdx.y, chunk = blockIdx.x;
  // (ti, tj), ti <= tj, from the row-major index over the upper triangle of tiles
  int ti = 0, start = 0;
  while (start + (ntiles - ti) <= tp) { start += ntiles - ti; ++ti; }
  const int tj = ti + (tp - start);
  const bool diag = ti == tj;
  const int n = map.total();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[8][8] = {};
  const int64_t r_beg = (int64_t)chunk * rows_per_chunk;
  const int64_t r_end = min(rows, r_beg + rows_per_chunk);
  float (*Bp)[kT] = diag ? As : Bs;
  for (int64_t r0 = r_beg; r0 < r_end; r0 += kR) {
#pragma unroll
    for (int q = 0; q < (kR * kT) / 256; ++q) {
      const int li = threadIdx.x + q * 256;
      const int rr = li / kT, cc = li % kT;
      const int64_t g = r0 + rr;
      const int ca = ti * kT + cc;
      As[rr][cc] = (g < r_end && ca < n) ? map.at(X, ldx, g, ca) : 0.f;
      if (!diag) {
        const int cb = tj * kT + cc;
        Bs[rr][cc] = (g < r_end && cb < n) ? map.at(X, ldx, g, cb) : 0.f;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < kR; ++rr) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[rr][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[rr][ty * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bp[rr][tx * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bp[rr][tx * 8 + 4]);
      fma8x8(acc, a0, a1, b0, b1);
    }
    __syncthreads();
  }
  float* out = partial + ((int64_t)chunk * npairs + tp) * (kT * kT);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float4* o = reinterpret_cast<float4*>(&out[(ty * 8 + i) * kT + tx * 8]);
    o[0] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    o[1] = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
  }
}

// G[e] = sum over chunks of the partial tiles. A block takes 32 consecutive
// output elements; its 8 warps each sum every 8th chunk (coalesced 128-byte
// reads per chunk), and the 8 warp sums are added in a fixed order, so the
// result does not depend on scheduling.
constexpr int kRedGroups = 8;

__global__ void __launch_bounds__(32 * kRedGroups)
    k_gram_reduce(const float* __restrict__ partial, int nchunks, int npairs, int ntiles, int n,
                  float* __restrict__ G) {
  __shared__ float sums[kRedGroups][33];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  const bool live = e < (int64_t)n * n;
  float acc = 0.f;
  if (live) {
    int a = (int)(e / n), c = (int)(e % n);
    if (a / kT > c / kT) { int t = a; a = c; c = t; }   // use the upper tile (ti <= tj)
    const int ti = a / kT, tj = c / kT;
    const int tp = ti * ntiles - ti * (ti - 1) / 2 + (tj - ti);
    const int off = (a % kT) * kT + (c % kT);
    const float* p = partial + (int64_t)tp * (kT * kT) + off;
    const int64_t stride = (int64_t)npairs * (kT * kT);
    // chunks grp, grp + 16, ... into s0 and grp + 8, grp + 24, ... into s1,
    // in that order; eight loads are issued before their adds
    float s0 = 0.f, s1 = 0.f;
    int ch = grp;
    for (; ch + 7 * kRedGroups < nchunks; ch += 8 * kRedGroups) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldg(p + (int64_t)(ch + u * kRedGroups) * stride);
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        s0 += v[u];
        s1 += v[u + 1];
      }
    }
    for (; ch + kRedGroups < nchunks; ch += 2 * kRedGroups) {
      s0 += p[ch * stride];
      s1 += p[(ch + kRedGroups) * stride];
    }
    if (ch < nchunks) s0 += p[ch * stride];
    acc = s0 + s1;
  }
  sums[grp][lane] = acc;
  __syncthreads();
  if (grp == 0 && live) {
    float t = 0.f;
#pragma unroll
    for (int g = 0; g < kRedGroups; ++g) t += sums[g][lane];
    G[e] = t;
  }
}

// ---------------------------------------------------------------- X * T
// Y[rows, 0:kout] = X[rows, map] T : 128-row x 128-column output tiles, the
// inner dimension staged 16 at a time (X tile stored transposed so each
// thread reads its 8 rows as two float4).
__global__ void __launch_bounds__(256, 2)
    k_gemm_ts(const float* __restrict__ X, int ldx, ColMap map, int64_t rows,
              const float* __restrict__ T, int kout, float* __restrict__ Y, int ldy) {
  __shared__ __align__(16) float Xs[kR][kT + 4];
  __shared__ __align__(16) float Ts[kR][kT];
  const int n = map.total();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * kT;
  const int col0 = blockIdx.y * kT;
  float acc[8][8] = {};
  for (int c0 = 0; c0 < n; c0 += kR) {
#pragma unroll
    for (int q = 0; q < (kT * kR) / 256; ++q) {
      const int li = threadIdx.x + q * 256;
      const int rr = li / kR, cc = li % kR;     // X tile: 128 rows x 16 inner
      const int64_t g = row0 + rr;
      const int c = c0 + cc;
      Xs[cc][rr] = (g < rows && c < n) ? map.at(X, ldx, g, c) : 0.f;
      const int tr = li / kT, tc = li % kT;     // T tile: 16 inner x 128 out
      const int cr = c0 + tr, oc = col0 + tc;
      Ts[tr][tc] = (cr < n && oc < kout) ? T[(int64_t)cr * kout + oc] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int cc = 0; cc < kR; ++cc) {
      const float4 a0 = *reinterpret_cast<const float4*>(&Xs[cc][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&Xs[cc][ty * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Ts[cc][tx * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Ts[cc][tx * 8 + 4]);
      fma8x8(acc, a0, a1, b0, b1);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t g = row0 + ty * 8 + i;
    if (g >= rows) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int oc = col0 + tx * 8 + j;
      if (oc < kout) Y[g * ldy + oc] = acc[i][j];
    }
  }
}

// --------------------------------------------------- Cholesky + inverse
__device__ float block_sum_f(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// One CTA of kCholThreads threads. G + s I = R^T R with s = 2^-20 trace(G)/k
// (shifted CholeskyQR: keeps the factorisation defined for a rank-deficient
// block; X R^-1 then spans the same columns), then Rinv = R^-1.
// A is k x lda (lda odd, so column walks hit distinct banks).
//  - Cholesky, right-looking, one barrier per column: step j writes
//    R[j][t] = L[t][j] into the upper triangle (never read by the update),
//    R[j][j] into rdiag, and updates the trailing lower triangle with the
//    scaled column computed on the fly.
//  - Inverse, one barrier per row: R X = I is solved for all columns at once
//    by back-substitution from the last row; the running right-hand sides B
//    (upper triangular, B[i][c] stored at A[c][i]) take the freed lower
//    triangle. Rinv[r][c] = B[r][c] / R[r][r].
constexpr int kCholThreads = 256;

__device__ __forceinline__ float c_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double c_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float c_ldexp(float x, int e) { return ldexpf(x, e); }
__device__ __forceinline__ double c_ldexp(double x, int e) { return ldexp(x, e); }

__device__ double block_sum_d(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}
__device__ __forceinline__ float block_sum_t(float v, float* red) { return block_sum_f(v, red); }
__device__ __forceinline__ double block_sum_t(double v, double* red) { return block_sum_d(v, red); }

// T: the arithmetic type (float; double for the FP64 factorisation of the
// accurate CholeskyQR passes). G is read and Rinv written as fp32 either way.
template <typename T>
__global__ void __launch_bounds__(kCholThreads)
    k_chol_inv(const float* __restrict__ G, int k, float* __restrict__ Rinv,
               T* __restrict__ gA, int* __restrict__ flags, int use_smem) {
  extern __shared__ __align__(16) unsigned char sh_raw[];
  T* sh = reinterpret_cast<T*>(sh_raw);
  __shared__ T red[33];
  __shared__ T rdiag[kMaxEll];
  const int lda = k | 1;
  T* A = use_smem ? sh : gA;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  T tr = 0;
  for (int e = tid; e < k * k; e += nt) {
    int i = e / k, j = e % k;
    T v = (T)G[e];
    A[i * lda + j] = v;
    if (i == j) tr += v;
  }
  tr = block_sum_t(tr, red);
  const T shift = tr > (T)0 ? c_ldexp(tr / (T)k, -20) : (T)1e-30f;
  for (int i = tid; i < k; i += nt) A[i * lda + i] += shift;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    T p = A[j * lda + j];
    if (!(p > (T)0)) p = shift;
    const T ljj = c_sqrt(p);
    const T inv = (T)1 / ljj;
    if (tid == 0) {
      rdiag[j] = ljj;
      if (!(A[j * lda + j] > (T)0)) atomicAdd(&flags[1], 1);
    }
    for (int t = j + 1 + tid; t < k; t += nt) A[j * lda + t] = A[t * lda + j] * inv;
    for (int i = j + 1 + warp; i < k; i += nw) {
      const T lij = A[i * lda + j] * inv;
      for (int t = j + 1 + lane; t <= i; t += 32) A[i * lda + t] -= lij * (A[t * lda + j] * inv);
    }
    __syncthreads();
  }
  // B = I in the lower triangle (B[i][c] at A[c][i], i <= c)
  for (int e = tid; e < k * k; e += nt) {
    int c = e / k, i = e % k;
    if (i <= c) A[c * lda + i] = i == c ? (T)1 : (T)0;
  }
  __syncthreads();
  for (int j = k - 1; j > 0; --j) {
    const T rj = (T)1 / rdiag[j];
    // B[i][c] -= R[i][j] * B[j][c] / R[j][j]   for i < j <= c
    for (int c = j + warp; c < k; c += nw) {
      const T xjc = A[c * lda + j] * rj;
      for (int i = lane; i < j; i += 32) A[c * lda + i] -= A[i * lda + j] * xjc;
    }
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += nt) {
    int r = e / k, c = e % k;
    Rinv[e] = c >= r ? (float)(A[c * lda + r] / rdiag[r]) : 0.f;
  }
}


// ------------------------------------------------------- shrink weights
__global__ void k_shrink_weights(const float* __restrict__ evals, const float* __restrict__ evecs,
                                 int n, int nwant, int nkeep, int thr_zero,
                                 float* __restrict__ T, double* __restrict__ scal) {
  __shared__ float s[kMaxEig];
  const float thr = thr_zero ? 0.f : fmaxf(evals[nkeep - 1], 0.f);
  for (int j = threadIdx.x; j < nkeep; j += blockDim.x) {
    float ev = evals[j];
    s[j] = (ev > thr && ev > 0.f) ? sqrtf(1.f - thr / ev) : 0.f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * nkeep; e += blockDim.x) {
    int i = e / nkeep, j = e % nkeep;
    T[e] = evecs[i * nwant + j] * s[j];
  }
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int j = 0; j < nkeep; ++j) acc += fmax((double)evals[j] - (double)thr, 0.0);
    scal[0] = acc;
    scal[1] = thr;
  }
}

// --------------------------------------------------------------- transpose
__global__ void k_transpose(const float* __restrict__ in, int64_t rows, int cols, int ld_in,
                            float* __restrict__ out, int64_t ld_out) {
  __shared__ float t[32][33];
  int64_t r0 = (int64_t)blockIdx.x * 32;
  int c0 = blockIdx.y * 32;
  int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    int64_t r = r0 + k;
    int c = c0 + tx;
    t[k][tx] = (r < rows && c < cols) ? in[r * ld_in + c] : 0.f;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    int c = c0 + k;
    int64_t r = r0 + tx;
    if (c < cols && r < rows) out[(int64_t)c * ld_out + r] = t[tx][k];
  }
}

__global__ void k_csr_to_dense_t(const int* __restrict__ ptr, const int* __restrict__ idx,
                                 const float* __restrict__ val, int rows, float* __restrict__ out,
                                 int ld) {
  int r = blockIdx.x;
  if (r >= rows) return;
  for (int p = ptr[r] + threadIdx.x; p < ptr[r + 1]; p += blockDim.x)
    atomicAdd(&out[(int64_t)idx[p] * ld + r], val[p]);
}

}  // namespace

// ======================================================================= API
void launch_gauss_fill(float* out, int64_t rows, int cols, int ld, uint64_t seed, uint64_t b,
                       uint64_t r, uint64_t tag, cudaStream_t s) {
  int64_t nblk = (rows * cols + 3) / 4;
  if (nblk == 0) return;
  k_gauss_fill<<<(unsigned)((nblk + 255) / 256), 256, 0, s>>>(out, rows, cols, ld, seed, b, r, tag);
  SFD_LAUNCH_CHECK();
}

void gram(const float* X, int ldx, ColMap map, int64_t rows, float* G, Workspace& ws,
          cudaStream_t s) {
  const int n = map.total();
  const int ntiles = (n + kT - 1) / kT;
  const int npairs = ntiles * (ntiles + 1) / 2;
  int nchunks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + kR - 1) / kR, kGramBlocks / npairs));
  int64_t rpc = (rows + nchunks - 1) / nchunks;
  rpc = ((rpc + kR - 1) / kR) * kR;
  nchunks = (int)std::max<int64_t>(1, (rows + rpc - 1) / rpc);
  float* partial = ws.gram_partial;
  if (rows > 0) {
    dim3 grid(nchunks, npairs);
    k_gram_tiles<<<grid, 256, 0, s>>>(X, ldx, map, rows, rpc, ntiles, npairs, partial);
    SFD_LAUNCH_CHECK();
  } else {
    nchunks = 0;
  }
  int64_t ne = (int64_t)n * n;
  k_gram_reduce<<<(unsigned)((ne + 31) / 32), 32 * kRedGroups, 0, s>>>(partial, nchunks, npairs, ntiles, n, G);
  SFD_LAUNCH_CHECK();
}

void gram_reduce_tiles(const float* partial, int nchunks, int n, float* G, cudaStream_t s) {
  int64_t ne = (int64_t)n * n;
  k_gram_reduce<<<(unsigned)((ne + 31) / 32), 32 * kRedGroups, 0, s>>>(partial, nchunks, 1, 1, n, G);
  SFD_LAUNCH_CHECK();
}

void gemm_ts(const float* X, int ldx, ColMap map, int64_t rows, const float* T, int kout, float* Y,
             int ldy, cudaStream_t s) {
  if (rows <= 0 || kout <= 0) return;
  dim3 grid((unsigned)((rows + kT - 1) / kT), (kout + kT - 1) / kT);
  k_gemm_ts<<<grid, 256, 0, s>>>(X, ldx, map, rows, T, kout, Y, ldy);
  SFD_LAUNCH_CHECK();
}

void chol_inv(const float* G, int k, float* Rinv, float* work, int* flags, cudaStream_t s,
              bool fp64) {
  if (chol_blk_supported(k, fp64)) {  // blocked one-CTA form: fp32 k <= 128, fp64 k <= 112
    chol_inv_blk(G, k, Rinv, flags, s, fp64);
    return;
  }
  const int lda = k | 1;
  const size_t bytes = (size_t)k * lda * (fp64 ? sizeof(double) : sizeof(float));
  const int use_smem = bytes <= 200 * 1024;
  static std::atomic<unsigned> attr_set{0};  // one bit per device
  int dev = 0;
  SFD_CUDA(cudaGetDevice(&dev));
  if (dev < 32 && !(attr_set.load() & (1u << dev))) {
    SFD_CUDA(cudaFuncSetAttribute(k_chol_inv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  200 * 1024));
    SFD_CUDA(cudaFuncSetAttribute(k_chol_inv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  200 * 1024));
    attr_set.fetch_or(1u << dev);
  }
  // work: k * lda scalars when the matrix does not fit in shared memory (the
  // eigensolver scratch, 256-byte aligned, is far larger)
  if (fp64)
    k_chol_inv<double><<<1, kCholThreads, use_smem ? bytes : 0, s>>>(
        G, k, Rinv, reinterpret_cast<double*>(work), flags, use_smem);
  else
    k_chol_inv<float><<<1, kCholThreads, use_smem ? bytes : 0, s>>>(G, k, Rinv, work, flags,
                                                                    use_smem);
  SFD_LAUNCH_CHECK();
}

void shrink_weights(const float* evals, const float* evecs, int n, int nwant, int nkeep,
                    int thr_zero, float* T, double* scal, cudaStream_t s) {
  k_shrink_weights<<<1, 1024, 0, s>>>(evals, evecs, n, nwant, nkeep, thr_zero, T, scal);
  SFD_LAUNCH_CHECK();
}

void transpose(const float* in, int64_t rows, int cols, int ld_in, float* out, int64_t ld_out,
               cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  dim3 grid((unsigned)((rows + 31) / 32), (cols + 31) / 32);
  k_transpose<<<grid, dim3(32, 8), 0, s>>>(in, rows, cols, ld_in, out, ld_out);
  SFD_LAUNCH_CHECK();
}

void csr_to_dense_t(const int* ptr, const int* idx, const float* val, int rows, int64_t d,
                    float* out, int ld, cudaStream_t s) {
  (void)d;
  if (rows <= 0) return;
  k_csr_to_dense_t<<<rows, 128, 0, s>>>(ptr, idx, val, rows, out, ld);
  SFD_LAUNCH_CHECK();
}

}  // namespace sfd
