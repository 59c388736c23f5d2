// Symmetric eigensolver for the small matrices of the method: P P^T (l x l)
// in SparseShrink (Alg. 3, svd(P, l)) and [B; B'][B; B']^T (2l x 2l) in
// DenseShrink (Alg. 5, svd([B; B'], l)). Only the `nwant` largest eigenpairs
// are formed.
//
// One CTA of 1024 threads, fp32:
//  1. Householder tridiagonalisation A = Q T Q^T (A in shared memory when it
//     fits, else in global scratch).
//  2. Bisection on Sturm counts of T for eigenvalues n-1 .. n-nwant
//     (one thread per eigenvalue).
//  3. Inverse iteration for their eigenvectors of T (one thread per vector,
//     LU with partial pivoting of T - lambda I), then classical Gram-Schmidt
//     twice over the whole set in descending order (fp32 inverse iteration
//     alone leaves a loss of orthogonality of u ||T|| / gap).
//  4. Back-transformation Z <- Q Z with the stored reflectors.
// A full Jacobi method costs ~6 n^3 flops per sweep over several sweeps; this
// path costs ~(4/3 + 2 nwant/n) n^3 and runs in a fraction of the time at the
// sizes used here (n <= 512).
#include <float.h>

#include <algorithm>
#include <atomic>

#include "sfd_internal.cuh"

namespace sfd {

namespace {

constexpr int kThreads = 1024;
constexpr int kSmemLimit = 200 * 1024;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ float block_reduce(float v, float* red, int op /*0 sum, 1 max, 2 min*/) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float t = __shfl_xor_sync(0xffffffffu, v, o);
    v = op == 0 ? v + t : (op == 1 ? fmaxf(v, t) : fminf(v, t));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : (op == 0 ? 0.f : red[0]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float u = __shfl_xor_sync(0xffffffffu, t, o);
      t = op == 0 ? t + u : (op == 1 ? fmaxf(t, u) : fminf(t, u));
    }
    if (threadIdx.x == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

__device__ __forceinline__ float hash_unit(int i, int j) {
  uint32_t h = (uint32_t)i * 0x9E3779B1u ^ ((uint32_t)j + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
  return (float)(h >> 8) * (2.0f / 16777216.0f) - 1.0f;   // [-1, 1)
}

// One inverse-iteration step on column z (stride nwp): solve with the stored
// LU of T - lambda I (row swaps P, multipliers Lm, U with three diagonals),
// then scale to max |z| = 1 and finally to unit length.
__device__ void tri_solve_scaled(const float* U0, const float* U1, const float* U2,
                                 const float* Lm, const float* P, float* Z, int n, int nwp) {
  for (int i = 0; i + 1 < n; ++i) {
    float ri = Z[i * nwp], rn = Z[(i + 1) * nwp];
    if (P[i * nwp] != 0.f) { float t = ri; ri = rn; rn = t; }
    Z[i * nwp] = ri;
    Z[(i + 1) * nwp] = rn - Lm[i * nwp] * ri;
  }
  // back substitution; near a cluster the solution can outgrow fp32, so when
  // an entry passes 2^100 the whole system (solved part, neighbours and the
  // remaining right-hand side) is scaled by 2^-100 and the entry redone
  float zmax = 0.f, z1 = 0.f, z2 = 0.f;
  for (int i = n - 1; i >= 0; --i) {
    float z = (Z[i * nwp] - U1[i * nwp] * z1 - U2[i * nwp] * z2) / U0[i * nwp];
    if (!(fabsf(z) <= 0x1p100f)) {
      for (int k = 0; k < n; ++k) Z[k * nwp] *= 0x1p-100f;
      z1 *= 0x1p-100f;
      z2 *= 0x1p-100f;
      zmax *= 0x1p-100f;
      z = (Z[i * nwp] - U1[i * nwp] * z1 - U2[i * nwp] * z2) / U0[i * nwp];
      if (!(fabsf(z) <= 0x1p100f)) z = 0.f;
    }
    Z[i * nwp] = z;
    z2 = z1;
    z1 = z;
    zmax = fmaxf(zmax, fabsf(z));
  }
  float inv = zmax > 0.f ? 1.f / zmax : 1.f;
  float nrm = 0.f;
  for (int i = 0; i < n; ++i) {
    float z = Z[i * nwp] * inv;
    nrm = fmaf(z, z, nrm);
  }
  inv *= nrm > 0.f ? rsqrtf(nrm) : 0.f;
  for (int i = 0; i < n; ++i) Z[i * nwp] *= inv;
}

// LU with partial pivoting of the tridiagonal T - lam I (diagonal d, off
// diagonal e): U has three diagonals (U0, U1, U2), Lm the multipliers, P the
// row swaps; pivots below tiny_piv are raised to +-tiny_piv.
__device__ void tri_factor(const float* d, const float* e, float lam, float* U0, float* U1,
                           float* U2, float* Lm, float* P, int n, int st, float tiny_piv) {
  float a_i = d[0] - lam, c_i = n > 1 ? e[0] : 0.f;
  for (int i = 0; i + 1 < n; ++i) {
    const float b = e[i];
    const float an = d[i + 1] - lam;
    const float cn = (i + 2 < n) ? e[i + 1] : 0.f;
    float a_nx, c_nx;
    if (fabsf(b) > fabsf(a_i)) {
      const float l = a_i / b;
      U0[i * st] = b; U1[i * st] = an; U2[i * st] = cn; P[i * st] = 1.f; Lm[i * st] = l;
      a_nx = c_i - l * an;
      c_nx = -l * cn;
    } else {
      float piv = a_i;
      if (fabsf(piv) < tiny_piv) piv = piv < 0.f ? -tiny_piv : tiny_piv;
      const float l = b / piv;
      U0[i * st] = piv; U1[i * st] = c_i; U2[i * st] = 0.f; P[i * st] = 0.f; Lm[i * st] = l;
      a_nx = an - l * c_i;
      c_nx = cn;
    }
    a_i = a_nx;
    c_i = c_nx;
  }
  // the last row has no super-diagonals, multiplier or swap; they are written
  // (not left as whatever the memory held) because the solve reads U1 and U2
  // of that row times 0, and a leftover NaN / Inf pattern would make it NaN
  U0[(n - 1) * st] = a_i;
  U1[(n - 1) * st] = 0.f;
  U2[(n - 1) * st] = 0.f;
  Lm[(n - 1) * st] = 0.f;
  P[(n - 1) * st] = 0.f;
  for (int i = 0; i < n; ++i) {
    float u = U0[i * st];
    if (fabsf(u) < tiny_piv) U0[i * st] = u < 0.f ? -tiny_piv : tiny_piv;
  }
}

// Sturm count: how many eigenvalues of the tridiagonal (d, e2 = e^2) lie below x.
// The quotient uses the fast reciprocal (2 ulp): a count is only wrong for x
// within a few ulps of an eigenvalue, which moves the bisection result by as
// much and no more. |q| >= pivmin keeps the divisor in range.
__device__ int sturm_count(const float* d, const float* e2, int n, float x, float pivmin) {
  int cnt = 0;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  cnt += q < 0.f;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += q < 0.f;
  }
  return cnt;
}

// 1. Householder tridiagonalisation and 2. bisection, one CTA of 1024 threads.
//
// Step k reflects column k below the diagonal. Two barriers per step: the
// reflector's scalars come from per-warp partial norms left by the previous
// step (every thread sums them), the product p = beta A22 u also leaves the
// per-warp partials of u^T p, and the rank-2 update A22 -= u w^T + w u^T
// (w = p - (beta u^T p / 2) u) copies the next column and its partial norms
// on the way. Reflector k goes to house[k n + i] (u_0 replaced) and beta[k].
//
// Bisection is a multisection: g threads per eigenvalue evaluate Sturm
// counts at g interior points and keep the sub-interval holding it, so each
// round gains log2(g + 1) bits with synchronisation inside the warp only.
__global__ void __launch_bounds__(kThreads)
    k_tridiag_bisect(const float* __restrict__ S, int n, int nwant, float* __restrict__ house,
                     float* __restrict__ beta_g, float* __restrict__ dg, float* __restrict__ eg,
                     float* __restrict__ evals, float* __restrict__ gA, int use_smem) {
  extern __shared__ float shA[];
  __shared__ float d[kMaxEig], e[kMaxEig], e2[kMaxEig], ubuf[2][kMaxEig], pv[kMaxEig];
  __shared__ float npart[32], kpart[32];
  __shared__ float red[33];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int lda = n | 1;
  float* A = use_smem ? shA : gA;

  float amax = 0.f;
  for (int i = warp; i < n; i += nw)
    for (int j = lane; j < n; j += 32) {
      const float v = S[(size_t)i * n + j];
      A[i * lda + j] = v;
      amax = fmaxf(amax, fabsf(v));
    }
  amax = block_reduce(amax, red, 1);
  // a column below this squared norm is at fp32 resolution of the matrix: its
  // reflector is skipped (and 2 / |u|^2 cannot overflow)
  const float negligible2 = fmaxf(1e-30f * amax * amax, 64.f * FLT_MIN);
  {
    float part = 0.f;
    for (int i = tid; i + 1 < n; i += nt) {
      const float x = A[(1 + i) * lda];
      ubuf[0][i] = x;
      part = fmaf(x, x, part);
    }
    part = warp_sum(part);
    if (lane == 0) npart[warp] = part;
  }
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    const int L = n - k - 1;
    const float* ub = ubuf[k & 1];
    float* ubn = ubuf[(k + 1) & 1];
    // every warp sums the 32 partial norms with one load and a shuffle tree
    const float norm2 = warp_sum(lane < nw ? npart[lane] : 0.f);
    const float x0 = ub[0];
    float bt = 0.f, u0 = x0, alpha = x0;
    if (norm2 - x0 * x0 > negligible2) {
      alpha = -copysignf(sqrtf(norm2), x0);
      u0 = x0 - alpha;
      bt = 2.f / (norm2 - x0 * x0 + u0 * u0);
    }
    const float du0 = u0 - x0;
    if (tid == 0) {
      d[k] = A[k * lda + k];
      e[k] = alpha;
      beta_g[k] = bt;
    }
    float kp = 0.f;
    for (int i = warp; i < L; i += nw) {
      const float* row = A + (k + 1 + i) * lda + (k + 1);
      float s = 0.f;
      for (int j = lane; j < L; j += 32) s = fmaf(row[j], ub[j], s);
      s = fmaf(row[0], du0, warp_sum(s));
      const float p = bt * s;
      if (lane == 0) pv[i] = p;
      kp = fmaf(i == 0 ? u0 : ub[i], p, kp);
    }
    if (lane == 0) kpart[warp] = kp;
    for (int i = tid; i < L; i += nt) house[(size_t)k * n + i] = i == 0 ? u0 : ub[i];
    __syncthreads();
    const float K = 0.5f * bt * warp_sum(lane < nw ? kpart[lane] : 0.f);
    float np = 0.f;
    for (int i = warp; i < L; i += nw) {
      float* row = A + (k + 1 + i) * lda + (k + 1);
      const float ui = i == 0 ? u0 : ub[i];
      const float wi = pv[i] - K * ui;
      for (int j = lane; j < L; j += 32) {
        const float uj = j == 0 ? u0 : ub[j];
        const float v = row[j] - (ui * (pv[j] - K * uj) + wi * uj);
        row[j] = v;
        if (j == 0 && i > 0) {
          ubn[i - 1] = v;
          np = fmaf(v, v, np);
        }
      }
    }
    if (lane == 0) npart[warp] = np;
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = A[(n - 2) * lda + (n - 2)];
      e[n - 2] = A[(n - 1) * lda + (n - 2)];
      d[n - 1] = A[(n - 1) * lda + (n - 1)];
    } else {
      d[0] = A[0];
    }
    e[n - 1] = 0.f;
  }
  __syncthreads();

  float lo_t = FLT_MAX, hi_t = -FLT_MAX, me2 = 0.f;
  for (int i = tid; i < n; i += nt) {
    const float r = fabsf(e[i]) + (i > 0 ? fabsf(e[i - 1]) : 0.f);
    lo_t = fminf(lo_t, d[i] - r);
    hi_t = fmaxf(hi_t, d[i] + r);
    if (i < n - 1) {
      e2[i] = e[i] * e[i];
      me2 = fmaxf(me2, e2[i]);
    }
    dg[i] = d[i];
    eg[i] = e[i];
  }
  float lo = block_reduce(lo_t, red, 2);
  float hi = block_reduce(hi_t, red, 1);
  me2 = block_reduce(me2, red, 1);
  const float tnorm = fmaxf(fmaxf(fabsf(lo), fabsf(hi)), FLT_MIN);
  const float pivmin = FLT_MIN * fmaxf(1.f, me2);
  const float abstol = FLT_EPSILON * tnorm;
  if (tid == 0) dg[n] = tnorm;
  lo -= 4.f * abstol + 2.f * pivmin;
  hi += 4.f * abstol + 2.f * pivmin;
  const int g = nwant <= 128 ? 8 : (nwant <= 256 ? 4 : 2);
  const int grp = tid / g, t = tid % g, l0 = (lane / g) * g;
  const int target = n - 1 - grp;  // ascending index of the grp-th largest
  float a = lo, b = hi;
  bool done = grp >= nwant;
  for (int round = 0; round < 64; ++round) {
    if (__all_sync(0xffffffffu, done)) break;
    const float h = (b - a) / (float)(g + 1);
    done = done || (b - a <= fmaxf(abstol, 2.f * FLT_EPSILON * fmaxf(fabsf(a), fabsf(b))));
    const int cnt = done ? 0 : sturm_count(d, e2, n, a + (float)(t + 1) * h, pivmin);
    const unsigned ball = __ballot_sync(0xffffffffu, !done && cnt > target);
    const unsigned gm = (ball >> l0) & ((1u << g) - 1u);
    if (!done) {
      if (gm) {
        const int ts = __ffs(gm) - 1;  // first point above the eigenvalue
        const float na = ts > 0 ? a + (float)ts * h : a;
        b = a + (float)(ts + 1) * h;
        a = na;
      } else {
        a = a + (float)g * h;
      }
    }
  }
  if (t == 0 && grp < nwant) evals[grp] = 0.5f * (a + b);
}

// 3. Inverse iteration: one thread per eigenvector, vpc per CTA, the LU of
// T - lambda I and the iterate in shared memory (interleaved by thread).
// Eigenvalues tied within fp32 resolution get distinct shifts.
__global__ void k_inviter(const float* __restrict__ dg, const float* __restrict__ eg,
                          const float* __restrict__ evals, int n, int nwant, float* __restrict__ Z,
                          int nwp) {
  extern __shared__ float sm[];
  const int vpc = blockDim.x;
  float* d = sm;
  float* e = d + n;
  for (int i = threadIdx.x; i < n; i += vpc) {
    d[i] = dg[i];
    e[i] = eg[i];
  }
  __syncthreads();
  const int j = blockIdx.x * vpc + threadIdx.x;
  if (j >= nwant) return;
  const float tnorm = dg[n];
  const float pertol = 10.f * FLT_EPSILON * tnorm;
  const float tiny_piv = FLT_EPSILON * tnorm;
  int rank = 0;
  for (int k = j; k > 0 && evals[k - 1] - evals[k] < pertol; --k) ++rank;
  const float lam = evals[j] - (float)rank * pertol;
  const size_t blk = (size_t)n * vpc;
  float* U0 = e + n + threadIdx.x;
  float* U1 = U0 + blk;
  float* U2 = U1 + blk;
  float* Lm = U2 + blk;
  float* P = Lm + blk;
  float* Zs = P + blk;
  tri_factor(d, e, lam, U0, U1, U2, Lm, P, n, vpc, tiny_piv);
  for (int i = 0; i < n; ++i) Zs[i * vpc] = hash_unit(i, j);
  for (int it = 0; it < 3; ++it) tri_solve_scaled(U0, U1, U2, Lm, P, Zs, n, vpc);
  // an iterate that collapsed (zero or non-finite) restarts as the hash
  // vector; the orthonormalisation then takes its component off the others
  float nz = 0.f;
  for (int i = 0; i < n; ++i) nz = fmaf(Zs[i * vpc], Zs[i * vpc], nz);
  const bool bad = !(nz > 0.f) || !isfinite(nz);
  for (int i = 0; i < n; ++i)
    Z[(size_t)i * nwp + j] = bad ? hash_unit(i, j) * rsqrtf((float)n) : Zs[i * vpc];
}

// 4. CholeskyQR of the eigenvector block Z (n x nwant, row-major, ld nwp):
// G = Z^T Z in 32 x 32 tiles (each CTA sums all n rows in order), then
// Z2 = Z R^-1 (R^-1 upper triangular) in 32 x 32 tiles.
constexpr int kZT = 32;

__global__ void __launch_bounds__(256)
    k_zgram(const float* __restrict__ Z, int n, int nwant, int nwp, float* __restrict__ G) {
  __shared__ float za[kZT][kZT + 1], zb[kZT][kZT + 1];
  const int a0 = blockIdx.y * kZT, c0 = blockIdx.x * kZT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 4 outputs
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int r0 = 0; r0 < n; r0 += kZT) {
    for (int e = threadIdx.x; e < kZT * kZT; e += 256) {
      const int rr = e / kZT, cc = e % kZT;
      const int r = r0 + rr;
      za[rr][cc] = (r < n && a0 + cc < nwant) ? Z[(size_t)r * nwp + a0 + cc] : 0.f;
      zb[rr][cc] = (r < n && c0 + cc < nwant) ? Z[(size_t)r * nwp + c0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < kZT; ++rr) {
      const float bv = zb[rr][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(za[rr][ty + 8 * q], bv, acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int a = a0 + ty + 8 * q, c = c0 + tx;
    if (a < nwant && c < nwant) G[(size_t)a * nwant + c] = acc[q];
  }
}

__global__ void __launch_bounds__(256)
    k_zmul(const float* __restrict__ Z, const float* __restrict__ R, int n, int nwant, int nwp,
           float* __restrict__ Y) {
  __shared__ float zt[kZT][kZT + 1], rt[kZT][kZT + 1];
  const int i0 = blockIdx.y * kZT, c0 = blockIdx.x * kZT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 <= c0 && k0 < nwant; k0 += kZT) {  // R is upper triangular
    for (int e = threadIdx.x; e < kZT * kZT; e += 256) {
      const int rr = e / kZT, cc = e % kZT;
      zt[rr][cc] = (i0 + rr < n && k0 + cc < nwant) ? Z[(size_t)(i0 + rr) * nwp + k0 + cc] : 0.f;
      rt[rr][cc] = (k0 + rr < nwant && c0 + cc < nwant) ? R[(size_t)(k0 + rr) * nwant + c0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kZT; ++kk) {
      const float rv = rt[kk][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(zt[ty + 8 * q][kk], rv, acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + ty + 8 * q, c = c0 + tx;
    if (i < n && c < nwant) Y[(size_t)i * nwp + c] = acc[q];
  }
}

// After the first CholeskyQR pass the block must be orthonormal to a few
// ulps times its condition number; if max |G - I| of the second pass's Gram
// exceeds 1e-2, inverse iteration left (nearly) dependent vectors (eigenvalues
// tied at fp32 resolution) and flags[3] selects the repair path.
__global__ void k_orth_check(const float* __restrict__ G, int nwant, int* __restrict__ flags) {
  __shared__ float red[33];
  float m = 0.f;
  for (int e = threadIdx.x; e < nwant * nwant; e += blockDim.x)
    m = fmaxf(m, fabsf(G[e] - (e / nwant == e % nwant ? 1.f : 0.f)));
  m = block_reduce(m, red, 1);
  if (threadIdx.x == 0 && !(m <= 1e-2f)) flags[3] = 1;
}

// Repair path (runs only when flags[3] is set): classical Gram-Schmidt twice
// over the inverse-iteration vectors in descending eigenvalue order; a vector
// left almost inside the span of the earlier ones gets one more solve with its
// own shifted factorisation from a perturbed start and is projected again.
// Zs (column j at Zs[j n]) and the factorisation scratch fw (6 n) are global.
__global__ void __launch_bounds__(kThreads)
    k_cgs_repair(const int* __restrict__ flags, const float* __restrict__ Zin, int nwp,
                 const float* __restrict__ dg, const float* __restrict__ eg,
                 const float* __restrict__ evals, int n, int nwant, float* __restrict__ Zs,
                 float* __restrict__ fw) {
  if (flags[3] == 0) return;
  __shared__ float d[kMaxEig], e[kMaxEig], tcoef[kMaxEig];
  __shared__ float red[33];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int i = tid; i < n; i += nt) {
    d[i] = dg[i];
    e[i] = eg[i];
  }
  for (int j = warp; j < nwant; j += nw)
    for (int i = lane; i < n; i += 32) Zs[(size_t)j * n + i] = Zin[(size_t)i * nwp + j];
  __syncthreads();
  const float tnorm = dg[n];
  const float pertol = 10.f * FLT_EPSILON * tnorm;
  const float tiny_piv = FLT_EPSILON * tnorm;
  for (int j = 0; j < nwant; ++j) {
    float* zj = Zs + (size_t)j * n;
    for (int attempt = 0; attempt < 4; ++attempt) {
      float n0 = 0.f;
      for (int i = tid; i < n; i += nt) n0 = fmaf(zj[i], zj[i], n0);
      n0 = block_reduce(n0, red, 0);
      for (int pass = 0; pass < 2; ++pass) {
        for (int c = warp; c < j; c += nw) {
          const float* zc = Zs + (size_t)c * n;
          float s = 0.f;
          for (int i = lane; i < n; i += 32) s = fmaf(zc[i], zj[i], s);
          s = warp_sum(s);
          if (lane == 0) tcoef[c] = s;
        }
        __syncthreads();
        for (int i = tid; i < n; i += nt) {
          float acc = zj[i];
          for (int c = 0; c < j; ++c) acc -= tcoef[c] * Zs[(size_t)c * n + i];
          zj[i] = acc;
        }
        __syncthreads();
      }
      float n1 = 0.f;
      for (int i = tid; i < n; i += nt) n1 = fmaf(zj[i], zj[i], n1);
      n1 = block_reduce(n1, red, 0);
      if (n1 > 1e-4f * n0 || attempt == 3) {
        const float inv = n1 > 0.f ? rsqrtf(n1) : 0.f;
        for (int i = tid; i < n; i += nt) zj[i] *= inv;
        __syncthreads();
        break;
      }
      if (tid == 0) {
        int rank = 0;
        for (int k = j; k > 0 && evals[k - 1] - evals[k] < pertol; --k) ++rank;
        float* col = fw + 5 * (size_t)n;
        tri_factor(d, e, evals[j] - rank * pertol, fw, fw + n, fw + 2 * n, fw + 3 * n, fw + 4 * n, n,
                   1, tiny_piv);
        for (int i = 0; i < n; ++i) col[i] = zj[i] + 1e-3f * hash_unit(i + 7919 * attempt, j);
        tri_solve_scaled(fw, fw + n, fw + 2 * n, fw + 3 * n, fw + 4 * n, col, n, 1);
        for (int i = 0; i < n; ++i) zj[i] = col[i];
      }
      __syncthreads();
    }
  }
}

// 5. Back-transformation Z <- H_0 ... H_{n-3} Z: a warp per eigenvector holds
// it in registers (NR per lane) and applies every reflector in turn; the
// vectors are independent, so no block barrier is needed.
template <int NR>
__global__ void __launch_bounds__(256)
    k_back(const float* __restrict__ house, const float* __restrict__ beta, int n, int nwant,
           const float* __restrict__ Z, int nwp, const float* __restrict__ Zrep,
           const int* __restrict__ flags, float* __restrict__ evecs) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= nwant) return;
  const bool rep = flags[3] != 0;  // the repair path produced Zrep (column j at Zrep[j n])
  float z[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int e = r * 32 + lane;
    z[r] = e < n ? (rep ? Zrep[(size_t)j * n + e] : Z[(size_t)e * nwp + j]) : 0.f;
  }
  for (int k = n - 3; k >= 0; --k) {
    const float bt = beta[k];
    if (bt == 0.f) continue;
    const float* u = house + (size_t)k * n;  // element e in [k+1, n) is u[e - k - 1]
    float s = 0.f;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int e = r * 32 + lane;
      if (e > k && e < n) s = fmaf(u[e - k - 1], z[r], s);
    }
    s = warp_sum(s) * bt;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int e = r * 32 + lane;
      if (e > k && e < n) z[r] = fmaf(-s, u[e - k - 1], z[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int e = r * 32 + lane;
    if (e < n) evecs[(size_t)e * nwant + j] = z[r];
  }
}

// ---------------------------------------------------------------------------
// PSD input, n <= kJacobiMax: one-sided Jacobi on the Cholesky factor.
// S + s I = L L^T (s = 2^-20 trace/n keeps a rank-deficient Gram factorable).
// Orthogonalising the columns of L by plane rotations (Hestenes) gives
// L J = U Sigma with U the eigenvectors of L L^T and Sigma^2 its eigenvalues,
// so no rotation product is accumulated: eigenvector i is column i / its norm,
// eigenvalue i its squared norm minus s. Pairs follow the round-robin
// tournament; one warp per pair, one barrier per round. Column walks are
// bank-conflict free because the row stride n|1 is odd.
constexpr int kJacobiMax = 64;   // measured: faster than the tridiagonal path only up to ~64
constexpr int kJacobiSweeps = 30;

__global__ void __launch_bounds__(kThreads)
    k_symeig_jacobi(const float* __restrict__ S, int n, int nwant, float* __restrict__ evals,
                    float* __restrict__ evecs) {
  extern __shared__ float A[];          // n x (n|1)
  __shared__ float nrm[kJacobiMax + 1], rdiag[kJacobiMax];
  __shared__ int rnk[kJacobiMax];
  __shared__ float red[33];
  __shared__ int rotations;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int lda = n | 1;
  // shift: 2^-20 trace/n for a positive semi-definite S (the Grams of the
  // method); if the factorisation meets a non-positive pivot, S is indefinite
  // and it restarts with the Gershgorin bound, which makes S + sI definite
  __shared__ int indefinite;
  __shared__ float shift_sh;
  float tr = 0.f, gersh = FLT_MAX;
  for (int i = warp; i < n; i += nw) {
    float off = 0.f;
    for (int j = lane; j < n; j += 32) {
      const float v = S[(size_t)i * n + j];
      if (j == i) tr += v; else off += fabsf(v);
    }
    off = warp_sum(off);
    if (lane == 0) gersh = fminf(gersh, S[(size_t)i * n + i] - off);
  }
  tr = block_reduce(tr, red, 0);
  gersh = block_reduce(gersh, red, 2);
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (tid == 0) {
      float sft = tr > 0.f ? ldexpf(tr / (float)n, -20) : FLT_MIN;
      if (attempt == 1) sft = fmaxf(sft, -gersh) * 1.01f + FLT_MIN;
      shift_sh = sft;
      indefinite = 0;
    }
    __syncthreads();
    const float sft = shift_sh;
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e % n;
      A[i * lda + j] = S[e] + (i == j ? sft : 0.f);
    }
    __syncthreads();
    // Cholesky, lower, in place; column j is scaled one step later (after the
    // barrier), so the trailing update can read it raw in the same step
    for (int j = 0; j < n; ++j) {
      float piv = A[j * lda + j];
      if (!(piv > 0.f)) {
        piv = sft;
        if (tid == 0 && attempt == 0 && j < n) indefinite = 1;
      }
      const float rinv = 1.f / piv;
      if (tid == 0) rdiag[j] = sqrtf(piv);
      if (j > 0) {
        const float sc = 1.f / rdiag[j - 1];
        for (int i = j + tid; i < n; i += nt) A[i * lda + (j - 1)] *= sc;
      }
      for (int i = j + 1 + warp; i < n; i += nw) {
        const float aij = A[i * lda + j] * rinv;
        for (int t = j + 1 + lane; t <= i; t += 32) A[i * lda + t] -= aij * A[t * lda + j];
      }
      __syncthreads();
    }
    if (!indefinite) break;
  }
  const float shift = shift_sh;
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e % n;
    if (j > i) A[i * lda + j] = 0.f;
    else if (j == i) A[i * lda + j] = rdiag[i];
  }
  __syncthreads();
  // one-sided Jacobi over the columns of L
  const int np = n + (n & 1);                 // even count; column n is a virtual zero
  const float tiny = ldexpf(fabsf(tr) + shift * n, -30);  // columns below this are zero
  const float tol = 4.f * FLT_EPSILON * sqrtf((float)n);  // attainable fp32 orthogonality
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    if (tid == 0) rotations = 0;
    __syncthreads();
    for (int r = 0; r < np - 1; ++r) {
      for (int w = warp; w < np / 2; w += nw) {
        int p, q;
        if (w == 0) { p = r; q = np - 1; }
        else { p = (r + w) % (np - 1); q = (r - w + (np - 1)) % (np - 1); }
        if (p >= n || q >= n) continue;
        float a = 0.f, b = 0.f, g = 0.f;
        for (int i = lane; i < n; i += 32) {
          const float x = A[i * lda + p], y = A[i * lda + q];
          a = fmaf(x, x, a);
          b = fmaf(y, y, b);
          g = fmaf(x, y, g);
        }
        a = warp_sum(a); b = warp_sum(b); g = warp_sum(g);
        if (fminf(a, b) <= tiny || fabsf(g) <= tol * sqrtf(a * b)) continue;
        const float zeta = (b - a) / (2.f * g);
        const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        const float c = rsqrtf(1.f + t * t), sn = c * t;
        for (int i = lane; i < n; i += 32) {
          const float x = A[i * lda + p], y = A[i * lda + q];
          A[i * lda + p] = c * x - sn * y;
          A[i * lda + q] = sn * x + c * y;
        }
        if (lane == 0) atomicAdd(&rotations, 1);
      }
      __syncthreads();
    }
    if (rotations == 0) break;
    __syncthreads();
  }
  // squared column norms, ranks (descending, ties by index), outputs
  for (int c = warp; c < n; c += nw) {
    float a = 0.f;
    for (int i = lane; i < n; i += 32) a = fmaf(A[i * lda + c], A[i * lda + c], a);
    a = warp_sum(a);
    if (lane == 0) nrm[c] = a;
  }
  __syncthreads();
  for (int c = tid; c < n; c += nt) {
    int r = 0;
    const float v = nrm[c];
    for (int c2 = 0; c2 < n; ++c2) r += (nrm[c2] > v) || (nrm[c2] == v && c2 < c);
    rnk[c] = r;
  }
  __syncthreads();
  for (int c = warp; c < n; c += nw) {
    const int r = rnk[c];
    if (r >= nwant) continue;
    const float v = nrm[c];
    const float inv = v > 0.f ? rsqrtf(v) : 0.f;
    for (int i = lane; i < n; i += 32) evecs[(size_t)i * nwant + r] = A[i * lda + c] * inv;
    if (lane == 0) evals[r] = v - shift;
  }
}

}  // namespace

namespace {
// Scratch of the tridiagonal path, carved from one float array.
struct EigScratch {
  float *house, *beta, *d, *e, *Z, *Z2, *Z3, *G, *R, *cw, *fw, *gA;
  int* flags;
  size_t floats;
};
EigScratch carve(float* w, int n, int nwant) {
  const size_t nwp = (size_t)((nwant + 31) & ~31);
  const size_t lda = (size_t)(n | 1);
  EigScratch c;
  size_t o = 0;
  auto take = [&](size_t k) {
    float* p = w ? w + o : nullptr;
    o += (k + 63) & ~(size_t)63;  // 256-byte aligned pieces
    return p;
  };
  c.house = take((size_t)n * n);
  c.beta = take(n);
  c.d = take(n + 2);
  c.e = take(n);
  c.Z = take(n * nwp);
  c.Z3 = take(n * nwp);
  c.G = take(nwp * nwp);
  c.R = take(nwp * nwp);
  c.cw = take(nwp * (nwp | 1));
  c.fw = take(6 * (size_t)n);
  c.flags = reinterpret_cast<int*>(take(16));
  // the tridiagonalisation's matrix (when it is not in shared memory) is dead
  // once stage 1 ends: the second eigenvector block reuses it
  c.gA = take(std::max(n * lda, n * nwp));
  c.Z2 = c.gA;
  c.floats = o;
  return c;
}
}  // namespace

size_t symeig_work_floats(int n, int nwant) { return carve(nullptr, n, nwant).floats; }

void symeig(const float* S, int n, int nwant, float* evals, float* evecs, float* work,
            cudaStream_t s, bool psd) {
  if (psd && n <= kJacobiMax) {
    static std::atomic<unsigned> jac_attr{0};  // one bit per device
    int dv = 0;
    SFD_CUDA(cudaGetDevice(&dv));
    if (dv < 32 && !(jac_attr.load() & (1u << dv))) {
      SFD_CUDA(cudaFuncSetAttribute(k_symeig_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kJacobiMax * (kJacobiMax | 1) * (int)sizeof(float)));
      jac_attr.fetch_or(1u << dv);
    }
    const size_t bytes = (size_t)n * (n | 1) * sizeof(float);
    k_symeig_jacobi<<<1, kThreads, bytes, s>>>(S, n, nwant, evals, evecs);
    SFD_LAUNCH_CHECK();
    return;
  }
  const int nwp = (nwant + 31) & ~31;
  EigScratch c = carve(work, n, nwant);
  const size_t abytes = (size_t)n * (n | 1) * sizeof(float);
  const int use_smem = abytes <= (size_t)kSmemLimit;
  static std::atomic<unsigned> attr{0};
  int dev = 0;
  SFD_CUDA(cudaGetDevice(&dev));
  if (dev < 32 && !(attr.load() & (1u << dev))) {
    SFD_CUDA(cudaFuncSetAttribute(k_tridiag_bisect, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kSmemLimit));
    SFD_CUDA(cudaFuncSetAttribute(k_inviter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kSmemLimit));
    attr.fetch_or(1u << dev);
  }
  SFD_CUDA(cudaMemsetAsync(c.flags, 0, 16 * sizeof(int), s));
  k_tridiag_bisect<<<1, kThreads, use_smem ? abytes : 0, s>>>(S, n, nwant, c.house, c.beta, c.d,
                                                              c.e, evals, c.gA, use_smem);
  SFD_LAUNCH_CHECK();
  int vpc = 32;
  while (vpc > 1 && (size_t)(2 * n + 6 * (size_t)n * vpc) * sizeof(float) > (size_t)kSmemLimit)
    vpc >>= 1;
  const size_t ibytes = (size_t)(2 * n + 6 * (size_t)n * vpc) * sizeof(float);
  k_inviter<<<(nwant + vpc - 1) / vpc, vpc, ibytes, s>>>(c.d, c.e, evals, n, nwant, c.Z, nwp);
  SFD_LAUNCH_CHECK();
  const dim3 gg((nwant + kZT - 1) / kZT, (nwant + kZT - 1) / kZT);
  const dim3 gm((nwant + kZT - 1) / kZT, (n + kZT - 1) / kZT);
  for (int pass = 0; pass < 2; ++pass) {  // CholeskyQR2: Z -> Z2 -> Z3 (Z is kept)
    const float* zin = pass == 0 ? c.Z : c.Z2;
    float* zout = pass == 0 ? c.Z2 : c.Z3;
    k_zgram<<<gg, 256, 0, s>>>(zin, n, nwant, nwp, c.G);
    SFD_LAUNCH_CHECK();
    if (pass == 1) {
      k_orth_check<<<1, 1024, 0, s>>>(c.G, nwant, c.flags);
      SFD_LAUNCH_CHECK();
    }
    chol_inv(c.G, nwant, c.R, c.cw, c.flags, s);
    k_zmul<<<gm, 256, 0, s>>>(zin, c.R, n, nwant, nwp, zout);
    SFD_LAUNCH_CHECK();
  }
  // Z2 is free again: the repair path (if flagged) writes its block there
  k_cgs_repair<<<1, kThreads, 0, s>>>(c.flags, c.Z, nwp, c.d, c.e, evals, n, nwant, c.Z2, c.fw);
  SFD_LAUNCH_CHECK();
  const int gb = (nwant + 7) / 8;
  if (n <= 128)
    k_back<4><<<gb, 256, 0, s>>>(c.house, c.beta, n, nwant, c.Z3, nwp, c.Z2, c.flags, evecs);
  else if (n <= 256)
    k_back<8><<<gb, 256, 0, s>>>(c.house, c.beta, n, nwant, c.Z3, nwp, c.Z2, c.flags, evecs);
  else
    k_back<16><<<gb, 256, 0, s>>>(c.house, c.beta, n, nwant, c.Z3, nwp, c.Z2, c.flags, evecs);
  SFD_LAUNCH_CHECK();
}

}  // namespace sfd
