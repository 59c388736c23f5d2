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
  float zmax = 0.f, z1 = 0.f, z2 = 0.f;
  for (int i = n - 1; i >= 0; --i) {
    float z = (Z[i * nwp] - U1[i * nwp] * z1 - U2[i * nwp] * z2) / U0[i * nwp];
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
  U0[(n - 1) * st] = a_i;
  for (int i = 0; i < n; ++i) {
    float u = U0[i * st];
    if (fabsf(u) < tiny_piv) U0[i * st] = u < 0.f ? -tiny_piv : tiny_piv;
  }
}

struct EigWork {
  float* house;   // n * n : reflector k at house[k * n + i], i < n - k - 1
  float* beta;    // n
  float* U0;      // n * nwp each, [i * nwp + j]
  float* U1;
  float* U2;
  float* Lm;
  float* Z;
  float* piv;
  float* gA;      // n * lda when A does not fit in shared memory
};

__device__ EigWork carve(float* w, int n, int nwp, int lda) {
  EigWork e;
  e.house = w; w += (size_t)n * n;
  e.beta = w; w += n;
  size_t blk = (size_t)n * nwp;
  e.U0 = w; w += blk;
  e.U1 = w; w += blk;
  e.U2 = w; w += blk;
  e.Lm = w; w += blk;
  e.Z = w; w += blk;
  e.piv = w; w += blk;
  e.gA = w;
  (void)lda;
  return e;
}

__global__ void __launch_bounds__(kThreads)
    k_symeig(const float* __restrict__ S, int n, int nwant, float* __restrict__ evals,
             float* __restrict__ evecs, float* __restrict__ work, int use_smem) {
  extern __shared__ float shA[];
  __shared__ float d[kMaxEig], e[kMaxEig], e2[kMaxEig], ub[kMaxEig], pv[kMaxEig], wv[kMaxEig];
  __shared__ float red[33];
  __shared__ float sc[4];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int lda = n | 1;
  const int nwp = (nwant + 31) & ~31;
  EigWork W = carve(work, n, nwp, lda);
  float* A = use_smem ? shA : W.gA;

  // ---------------------------------------------------------------- load
  float amax = 0.f;
  for (int i = warp; i < n; i += nw)
    for (int j = lane; j < n; j += 32) {
      float v = S[(size_t)i * n + j];
      A[i * lda + j] = v;
      amax = fmaxf(amax, fabsf(v));
    }
  amax = block_reduce(amax, red, 1);
  // columns below this squared norm are at or below fp32 resolution of the
  // matrix: their reflector is skipped (and 2/|u|^2 cannot overflow)
  const float negligible2 = fmaxf(1e-30f * amax * amax, 64.f * FLT_MIN);

  // ------------------------------------------------- 1. tridiagonalise
  for (int k = 0; k + 2 < n; ++k) {
    const int L = n - k - 1;
    float part = 0.f;
    for (int i = tid; i < L; i += nt) {
      float x = A[(k + 1 + i) * lda + k];
      ub[i] = x;
      part = fmaf(x, x, part);
    }
    const float norm2 = block_reduce(part, red, 0);
    if (tid == 0) {
      float x0 = ub[0];
      if (norm2 - x0 * x0 <= negligible2) {
        // nothing below the subdiagonal worth a reflector
        sc[0] = 0.f;
        e[k] = x0;
      } else {
        float alpha = -copysignf(sqrtf(norm2), x0);
        float u0 = x0 - alpha;
        float un2 = norm2 - x0 * x0 + u0 * u0;
        ub[0] = u0;
        sc[0] = 2.f / un2;
        e[k] = alpha;
      }
      d[k] = A[k * lda + k];
    }
    __syncthreads();
    const float bt = sc[0];
    for (int i = warp; i < L; i += nw) {
      const float* row = A + (k + 1 + i) * lda + (k + 1);
      float s = 0.f;
      for (int j = lane; j < L; j += 32) s = fmaf(row[j], ub[j], s);
      s = warp_sum(s);
      if (lane == 0) pv[i] = bt * s;
    }
    __syncthreads();
    part = 0.f;
    for (int i = tid; i < L; i += nt) part = fmaf(ub[i], pv[i], part);
    const float K = 0.5f * bt * block_reduce(part, red, 0);
    for (int i = tid; i < L; i += nt) pv[i] -= K * ub[i];
    __syncthreads();
    for (int i = warp; i < L; i += nw) {
      float* row = A + (k + 1 + i) * lda + (k + 1);
      const float ui = ub[i], wi = pv[i];
      for (int j = lane; j < L; j += 32) row[j] -= ui * pv[j] + wi * ub[j];
    }
    for (int i = tid; i < L; i += nt) W.house[(size_t)k * n + i] = ub[i];
    if (tid == 0) W.beta[k] = bt;
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

  // ----------------------------------------------------- 2. bisection
  float lo_t = FLT_MAX, hi_t = -FLT_MAX, me2 = 0.f;
  for (int i = tid; i < n; i += nt) {
    float r = fabsf(e[i]) + (i > 0 ? fabsf(e[i - 1]) : 0.f);
    lo_t = fminf(lo_t, d[i] - r);
    hi_t = fmaxf(hi_t, d[i] + r);
    if (i < n - 1) {
      e2[i] = e[i] * e[i];
      me2 = fmaxf(me2, e2[i]);
    }
  }
  float lo = block_reduce(lo_t, red, 2);
  float hi = block_reduce(hi_t, red, 1);
  me2 = block_reduce(me2, red, 1);
  const float tnorm = fmaxf(fmaxf(fabsf(lo), fabsf(hi)), FLT_MIN);
  const float pivmin = FLT_MIN * fmaxf(1.f, me2);
  const float abstol = FLT_EPSILON * tnorm;
  lo -= 4.f * abstol + 2.f * pivmin;
  hi += 4.f * abstol + 2.f * pivmin;
  if (tid < nwant) {
    const int target = n - 1 - tid;  // ascending index of the tid-th largest
    float a = lo, b = hi;
    for (int it = 0; it < 128; ++it) {
      float mid = 0.5f * (a + b);
      if (b - a <= fmaxf(abstol, 2.f * FLT_EPSILON * fmaxf(fabsf(a), fabsf(b)))) break;
      int cnt = 0;
      float q = d[0] - mid;
      if (fabsf(q) < pivmin) q = -pivmin;
      cnt += q < 0.f;
      for (int i = 1; i < n; ++i) {
        q = (d[i] - mid) - e2[i - 1] / q;
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt += q < 0.f;
      }
      if (cnt > target) b = mid; else a = mid;
    }
    wv[tid] = 0.5f * (a + b);
  }
  __syncthreads();

  // ------------------------------------------------ 3. inverse iteration
  const float pertol = 10.f * FLT_EPSILON * tnorm;
  const float tiny_piv = FLT_EPSILON * tnorm;
  {
    // batches of eigenvectors whose factorisation and iterate fit in the A
    // region (six vectors of n floats per eigenvector, interleaved by thread)
    const int region = n * lda;
    const int bsz = use_smem ? max(1, min(nwant, region / (6 * n))) : nwant;
    for (int b0 = 0; b0 < nwant; b0 += bsz) {
      const int j = b0 + tid;
      if (tid < bsz && j < nwant) {
        int rank = 0;  // eigenvalues tied within fp32 resolution get distinct shifts
        for (int k = j; k > 0 && wv[k - 1] - wv[k] < pertol; --k) ++rank;
        const float lam = wv[j] - rank * pertol;
        float *U0, *U1, *U2, *Lm, *P, *Z;
        int st;
        if (use_smem) {
          st = bsz;
          U0 = A + tid; U1 = U0 + n * bsz; U2 = U1 + n * bsz; Lm = U2 + n * bsz;
          P = Lm + n * bsz; Z = P + n * bsz;
        } else {
          st = nwp;
          U0 = W.U0 + j; U1 = W.U1 + j; U2 = W.U2 + j; Lm = W.Lm + j; P = W.piv + j; Z = W.Z + j;
        }
        tri_factor(d, e, lam, U0, U1, U2, Lm, P, n, st, tiny_piv);
        for (int i = 0; i < n; ++i) Z[i * st] = hash_unit(i, j);
        for (int it = 0; it < 3; ++it) tri_solve_scaled(U0, U1, U2, Lm, P, Z, n, st);
        if (use_smem)
          for (int i = 0; i < n; ++i) W.Z[i * nwp + j] = Z[i * st];
      }
      __syncthreads();
    }
  }
  // eigenvectors into shared memory (or the global A region), column j contiguous
  float* Zs = A;
  for (int j = warp; j < nwant; j += nw)
    for (int i = lane; i < n; i += 32) Zs[j * n + i] = W.Z[i * nwp + j];
  __syncthreads();
  // classical Gram-Schmidt twice, in descending eigenvalue order: makes the
  // set orthonormal to fp32 precision (inverse iteration alone leaves
  // u ||T|| / gap); a vector left almost parallel to earlier ones (tied
  // eigenvalues) is refined by further solves inside that complement
  float* tcoef = pv;  // nwant <= kMaxEig coefficients
  for (int j = 0; j < nwant; ++j) {
    float* zj = Zs + j * n;
    for (int attempt = 0; attempt < 4; ++attempt) {
      float n0 = 0.f;
      for (int i = tid; i < n; i += nt) n0 = fmaf(zj[i], zj[i], n0);
      n0 = block_reduce(n0, red, 0);
      for (int pass = 0; pass < 2; ++pass) {
        for (int c = warp; c < j; c += nw) {
          const float* zc = Zs + c * n;
          float s = 0.f;
          for (int i = lane; i < n; i += 32) s = fmaf(zc[i], zj[i], s);
          s = warp_sum(s);
          if (lane == 0) tcoef[c] = s;
        }
        __syncthreads();
        for (int i = tid; i < n; i += nt) {
          float acc = zj[i];
          for (int c = 0; c < j; ++c) acc -= tcoef[c] * Zs[c * n + i];
          zj[i] = acc;
        }
        __syncthreads();
      }
      float n1 = 0.f;
      for (int i = tid; i < n; i += nt) n1 = fmaf(zj[i], zj[i], n1);
      n1 = block_reduce(n1, red, 0);
      const bool ok = n1 > 1e-4f * n0 || attempt == 3;
      if (ok) {
        const float inv = n1 > 0.f ? rsqrtf(n1) : 0.f;
        for (int i = tid; i < n; i += nt) zj[i] *= inv;
        __syncthreads();
        break;
      }
      // repair: one more solve with this vector's factorisation, then project again
      if (tid == 0) {
        int rank = 0;
        for (int k = j; k > 0 && wv[k - 1] - wv[k] < pertol; --k) ++rank;
        float* col = W.Z + j;
        tri_factor(d, e, wv[j] - rank * pertol, W.U0 + j, W.U1 + j, W.U2 + j, W.Lm + j,
                   W.piv + j, n, nwp, tiny_piv);
        for (int i = 0; i < n; ++i) col[i * nwp] = zj[i] + 1e-3f * hash_unit(i + 7919 * attempt, j);
        tri_solve_scaled(W.U0 + j, W.U1 + j, W.U2 + j, W.Lm + j, W.piv + j, col, n, nwp);
        for (int i = 0; i < n; ++i) zj[i] = col[i * nwp];
      }
      __syncthreads();
    }
  }

  // ---------------------------------------------- 4. back-transformation
  for (int k = n - 3; k >= 0; --k) {
    const int L = n - k - 1;
    for (int i = tid; i < L; i += nt) ub[i] = W.house[(size_t)k * n + i];
    if (tid == 0) sc[1] = W.beta[k];
    __syncthreads();
    const float bt = sc[1];
    if (bt != 0.f) {
      for (int j = warp; j < nwant; j += nw) {
        float* z = Zs + j * n + (k + 1);
        float s = 0.f;
        for (int i = lane; i < L; i += 32) s = fmaf(ub[i], z[i], s);
        s = warp_sum(s) * bt;
        for (int i = lane; i < L; i += 32) z[i] -= ub[i] * s;
      }
    }
    __syncthreads();
  }
  for (int i = warp; i < n; i += nw)
    for (int j = lane; j < nwant; j += 32) evecs[(size_t)i * nwant + j] = Zs[j * n + i];
  for (int j = tid; j < nwant; j += nt) evals[j] = wv[j];
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

size_t symeig_work_floats(int n, int nwant) {
  const int nwp = (nwant + 31) & ~31;
  const int lda = n | 1;
  return (size_t)n * n + n + 6 * (size_t)n * nwp + (size_t)n * lda;
}

void symeig(const float* S, int n, int nwant, float* evals, float* evecs, float* work,
            cudaStream_t s, bool psd) {
  if (psd && n <= kJacobiMax) {
    static unsigned jac_attr = 0;  // one bit per device
    int dv = 0;
    SFD_CUDA(cudaGetDevice(&dv));
    if (dv < 32 && !(jac_attr & (1u << dv))) {
      SFD_CUDA(cudaFuncSetAttribute(k_symeig_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kJacobiMax * (kJacobiMax | 1) * (int)sizeof(float)));
      jac_attr |= 1u << dv;
    }
    const size_t bytes = (size_t)n * (n | 1) * sizeof(float);
    k_symeig_jacobi<<<1, kThreads, bytes, s>>>(S, n, nwant, evals, evecs);
    SFD_LAUNCH_CHECK();
    return;
  }
  const int lda = n | 1;
  size_t bytes = (size_t)n * lda * sizeof(float);
  int use_smem = bytes <= (size_t)kSmemLimit;
  static unsigned attr_set = 0;
  int dev = 0;
  SFD_CUDA(cudaGetDevice(&dev));
  if (dev < 32 && !(attr_set & (1u << dev))) {
    SFD_CUDA(cudaFuncSetAttribute(k_symeig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kSmemLimit));
    attr_set |= 1u << dev;
  }
  k_symeig<<<1, kThreads, use_smem ? bytes : 0, s>>>(S, n, nwant, evals, evecs, work, use_smem);
  SFD_LAUNCH_CHECK();
}

}  // namespace sfd
