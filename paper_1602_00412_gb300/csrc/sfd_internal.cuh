// Internal declarations shared by the translation units of libsfd.so.
// Nothing here is part of the C ABI (include/sfd.h).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>

#include "../../include/sfd.h"

namespace sfd {

// Schedules of the method (readings shared with the oracle):
// q = ceil(c_q ln(m / eps) / eps), eps = 1/4 (Alg. 1 with the eps of Alg. 3)
inline int q_for(const sfd_options& o, int m) {
  if (o.q_override >= 0) return o.q_override;
  double q = ceil(o.c_q * log((double)m / 0.25) / 0.25);
  return q > 0 ? (int)q : 0;
}
// delta_{b,r} = delta (6/pi^2) / (b+1)^2 / 2^(r+1): the VS budget of buffer b, attempt r
inline double delta_br(double delta, int64_t b, int r) {
  return delta * (6.0 / (M_PI * M_PI)) / ((double)(b + 1) * (double)(b + 1)) / ldexp(1.0, r + 1);
}
// power steps p = ceil(log2(sqrt(2d/pi) / delta_i)) (Lemma 4.1)
inline int vs_steps(int64_t d, double di) {
  int p = (int)ceil(log2(sqrt(2.0 * (double)d / M_PI) / di));
  return p > 1 ? p : 1;
}

// Dense blocks are row-major with the leading dimension padded to a multiple
// of 8 floats, so every row starts on a 32-byte sector and float4 accesses
// are aligned. Padding columns are kept at zero.
inline int ld_of(int k) { return (k + 7) & ~7; }

constexpr int kMaxEll = 256;      // largest sketch size l
constexpr int kMaxEig = 512;      // largest symmetric eigenproblem (2 l)
constexpr int kSplit = 256;       // entries per work item of the sparse products
constexpr float kAlpha = 6.0f / 41.0f;  // alpha of Alg. 4

struct CudaError {
  cudaError_t err;
  const char* where;
};

// Throwing check used inside the library; the C ABI layer catches it.
#define SFD_CUDA(call)                                        \
  do {                                                        \
    cudaError_t e__ = (call);                                 \
    if (e__ != cudaSuccess) throw ::sfd::CudaError{e__, #call}; \
  } while (0)

// Every kernel launch is followed by this check; it also counts launches
// (process-wide) so callers can report how many kernels ran.
extern unsigned long long g_kernel_launches;
#define SFD_LAUNCH_CHECK()                 \
  do {                                     \
    __atomic_add_fetch(&::sfd::g_kernel_launches, 1ull, __ATOMIC_RELAXED); \
    SFD_CUDA(cudaGetLastError());          \
  } while (0)

// A CSR-like structure on the device (rows of A' for the CSR copy, columns
// for the CSC copy) plus the work list that splits long segments.
// The item and split counts stay on the device (no host round trip): kernels
// are launched for the capacities and read the counts.
struct SegWork {
  int4* items = nullptr;     // (segment, begin, end, partial slot or -1), end - begin <= kSplit
  int* item_slot = nullptr;  // -1: item covers its whole segment, else partial slot
  int* item_split = nullptr; // -1, else the split segment (index into split_*) of the item
  unsigned* split_ticket = nullptr;  // per split segment: items done (0 between launches)
  int* split_seg = nullptr;  // segments cut into several items
  int* split_first = nullptr;// first item of each split segment
  int* split_count = nullptr;// items of each split segment
  int* counters = nullptr;   // offsets / scan scratch
  const int* d_n_items = nullptr;  // device: number of items
  const int* d_n_split = nullptr;  // device: number of split segments
  int cap_items = 0, cap_split = 0;
};

struct Csr {
  int* ptr = nullptr;   // nseg + 1
  int* idx = nullptr;   // nnz
  float* val = nullptr; // nnz
  int nseg = 0;
  int64_t nnz = 0;
  // host: false only when no segment is longer than kSplit (known from the
  // host's copy of the row pointers), so no item writes a partial row and the
  // products skip their split fix-up launch
  bool may_split = true;
  SegWork work;
};

// Scratch owned by a context (or by a one-shot call).
struct Workspace {
  // small dense
  float* gram_partial = nullptr;  // [chunks][tiles] 64x64 partial tiles
  int gram_partial_cap = 0;       // floats
  float* small_a = nullptr;       // kMaxEig^2 floats: Gram / eigen input
  float* small_b = nullptr;       // kMaxEig^2 floats: R^-1 / eigenvectors / weights
  float* evals = nullptr;         // kMaxEig
  float* eig_work = nullptr;      // eigensolver scratch
  double* scalars = nullptr;      // device scalars (norms, logs)
  int* flags = nullptr;           // device status words (16): [0] bad input entry,
                                  // [1] clamped Cholesky pivots, [2] a bounded wait
                                  // expired, [8] VerifySpectral's block tickets
  // sparse helpers
  int* tmp_i0 = nullptr;
  int* tmp_i1 = nullptr;
  float* tmp_f0 = nullptr;
  int* hist = nullptr;
  int hist_cap = 0;
  int* scan_tmp = nullptr;
  float* partial_rows = nullptr;  // split-segment partial outputs [slots][ld]
  int partial_rows_cap = 0;       // rows
  float* vec0 = nullptr;          // VS vectors
  float* vec1 = nullptr;
  float* vec2 = nullptr;
  float* wpart = nullptr;         // VS B'x partials
};

// ---------------------------------------------------------------- sparse ops
// Row ids of each entry of a CSR (expand ptr).
void launch_row_ids(const int* ptr, int nseg, int* rows, cudaStream_t s);
// Validate a buffer slice: indices in [0,d), finite values; sum of squares
// into fro2_out[0]; column counts (atomic) when col_count is not null. Sets
// flags[0] on a bad index/value.
void launch_check_entries(const int* idx, const float* val, int64_t nnz, int d, int* col_count,
                          double* fro2_out, int* flags, cudaStream_t s);
// ptr[c] = first position of column c in the column-sorted keys (ptr[d] = n).
void colptr_from_sorted(const int* keys, int64_t n, int d, int* ptr, cudaStream_t s);
// Exclusive scan of n ints (n >= 0) into out[0..n]; out[n] = total.
void exclusive_scan(const int* in, int n, int* out, int* tmp, cudaStream_t s);
// Stable LSD radix sort of (key, a, b) by key in [0, 2^bits): CSR -> CSC.
void radix_sort_by_key(int* key, int* a, float* b, int* key_alt, int* a_alt, float* b_alt,
                       int64_t n, int bits, int* hist, int* scan_tmp, cudaStream_t s);
// Work list of a segmented structure (split segments longer than kSplit).
void build_work(Csr& c, cudaStream_t s);
// Y[seg, 0:k] = sum over entries of seg: val * X[idx, 0:k]  (k <= 256, lds % 4 == 0)
// variant: how many gathers each lane keeps in flight (0: the default; the
// variants differ only in unrolling, never in results; spmm_variants(true)
// tells how many the fp16 form has)
void spmm(const Csr& c, const float* X, int ldx, int k, float* Y, int ldy, float* partial,
          cudaStream_t s, int variant = 0);
inline int spmm_variants(bool half) { return half ? 3 : 2; }
// Same with X stored as fp16 (k <= 128, ldx % 8 == 0): the gather moves half
// the bytes; products and sums are fp32.
void spmm_h(const Csr& c, const __half* X, int ldx, int k, float* Y, int ldy, float* partial,
            cudaStream_t s, int variant = 0);
// y[seg] = scale_ptr? * sum val * x[idx]
// xscale (nullable): x is read as x * (float)xscale[1] (a pending normalisation)
void spmv(const Csr& c, const float* x, float* y, float* partial, cudaStream_t s,
          const double* xscale = nullptr);

// Bounded waits of the tensor-core stages (failure detection without a GPU
// fault): set the iteration limit of every stage's first waits for the
// launches that follow, process-wide (spins < 0: the default; 0: such a wait
// gives up at once), and run one wait that nothing ends with the given
// limit (returns 1 when it ran out, as it must; *ms: its duration).
void set_wait_limit(int64_t spins);
int wait_selftest(int64_t spins, float* ms);

// ----------------------------------------------------------------- dense ops
// Philox4x64-10 Gaussian fill: out[i*ld + j] = normal #(i*cols + j) of (seed,b,r,tag).
void launch_gauss_fill(float* out, int64_t rows, int cols, int ld, uint64_t seed, uint64_t b,
                       uint64_t r, uint64_t tag, cudaStream_t s);
// Column map of a dense operand made of two blocks: columns [0, k0) are
// columns of X (leading dimension ldx), columns [k0, k0+k1) are columns of x1
// (leading dimension ld1). Single blocks use k1 = 0.
struct ColMap {
  int k0, k1;
  const float* x1;
  int ld1;
  __host__ __device__ int total() const { return k0 + k1; }
  __device__ float at(const float* X, int ldx, int64_t g, int c) const {
    return c < k0 ? X[g * ldx + c] : x1[g * ld1 + (c - k0)];
  }
};
inline ColMap single_map(int k) { return ColMap{k, 0, nullptr, 0}; }
// G = X^T X (n x n, n = map.total(), row-major ld n) over `rows` rows.
void gram(const float* X, int ldx, ColMap map, int64_t rows, float* G, Workspace& ws,
          cudaStream_t s);
// Y[:, 0:kout] = X[:, map] * T (T: n x kout row-major, ld kout).
void gemm_ts(const float* X, int ldx, ColMap map, int64_t rows, const float* T, int kout, float* Y,
             int ldy, cudaStream_t s);
// G = X^T X reduced from 128 x 128 partial tiles (one per chunk of rows).
void gram_reduce_tiles(const float* partial, int nchunks, int n, float* G, cudaStream_t s);
// Tensor-core (tcgen05 kind::tf32, FP32 accumulate) forms of gram and
// gemm_ts for n, kout <= 128. A wait that expires sets flags[2].
// split: the fp32-accurate form (each value split into TF32 hi and lo parts,
// hi*hi + hi*lo + lo*hi accumulated; ~21 significant bits); the split X * T
// needs tc_split_supported (its operands' hi and lo parts fill shared memory).
bool tc_supported(int n, int kout);
bool tc_split_supported(int n, int kout);
void gram_tc(const float* X, int ldx, ColMap map, int64_t rows, float* G, Workspace& ws,
             cudaStream_t s, bool split = false);
// G = [X1 X2]^T [X1 X2] ((n1 + n2) x (n1 + n2) row-major) for blocks whose
// columns are mutually orthogonal within each block: only the cross block
// X1^T X2 (split TF32) and the squared column norms are formed; the other
// entries of the diagonal blocks are 0. n1 in [1, 128], n2 in [0, 128].
void cross_gram_tc(const float* X1, int ld1, int n1, const float* X2, int ld2, int n2,
                   int64_t rows, float* G, Workspace& ws, cudaStream_t s);
// Yh (optional): write Y as fp16 into Yh (ld ldy, a multiple of 8, >= kout;
// columns kout..ldy-1 get 0) instead of fp32 into Y; for |entries| <= 1.
// accumulate (split form only): Y += X T instead of Y = X T.
void gemm_ts_tc(const float* X, int ldx, ColMap map, int64_t rows, const float* T, int kout,
                float* Y, int ldy, Workspace& ws, cudaStream_t s, __half* Yh = nullptr,
                bool split = false, bool accumulate = false);
// Cholesky of G + shift (k x k) and the inverse of the factor: Rinv (k x k
// row-major, upper triangular) with G + shift = R^T R. flags[1] counts pivots
// clamped. fp64: factorisation and inverse in double (one CTA; work holds
// k (k|1) doubles when they do not fit in shared memory), else fp32.
void chol_inv(const float* G, int k, float* Rinv, float* work, int* flags, cudaStream_t s,
              bool fp64 = false);
// The blocked one-CTA form used by chol_inv for k <= 128.
void chol_inv_blk(const float* G, int k, float* Rinv, int* flags, cudaStream_t s,
                  bool fp64 = false);
// Whether the blocked form fits one CTA's shared memory (fp64: k <= 112).
bool chol_blk_supported(int k, bool fp64);
// Largest nwant eigenpairs of the symmetric n x n S: evals (descending),
// evecs n x nwant row-major. psd: S is a Gram matrix (positive semi-definite),
// which allows the one-sided Jacobi path for n <= 128; otherwise (or for
// larger n) tridiagonalisation + bisection + inverse iteration.
void symeig(const float* S, int n, int nwant, float* evals, float* evecs, float* work,
            cudaStream_t s, bool psd = false);
size_t symeig_work_floats(int n, int nwant);
// Shrink weights with threshold thr = ev[nkeep-1] (thr_zero: thr = 0, the
// case of fewer than l rows): T[i][j] = evecs[i][j] * sqrt(max(0, 1 - thr/ev[j]))
// for j < nkeep (0 where ev[j] <= thr or ev[j] <= 0); scal[0] =
// sum_j max(0, ev[j] - thr), the squared Frobenius norm of the shrunk sketch.
void shrink_weights(const float* evals, const float* evecs, int n, int nwant, int nkeep,
                    int thr_zero, float* T, double* scal, cudaStream_t s);
// out (cols x rows, row-major, ld_out) = in^T  (in: rows x cols, ld_in)
void transpose(const float* in, int64_t rows, int cols, int ld_in, float* out, int64_t ld_out,
               cudaStream_t s);
// Scatter a CSR block (rows x d) densely and transposed into out (d x ld, zeroed first).
void csr_to_dense_t(const int* ptr, const int* idx, const float* val, int rows, int64_t d,
                    float* out, int ld, cudaStream_t s);

// ------------------------------------------------------------ VerifySpectral
struct VsArgs {
  const Csr* csr;
  const Csr* csc;
  const float* Bt;  // d x ld (B'^T)
  int ld, ell;
  int64_t d, m;
  const double* scale_dev;  // device: 2 / Delta
  int p;
  uint64_t seed, b, r;
};
// CUDA graphs of one and of two power steps (the step's arguments are fixed
// for the workspace and the CSR/CSC copies it is used with), captured on first
// use and replayed; owned by the caller.
struct VsGraphs {
  cudaGraphExec_t one = nullptr, two = nullptr;
  int kernels_per_step = 0;
  void release() {
    if (one) cudaGraphExecDestroy(one);
    if (two) cudaGraphExecDestroy(two);
    one = two = nullptr;
  }
};
// Enqueues p power steps; log ||C^p x|| lands in ws.scalars[kSlogsum],
// ws.scalars[kSzero] = 1 if some C x_t vanished. No host synchronisation.
// With graphs (not null) the steps are replayed from its CUDA graphs.
void verify_spectral(const VsArgs& a, Workspace& ws, cudaStream_t s, VsGraphs* graphs = nullptr);

// Device scalars of one SparseShrink attempt (ws.scalars[...]).
enum : int {
  kSfro2b = 0,   // ||B'||_F^2 (shrink_weights)
  kSthr = 1,     // lambda_l^2
  kSlogsum = 8,  // VerifySpectral log-sum
  kSinvn = 9,    // its running inverse norm
  kSzero = 10,   // some C x_t was zero
  kSdelta = 16,  // Delta of Alg. 4
  kSscale = 17,  // 2 / Delta
  kSsmall = 18,  // Delta/2 at the fp32 resolution of ||A'||_F^2: accepted
};
// Verdict of one attempt, copied to pinned host memory.
struct Verdict {
  double fro2a, fro2b, delta, logsum;
  double captured;  // ||P||_F^2 = sum of the eigenvalues of P P^T
  int ok, small, zero, timeout;  // timeout: a bounded device wait expired (flags[2])
};
// Delta = (fro2a - fro2b) / (alpha l), scale = 2 / Delta, small flag.
void launch_delta(const double* fro2a, double* scal, int ell, cudaStream_t s);
// Verdict from the device scalars (verify = 0: accepted).
void launch_verdict(const double* fro2a, const double* scal, const int* flags,
                    const float* evals, int ell, int verify, Verdict* out,
                    cudaStream_t s);

// ------------------------------------------------------------- learned q
constexpr int kQF = 16;   // features
constexpr int kQH = 64;   // hidden width
constexpr int kQParams = kQF * kQH + kQH + kQH * kQH + kQH + kQH + 1;
constexpr int kQAccWords = 8;  // scratch of q_features (unsigned words)
// The 16 features of a buffer (CSR + CSC built, fro2 = ||A'||_F^2 on the
// device, S0 = Gram of A'G, l x l) into feat[16].
void q_features(const Csr& csr, const Csr& csc, int64_t d, int ell, int q_fixed,
                const double* fro2, const float* S0, float* feat, unsigned* acc_dev,
                cudaStream_t s);
// y[s] = network(X[s]) (X: n x 16 row-major).
void mlp_forward(const float* P, const float* X, int n, float* y, cudaStream_t s);
// q_out[0] = clamp(ceil(network(feat) + margin), 1, q_fixed); y_tmp: 1 float.
void predict_q(const float* P, const float* feat, float margin, int q_fixed, float* y_tmp,
               int* q_out, cudaStream_t s);
// grad = d/dP of (1/2n) sum (network(X) - T)^2, loss (nullable) = that value.
void mlp_grad(const float* P, const float* X, const float* T, int n, float* grad, float* loss,
              cudaStream_t s);
// Adam step number `step` (>= 1) on P with moments m1, m2.
void adam_update(float* P, const float* grad, float* m1, float* m2, int step, float lr,
                 cudaStream_t s);

}  // namespace sfd
