/*
 * sfd.h - C ABI of the GB300 Sparse Frequent Directions library (libsfd.so).
 *
 * Sparse Frequent Directions (Ghashami, Liberty, Phillips): rows of a sparse
 * matrix A (n x d) arrive one at a time (Sec. 1, the row-streaming model);
 * the library keeps an l x d sketch B with O(d l) memory (Fact in Sec. 4.2).
 * Rows are buffered until the buffer A' holds l*d non-zeros or d rows
 * (Alg. 2); then B' = BoostedSparseShrink(A') (Alg. 4: SparseShrink of Alg. 3
 * on top of SimultaneousIteration of Alg. 1, checked by VerifySpectral of
 * Alg. 6) and B = DenseShrink([B; B']) (Alg. 5). Sketches are mergeable
 * (Sec. 3.1): merge(B1, B2) = DenseShrink([B1; B2]).
 *
 * Conventions for every entry point
 *  - Return value: SFD_OK (0) or one of the SFD_E* codes below. No C++
 *    exception crosses this boundary. After SFD_EINVAL the context is
 *    unchanged and usable; after SFD_ECUDA / SFD_ETIMEOUT it must be destroyed.
 *  - `where` says where caller arrays live: SFD_HOST (0) or SFD_DEVICE (1,
 *    memory of the current CUDA device). Caller arrays stay the caller's; the
 *    library copies what it keeps before the call returns.
 *  - Dense matrices are row-major float32 with the leading dimension stated.
 *  - A context is bound to the CUDA device current at sfd_create. Its work is
 *    ordered after the work already queued on options.cuda_stream when a call
 *    starts, and that stream waits for the call's work before the call returns
 *    (internally a context runs several streams). Calls on one context must
 *    not overlap; distinct contexts are independent.
 *  - Every call returns with its work finished on the device (results
 *    written, stream synchronised), except where stated.
 */
#ifndef SFD_H
#define SFD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SFD_ABI_VERSION 4u

#define SFD_OK 0
#define SFD_EINVAL 1   /* bad argument: l < 1, l > d, index outside [0,d), non-monotone indptr, NaN/Inf value, ... */
#define SFD_ENOMEM 2   /* device or host allocation failed */
#define SFD_ECUDA 3    /* CUDA runtime error (message in sfd_last_error) */
#define SFD_EVERIFY 4  /* strict mode: a buffer stayed unverified after retry_cap attempts */
#define SFD_ETIMEOUT 5 /* a bounded device-side wait ran out */

#define SFD_HOST 0
#define SFD_DEVICE 1

typedef struct sfd_ctx sfd_ctx; /* opaque, library-owned */

/* Options. Initialise with sfd_options_init(), then change fields. */
typedef struct sfd_options {
  uint32_t abi_version; /* must be SFD_ABI_VERSION */
  double delta;         /* failure probability delta of Alg. 4 / Theorem 4.1 (default 0.01) */
  int32_t verify;       /* 1: BoostedSparseShrink with VerifySpectral (Alg. 4, default);
                           0: SparseShrink called directly, as in the paper's experiments (Sec. 5) */
  double c_q;           /* power count q = ceil(c_q * ln(m/eps)/eps), eps = 1/4 (Alg. 1 with the
                           eps of Alg. 3); default 0.25, i.e. q = ceil(ln(4m)) */
  int32_t q_override;   /* >= 0: use this q for every buffer; -1 (default): the schedule above */
  int32_t retry_cap;    /* SparseShrink attempts per buffer before it is kept unverified (default 8) */
  int32_t precision;    /* 0: plain fp32 (default); 1: mixed: for l <= 128 the orthonormalisations
                           of every power iteration of Alg. 1 but the last form their Gram and
                           X R^-1 on tcgen05 tensor cores (TF32 inputs, FP32 accumulation);
                           the other dense products (last iteration, second CholeskyQR pass,
                           P P^T and B'^T of Alg. 3) keep FP32 accuracy: tensor cores in the
                           split form of sfd_gram (precision 2) where l allows, else CUDA
                           cores; the sparse products and eigensolvers stay FP32 */
  int32_t q_mode;       /* power count per buffer. 0: the fixed schedule (default); 1: learned:
                           q = clamp(ceil(network(features) + q_margin), 1, q_fixed) with the
                           network set by sfd_set_q_model (fixed schedule until one is set); a
                           buffer whose attempt VerifySpectral rejects is retried with q_fixed;
                           2: fixed schedule, and every buffer whose first attempt is accepted
                           is labelled for training (sfd_q_log) */
  int32_t strict;       /* 1: a buffer left unverified makes sfd_append_rows return SFD_EVERIFY */
  int32_t inject_vs_fail; /* testing: force this many VerifySpectral verdicts to False (host-side) */
  void* cuda_stream;    /* cudaStream_t to run on; NULL: the context creates its own */
  int32_t profile;      /* 1: time every sparse-product launch with CUDA events (sfd_stats.spmm_*) */
  int32_t slots;        /* buffers in flight: each slot runs one buffer's BoostedSparseShrink on its
                           own stream while DenseShrink folds finished buffers in order; 0: 6 */
  float q_margin;       /* q_mode 1: added to the network's output before rounding up (default 1) */
  float q_tau;          /* q_mode 2: a buffer's label is the smallest q of the ladder
                           {1,2,3,4,6,8,11,16,23,32,45,64} below q_fixed whose attempt passes
                           VerifySpectral and keeps ||P||_F^2 >= (1 - q_tau) times its value at
                           q_fixed (same G); q_fixed if none does (default 1e-2) */
  int32_t autotune;     /* 1 (default): each slot times the unroll variants of its sparse
                           products on first use and keeps the fastest per pass (the variants
                           give identical results); 0: the default variant */
  int32_t mode;         /* 0: Sparse Frequent Directions (Alg. 2, default); 1: the classical
                           FrequentDirections of Sec. 3.1, for comparison (Sec. 5): every l rows
                           B = DenseShrink([B; rows]) (Alg. 5), no SparseShrink */
} sfd_options;

/* Counters of a context (Alg. 2 / Alg. 4 bookkeeping). */
typedef struct sfd_stats {
  int64_t rows_seen;    /* rows appended */
  int64_t nnz_seen;     /* entries appended */
  int64_t buffers;      /* buffers closed (SparseShrink path or small-buffer DenseShrink) */
  int64_t attempts;     /* SparseShrink runs (>= verified buffers) */
  int64_t vs_rejects;   /* VerifySpectral verdicts that were False */
  int64_t unverified;   /* buffers kept after retry_cap failed attempts */
  int64_t q_total;      /* sum of q over all SparseShrink runs */
  int64_t pending_rows; /* rows in the open buffer */
  int64_t pending_nnz;  /* entries in the open buffer */
  double last_delta;    /* Delta of the last accepted buffer (Alg. 4) */
  double last_logsum;   /* log ||C^p x|| of the last VerifySpectral call */
  double last_fro2;     /* ||A'||_F^2 of the last buffer */
  int64_t kernel_launches; /* CUDA kernels this context launched */
  int64_t spmm_launches;   /* profile: sparse x dense products timed (A' X and A'^T Y) */
  double spmm_ms;          /* profile: their summed device time (CUDA events, ms) */
  double spmm_bytes;       /* profile: their algorithmic bytes: entries (8 B each) + row
                              pointers + dense input + dense output, fp32 */
} sfd_stats;

/* Per-buffer result of sfd_bssh_buffer. */
typedef struct sfd_shrink_info {
  int32_t q;            /* power count used */
  int32_t attempts;     /* SparseShrink runs */
  int32_t verified;     /* 1 if VerifySpectral accepted (or verify == 0) */
  int32_t vs_steps;     /* power steps p of the last VerifySpectral */
  double delta_shrink;  /* Delta = (||A'||_F^2 - ||B'||_F^2) / (alpha l), alpha = 6/41 */
  double logsum;        /* log ||C^p x|| of the last VerifySpectral */
  double fro2_a;        /* ||A'||_F^2 */
  double fro2_b;        /* ||B'||_F^2 */
  double captured;      /* ||P||_F^2 = ||Z^T A'||_F^2, the energy the subspace Z captures */
} sfd_shrink_info;

/* Fill `opt` with the defaults listed above. */
void sfd_options_init(sfd_options* opt);

/* Create a context for rows of dimension d and sketch size l (1 <= l <= d),
 * Alg. 2 initial state B = 0^{l x d}, empty buffer. `seed` keys every random
 * draw: G of Alg. 1 and x of Alg. 6 use Philox4x64-10 with
 * counter (block, buffer index, attempt, tag). opt may be NULL (defaults).
 * All device memory of the context is allocated here (O(d l) dense plus a
 * buffer of at most l*d + d entries). Errors: SFD_EINVAL, SFD_ENOMEM, SFD_ECUDA. */
int sfd_create(int64_t d, int32_t ell, uint64_t seed, const sfd_options* opt, sfd_ctx** out);

/* Append `nrows` rows given in CSR form (Alg. 2 loop body, one row at a time):
 *   indptr  nrows+1 int64, non-decreasing; row i holds entries
 *           [indptr[i], indptr[i+1]) of indices/values (indptr[0] may be != 0)
 *   indices int32 column indices in [0, d); duplicates within a row are summed
 *   values  float32, finite
 * All three arrays live in `where` memory. A row may hold at most d entries.
 * Every full buffer met on the way is shrunk and merged into B before the call
 * returns. The whole call is validated first: on SFD_EINVAL nothing of it is
 * applied. SFD_EVERIFY only in strict mode (the rows are applied). */
int sfd_append_rows(sfd_ctx* ctx, int64_t nrows, const int64_t* indptr, const int32_t* indices,
                    const float* values, int where);

/* Write the sketch B (l x d, row-major, leading dimension d) to B_out in
 * `where` memory. Rows still in the open buffer are flushed first: with at
 * least l rows they take BoostedSparseShrink + DenseShrink, with fewer
 * DenseShrink([B; A']) (Alg. 2 returns B without them; this closes the stream
 * the same way at any point). Rows of B are orthogonal; the last is zero. */
int sfd_sketch(sfd_ctx* ctx, float* B_out, int where);

/* Mergeability (Sec. 3.1): dst.B <- DenseShrink([dst.B; src.B]), after both
 * open buffers are flushed as in sfd_sketch. src keeps its (flushed) sketch.
 * Requires equal d and l and the same device. */
int sfd_merge(sfd_ctx* dst, sfd_ctx* src);

/* Checkpoint (no counterpart in the paper; the stream state of Alg. 2 between
 * rows is the sketch B, the open buffer A' and the buffer counter b). sfd_save
 * writes the context's state to `buf` (host memory, `cap` bytes) and its size
 * to *size_out; buf = NULL only reports the size. Nothing is flushed: the
 * state is taken as it stands after the last call (every call leaves no
 * buffer in flight). The blob holds d, l, seed, b, the options that decide
 * the result (delta, verify, c_q, q_override, retry_cap, precision, q_mode,
 * strict, q_margin, q_tau, mode), the counters, B (l x d float32), the open buffer
 * (int32 row pointer, int32 columns, float32 values), the learned-q network
 * when one is set (not the q_mode 2 label log), and an FNV-1a hash; host
 * byte order. Errors: SFD_EINVAL (cap too small), SFD_ENOMEM, SFD_ECUDA. */
int sfd_save(sfd_ctx* ctx, void* buf, int64_t cap, int64_t* size_out);

/* A new context on the current device from a blob of sfd_save: appending the
 * same rows to it gives the same sketch, bit for bit, as appending them to the
 * saved context. The computing options come from the blob; `runtime`
 * (nullable) supplies only cuda_stream, slots, profile and autotune.
 * Errors: SFD_EINVAL (bad size, magic, version, hash or contents), SFD_ENOMEM,
 * SFD_ECUDA. */
int sfd_load(const void* buf, int64_t size, const sfd_options* runtime, sfd_ctx** out);

/* Counters; see sfd_stats. */
int sfd_get_stats(const sfd_ctx* ctx, sfd_stats* out);

/* Start a new stream on the same context: B = 0, the open buffer is dropped,
 * the buffer counter (and so every Philox key) restarts at 0, counters are
 * cleared. Device memory is kept. */
int sfd_reset(sfd_ctx* ctx);

/* Release every resource of the context (NULL is a no-op). */
void sfd_destroy(sfd_ctx* ctx);

/* Static text for a status code. */
const char* sfd_strerror(int status);

/* Text of the last error seen by this context ("" if none). */
const char* sfd_last_error(const sfd_ctx* ctx);

/* ------------------------------------------------------------------------
 * One buffer / one stack (the per-step calls used to check each stage).
 * Device pointers only; the stream is the default stream of the calling
 * thread's current device. Each call allocates its own scratch.
 * ------------------------------------------------------------------------ */

/* BoostedSparseShrink (Alg. 4) of one buffer A' (m x d CSR with int32
 * rowptr[m+1] starting at 0, colidx[nnz], vals[nnz], device memory), with the
 * randomness of buffer index b under `seed` (same keys as a context).
 * l <= m is required (Alg. 3). Output Bp_out: l x d row-major (device), the
 * shrunk sketch B' = Lambda~ V^T. info may be NULL. opt may be NULL. */
int sfd_bssh_buffer(int64_t m, int64_t d, int32_t ell, const int32_t* rowptr, const int32_t* colidx,
                    const float* vals, uint64_t seed, int64_t b, const sfd_options* opt,
                    float* Bp_out, sfd_shrink_info* info);

/* DenseShrink (Alg. 5) of a rows x d matrix M (row-major, device), rows <= 2*l
 * and l <= 256: B_out (l x d, device) = sqrt(Lambda^2 - lambda_l^2) V^T. */
int sfd_dense_shrink(int64_t rows, int64_t d, int32_t ell, const float* M, float* B_out);

/* Sparse x dense product of Alg. 1: Y = A X (transpose = 0) or Y = A^T X
 * (transpose = 1) for A (m x d CSR as in sfd_bssh_buffer), X (d x k or m x k,
 * leading dimension ldx), Y (m x k or d x k, leading dimension ldy), k <= 256,
 * ldx, ldy multiples of 4 and >= k, all device memory. */
int sfd_csr_spmm(int64_t m, int64_t d, const int32_t* rowptr, const int32_t* colidx,
                 const float* vals, int32_t k, const float* X, int32_t ldx, float* Y, int32_t ldy,
                 int32_t transpose);

/* The same product with the kernel form chosen (for testing the autotuned
 * forms, which give bit-identical results): X is fp32 (x_fp16 = 0; k <= 256,
 * ldx, ldy multiples of 4) or fp16 (x_fp16 = 1, X holds IEEE binary16 values;
 * k <= 128, ldx, ldy multiples of 8; products and sums in fp32); variant in
 * [0, sfd_spmm_variant_count(x_fp16)): the forms differ in how many gathered
 * rows each lane keeps in flight. Errors: SFD_EINVAL, SFD_ENOMEM, SFD_ECUDA. */
int sfd_spmm_variant_count(int32_t x_fp16);
int sfd_csr_spmm_ex(int64_t m, int64_t d, const int32_t* rowptr, const int32_t* colidx,
                    const float* vals, int32_t k, const void* X, int32_t x_fp16, int32_t ldx,
                    float* Y, int32_t ldy, int32_t transpose, int32_t variant);

/* Orthonormalise the columns of X (rows x k, leading dimension ld, device) in
 * place (the GramSchmidt step of Alg. 1), k <= 256, by shifted CholeskyQR3:
 * three passes of Gram (FP32, fixed summation order), Cholesky factor of the
 * shifted Gram and its inverse (FP64), X R^-1 (FP32). */
int sfd_orthonormalize(int64_t rows, int32_t k, float* X, int32_t ld);

/* ------------------------------------------------------------ many streams
 * A batch of independent SFD streams on the current device (Alg. 2 each;
 * no counterpart in the paper beyond mergeability, Sec. 3.1): stream i has
 * d[i] columns, l = ell[i], Philox seed `seed + i`, and the options `opt`
 * (NULL: defaults; cuda_stream must be NULL; slots 0 means 1 here). Worker
 * threads (`workers`, 0: min(nstreams, 8)) drive the streams so that their
 * buffers run concurrently; stream i belongs to worker i % workers, so its
 * rows are processed in append order. Host arrays are copied before
 * sfd_batch_append returns; device arrays are read later and must stay valid
 * until sfd_batch_wait (or a call that waits) returns. Errors of queued work
 * are reported by the next call that waits (first error only). */
typedef struct sfd_batch sfd_batch;
int sfd_batch_create(int32_t nstreams, const int64_t* d, const int32_t* ell, uint64_t seed,
                     const sfd_options* opt, int32_t workers, sfd_batch** out);
/* Queue rows for one stream (arguments as in sfd_append_rows). */
int sfd_batch_append(sfd_batch* batch, int32_t stream, int64_t nrows, const int64_t* indptr,
                     const int32_t* indices, const float* values, int where);
/* Wait for all queued work. */
int sfd_batch_wait(sfd_batch* batch);
/* Wait, then the sketch of one stream (as sfd_sketch). */
int sfd_batch_sketch(sfd_batch* batch, int32_t stream, float* B_out, int where);
/* Chunk-parallel sketch: wait, then fold every stream into stream 0 by a
 * binary tree of merges (level s merges stream i + s into stream i for i a
 * multiple of 2s, pairs of a level in parallel); all streams must have the same
 * d and l. Streams other than 0 keep partial unions. B_out (nullable) gets
 * stream 0's sketch (l x d row-major, where as in sfd_sketch). */
int sfd_batch_merge_tree(sfd_batch* batch, float* B_out, int where);
int sfd_batch_stats(const sfd_batch* batch, int32_t stream, sfd_stats* out);
void sfd_batch_destroy(sfd_batch* batch);

/* ---------------------------------------------------------------- learned q
 * The power count q of Alg. 1 is fixed by Sec. 3.2 only up to a constant, and
 * Alg. 4 verifies every result; the learned form predicts q per buffer (no
 * counterpart in the paper). The predictor is a 16 -> 64 -> 64 -> 1 ReLU
 * network over SFD_QF buffer features; its SFD_QPARAMS float parameters are
 * laid out as W1 [16][64] (input-major), b1[64], W2 [64][64] (input-major),
 * b2[64], w3[64], b3. Features (all computed on the device):
 *   0 1;  1 ln m / 10;  2 ln N / 20 (N = nnz);  3 ln d / 15;  4 l / 256;
 *   5 ln(N/m) / 5;  6 ln(||A'||_F^2 / N) / 10;  7 max row norm^2 / ||A'||_F^2;
 *   8 max column count / N;  9 sum of column counts^2 / N^2;
 *  10 m * sum of row counts^2 / N^2 - 1;  11 ln q_fixed / 3;
 *  12 ||S0||_F^2 / tr(S0)^2;  13 max diag(S0) / tr(S0)  (S0 = (A'G)^T (A'G),
 *     G the start block of attempt 0);  14 ln(1 + N / (m l));
 *  15 1 - (nonempty columns) / d.
 * All arrays below are host memory; errors: SFD_EINVAL, SFD_ENOMEM, SFD_ECUDA. */
#define SFD_QF 16
#define SFD_QPARAMS 5313
/* Use `params` (host, copied) for q_mode 1; NULL removes the model. */
int sfd_set_q_model(sfd_ctx* ctx, const float* params);
/* The label log of q_mode 2: up to `cap` rows of features (cap x 16), labels
 * and the buffers' q_fixed (nullable); *n_out = rows logged so far. */
int sfd_q_log(const sfd_ctx* ctx, int64_t cap, float* features, float* labels, int32_t* q_fixed,
              int64_t* n_out);
/* The features of one buffer (device CSR as in sfd_bssh_buffer, key (seed, b)). */
int sfd_q_features(int64_t m, int64_t d, int32_t ell, const int32_t* rowptr, const int32_t* colidx,
                   const float* vals, uint64_t seed, int64_t b, int32_t q_fixed, float* features);
/* y[i] = network(features[i]) for n rows (n x 16). */
int sfd_q_predict(int64_t n, const float* features, const float* params, float* y_out);
/* Gradient (SFD_QPARAMS floats) of L = (1/2n) sum (network(features[i]) - targets[i])^2,
 * and L (nullable). */
int sfd_q_grad(int64_t n, const float* features, const float* targets, const float* params,
               float* grad_out, float* loss_out);
/* Adam (lr, betas 0.9 / 0.999, eps 1e-8) on L over `epochs` passes in minibatches of
 * `batch` rows, each pass in an order drawn from `seed`; params is updated in place
 * and *loss_out (nullable) is L of the result over all n rows. */
int sfd_q_train(int64_t n, const float* features, const float* targets, int32_t epochs,
                int32_t batch, float lr, uint64_t seed, float* params, float* loss_out);

/* The two dense products of a CholeskyQR step (the GramSchmidt of Alg. 1):
 * G = X^T X (k x k row-major, leading dimension k) over X (rows x k, leading
 * dimension ldx), and Y = X T for T (n x kout row-major, leading dimension
 * kout), X (rows x n, ldx), Y (rows x kout, ldy). All device memory; rows may
 * be 0 (G = 0, Y untouched). precision 0: FP32 on the CUDA cores, sums in a
 * fixed order (bit-reproducible); precision 1: tcgen05 tensor cores, inputs
 * rounded to TF32 (10-bit mantissa), FP32 accumulation, for k, n, kout <= 128
 * (larger returns SFD_EINVAL); precision 2: tensor cores in the split form
 * (each input x = x_hi + x_lo, x_hi = x with its 13 low mantissa bits
 * cleared; x_hi y_hi + x_hi y_lo + x_lo y_hi accumulated in FP32: about 21
 * significant bits), for k <= 128 in sfd_gram and n, kout <= 112 in
 * sfd_gemm_ts (larger returns SFD_EINVAL). Errors: SFD_EINVAL, SFD_ENOMEM, SFD_ECUDA,
 * SFD_ETIMEOUT (a bounded tensor-core wait ran out; the outputs are not valid). */
int sfd_gram(int64_t rows, int32_t k, const float* X, int32_t ldx, float* G, int32_t precision);
int sfd_gemm_ts(int64_t rows, int32_t n, const float* X, int32_t ldx, const float* T, int32_t kout,
                float* Y, int32_t ldy, int32_t precision);

/* Failure detection of the bounded device waits (not an operation of the
 * paper: the tensor-core stages of Alg. 1, 3 and 5 wait on mbarriers for their
 * copies and MMAs, and every such wait gives up after an iteration limit,
 * raising SFD_ETIMEOUT instead of hanging).
 * sfd_set_wait_limit: the limit of each stage's first waits, process-wide,
 * for every tensor-core launch made after the call: spins < 0 restores the
 * default (2^18 tries, about one second on GB300); 0 makes every such wait
 * give up at once, so the next tensor-core stage reports SFD_ETIMEOUT. The
 * waits that drain a failed stage (its copies and MMAs in flight) always keep
 * the default, so a stage that gave up still leaves nothing running. A
 * one-shot call (sfd_gram, sfd_gemm_ts) that returned SFD_ETIMEOUT may simply
 * be repeated; a context that did must be destroyed.
 * sfd_wait_selftest: one CTA waits, with limit `spins` (< 0: the default), on
 * an mbarrier that nothing arrives at; returns SFD_ETIMEOUT when the wait ran
 * out (the expected outcome), SFD_OK otherwise; *ms_out (nullable) receives
 * its duration in milliseconds. Errors: SFD_ECUDA. */
int sfd_set_wait_limit(int64_t spins);
int sfd_wait_selftest(int64_t spins, float* ms_out);

/* Symmetric eigendecomposition used by Alg. 3 / Alg. 5: the `nwant` largest
 * eigenvalues (descending, evals[nwant]) and their eigenvectors (evecs,
 * n x nwant row-major) of the symmetric n x n matrix S (row-major), n <= 512,
 * all device memory. */
int sfd_symeig(int32_t n, const float* S, int32_t nwant, float* evals, float* evecs);

/* The eigensolver of sfd_symeig without any allocation (no counterpart in the
 * paper; this is a library service). For callers that must not let a library
 * allocate device memory: a process whose caching allocator already holds the
 * device's memory budget, or a latency-critical loop that cannot take the
 * device-wide synchronisation cudaMalloc / cudaFree may cause. Its scratch is
 * a fixed array inside libsfd.so (~2.1 MB), so n <= 256 (1 <= nwant <= n);
 * larger n returns SFD_EINVAL. S, evals, evecs are caller-owned device memory
 * as in sfd_symeig. Runs on the legacy default stream (0) of the current
 * device and returns after that stream has finished.
 * The first call on each device (and again after the device's context was
 * reset) loads the part of the library that holds the array and looks up its
 * device address: with CUDA's lazy module loading (the default) that first
 * call is when the array (~2.1 MB) and that code take device memory, and it
 * may synchronise the device. Make one warm-up call per device before handing
 * the memory budget to an allocator and before any stream capture; from then
 * on calls allocate nothing and the device holds the array until its context
 * ends. All calls share the one array, which keeps the last call's contents:
 * calls that overlap on the GPU (from several host threads or streams) race
 * and must be serialised by the caller.
 * Errors: SFD_EINVAL, SFD_ECUDA. */
int sfd_symeig_noalloc(int32_t n, const float* S, int32_t nwant, float* evals, float* evecs);

#ifdef __cplusplus
}
#endif

#endif /* SFD_H */
