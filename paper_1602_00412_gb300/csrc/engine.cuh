// Device-side engine of Sparse Frequent Directions (internal, not the C ABI).
//
// A Slot owns everything one buffer's BoostedSparseShrink needs (Alg. 3, 4,
// 1, 6): the CSR and CSC copies of A', the work lists, the dense blocks of
// SimultaneousIteration, B'^T, scratch, a CUDA stream and pinned memory for
// the verdict. Several slots run different buffers concurrently, so the
// one-CTA steps (Cholesky, eigensolver) of one buffer overlap the
// whole-GPU steps (sparse products, Grams) of another.
//
// The Merger owns the sketch B (as B^T, d x ld, ping-pong pair) and runs
// DenseShrink (Alg. 5) on its own stream, in buffer order.
//
// Nothing on a slot's stream synchronises the host: counts, norms, Delta and
// the VerifySpectral verdict stay on the device until the verdict is copied
// to pinned host memory at the end of an attempt.
#pragma once

#include <vector>

#include "sfd_internal.cuh"

namespace sfd {

// Device allocations of one owner, freed together.
struct DevArena {
  std::vector<void*> ptrs;
  template <typename T>
  T* alloc(size_t n) {
    void* p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) throw CudaError{e, "cudaMalloc"};
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

// Scratch of the dense stages (Gram, Cholesky, eigensolver, weights).
void alloc_dense_scratch(DevArena& A, Workspace& ws);

// How an attempt chooses its power count (the learned form; Alg. 1's q).
struct QControl {
  const float* params = nullptr;  // device network parameters (kQParams), predict only
  float margin = 1.f;
  int q_fixed = 0;
  bool predict = false;   // q = network(features), clamped to [1, q_fixed]
  bool features = false;  // compute the features (copied to qfeat_host) without predicting
};

struct Slot {
  int64_t d = 0, cap_rows = 0, cap_nnz = 0;
  int ell = 0, ld = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t done = nullptr;   // recorded after the verdict copy of an attempt
  cudaEvent_t freed = nullptr;  // recorded on the merge stream after DenseShrink read B'^T
  bool freed_pending = false;   // `freed` has been recorded and not yet waited on
  DevArena arena;
  Csr csr, csc;
  int *key = nullptr, *key2 = nullptr, *a_alt = nullptr;
  float* b_alt = nullptr;
  float *W = nullptr, *W2 = nullptr, *Y = nullptr, *Y2 = nullptr;
  __half *Wh = nullptr, *Yh = nullptr;  // fp16 copies of orthonormal blocks (mixed precision)
  float* Bpt = nullptr;         // B'^T, d x ld
  Workspace ws;
  double* fro2 = nullptr;       // [0] ||A'||_F^2, [1..] partials
  Verdict* verdict_dev = nullptr;
  Verdict* verdict_host = nullptr;  // pinned
  // learned q: features and prediction of the current buffer
  float* qfeat = nullptr;           // device, kQF
  unsigned* qacc = nullptr;         // device, kQAccWords
  float* qy = nullptr;              // device, 1
  int* q_dev = nullptr;             // device, 1
  float* qfeat_host = nullptr;      // pinned, kQF
  int* q_host = nullptr;            // pinned, 1
  int* ptr_host = nullptr;          // pinned staging of the local row pointer
  // precision 1: the orthonormalisations inside the power iterations run their
  // Gram and X R^-1 on tensor cores (TF32 inputs, FP32 accumulate), the
  // accurate stages in the split TF32 form
  bool mixed = false;
  // autotuning of the sparse products: the unroll variant of each pass
  // ([A' X (CSR), A'^T Y (CSC)] x [fp32, fp16 X]), timed on its first use
  bool autotune = false;
  int spmm_choice[2][2] = {{-1, -1}, {-1, -1}};
  // the choices in use: this slot's own, or those of the context's first slot
  // (slots of one context share their shapes, so one slot tunes for all)
  int (*choice)[2] = spmm_choice;
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  VsGraphs vs_graphs;  // VerifySpectral steps, captured on first use
  // profiling of the sparse products
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, double>> ev_pending;
  int ev_used = 0;
  int64_t prof_launches = 0;
  double prof_ms = 0, prof_bytes = 0;

  Slot(int64_t d, int ell, int64_t cap_rows, int64_t cap_nnz, cudaStream_t s);
  ~Slot();
  Slot(const Slot&) = delete;
  Slot& operator=(const Slot&) = delete;

  // the stream must not overwrite B'^T before DenseShrink has read it
  void wait_freed();
  // CSR structure + CSC copy + work lists of the buffer already in csr.{ptr,idx,val}
  // max_row: the longest row of the buffer when the host knows it, else -1
  void build(int m, int64_t nnz, int64_t max_row = -1);
  // One SparseShrink attempt (Alg. 3) + Delta + VerifySpectral (Alg. 6) +
  // verdict copy; `done` is recorded at the end. With qc->predict the power
  // count comes from the network: the host waits for the first product's
  // Gram and the prediction before it enqueues the power loop. Returns the q
  // used.
  int enqueue_attempt(int m, int q, uint64_t seed, uint64_t b, uint64_t r, int p, int verify,
                      const QControl* qc = nullptr);
  void collect_profile();  // host: needs `done`

 private:
  void cleanup();
  // CholeskyQR step X -> Xout. form 0: CUDA cores, FP32; 1: tensor cores,
  // TF32 inputs; 2: tensor cores, split TF32 (FP32-accurate) and the l x l
  // Cholesky in FP64. The tensor-core Grams need l <= 128 (else the CUDA-core
  // Gram runs; form 2 keeps its FP64 Cholesky). With form 1 and Xh, the result
  // goes to Xh as fp16 only (returns true then).
  bool orth_pass(const float* X, int64_t rows, float* Xout, int form, __half* Xh = nullptr);
  void spmm_timed(const Csr& c, const float* X, float* Yo, int64_t rows_in,
                  const __half* Xh = nullptr);
  int tune_spmm(const Csr& c, const float* X, const __half* Xh, float* Yo);
};

struct Merger {
  int64_t d = 0;
  int ell = 0, ld = 0;
  cudaStream_t stream = nullptr;
  DevArena arena;
  float* Bt[2] = {nullptr, nullptr};  // d x ld
  float* out = nullptr;               // l x d: the sketch, transposed for a host copy
  int cur = 0;
  Workspace ws;

  Merger(int64_t d, int ell);
  ~Merger();
  Merger(const Merger&) = delete;
  Merger& operator=(const Merger&) = delete;

  // precision 1: when both blocks have orthogonal rows, the Gram of the stack
  // is formed on tensor cores from its cross block (split TF32, cross_gram_tc)
  bool mixed = false;

  float* B() { return Bt[cur]; }
  void zero();
  // B <- DenseShrink([B; X]) with X^T given as d x k1 (leading dimension ldx).
  // orthogonal_rows: X has orthogonal rows (a sketch, or the B' of
  // SparseShrink), as B always has (it is a DenseShrink output, or 0).
  void dense_shrink(const float* Xt, int ldx, int k1, bool orthogonal_rows = false);

 private:
  void cleanup();
};

}  // namespace sfd
