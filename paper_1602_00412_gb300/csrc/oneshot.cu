// Per-stage entry points of include/sfd.h (one buffer / one stack / one
// matrix), used to check each stage against the oracle. Each call allocates
// its own scratch and runs synchronously.
#include <string.h>

#include <algorithm>
#include <vector>

#include "engine.cuh"

using namespace sfd;

namespace {

int code_of(const CudaError& e) {
  return e.err == cudaErrorMemoryAllocation ? SFD_ENOMEM : SFD_ECUDA;
}

// Order a library stream after the work the caller queued on the legacy
// default stream (e.g. the fill of an output or input array).
void after_caller(cudaStream_t s) {
  cudaEvent_t ev;
  SFD_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e1 = cudaEventRecord(ev, 0);
  cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(s, ev, 0) : e1;
  cudaEventDestroy(ev);
  if (e2 != cudaSuccess) throw CudaError{e2, "order after the caller's stream"};
}

// host copy of a device row pointer, checked (starts at 0, non-decreasing,
// rows of at most max_row entries); returns nnz or -1
int64_t checked_rowptr(const int32_t* rowptr, int64_t m, int64_t max_row) {
  std::vector<int> hp(m + 1);
  SFD_CUDA(cudaMemcpy(hp.data(), rowptr, (m + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  if (hp[0] != 0) return -1;
  for (int64_t i = 0; i < m; ++i)
    if (hp[i + 1] < hp[i] || hp[i + 1] - hp[i] > max_row) return -1;
  return hp[m];
}

// copy a device CSR into a slot and build its CSC / work lists; false on bad entries
bool load_slot(Slot& S, int64_t m, int64_t nnz, const int32_t* rowptr, const int32_t* colidx,
               const float* vals) {
  after_caller(S.stream);
  SFD_CUDA(cudaMemcpyAsync(S.csr.ptr, rowptr, (m + 1) * sizeof(int), cudaMemcpyDeviceToDevice,
                           S.stream));
  if (nnz > 0) {
    SFD_CUDA(cudaMemcpyAsync(S.csr.idx, colidx, nnz * sizeof(int), cudaMemcpyDeviceToDevice,
                             S.stream));
    SFD_CUDA(cudaMemcpyAsync(S.csr.val, vals, nnz * sizeof(float), cudaMemcpyDeviceToDevice,
                             S.stream));
  }
  SFD_CUDA(cudaMemsetAsync(S.ws.flags, 0, sizeof(int), S.stream));
  S.build((int)m, nnz);
  int bad = 0;
  SFD_CUDA(cudaMemcpyAsync(&bad, S.ws.flags, sizeof(int), cudaMemcpyDeviceToHost, S.stream));
  SFD_CUDA(cudaStreamSynchronize(S.stream));
  return bad == 0;
}

// Shared body of the two dense products: scratch, stream, timeout flag.
template <typename F>
int run_dense(F&& f) {
  DevArena A;
  cudaStream_t s = nullptr;
  try {
    SFD_CUDA(cudaStreamCreate(&s));
    Workspace ws;
    alloc_dense_scratch(A, ws);
    f(ws, s);
    int flags[4] = {0, 0, 0, 0};
    SFD_CUDA(cudaMemcpyAsync(flags, ws.flags, sizeof(flags), cudaMemcpyDeviceToHost, s));
    SFD_CUDA(cudaStreamSynchronize(s));
    A.release();
    cudaStreamDestroy(s);
    return flags[2] ? SFD_ETIMEOUT : SFD_OK;
  } catch (const CudaError& e) {
    A.release();
    if (s) cudaStreamDestroy(s);
    return code_of(e);
  }
}

}  // namespace

extern "C" {

int sfd_bssh_buffer(int64_t m, int64_t d, int32_t ell, const int32_t* rowptr, const int32_t* colidx,
                    const float* vals, uint64_t seed, int64_t b, const sfd_options* opt,
                    float* Bp_out, sfd_shrink_info* info) {
  if (m < 1 || d < 1 || ell < 1 || ell > m || m > d || ell > kMaxEll || !rowptr || !Bp_out || b < 0)
    return SFD_EINVAL;
  sfd_options o;
  if (opt) o = *opt; else sfd_options_init(&o);
  try {
    const int64_t nnz = checked_rowptr(rowptr, m, d);
    if (nnz < 0 || (nnz > 0 && (!colidx || !vals))) return SFD_EINVAL;
    Slot S(d, ell, m, nnz, nullptr);
    if (!load_slot(S, m, nnz, rowptr, colidx, vals)) return SFD_EINVAL;
    const int q = q_for(o, (int)m);
    int inject = o.inject_vs_fail, r = 0, p = 0;
    Verdict v{};
    bool ok = false;
    for (; r < std::max(1, o.retry_cap); ++r) {
      p = o.verify ? vs_steps(d, delta_br(o.delta, b, r)) : 0;
      S.enqueue_attempt((int)m, q, seed, (uint64_t)b, (uint64_t)r, std::max(p, 1), o.verify);
      SFD_CUDA(cudaEventSynchronize(S.done));
      v = *S.verdict_host;
      ok = v.ok != 0;
      if (o.verify && inject > 0) {
        ok = false;
        --inject;
      }
      if (ok) break;
    }
    transpose(S.Bpt, d, ell, S.ld, Bp_out, d, S.stream);
    SFD_CUDA(cudaStreamSynchronize(S.stream));
    if (info) {
      info->q = q;
      info->attempts = std::min(r + 1, std::max(1, o.retry_cap));
      info->verified = ok ? 1 : 0;
      info->vs_steps = p;
      info->delta_shrink = v.delta;
      info->logsum = v.logsum;
      info->fro2_a = v.fro2a;
      info->fro2_b = v.fro2b;
      info->captured = v.captured;
    }
    return SFD_OK;
  } catch (const CudaError& e) {
    return code_of(e);
  }
}

int sfd_q_features(int64_t m, int64_t d, int32_t ell, const int32_t* rowptr, const int32_t* colidx,
                   const float* vals, uint64_t seed, int64_t b, int32_t q_fixed, float* features) {
  if (m < 1 || d < 1 || ell < 1 || ell > m || m > d || ell > kMaxEll || !rowptr || !features ||
      b < 0 || q_fixed < 1)
    return SFD_EINVAL;
  try {
    const int64_t nnz = checked_rowptr(rowptr, m, d);
    if (nnz < 0 || (nnz > 0 && (!colidx || !vals))) return SFD_EINVAL;
    Slot S(d, ell, m, nnz, nullptr);
    if (!load_slot(S, m, nnz, rowptr, colidx, vals)) return SFD_EINVAL;
    // S0 = (A'G)^T (A'G) for the G of attempt 0 (Alg. 1's start block)
    launch_gauss_fill(S.W, d, ell, S.ld, seed, (uint64_t)b, 0, 1, S.stream);
    spmm(S.csr, S.W, S.ld, S.ld, S.Y, S.ld, S.ws.partial_rows, S.stream);
    gram(S.Y, S.ld, single_map(ell), m, S.ws.small_a, S.ws, S.stream);
    q_features(S.csr, S.csc, d, ell, q_fixed, S.fro2, S.ws.small_a, S.qfeat, S.qacc, S.stream);
    SFD_CUDA(cudaMemcpyAsync(features, S.qfeat, kQF * sizeof(float), cudaMemcpyDeviceToHost,
                             S.stream));
    SFD_CUDA(cudaStreamSynchronize(S.stream));
    return SFD_OK;
  } catch (const CudaError& e) {
    return code_of(e);
  }
}

int sfd_dense_shrink(int64_t rows, int64_t d, int32_t ell, const float* M, float* B_out) {
  if (rows < 1 || d < 1 || ell < 1 || ell > kMaxEll || rows > 2 * (int64_t)ell || !M || !B_out ||
      d > 2000000)
    return SFD_EINVAL;
  try {
    Merger G(d, ell);
    after_caller(G.stream);
    // rows 0..min(rows,l) are the "B" block, the rest the stacked block
    const int k0 = (int)std::min<int64_t>(rows, ell);
    const int k1 = (int)(rows - k0);
    transpose(M, k0, (int)d, (int)d, G.B(), G.ld, G.stream);
    float* X = G.arena.alloc<float>((size_t)d * G.ld);
    SFD_CUDA(cudaMemsetAsync(X, 0, (size_t)d * G.ld * sizeof(float), G.stream));
    if (k1 > 0) transpose(M + (size_t)k0 * d, k1, (int)d, (int)d, X, G.ld, G.stream);
    G.dense_shrink(X, G.ld, k1);
    transpose(G.B(), d, ell, G.ld, B_out, d, G.stream);
    SFD_CUDA(cudaStreamSynchronize(G.stream));
    return SFD_OK;
  } catch (const CudaError& e) {
    return code_of(e);
  }
}

int sfd_csr_spmm(int64_t m, int64_t d, const int32_t* rowptr, const int32_t* colidx,
                 const float* vals, int32_t k, const float* X, int32_t ldx, float* Y, int32_t ldy,
                 int32_t transpose_flag) {
  if (m < 1 || d < 1 || k < 1 || k > kMaxEll || ldx < k || ldy < k || (ldx & 3) || (ldy & 3) ||
      !rowptr || !X || !Y)
    return SFD_EINVAL;
  try {
    const int64_t nnz = checked_rowptr(rowptr, m, INT32_MAX);
    if (nnz < 0 || (nnz > 0 && (!colidx || !vals))) return SFD_EINVAL;
    Slot S(d, 1, m, nnz, nullptr);
    if (!load_slot(S, m, nnz, rowptr, colidx, vals)) return SFD_EINVAL;
    const int64_t slots = 2 * (nnz / kSplit) + 4;
    float* partial = S.arena.alloc<float>((size_t)slots * std::max(ldx, ldy));
    spmm(transpose_flag ? S.csc : S.csr, X, ldx, k, Y, ldy, partial, S.stream);
    SFD_CUDA(cudaStreamSynchronize(S.stream));
    return SFD_OK;
  } catch (const CudaError& e) {
    return code_of(e);
  }
}

int sfd_spmm_variant_count(int32_t x_fp16) { return spmm_variants(x_fp16 != 0); }

int sfd_csr_spmm_ex(int64_t m, int64_t d, const int32_t* rowptr, const int32_t* colidx,
                    const float* vals, int32_t k, const void* X, int32_t x_fp16, int32_t ldx,
                    float* Y, int32_t ldy, int32_t transpose_flag, int32_t variant) {
  if (m < 1 || d < 1 || k < 1 || ldx < k || ldy < k || !rowptr || !X || !Y ||
      variant < 0 || variant >= spmm_variants(x_fp16 != 0))
    return SFD_EINVAL;
  if (x_fp16 ? (k > 128 || (ldx & 7) || (ldy & 7)) : (k > kMaxEll || (ldx & 3) || (ldy & 3)))
    return SFD_EINVAL;
  try {
    const int64_t nnz = checked_rowptr(rowptr, m, INT32_MAX);
    if (nnz < 0 || (nnz > 0 && (!colidx || !vals))) return SFD_EINVAL;
    Slot S(d, 1, m, nnz, nullptr);
    if (!load_slot(S, m, nnz, rowptr, colidx, vals)) return SFD_EINVAL;
    const int64_t slots = 2 * (nnz / kSplit) + 4;
    float* partial = S.arena.alloc<float>((size_t)slots * std::max(ldx, ldy));
    const Csr& c = transpose_flag ? S.csc : S.csr;
    if (x_fp16)
      spmm_h(c, static_cast<const __half*>(X), ldx, k, Y, ldy, partial, S.stream, variant);
    else
      spmm(c, static_cast<const float*>(X), ldx, k, Y, ldy, partial, S.stream, variant);
    SFD_CUDA(cudaStreamSynchronize(S.stream));
    return SFD_OK;
  } catch (const CudaError& e) {
    return code_of(e);
  }
}

int sfd_orthonormalize(int64_t rows, int32_t k, float* X, int32_t ld) {
  if (rows < 1 || k < 1 || k > kMaxEll || ld < k || !X) return SFD_EINVAL;
  DevArena A;
  cudaStream_t s = nullptr;
  try {
    SFD_CUDA(cudaStreamCreate(&s));
    Workspace ws;
    alloc_dense_scratch(A, ws);
    float* tmp = A.alloc<float>((size_t)rows * ld);
    const ColMap map = single_map(k);
    // shifted CholeskyQR3: the first (shifted) pass leaves a block of condition
    // number about sqrt(||X||^2 / shift) <= 2^10 whatever cond(X) was; the
    // next two make it orthonormal to fp32 accuracy
    for (int pass = 0; pass < 3; ++pass) {
      gram(X, ld, map, rows, ws.small_a, ws, s);
      chol_inv(ws.small_a, k, ws.small_b, ws.eig_work, ws.flags, s, true);  // FP64 factor
      gemm_ts(X, ld, map, rows, ws.small_b, k, tmp, ld, s);
      SFD_CUDA(cudaMemcpy2DAsync(X, ld * sizeof(float), tmp, ld * sizeof(float), k * sizeof(float),
                                 rows, cudaMemcpyDeviceToDevice, s));
    }
    SFD_CUDA(cudaStreamSynchronize(s));
    A.release();
    cudaStreamDestroy(s);
    return SFD_OK;
  } catch (const CudaError& e) {
    A.release();
    if (s) cudaStreamDestroy(s);
    return code_of(e);
  }
}

int sfd_set_wait_limit(int64_t spins) {
  try {
    set_wait_limit(spins);
    return SFD_OK;
  } catch (const CudaError& e) {
    return code_of(e);
  }
}

int sfd_wait_selftest(int64_t spins, float* ms_out) {
  try {
    return wait_selftest(spins, ms_out) ? SFD_ETIMEOUT : SFD_OK;
  } catch (const CudaError& e) {
    return code_of(e);
  }
}

int sfd_gram(int64_t rows, int32_t k, const float* X, int32_t ldx, float* G, int32_t precision) {
  if (rows < 0 || k < 1 || k > kMaxEll || ldx < k || !G || (rows > 0 && !X)) return SFD_EINVAL;
  if (precision != 0 && !((precision == 1 || precision == 2) && tc_supported(k, k)))
    return SFD_EINVAL;
  return run_dense([&](Workspace& ws, cudaStream_t s) {
    if (precision) gram_tc(X, ldx, single_map(k), rows, G, ws, s, precision == 2);
    else gram(X, ldx, single_map(k), rows, G, ws, s);
  });
}

int sfd_gemm_ts(int64_t rows, int32_t n, const float* X, int32_t ldx, const float* T, int32_t kout,
                float* Y, int32_t ldy, int32_t precision) {
  if (rows < 0 || n < 1 || n > kMaxEll || kout < 1 || kout > kMaxEll || ldx < n || ldy < kout ||
      !T || (rows > 0 && (!X || !Y)))
    return SFD_EINVAL;
  if (precision != 0 && !(precision == 1 && tc_supported(n, kout)) &&
      !(precision == 2 && tc_split_supported(n, kout)))
    return SFD_EINVAL;
  return run_dense([&](Workspace& ws, cudaStream_t s) {
    if (precision) gemm_ts_tc(X, ldx, single_map(n), rows, T, kout, Y, ldy, ws, s, nullptr,
                              precision == 2);
    else gemm_ts(X, ldx, single_map(n), rows, T, kout, Y, ldy, s);
  });
}

int sfd_symeig(int32_t n, const float* S, int32_t nwant, float* evals, float* evecs) {
  if (n < 1 || n > kMaxEig || nwant < 1 || nwant > n || !S || !evals || !evecs) return SFD_EINVAL;
  DevArena A;
  cudaStream_t s = nullptr;
  try {
    SFD_CUDA(cudaStreamCreate(&s));
    float* work = A.alloc<float>(symeig_work_floats(kMaxEig, kMaxEig));
    symeig(S, n, nwant, evals, evecs, work, s);
    SFD_CUDA(cudaStreamSynchronize(s));
    A.release();
    cudaStreamDestroy(s);
    return SFD_OK;
  } catch (const CudaError& e) {
    A.release();
    if (s) cudaStreamDestroy(s);
    return code_of(e);
  }
}

}  // extern "C"
