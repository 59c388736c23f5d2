// Host orchestration of Sparse Frequent Directions on one GPU and the C ABI
// of include/sfd.h.
//
// Alg. 2 (SFD): rows are appended to a device buffer A' (CSR); when the
// buffer holds l*d entries or d rows it is closed: the CSC copy is built,
// BoostedSparseShrink (Alg. 4) computes B' (SparseShrink of Alg. 3 over
// SimultaneousIteration of Alg. 1, checked by VerifySpectral of Alg. 6), and
// DenseShrink (Alg. 5) folds B' into B.
//
// Device layout of a context (d rows of every dense block, ld = l rounded up
// to a multiple of 8, padding columns kept at zero):
//   Mt[2]   d x 2ld : ping-pong stacks [B^T | B'^T]; DenseShrink reads Mt[cur]
//           and writes the new B^T into the left half of Mt[1-cur]
//   W, W2   d x ld  : A'^T Y products and their orthonormalised copies
//   Y, Y2   d x ld  : A' W products (m <= d rows used)
//   csr/csc buffer  : at most l*d + d entries
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "sfd_internal.cuh"

namespace sfd {

unsigned long long g_kernel_launches = 0;

namespace {

template <typename T>
T* dalloc(size_t n) {
  void* p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(&p, n * sizeof(T));
  if (e != cudaSuccess) throw CudaError{e, "cudaMalloc"};
  return static_cast<T*>(p);
}

int bits_for(int64_t d) {
  int b = 1;
  while ((int64_t(1) << b) < d) ++b;
  return b;
}

}  // namespace

struct Engine {
  int dev = 0;
  int64_t d = 0;
  int ell = 0, ld = 0;
  int64_t cap_rows = 0, cap_nnz = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<void*> allocs;

  Csr csr, csc;
  int* row_ids = nullptr;        // cap_nnz
  int* key_alt = nullptr;        // radix keys (a copy of the CSR column indices)
  int* key_alt2 = nullptr;       // radix ping-pong partners
  int* a_alt = nullptr;
  float* b_alt = nullptr;
  int* col_count = nullptr;      // d
  float* Mt[2] = {nullptr, nullptr};
  int cur = 0;
  float *W = nullptr, *W2 = nullptr, *Y = nullptr, *Y2 = nullptr;
  Workspace ws;
  double* fro2_dev = nullptr;    // [0] total, [1..] partials

  // optional per-launch timing of the sparse products
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, double>> ev_pending;  // (event pair index, algorithmic bytes)
  int ev_used = 0;
  int64_t prof_launches = 0;
  double prof_ms = 0, prof_bytes = 0;

  // A' X (csr) or A'^T Y (csc), timed when profiling
  void spmm_timed(const Csr& c, const float* X, float* Yo, int64_t rows_in) {
    if (!profile) {
      spmm(c, X, ld, ld, Yo, ld, ws.partial_rows, stream);
      return;
    }
    if (ev_used + 2 > (int)ev_pool.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        SFD_CUDA(cudaEventCreate(&e));
        ev_pool.push_back(e);
      }
    }
    const int i0 = ev_used;
    ev_used += 2;
    SFD_CUDA(cudaEventRecord(ev_pool[i0], stream));
    spmm(c, X, ld, ld, Yo, ld, ws.partial_rows, stream);
    SFD_CUDA(cudaEventRecord(ev_pool[i0 + 1], stream));
    double bytes = 8.0 * (double)c.nnz + 4.0 * (c.nseg + 1) + 4.0 * ell * (double)rows_in +
                   4.0 * ell * (double)c.nseg;
    ev_pending.push_back({i0, bytes});
  }
  void collect_profile() {
    if (!profile || ev_pending.empty()) return;
    SFD_CUDA(cudaStreamSynchronize(stream));
    for (auto& pb : ev_pending) {
      float ms = 0;
      SFD_CUDA(cudaEventElapsedTime(&ms, ev_pool[pb.first], ev_pool[pb.first + 1]));
      prof_ms += ms;
      prof_bytes += pb.second;
      prof_launches += 1;
    }
    ev_pending.clear();
    ev_used = 0;
  }

  template <typename T>
  T* alloc(size_t n) {
    T* p = dalloc<T>(n);
    allocs.push_back(p);
    return p;
  }

  void alloc_work(SegWork& w, int nseg, int64_t nnz) {
    w.cap_items = (int)(nseg + nnz / kSplit + 2);
    w.items = alloc<int2>(w.cap_items);
    w.item_slot = alloc<int>(w.cap_items);
    w.split_seg = alloc<int>(std::max<int64_t>(nseg, 1) + 1);
    w.split_first = alloc<int>(std::max<int64_t>(nseg, 1) + 1);
    w.split_count = alloc<int>(std::max<int64_t>(nseg, 1) + 1);
    w.counters = alloc<int>(8 + 4 * ((size_t)nseg + 1) + nseg / 4096 + 16);
  }

  Engine(int64_t d_, int ell_, int64_t cap_rows_, int64_t cap_nnz_, cudaStream_t s) {
    SFD_CUDA(cudaGetDevice(&dev));
    d = d_;
    ell = ell_;
    ld = ld_of(ell);
    cap_rows = cap_rows_;
    cap_nnz = std::max<int64_t>(cap_nnz_, 1);
    if (s) {
      stream = s;
    } else {
      SFD_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
      own_stream = true;
    }
    try {
      csr.ptr = alloc<int>(cap_rows + 1);
      csr.idx = alloc<int>(cap_nnz);
      csr.val = alloc<float>(cap_nnz);
      csc.ptr = alloc<int>(d + 1);
      csc.idx = alloc<int>(cap_nnz);
      csc.val = alloc<float>(cap_nnz);
      row_ids = csc.idx;  // row ids are sorted in place into the CSC arrays
      key_alt = alloc<int>(cap_nnz);
      key_alt2 = alloc<int>(cap_nnz);
      a_alt = alloc<int>(cap_nnz);
      b_alt = alloc<float>(cap_nnz);
      col_count = alloc<int>(d + 1);
      alloc_work(csr.work, (int)cap_rows, cap_nnz);
      alloc_work(csc.work, (int)d, cap_nnz);
      size_t dense = (size_t)d * ld;
      for (int i = 0; i < 2; ++i) {
        Mt[i] = alloc<float>(2 * dense);
        SFD_CUDA(cudaMemsetAsync(Mt[i], 0, 2 * dense * sizeof(float), stream));
      }
      W = alloc<float>(dense);
      W2 = alloc<float>(dense);
      Y = alloc<float>(dense);
      Y2 = alloc<float>(dense);
      for (float* p : {W, W2, Y, Y2}) SFD_CUDA(cudaMemsetAsync(p, 0, dense * sizeof(float), stream));
      ws.gram_partial = alloc<float>((size_t)320 * 128 * 128);
      ws.small_a = alloc<float>((size_t)kMaxEig * kMaxEig);
      ws.small_b = alloc<float>((size_t)kMaxEig * kMaxEig);
      ws.evals = alloc<float>(kMaxEig);
      ws.eig_work = alloc<float>(symeig_work_floats(kMaxEig, kMaxEig));
      ws.scalars = alloc<double>(64);
      ws.flags = alloc<int>(16);
      SFD_CUDA(cudaMemsetAsync(ws.flags, 0, 16 * sizeof(int), stream));
      int64_t ntiles = (cap_nnz + 4095) / 4096 + 1;
      ws.hist_cap = (int)(512 * ntiles + 8);
      ws.hist = alloc<int>(ws.hist_cap);
      // block sums of every scan: radix histograms, colptr (d + 1), work lists
      ws.scan_tmp = alloc<int>(std::max<int64_t>(ws.hist_cap, d + cap_rows + 2) / 4096 + 64);
      int64_t slots = 2 * (cap_nnz / kSplit) + 4;
      ws.partial_rows_cap = (int)slots;
      ws.partial_rows = alloc<float>((size_t)slots * ld);
      ws.vec0 = alloc<float>(d);
      ws.vec1 = alloc<float>(std::max<int64_t>(d, cap_rows));
      ws.vec2 = alloc<float>(d);
      ws.wpart = alloc<float>(512 * kMaxEll + kMaxEll + 512);
      fro2_dev = alloc<double>(1024 + 8);
      SFD_CUDA(cudaStreamSynchronize(stream));
    } catch (...) {
      release();
      throw;
    }
  }

  void release() {
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    ev_pool.clear();
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    if (own_stream && stream) cudaStreamDestroy(stream);
    stream = nullptr;
  }
  ~Engine() { release(); }

  float* Bt() { return Mt[cur]; }            // d x ld view, leading dimension 2 ld
  float* Bpt() { return Mt[cur] + ld; }      // right half

  // ---------------------------------------------------------- orthonormalise
  // X (rows x l, ld) -> X R^-1 written to Xout, one CholeskyQR pass with shift.
  void orth_pass(const float* X, int64_t rows, float* Xout) {
    ColMap map{ell, 0, 0};
    gram(X, ld, map, rows, ws.small_a, ws, stream);
    chol_inv(ws.small_a, ell, ws.small_b, ws.eig_work, ws.flags, stream);
    gemm_ts(X, ld, map, rows, ws.small_b, ell, Xout, ld, stream);
  }

  // ---------------------------------------------------- CSC of the buffer
  double build_structures(int m, int64_t nnz) {
    csr.nseg = m;
    csr.nnz = nnz;
    launch_check_entries(csr.idx, csr.val, nnz, (int)d, nullptr, fro2_dev, ws.flags, stream);
    build_work(csr, stream);  // syncs the stream (reads work-list sizes)
    // CSC by a stable radix sort of (col, row, val) by col
    int* key = key_alt;
    int* rows = csc.idx;
    float* vals = csc.val;
    SFD_CUDA(cudaMemcpyAsync(key, csr.idx, nnz * sizeof(int), cudaMemcpyDeviceToDevice, stream));
    SFD_CUDA(cudaMemcpyAsync(vals, csr.val, nnz * sizeof(float), cudaMemcpyDeviceToDevice, stream));
    launch_row_ids(csr.ptr, m, rows, stream);
    // ping-pong partners: the CSR arrays stay intact, so use dedicated alternates
    radix_sort_by_key(key, rows, vals, key_alt2, a_alt, b_alt, nnz, bits_for(d), ws.hist,
                      ws.scan_tmp, stream);
    colptr_from_sorted(key, nnz, (int)d, csc.ptr, stream);  // keys now sorted by column
    csc.nseg = (int)d;
    csc.nnz = nnz;
    build_work(csc, stream);
    double h = 0;
    SFD_CUDA(cudaMemcpyAsync(&h, fro2_dev, sizeof(double), cudaMemcpyDeviceToHost, stream));
    SFD_CUDA(cudaStreamSynchronize(stream));
    return h;
  }

  // -------------------------------------------------------- SparseShrink
  // Alg. 3 for attempt r of buffer b: leaves B'^T in Bpt() (ld 2 ld) and
  // returns ||B'||_F^2.
  double sparse_shrink(int m, int q, uint64_t seed, uint64_t b, uint64_t r) {
    // G ~ N(0,1)^{d x l} (Alg. 1)
    launch_gauss_fill(W, d, ell, ld, seed, b, r, 1, stream);
    spmm_timed(csr, W, Y, d);                                       // Y = A' G
    orth_pass(Y, m, Y2);
    std::swap(Y, Y2);
    for (int t = 0; t < q; ++t) {
      spmm_timed(csc, Y, W, m);                                     // W = A'^T Y
      orth_pass(W, d, W2);
      std::swap(W, W2);
      spmm_timed(csr, W, Y, d);                                     // Y = A' W
      orth_pass(Y, m, Y2);
      std::swap(Y, Y2);
    }
    orth_pass(Y, m, Y2);                                            // second CholeskyQR pass: Z
    std::swap(Y, Y2);
    spmm_timed(csc, Y, W, m);                                       // W = A'^T Z = P^T
    ColMap map{ell, 0, 0};
    gram(W, ld, map, d, ws.small_a, ws, stream);                    // P P^T
    symeig(ws.small_a, ell, ell, ws.evals, ws.small_b, ws.eig_work, stream);
    shrink_weights(ws.evals, ws.small_b, ell, ell, ell, 0, ws.small_a, ws.scalars, stream);
    gemm_ts(W, ld, map, d, ws.small_a, ell, Bpt(), 2 * ld, stream); // B'^T = P^T H diag(s)
    double fro2b = 0;
    SFD_CUDA(cudaMemcpyAsync(&fro2b, ws.scalars, sizeof(double), cudaMemcpyDeviceToHost, stream));
    SFD_CUDA(cudaStreamSynchronize(stream));
    collect_profile();
    return fro2b;
  }

  // ------------------------------------------------------- DenseShrink
  // Alg. 5 on the stack [B; B'] held in Mt[cur] (columns 0..l and ld..ld+k1).
  void dense_shrink(int k1) {
    ColMap map{ell, k1, ld};
    const int n = ell + k1;
    gram(Mt[cur], 2 * ld, map, d, ws.small_a, ws, stream);
    symeig(ws.small_a, n, ell, ws.evals, ws.small_b, ws.eig_work, stream);
    shrink_weights(ws.evals, ws.small_b, n, ell, ell, 0, ws.small_a, ws.scalars, stream);
    gemm_ts(Mt[cur], 2 * ld, map, d, ws.small_a, ell, Mt[1 - cur], 2 * ld, stream);
    cur = 1 - cur;
  }
};

// ============================================================== the context
struct Ctx {
  Engine* eng = nullptr;
  sfd_options opt;
  uint64_t seed = 0;
  int64_t b = 0;               // buffer counter
  int inject_left = 0;
  int pend_rows = 0;
  int64_t pend_nnz = 0;
  std::vector<int> h_ptr;      // host copy of the open buffer's local rowptr
  sfd_stats st{};
  std::string last_error;
  // staging for host input
  int* stage_idx = nullptr;
  float* stage_val = nullptr;
  int64_t stage_cap = 0;
};

}  // namespace sfd

struct sfd_ctx {
  sfd::Ctx c;
};

namespace sfd {

namespace {

int q_for(const sfd_options& o, int m) {
  if (o.q_override >= 0) return o.q_override;
  double q = ceil(o.c_q * log((double)m / 0.25) / 0.25);
  return (int)std::max(0.0, q);
}

double delta_br(double delta, int64_t b, int r) {
  return delta * (6.0 / (M_PI * M_PI)) / ((double)(b + 1) * (double)(b + 1)) / ldexp(1.0, r + 1);
}

int vs_steps(int64_t d, double di) {
  return std::max(1, (int)ceil(log2(sqrt(2.0 * (double)d / M_PI) / di)));
}

// Close the open buffer: BSSh + DSh (m >= l) or DSh([B; A']) (m < l).
int close_buffer(Ctx& C) {
  Engine& E = *C.eng;
  const int m = C.pend_rows;
  const int64_t nnz = C.pend_nnz;
  if (m == 0) return SFD_OK;
  SFD_CUDA(cudaMemcpyAsync(E.csr.ptr, C.h_ptr.data(), (m + 1) * sizeof(int), cudaMemcpyHostToDevice,
                           E.stream));
  int status = SFD_OK;
  if (m >= E.ell) {
    const double fro2a = E.build_structures(m, nnz);
    const int q = q_for(C.opt, m);
    bool ok = false;
    int r = 0;
    double Delta = 0, logsum = 0;
    for (; r < std::max(1, C.opt.retry_cap); ++r) {
      const double fro2b = E.sparse_shrink(m, q, C.seed, (uint64_t)C.b, (uint64_t)r);
      C.st.attempts++;
      C.st.q_total += q;
      Delta = (fro2a - fro2b) / ((double)kAlpha * E.ell);
      if (!C.opt.verify) { ok = true; break; }
      const double di = delta_br(C.opt.delta, C.b, r);
      const int p = vs_steps(E.d, di);
      if (Delta / 2.0 <= 64.0 * ldexp(1.0, -24) * fro2a) {
        ok = true;
        logsum = -INFINITY;
      } else {
        VsArgs a{&E.csr, &E.csc, E.Bpt(), 2 * E.ld, E.ell, E.d, m, 2.0 / Delta, p,
                 C.seed, (uint64_t)C.b, (uint64_t)r};
        logsum = verify_spectral(a, E.ws, E.stream);
        ok = logsum <= 0.0;
      }
      if (C.inject_left > 0) {
        ok = false;
        C.inject_left--;
      }
      C.st.last_logsum = logsum;
      if (ok) break;
      C.st.vs_rejects++;
    }
    if (!ok) {
      C.st.unverified++;
      if (C.opt.strict) status = SFD_EVERIFY;
    }
    C.st.last_delta = Delta;
    C.st.last_fro2 = fro2a;
    E.dense_shrink(E.ell);
  } else {
    // too few rows for SparseShrink: DenseShrink of [B; A'] with A' dense
    float* right = E.Bpt();
    SFD_CUDA(cudaMemset2DAsync(right, 2 * E.ld * sizeof(float), 0, E.ld * sizeof(float), E.d,
                               E.stream));
    csr_to_dense_t(E.csr.ptr, E.csr.idx, E.csr.val, m, E.d, right, 2 * E.ld, E.stream);
    E.dense_shrink(m);
  }
  SFD_CUDA(cudaStreamSynchronize(E.stream));
  C.st.buffers++;
  C.b++;
  C.pend_rows = 0;
  C.pend_nnz = 0;
  C.h_ptr.assign(1, 0);
  return status;
}

int fail(Ctx* C, int code, const std::string& msg) {
  if (C) C->last_error = msg;
  return code;
}

int from_cuda(Ctx* C, const CudaError& e) {
  std::string m = std::string(e.where) + ": " + cudaGetErrorString(e.err);
  if (e.err == cudaErrorMemoryAllocation) return fail(C, SFD_ENOMEM, m);
  return fail(C, SFD_ECUDA, m);
}

}  // namespace

}  // namespace sfd

using namespace sfd;

extern "C" {

void sfd_options_init(sfd_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->abi_version = SFD_ABI_VERSION;
  o->delta = 0.01;
  o->verify = 1;
  o->c_q = 0.25;
  o->q_override = -1;
  o->retry_cap = 8;
  o->precision = 0;
  o->q_mode = 0;
  o->strict = 0;
  o->inject_vs_fail = 0;
  o->cuda_stream = nullptr;
  o->profile = 0;
}

const char* sfd_strerror(int s) {
  switch (s) {
    case SFD_OK: return "ok";
    case SFD_EINVAL: return "invalid argument";
    case SFD_ENOMEM: return "out of memory";
    case SFD_ECUDA: return "CUDA error";
    case SFD_EVERIFY: return "buffer left unverified after retry_cap attempts";
    case SFD_ETIMEOUT: return "bounded device wait expired";
    default: return "unknown status";
  }
}

const char* sfd_last_error(const sfd_ctx* ctx) { return ctx ? ctx->c.last_error.c_str() : ""; }

int sfd_create(int64_t d, int32_t ell, uint64_t seed, const sfd_options* opt, sfd_ctx** out) {
  if (!out) return SFD_EINVAL;
  *out = nullptr;
  if (d < 1 || ell < 1 || ell > d || ell > kMaxEll || d > (int64_t)1 << 30) return SFD_EINVAL;
  if (opt && opt->abi_version != SFD_ABI_VERSION) return SFD_EINVAL;
  sfd_ctx* ctx = new (std::nothrow) sfd_ctx();
  if (!ctx) return SFD_ENOMEM;
  Ctx& C = ctx->c;
  if (opt) C.opt = *opt; else sfd_options_init(&C.opt);
  if (C.opt.delta <= 0 || C.opt.delta >= 1 || C.opt.c_q < 0) { delete ctx; return SFD_EINVAL; }
  C.seed = seed;
  C.inject_left = C.opt.inject_vs_fail;
  C.h_ptr.assign(1, 0);
  try {
    int64_t cap_nnz = (int64_t)ell * d + d;
    if (cap_nnz > INT32_MAX - 1) { delete ctx; return SFD_EINVAL; }
    C.eng = new Engine(d, ell, d, cap_nnz, (cudaStream_t)C.opt.cuda_stream);
    C.eng->profile = C.opt.profile != 0;
  } catch (const CudaError& e) {
    int rc = e.err == cudaErrorMemoryAllocation ? SFD_ENOMEM : SFD_ECUDA;
    delete ctx;
    return rc;
  } catch (const std::bad_alloc&) {
    delete ctx;
    return SFD_ENOMEM;
  }
  *out = ctx;
  return SFD_OK;
}

void sfd_destroy(sfd_ctx* ctx) {
  if (!ctx) return;
  Ctx& C = ctx->c;
  if (C.stage_idx) cudaFree(C.stage_idx);
  if (C.stage_val) cudaFree(C.stage_val);
  delete C.eng;
  delete ctx;
}

struct LaunchCount {
  sfd_stats& st;
  unsigned long long start;
  explicit LaunchCount(sfd_stats& s) : st(s), start(__atomic_load_n(&g_kernel_launches, __ATOMIC_RELAXED)) {}
  ~LaunchCount() { st.kernel_launches += (int64_t)(__atomic_load_n(&g_kernel_launches, __ATOMIC_RELAXED) - start); }
};

int sfd_append_rows(sfd_ctx* ctx, int64_t nrows, const int64_t* indptr, const int32_t* indices,
                    const float* values, int where) {
  if (!ctx) return SFD_EINVAL;
  Ctx& C = ctx->c;
  LaunchCount lc(C.st);
  if (nrows < 0 || (where != SFD_HOST && where != SFD_DEVICE)) return fail(&C, SFD_EINVAL, "bad nrows/where");
  if (nrows == 0) return SFD_OK;
  if (!indptr) return fail(&C, SFD_EINVAL, "null indptr");
  Engine& E = *C.eng;
  try {
    SFD_CUDA(cudaSetDevice(E.dev));
    // 1. indptr on the host, checked
    std::vector<int64_t> ip(nrows + 1);
    if (where == SFD_DEVICE)
      SFD_CUDA(cudaMemcpy(ip.data(), indptr, (nrows + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    else
      memcpy(ip.data(), indptr, (nrows + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < nrows; ++i) {
      int64_t c = ip[i + 1] - ip[i];
      if (c < 0 || c > E.d) return fail(&C, SFD_EINVAL, "indptr not non-decreasing or row longer than d");
    }
    const int64_t base = ip[0], total = ip[nrows] - ip[0];
    if (base < 0) return fail(&C, SFD_EINVAL, "negative indptr");
    if (total > 0 && (!indices || !values)) return fail(&C, SFD_EINVAL, "null indices/values");
    // 2. the entries on the device (staged for host input), checked
    const int* didx;
    const float* dval;
    if (where == SFD_HOST) {
      if (total > C.stage_cap) {
        if (C.stage_idx) cudaFree(C.stage_idx);
        if (C.stage_val) cudaFree(C.stage_val);
        C.stage_idx = nullptr;
        C.stage_val = nullptr;
        C.stage_cap = 0;
        C.stage_idx = dalloc<int>(total);
        C.stage_val = dalloc<float>(total);
        C.stage_cap = total;
      }
      if (total > 0) {
        SFD_CUDA(cudaMemcpyAsync(C.stage_idx, indices + base, total * sizeof(int),
                                 cudaMemcpyHostToDevice, E.stream));
        SFD_CUDA(cudaMemcpyAsync(C.stage_val, values + base, total * sizeof(float),
                                 cudaMemcpyHostToDevice, E.stream));
      }
      didx = C.stage_idx;
      dval = C.stage_val;
    } else {
      didx = indices + base;
      dval = values + base;
    }
    if (total > 0) {
      SFD_CUDA(cudaMemsetAsync(E.ws.flags, 0, sizeof(int), E.stream));
      launch_check_entries(didx, dval, total, (int)E.d, nullptr, E.fro2_dev, E.ws.flags, E.stream);
      int bad = 0;
      SFD_CUDA(cudaMemcpyAsync(&bad, E.ws.flags, sizeof(int), cudaMemcpyDeviceToHost, E.stream));
      SFD_CUDA(cudaStreamSynchronize(E.stream));
      if (bad) return fail(&C, SFD_EINVAL, "column index outside [0, d) or non-finite value");
    }
    // 3. Alg. 2: one row at a time, close the buffer when nnz >= l d or rows = d
    const int64_t thresh = (int64_t)E.ell * E.d;
    int status = SFD_OK;
    int64_t seg_start = 0;  // first row of the current copy segment
    auto copy_rows = [&](int64_t r0, int64_t r1) {
      // rows [r0, r1) of this call into the open buffer
      int64_t e0 = ip[r0] - base, e1 = ip[r1] - base;
      if (e1 > e0) {
        SFD_CUDA(cudaMemcpyAsync(E.csr.idx + C.pend_nnz, didx + e0, (e1 - e0) * sizeof(int),
                                 cudaMemcpyDeviceToDevice, E.stream));
        SFD_CUDA(cudaMemcpyAsync(E.csr.val + C.pend_nnz, dval + e0, (e1 - e0) * sizeof(float),
                                 cudaMemcpyDeviceToDevice, E.stream));
      }
      for (int64_t r = r0; r < r1; ++r) {
        C.pend_nnz += ip[r + 1] - ip[r];
        C.pend_rows += 1;
        C.h_ptr.push_back((int)C.pend_nnz);
      }
    };
    int64_t rows_in_buf = C.pend_rows, nnz_in_buf = C.pend_nnz;
    for (int64_t i = 0; i < nrows; ++i) {
      rows_in_buf += 1;
      nnz_in_buf += ip[i + 1] - ip[i];
      if (nnz_in_buf >= thresh || rows_in_buf == E.d) {
        copy_rows(seg_start, i + 1);
        seg_start = i + 1;
        int rc = close_buffer(C);
        if (rc != SFD_OK) status = rc;
        rows_in_buf = 0;
        nnz_in_buf = 0;
      }
    }
    if (seg_start < nrows) copy_rows(seg_start, nrows);
    SFD_CUDA(cudaStreamSynchronize(E.stream));
    C.st.rows_seen += nrows;
    C.st.nnz_seen += total;
    C.st.pending_rows = C.pend_rows;
    C.st.pending_nnz = C.pend_nnz;
    return status;
  } catch (const CudaError& e) {
    return from_cuda(&C, e);
  } catch (const std::bad_alloc&) {
    return fail(&C, SFD_ENOMEM, "host allocation");
  }
}

static int flush(Ctx& C) {
  int rc = close_buffer(C);
  C.st.pending_rows = 0;
  C.st.pending_nnz = 0;
  return rc;
}

int sfd_sketch(sfd_ctx* ctx, float* B_out, int where) {
  if (!ctx || !B_out || (where != SFD_HOST && where != SFD_DEVICE)) return SFD_EINVAL;
  Ctx& C = ctx->c;
  LaunchCount lc(C.st);
  Engine& E = *C.eng;
  try {
    SFD_CUDA(cudaSetDevice(E.dev));
    int rc = flush(C);
    if (where == SFD_DEVICE) {
      transpose(E.Bt(), E.d, E.ell, 2 * E.ld, B_out, E.d, E.stream);
    } else {
      float* tmp = E.W2;  // d x ld scratch holds l x d
      transpose(E.Bt(), E.d, E.ell, 2 * E.ld, tmp, E.d, E.stream);
      SFD_CUDA(cudaMemcpyAsync(B_out, tmp, (size_t)E.ell * E.d * sizeof(float),
                               cudaMemcpyDeviceToHost, E.stream));
    }
    SFD_CUDA(cudaStreamSynchronize(E.stream));
    return rc;
  } catch (const CudaError& e) {
    return from_cuda(&C, e);
  }
}

int sfd_merge(sfd_ctx* dst, sfd_ctx* src) {
  if (!dst || !src || dst == src) return SFD_EINVAL;
  Ctx& D = dst->c;
  Ctx& S = src->c;
  LaunchCount lc(D.st);
  Engine& ED = *D.eng;
  Engine& ES = *S.eng;
  if (ED.d != ES.d || ED.ell != ES.ell || ED.dev != ES.dev) return fail(&D, SFD_EINVAL, "shape/device mismatch");
  try {
    SFD_CUDA(cudaSetDevice(ED.dev));
    int rc1 = flush(S);
    int rc2 = flush(D);
    SFD_CUDA(cudaStreamSynchronize(ES.stream));
    SFD_CUDA(cudaMemcpy2DAsync(ED.Bpt(), 2 * ED.ld * sizeof(float), ES.Bt(), 2 * ES.ld * sizeof(float),
                               ED.ld * sizeof(float), ED.d, cudaMemcpyDeviceToDevice, ED.stream));
    ED.dense_shrink(ED.ell);
    SFD_CUDA(cudaStreamSynchronize(ED.stream));
    return rc1 != SFD_OK ? rc1 : rc2;
  } catch (const CudaError& e) {
    return from_cuda(&D, e);
  }
}

int sfd_get_stats(const sfd_ctx* ctx, sfd_stats* out) {
  if (!ctx || !out) return SFD_EINVAL;
  *out = ctx->c.st;
  const Engine& E = *ctx->c.eng;
  out->spmm_launches = E.prof_launches;
  out->spmm_ms = E.prof_ms;
  out->spmm_bytes = E.prof_bytes;
  return SFD_OK;
}

int sfd_reset(sfd_ctx* ctx) {
  if (!ctx) return SFD_EINVAL;
  Ctx& C = ctx->c;
  Engine& E = *C.eng;
  try {
    SFD_CUDA(cudaSetDevice(E.dev));
    size_t dense = (size_t)E.d * E.ld;
    for (int i = 0; i < 2; ++i)
      SFD_CUDA(cudaMemsetAsync(E.Mt[i], 0, 2 * dense * sizeof(float), E.stream));
    SFD_CUDA(cudaStreamSynchronize(E.stream));
    E.cur = 0;
    E.prof_launches = 0;
    E.prof_ms = E.prof_bytes = 0;
    C.b = 0;
    C.pend_rows = 0;
    C.pend_nnz = 0;
    C.h_ptr.assign(1, 0);
    C.inject_left = C.opt.inject_vs_fail;
    C.st = sfd_stats{};
    return SFD_OK;
  } catch (const CudaError& e) {
    return from_cuda(&C, e);
  }
}

// ------------------------------------------------------- one-shot entries
int sfd_bssh_buffer(int64_t m, int64_t d, int32_t ell, const int32_t* rowptr, const int32_t* colidx,
                    const float* vals, uint64_t seed, int64_t b, const sfd_options* opt,
                    float* Bp_out, sfd_shrink_info* info) {
  if (m < 1 || d < 1 || ell < 1 || ell > m || ell > d || ell > kMaxEll || !rowptr || !Bp_out || b < 0)
    return SFD_EINVAL;
  if (m > d) return SFD_EINVAL;
  sfd_options o;
  if (opt) o = *opt; else sfd_options_init(&o);
  try {
    std::vector<int> hp(m + 1);
    SFD_CUDA(cudaMemcpy(hp.data(), rowptr, (m + 1) * sizeof(int), cudaMemcpyDeviceToHost));
    if (hp[0] != 0) return SFD_EINVAL;
    for (int64_t i = 0; i < m; ++i)
      if (hp[i + 1] < hp[i] || hp[i + 1] - hp[i] > d) return SFD_EINVAL;
    const int64_t nnz = hp[m];
    if (nnz > 0 && (!colidx || !vals)) return SFD_EINVAL;
    Engine E(d, ell, m, nnz, nullptr);
    SFD_CUDA(cudaMemcpyAsync(E.csr.ptr, rowptr, (m + 1) * sizeof(int), cudaMemcpyDeviceToDevice, E.stream));
    if (nnz > 0) {
      SFD_CUDA(cudaMemcpyAsync(E.csr.idx, colidx, nnz * sizeof(int), cudaMemcpyDeviceToDevice, E.stream));
      SFD_CUDA(cudaMemcpyAsync(E.csr.val, vals, nnz * sizeof(float), cudaMemcpyDeviceToDevice, E.stream));
    }
    SFD_CUDA(cudaMemsetAsync(E.ws.flags, 0, sizeof(int), E.stream));
    const double fro2a = E.build_structures((int)m, nnz);
    int bad = 0;
    SFD_CUDA(cudaMemcpy(&bad, E.ws.flags, sizeof(int), cudaMemcpyDeviceToHost));
    if (bad) return SFD_EINVAL;
    const int q = q_for(o, (int)m);
    int inject = o.inject_vs_fail;
    bool ok = false;
    int r = 0, p = 0;
    double Delta = 0, logsum = 0, fro2b = 0;
    for (; r < std::max(1, o.retry_cap); ++r) {
      fro2b = E.sparse_shrink((int)m, q, seed, (uint64_t)b, (uint64_t)r);
      Delta = (fro2a - fro2b) / ((double)kAlpha * ell);
      if (!o.verify) { ok = true; break; }
      p = vs_steps(d, delta_br(o.delta, b, r));
      if (Delta / 2.0 <= 64.0 * ldexp(1.0, -24) * fro2a) {
        ok = true;
        logsum = -INFINITY;
      } else {
        VsArgs a{&E.csr, &E.csc, E.Bpt(), 2 * E.ld, ell, d, m, 2.0 / Delta, p, seed, (uint64_t)b,
                 (uint64_t)r};
        logsum = verify_spectral(a, E.ws, E.stream);
        ok = logsum <= 0.0;
      }
      if (inject > 0) { ok = false; --inject; }
      if (ok) break;
    }
    transpose(E.Bpt(), d, ell, 2 * E.ld, Bp_out, d, E.stream);
    SFD_CUDA(cudaStreamSynchronize(E.stream));
    if (info) {
      info->q = q;
      info->attempts = std::min(r + 1, std::max(1, o.retry_cap));
      info->verified = ok ? 1 : 0;
      info->vs_steps = p;
      info->delta_shrink = Delta;
      info->logsum = logsum;
      info->fro2_a = fro2a;
      info->fro2_b = fro2b;
    }
    return SFD_OK;
  } catch (const CudaError& e) {
    return e.err == cudaErrorMemoryAllocation ? SFD_ENOMEM : SFD_ECUDA;
  }
}

int sfd_dense_shrink(int64_t rows, int64_t d, int32_t ell, const float* M, float* B_out) {
  if (rows < 1 || d < 1 || ell < 1 || ell > kMaxEll || rows > 2 * (int64_t)ell || !M || !B_out)
    return SFD_EINVAL;
  try {
    Engine E(d, ell, 1, 1, nullptr);
    // stack rows 0..min(rows,l) into B^T, the rest into B'^T
    int k0 = (int)std::min<int64_t>(rows, ell);
    int k1 = (int)(rows - k0);
    transpose(M, k0, (int)d, (int)d, E.Mt[E.cur], 2 * E.ld, E.stream);
    if (k1 > 0) transpose(M + (size_t)k0 * d, k1, (int)d, (int)d, E.Mt[E.cur] + E.ld, 2 * E.ld, E.stream);
    // rows of M are columns of Mt: ColMap {k0, k1, ld}
    ColMap map{k0, k1, E.ld};
    const int n = k0 + k1;
    gram(E.Mt[E.cur], 2 * E.ld, map, d, E.ws.small_a, E.ws, E.stream);
    int nwant = std::min(ell, n);
    symeig(E.ws.small_a, n, nwant, E.ws.evals, E.ws.small_b, E.ws.eig_work, E.stream);
    // fewer rows than l: lambda_l = 0, nothing is shrunk
    shrink_weights(E.ws.evals, E.ws.small_b, n, nwant, nwant, nwant < ell ? 1 : 0, E.ws.small_a,
                   E.ws.scalars, E.stream);
    SFD_CUDA(cudaMemsetAsync(E.W, 0, (size_t)d * E.ld * sizeof(float), E.stream));
    gemm_ts(E.Mt[E.cur], 2 * E.ld, map, d, E.ws.small_a, nwant, E.W, E.ld, E.stream);
    transpose(E.W, d, ell, E.ld, B_out, d, E.stream);
    SFD_CUDA(cudaStreamSynchronize(E.stream));
    return SFD_OK;
  } catch (const CudaError& e) {
    return e.err == cudaErrorMemoryAllocation ? SFD_ENOMEM : SFD_ECUDA;
  }
}

int sfd_csr_spmm(int64_t m, int64_t d, const int32_t* rowptr, const int32_t* colidx,
                 const float* vals, int32_t k, const float* X, int32_t ldx, float* Y, int32_t ldy,
                 int32_t transpose_flag) {
  if (m < 1 || d < 1 || k < 1 || k > kMaxEll || ldx < k || ldy < k || (ldx & 3) || (ldy & 3) ||
      !rowptr || !X || !Y)
    return SFD_EINVAL;
  try {
    std::vector<int> hp(m + 1);
    SFD_CUDA(cudaMemcpy(hp.data(), rowptr, (m + 1) * sizeof(int), cudaMemcpyDeviceToHost));
    if (hp[0] != 0) return SFD_EINVAL;
    for (int64_t i = 0; i < m; ++i)
      if (hp[i + 1] < hp[i]) return SFD_EINVAL;
    const int64_t nnz = hp[m];
    if (nnz > 0 && (!colidx || !vals)) return SFD_EINVAL;
    Engine E(d, 1, m, nnz, nullptr);
    SFD_CUDA(cudaMemcpyAsync(E.csr.ptr, rowptr, (m + 1) * sizeof(int), cudaMemcpyDeviceToDevice, E.stream));
    if (nnz > 0) {
      SFD_CUDA(cudaMemcpyAsync(E.csr.idx, colidx, nnz * sizeof(int), cudaMemcpyDeviceToDevice, E.stream));
      SFD_CUDA(cudaMemcpyAsync(E.csr.val, vals, nnz * sizeof(float), cudaMemcpyDeviceToDevice, E.stream));
    }
    SFD_CUDA(cudaMemsetAsync(E.ws.flags, 0, sizeof(int), E.stream));
    E.build_structures((int)m, nnz);
    int bad = 0;
    SFD_CUDA(cudaMemcpy(&bad, E.ws.flags, sizeof(int), cudaMemcpyDeviceToHost));
    if (bad) return SFD_EINVAL;
    // partial rows sized for ld = 4 * ceil(k/4) <= ldy
    float* partial = nullptr;
    int64_t slots = 2 * (nnz / kSplit) + 4;
    SFD_CUDA(cudaMalloc(&partial, (size_t)slots * std::max(ldy, ldx) * sizeof(float)));
    if (transpose_flag)
      spmm(E.csc, X, ldx, k, Y, ldy, partial, E.stream);
    else
      spmm(E.csr, X, ldx, k, Y, ldy, partial, E.stream);
    SFD_CUDA(cudaStreamSynchronize(E.stream));
    cudaFree(partial);
    return SFD_OK;
  } catch (const CudaError& e) {
    return e.err == cudaErrorMemoryAllocation ? SFD_ENOMEM : SFD_ECUDA;
  }
}

int sfd_orthonormalize(int64_t rows, int32_t k, float* X, int32_t ld) {
  if (rows < 1 || k < 1 || k > kMaxEll || ld < k || !X) return SFD_EINVAL;
  try {
    Engine E(1, 1, 1, 1, nullptr);
    float* tmp = nullptr;
    SFD_CUDA(cudaMalloc(&tmp, (size_t)rows * ld * sizeof(float)));
    ColMap map{k, 0, 0};
    for (int pass = 0; pass < 2; ++pass) {
      gram(X, ld, map, rows, E.ws.small_a, E.ws, E.stream);
      chol_inv(E.ws.small_a, k, E.ws.small_b, E.ws.eig_work, E.ws.flags, E.stream);
      gemm_ts(X, ld, map, rows, E.ws.small_b, k, tmp, ld, E.stream);
      SFD_CUDA(cudaMemcpy2DAsync(X, ld * sizeof(float), tmp, ld * sizeof(float), k * sizeof(float),
                                 rows, cudaMemcpyDeviceToDevice, E.stream));
    }
    SFD_CUDA(cudaStreamSynchronize(E.stream));
    cudaFree(tmp);
    return SFD_OK;
  } catch (const CudaError& e) {
    return e.err == cudaErrorMemoryAllocation ? SFD_ENOMEM : SFD_ECUDA;
  }
}

int sfd_symeig(int32_t n, const float* S, int32_t nwant, float* evals, float* evecs) {
  if (n < 1 || n > kMaxEig || nwant < 1 || nwant > n || !S || !evals || !evecs) return SFD_EINVAL;
  try {
    Engine E(1, 1, 1, 1, nullptr);
    symeig(S, n, nwant, evals, evecs, E.ws.eig_work, E.stream);
    SFD_CUDA(cudaStreamSynchronize(E.stream));
    return SFD_OK;
  } catch (const CudaError& e) {
    return e.err == cudaErrorMemoryAllocation ? SFD_ENOMEM : SFD_ECUDA;
  }
}

}  // extern "C"
