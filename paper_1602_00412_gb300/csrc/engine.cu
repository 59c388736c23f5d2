// Slot (one buffer's BoostedSparseShrink) and Merger (DenseShrink chain) of
// the GB300 Sparse Frequent Directions engine. See engine.cuh.
//
// Device layout of a slot (ld = l rounded up to 8; padding columns stay 0):
//   CSR copy of A' (rowptr, col, val), CSC copy (stable radix sort by column),
//   work lists, radix ping-pong arrays  ~ 8 x 4 B per buffer entry
//   W, W2 (d x ld), Y, Y2 (m_max x ld): SimultaneousIteration blocks
//   Bpt (d x ld): B'^T, read by VerifySpectral and by the Merger
// The Merger holds B^T twice (d x ld, ping-pong): DenseShrink reads one and
// writes the other.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "engine.cuh"

namespace sfd {

unsigned long long g_kernel_launches = 0;

namespace {

int bits_for(int64_t d) {
  int b = 1;
  while ((int64_t(1) << b) < d) ++b;
  return b;
}

void alloc_work(DevArena& A, SegWork& w, int64_t nseg, int64_t nnz) {
  w.cap_items = (int)(nseg + nnz / kSplit + 2);
  w.cap_split = (int)std::min<int64_t>(nseg, nnz / kSplit + 1) + 1;
  w.items = A.alloc<int4>(w.cap_items);
  w.item_slot = A.alloc<int>(w.cap_items);
  w.item_split = A.alloc<int>(w.cap_items);
  w.split_ticket = A.alloc<unsigned>(w.cap_split);
  SFD_CUDA(cudaMemset(w.split_ticket, 0, (size_t)w.cap_split * sizeof(unsigned)));
  w.split_seg = A.alloc<int>(std::max<int64_t>(nseg, 1) + 1);
  w.split_first = A.alloc<int>(std::max<int64_t>(nseg, 1) + 1);
  w.split_count = A.alloc<int>(std::max<int64_t>(nseg, 1) + 1);
  w.counters = A.alloc<int>(8 + 4 * ((size_t)nseg + 1) + nseg / 4096 + 16);
}

}  // namespace

void alloc_dense_scratch(DevArena& A, Workspace& ws) {
  ws.gram_partial = A.alloc<float>((size_t)320 * 128 * 128);
  ws.small_a = A.alloc<float>((size_t)kMaxEig * kMaxEig);
  ws.small_b = A.alloc<float>((size_t)kMaxEig * kMaxEig);
  ws.evals = A.alloc<float>(kMaxEig);
  ws.eig_work = A.alloc<float>(symeig_work_floats(kMaxEig, kMaxEig));
  ws.scalars = A.alloc<double>(64);
  ws.flags = A.alloc<int>(16);
  SFD_CUDA(cudaMemset(ws.scalars, 0, 64 * sizeof(double)));
  SFD_CUDA(cudaMemset(ws.flags, 0, 16 * sizeof(int)));
}

// ======================================================================= Slot
Slot::Slot(int64_t d_, int ell_, int64_t cap_rows_, int64_t cap_nnz_, cudaStream_t s) {
  d = d_;
  ell = ell_;
  ld = ld_of(ell);
  cap_rows = std::max<int64_t>(cap_rows_, 1);
  cap_nnz = std::max<int64_t>(cap_nnz_, 1);
  try {
    if (s) {
      stream = s;
    } else {
      SFD_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
      own_stream = true;
    }
    SFD_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    SFD_CUDA(cudaEventCreateWithFlags(&freed, cudaEventDisableTiming));
    DevArena& A = arena;
    csr.ptr = A.alloc<int>(cap_rows + 1);
    csr.idx = A.alloc<int>(cap_nnz);
    csr.val = A.alloc<float>(cap_nnz);
    csc.ptr = A.alloc<int>(d + 1);
    csc.idx = A.alloc<int>(cap_nnz);
    csc.val = A.alloc<float>(cap_nnz);
    key = A.alloc<int>(cap_nnz);
    key2 = A.alloc<int>(cap_nnz);
    a_alt = A.alloc<int>(cap_nnz);
    b_alt = A.alloc<float>(cap_nnz);
    alloc_work(A, csr.work, cap_rows, cap_nnz);
    alloc_work(A, csc.work, d, cap_nnz);
    const size_t dense_d = (size_t)d * ld, dense_m = (size_t)cap_rows * ld;
    W = A.alloc<float>(dense_d);
    W2 = A.alloc<float>(dense_d);
    Bpt = A.alloc<float>(dense_d);
    Y = A.alloc<float>(dense_m);
    Y2 = A.alloc<float>(dense_m);
    Wh = A.alloc<__half>(dense_d);
    Yh = A.alloc<__half>(dense_m);
    SFD_CUDA(cudaMemset(Wh, 0, dense_d * sizeof(__half)));
    SFD_CUDA(cudaMemset(Yh, 0, dense_m * sizeof(__half)));
    for (float* p : {W, W2, Bpt}) SFD_CUDA(cudaMemset(p, 0, dense_d * sizeof(float)));
    for (float* p : {Y, Y2}) SFD_CUDA(cudaMemset(p, 0, dense_m * sizeof(float)));
    alloc_dense_scratch(A, ws);
    int64_t ntiles = (cap_nnz + 4095) / 4096 + 1;
    ws.hist_cap = (int)(512 * ntiles + 8);
    ws.hist = A.alloc<int>(ws.hist_cap);
    ws.scan_tmp = A.alloc<int>(std::max<int64_t>(ws.hist_cap, d + cap_rows + 2) / 4096 + 64);
    int64_t slots = 2 * (cap_nnz / kSplit) + 4;
    ws.partial_rows_cap = (int)slots;
    ws.partial_rows = A.alloc<float>((size_t)slots * ld);
    ws.vec0 = A.alloc<float>(d);
    ws.vec1 = A.alloc<float>(std::max<int64_t>(d, cap_rows));
    ws.vec2 = A.alloc<float>(d);
    ws.wpart = A.alloc<float>(512 * kMaxEll + kMaxEll + 512);
    fro2 = A.alloc<double>(1024 + 8);
    verdict_dev = A.alloc<Verdict>(1);
    qfeat = A.alloc<float>(kQF);
    qacc = A.alloc<unsigned>(kQAccWords);
    qy = A.alloc<float>(1);
    q_dev = A.alloc<int>(1);
    SFD_CUDA(cudaMallocHost(&verdict_host, sizeof(Verdict)));
    SFD_CUDA(cudaMallocHost(&qfeat_host, kQF * sizeof(float)));
    SFD_CUDA(cudaMallocHost(&q_host, sizeof(int)));
    SFD_CUDA(cudaMallocHost(&ptr_host, (cap_rows + 1) * sizeof(int)));
    SFD_CUDA(cudaDeviceSynchronize());
  } catch (...) {
    cleanup();
    throw;
  }
}

Slot::~Slot() { cleanup(); }

void Slot::cleanup() {
  for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  ev_pool.clear();
  for (cudaEvent_t& e : tune_ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  vs_graphs.release();
  arena.release();
  if (verdict_host) cudaFreeHost(verdict_host);
  if (ptr_host) cudaFreeHost(ptr_host);
  if (qfeat_host) cudaFreeHost(qfeat_host);
  if (q_host) cudaFreeHost(q_host);
  verdict_host = nullptr;
  ptr_host = nullptr;
  qfeat_host = nullptr;
  q_host = nullptr;
  if (done) cudaEventDestroy(done);
  if (freed) cudaEventDestroy(freed);
  done = freed = nullptr;
  if (own_stream && stream) cudaStreamDestroy(stream);
  stream = nullptr;
}

void Slot::wait_freed() {
  if (freed_pending) {
    SFD_CUDA(cudaStreamWaitEvent(stream, freed, 0));
    freed_pending = false;
  }
}

void Slot::build(int m, int64_t nnz, int64_t max_row) {
  csr.nseg = m;
  csr.nnz = nnz;
  csr.may_split = max_row < 0 || max_row > kSplit;
  launch_check_entries(csr.idx, csr.val, nnz, (int)d, nullptr, fro2, ws.flags, stream);
  build_work(csr, stream);
  // CSC by a stable radix sort of (col, row, val) by col
  SFD_CUDA(cudaMemcpyAsync(key, csr.idx, nnz * sizeof(int), cudaMemcpyDeviceToDevice, stream));
  SFD_CUDA(cudaMemcpyAsync(csc.val, csr.val, nnz * sizeof(float), cudaMemcpyDeviceToDevice, stream));
  launch_row_ids(csr.ptr, m, csc.idx, stream);
  radix_sort_by_key(key, csc.idx, csc.val, key2, a_alt, b_alt, nnz, bits_for(d), ws.hist,
                    ws.scan_tmp, stream);
  colptr_from_sorted(key, nnz, (int)d, csc.ptr, stream);
  csc.nseg = (int)d;
  csc.nnz = nnz;
  build_work(csc, stream);
}

bool Slot::orth_pass(const float* X, int64_t rows, float* Xout, int form, __half* Xh) {
  const ColMap map = single_map(ell);
  // the accurate passes of mixed precision (form 2) factor their Gram in FP64,
  // also where l is too wide for the tensor-core Gram
  const bool fp64 = form == 2;
  if (!tc_supported(ell, ell)) form = 0;
  const bool split = form == 2;
  if (form) gram_tc(X, ld, map, rows, ws.small_a, ws, stream, split);
  else gram(X, ld, map, rows, ws.small_a, ws, stream);
  chol_inv(ws.small_a, ell, ws.small_b, ws.eig_work, ws.flags, stream, fp64);
  if (form == 1) gemm_ts_tc(X, ld, map, rows, ws.small_b, ell, Xout, ld, ws, stream, Xh);
  else if (split && tc_split_supported(ell, ell))
    gemm_ts_tc(X, ld, map, rows, ws.small_b, ell, Xout, ld, ws, stream, nullptr, true);
  else gemm_ts(X, ld, map, rows, ws.small_b, ell, Xout, ld, stream);
  return form == 1 && Xh;
}

// Time every unroll variant of this pass once (after one warm-up launch each)
// and keep the fastest. The variants give identical results, so tuning never
// changes the sketch; it costs one host wait per variant on a slot's first
// products.
int Slot::tune_spmm(const Csr& c, const float* X, const __half* Xh, float* Yo) {
  if (!tune_ev[0]) {
    SFD_CUDA(cudaEventCreate(&tune_ev[0]));
    SFD_CUDA(cudaEventCreate(&tune_ev[1]));
  }
  int best = 0;
  float best_ms = 0.f;
  for (int v = 0; v < spmm_variants(Xh != nullptr); ++v) {
    for (int rep = 0; rep < 2; ++rep) {
      SFD_CUDA(cudaEventRecord(tune_ev[0], stream));
      if (Xh) spmm_h(c, Xh, ld, ld, Yo, ld, ws.partial_rows, stream, v);
      else spmm(c, X, ld, ld, Yo, ld, ws.partial_rows, stream, v);
      SFD_CUDA(cudaEventRecord(tune_ev[1], stream));
    }
    SFD_CUDA(cudaEventSynchronize(tune_ev[1]));
    float ms = 0.f;
    SFD_CUDA(cudaEventElapsedTime(&ms, tune_ev[0], tune_ev[1]));
    if (v == 0 || ms < best_ms) {
      best = v;
      best_ms = ms;
    }
  }
  return best;
}

void Slot::spmm_timed(const Csr& c, const float* X, float* Yo, int64_t rows_in, const __half* Xh) {
  int& choice = this->choice[&c == &csc ? 1 : 0][Xh ? 1 : 0];
  if (choice < 0) choice = autotune ? tune_spmm(c, X, Xh, Yo) : 0;
  const int variant = choice;
  auto run = [&] {
    if (Xh) spmm_h(c, Xh, ld, ld, Yo, ld, ws.partial_rows, stream, variant);
    else spmm(c, X, ld, ld, Yo, ld, ws.partial_rows, stream, variant);
  };
  if (!profile) {
    run();
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
  run();
  SFD_CUDA(cudaEventRecord(ev_pool[i0 + 1], stream));
  const double in_bytes = Xh ? 2.0 : 4.0;
  const double bytes = 8.0 * (double)c.nnz + 4.0 * (c.nseg + 1) +
                       in_bytes * ell * (double)rows_in + 4.0 * ell * (double)c.nseg;
  ev_pending.push_back({i0, bytes});
}

void Slot::collect_profile() {
  if (!profile || ev_pending.empty()) return;
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

int Slot::enqueue_attempt(int m, int q, uint64_t seed, uint64_t b, uint64_t r, int p, int verify,
                          const QControl* qc) {
  // Alg. 1: G ~ N(0,1)^{d x l}; Y = orth(A' G); q x { W = orth(A'^T Y); Y = orth(A' W) }
  launch_gauss_fill(W, d, ell, ld, seed, b, r, 1, stream);
  // mixed precision: the orthonormalisations of every power iteration but the
  // last run on tensor cores in TF32 (form 1); the last iteration, the second
  // CholeskyQR pass on Z and the products of Alg. 3 keep FP32 accuracy, so the
  // TF32 perturbation of the subspace is damped by one more accurate iteration
  // and Z is orthonormal to FP32 accuracy. Those accurate stages run on tensor
  // cores as well, in the split form (form 2: hi and lo TF32 parts, three
  // MMAs, ~21 significant bits), where l allows; else on the CUDA cores.
  // Mixed precision also stores the orthonormal blocks between a TF32
  // orthonormalisation and the next sparse product as fp16 (|entries| <= 1,
  // the TF32 inputs' precision), so the product's gather moves half the bytes.
  const int exact_form = mixed ? 2 : 0;
  spmm_timed(csr, W, Y, d);
  // leaves S0 = (A'G)^T (A'G) in ws.small_a
  bool y_half = orth_pass(Y, m, Y2, mixed ? (q > 0 ? 1 : 2) : 0, Yh);
  if (!y_half) std::swap(Y, Y2);
  if (qc && (qc->predict || qc->features)) {
    q_features(csr, csc, d, ell, qc->q_fixed, fro2, ws.small_a, qfeat, qacc, stream);
    SFD_CUDA(cudaMemcpyAsync(qfeat_host, qfeat, kQF * sizeof(float), cudaMemcpyDeviceToHost,
                             stream));
    if (qc->predict) {
      predict_q(qc->params, qfeat, qc->margin, qc->q_fixed, qy, q_dev, stream);
      SFD_CUDA(cudaMemcpyAsync(q_host, q_dev, sizeof(int), cudaMemcpyDeviceToHost, stream));
      SFD_CUDA(cudaStreamSynchronize(stream));
      q = *q_host;
    }
  }
  for (int t = 0; t < q; ++t) {
    const int tc = t + 1 < q && mixed ? 1 : exact_form;
    spmm_timed(csc, Y, W, m, y_half ? Yh : nullptr);
    const bool w_half = orth_pass(W, d, W2, tc, Wh);
    if (!w_half) std::swap(W, W2);
    spmm_timed(csr, W, Y, d, w_half ? Wh : nullptr);
    y_half = orth_pass(Y, m, Y2, tc, Yh);
    if (!y_half) std::swap(Y, Y2);
  }
  // here Y is fp32: a tensor-core first pass implies q >= 1 (the predicted q
  // is at least 1 as well), and the last iteration is fp32
  orth_pass(Y, m, Y2, exact_form);  // second CholeskyQR pass on Z
  std::swap(Y, Y2);
  // Alg. 3: P^T = A'^T Z, svd(P, l) through P P^T, B'^T = P^T H diag(s)
  spmm_timed(csc, Y, W, m);
  const ColMap map = single_map(ell);
  if (mixed && tc_supported(ell, ell)) gram_tc(W, ld, map, d, ws.small_a, ws, stream, true);
  else gram(W, ld, map, d, ws.small_a, ws, stream);
  symeig(ws.small_a, ell, ell, ws.evals, ws.small_b, ws.eig_work, stream, true);
  shrink_weights(ws.evals, ws.small_b, ell, ell, ell, 0, ws.small_a, ws.scalars, stream);
  wait_freed();  // DenseShrink of this slot's previous buffer must have read B'^T
  if (mixed && tc_split_supported(ell, ell))
    gemm_ts_tc(W, ld, map, d, ws.small_a, ell, Bpt, ld, ws, stream, nullptr, true);
  else gemm_ts(W, ld, map, d, ws.small_a, ell, Bpt, ld, stream);
  // Alg. 4: Delta; Alg. 6: VerifySpectral
  launch_delta(fro2, ws.scalars, ell, stream);
  if (verify) {
    VsArgs a{&csr, &csc, Bpt, ld, ell, d, m, ws.scalars + kSscale, p, seed, b, r};
    verify_spectral(a, ws, stream, &vs_graphs);
  }
  launch_verdict(fro2, ws.scalars, ws.flags, ws.evals, ell, verify, verdict_dev, stream);
  SFD_CUDA(cudaMemcpyAsync(verdict_host, verdict_dev, sizeof(Verdict), cudaMemcpyDeviceToHost,
                           stream));
  SFD_CUDA(cudaEventRecord(done, stream));
  return q;
}

// ===================================================================== Merger
Merger::Merger(int64_t d_, int ell_) {
  d = d_;
  ell = ell_;
  ld = ld_of(ell);
  try {
    SFD_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) Bt[i] = arena.alloc<float>((size_t)d * ld);
    out = arena.alloc<float>((size_t)d * ell);
    alloc_dense_scratch(arena, ws);
    zero();
    SFD_CUDA(cudaStreamSynchronize(stream));
  } catch (...) {
    cleanup();
    throw;
  }
}

Merger::~Merger() { cleanup(); }

void Merger::cleanup() {
  arena.release();
  if (stream) cudaStreamDestroy(stream);
  stream = nullptr;
}

void Merger::zero() {
  for (int i = 0; i < 2; ++i)
    SFD_CUDA(cudaMemsetAsync(Bt[i], 0, (size_t)d * ld * sizeof(float), stream));
  cur = 0;
}

void Merger::dense_shrink(const float* Xt, int ldx, int k1, bool orthogonal_rows) {
  // Alg. 5 on the stack [B; X]: K = M M^T, top-l eigenpairs, B^T <- M^T U_l diag(s)
  const ColMap map{ell, k1, Xt, ldx};
  const int n = ell + k1;
  // B B^T and X X^T are diagonal when both have orthogonal rows (B = diag(s) V^T
  // after Alg. 5, B' = diag(s) H^T P after Alg. 3): only B X^T and the row
  // norms are formed then
  if (mixed && orthogonal_rows && k1 >= 1 && ell <= 128 && k1 <= 128)
    cross_gram_tc(Bt[cur], ld, ell, Xt, ldx, k1, d, ws.small_a, ws, stream);
  else
    gram(Bt[cur], ld, map, d, ws.small_a, ws, stream);
  symeig(ws.small_a, n, ell, ws.evals, ws.small_b, ws.eig_work, stream, true);
  shrink_weights(ws.evals, ws.small_b, n, ell, ell, 0, ws.small_a, ws.scalars, stream);
  // B^T <- M^T T with M^T = [B^T | X^T] (T: n x l, row-major): in mixed
  // precision as B^T T[0:l] + X^T T[l:n] on the tensor cores (split TF32,
  // each block within one K tile), else in FP32 on the CUDA cores
  if (mixed && k1 >= 1 && tc_split_supported(ell, ell) && tc_split_supported(k1, ell)) {
    gemm_ts_tc(Bt[cur], ld, single_map(ell), d, ws.small_a, ell, Bt[1 - cur], ld, ws, stream,
               nullptr, true);
    gemm_ts_tc(Xt, ldx, single_map(k1), d, ws.small_a + (size_t)ell * ell, ell, Bt[1 - cur], ld,
               ws, stream, nullptr, true, true);
  } else {
    gemm_ts(Bt[cur], ld, map, d, ws.small_a, ell, Bt[1 - cur], ld, stream);
  }
  cur = 1 - cur;
}

}  // namespace sfd
