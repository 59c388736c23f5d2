// C ABI of include/sfd.h: the SFD stream (Alg. 2) over a pipeline of slots.
//
// Rows are copied into the slot being filled. When the buffer closes
// (l*d entries or d rows), its BoostedSparseShrink attempt is queued on that
// slot's stream and the buffer joins a FIFO; the next buffer fills the next
// slot. Before a slot is refilled, the FIFO is harvested in buffer order: the
// host reads the attempt's verdict (pinned memory, one wait per attempt),
// retries with the next Philox key if VerifySpectral rejected, and queues
// DenseShrink on the merge stream, which the slot's next B'^T write waits for.
// Every call drains the pipeline before it returns.
#include <string.h>

#include <algorithm>

#include <cmath>
#include <deque>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "context.cuh"


namespace sfd {
namespace {

int fail(Ctx* C, int code, const std::string& msg) {
  if (C) C->last_error = msg;
  return code;
}

int from_cuda(Ctx* C, const CudaError& e) {
  std::string m = std::string(e.where) + ": " + cudaGetErrorString(e.err);
  if (e.err == cudaErrorMemoryAllocation) return fail(C, SFD_ENOMEM, m);
  return fail(C, SFD_ECUDA, m);
}

struct LaunchCount {
  sfd_stats& st;
  unsigned long long start;
  explicit LaunchCount(sfd_stats& s)
      : st(s), start(__atomic_load_n(&g_kernel_launches, __ATOMIC_RELAXED)) {}
  ~LaunchCount() {
    st.kernel_launches +=
        (int64_t)(__atomic_load_n(&g_kernel_launches, __ATOMIC_RELAXED) - start);
  }
};

// Order the context's streams after the caller's stream.
void join_user_stream(Ctx& C) {
  cudaStream_t us = (cudaStream_t)C.opt.cuda_stream;
  SFD_CUDA(cudaEventRecord(C.user_ev, us));
  SFD_CUDA(cudaStreamWaitEvent(C.in_stream, C.user_ev, 0));
  SFD_CUDA(cudaStreamWaitEvent(C.merger->stream, C.user_ev, 0));
  for (auto& s : C.slots) SFD_CUDA(cudaStreamWaitEvent(s->stream, C.user_ev, 0));
}

// Make the caller's stream wait for everything the context queued.
void release_user_stream(Ctx& C) {
  cudaStream_t us = (cudaStream_t)C.opt.cuda_stream;
  SFD_CUDA(cudaEventRecord(C.user_ev, C.merger->stream));
  SFD_CUDA(cudaStreamWaitEvent(us, C.user_ev, 0));
  for (auto& s : C.slots) {
    SFD_CUDA(cudaEventRecord(C.user_ev, s->stream));
    SFD_CUDA(cudaStreamWaitEvent(us, C.user_ev, 0));
  }
}

// Training label of a buffer whose first attempt (q_fixed) was accepted: rerun
// SparseShrink + VerifySpectral with the same G at each smaller q of the
// ladder; the label is the smallest q that passes VerifySpectral and keeps
// ||P||_F^2 within a fraction q_tau of the q_fixed run. The reruns come after
// DenseShrink has read B'^T (enqueue_attempt waits for `freed`), so the sketch
// is unchanged.
void label_buffer(Ctx& C, Slot& S, const Ctx::Pend& e, const Verdict& v) {
  const float* f = S.qfeat_host;  // features of attempt 0, copied before `done`
  const int p = vs_steps(C.d, delta_br(C.opt.delta, e.b, 0));
  int lab = e.q_fixed;
  for (int q : kLadder) {
    if (q >= e.q_fixed) break;
    S.enqueue_attempt(e.m, q, C.seed, (uint64_t)e.b, 0, p, C.opt.verify);
    SFD_CUDA(cudaEventSynchronize(S.done));
    const Verdict& w = *S.verdict_host;
    if (w.timeout) return;
    if ((w.ok || !C.opt.verify) && w.captured >= (1.0 - C.opt.q_tau) * v.captured) {
      lab = q;
      break;
    }
  }
  C.qlog_feat.insert(C.qlog_feat.end(), f, f + kQF);
  C.qlog_label.push_back((float)lab);
  C.qlog_qfixed.push_back(e.q_fixed);
}

// Read the verdict of the oldest closed buffer, retry it until accepted or
// out of attempts, then queue its DenseShrink.
int harvest_front(Ctx& C) {
  Ctx::Pend e = C.fifo.front();
  Slot& S = *C.slots[e.slot];
  int status = SFD_OK;
  Verdict v{};
  for (;;) {
    SFD_CUDA(cudaEventSynchronize(S.done));
    v = *S.verdict_host;
    if (v.timeout) {  // a tensor-core wait expired: the attempt's result is not usable
      C.st.attempts++;
      status = SFD_ETIMEOUT;
      break;
    }
    C.st.attempts++;
    C.st.q_total += e.q;
    bool ok = v.ok != 0;
    if (C.opt.verify && C.inject_left > 0) {
      ok = false;
      C.inject_left--;
    }
    C.st.last_logsum = v.logsum;
    if (ok) break;
    C.st.vs_rejects++;
    if (e.r + 1 >= std::max(1, C.opt.retry_cap)) {
      C.st.unverified++;
      if (C.opt.strict) status = SFD_EVERIFY;
      break;
    }
    e.r++;
    e.q = e.q_fixed;  // a rejected attempt is retried on the fixed schedule
    S.enqueue_attempt(e.m, e.q, C.seed, (uint64_t)e.b, (uint64_t)e.r,
                      vs_steps(C.d, delta_br(C.opt.delta, e.b, e.r)), C.opt.verify);
  }
  S.collect_profile();
  C.st.last_delta = v.delta;
  C.st.last_fro2 = v.fro2a;
  Merger& M = *C.merger;
  SFD_CUDA(cudaStreamWaitEvent(M.stream, S.done, 0));
  M.dense_shrink(S.Bpt, S.ld, C.ell, true);
  SFD_CUDA(cudaEventRecord(S.freed, M.stream));
  S.freed_pending = true;
  C.st.buffers++;
  C.fifo.pop_front();
  if (C.opt.q_mode == 2 && status == SFD_OK && e.r == 0 && !v.timeout && (v.ok || !C.opt.verify))
    label_buffer(C, S, e, v);
  return status;
}

int drain(Ctx& C) {
  int status = SFD_OK;
  while (!C.fifo.empty()) {
    int rc = harvest_front(C);
    if (rc != SFD_OK) status = rc;
  }
  SFD_CUDA(cudaStreamSynchronize(C.merger->stream));
  return status;
}

// Pick the slot for the next buffer; its previous buffer must be harvested
// first (a retry would still need its CSR copy).
int acquire_fill_slot(Ctx& C) {
  int status = SFD_OK;
  if (C.fill >= 0) return status;
  const int s = C.next_slot;
  C.next_slot = (C.next_slot + 1) % (int)C.slots.size();
  for (;;) {
    bool busy = false;
    for (auto& e : C.fifo) busy |= e.slot == s;
    if (!busy) break;
    int rc = harvest_front(C);
    if (rc != SFD_OK) status = rc;
  }
  // the slot's last queued work (attempt or small-buffer path) read its
  // pinned row-pointer staging; it must be done before that is rewritten
  SFD_CUDA(cudaEventSynchronize(C.slots[s]->done));
  C.fill = s;
  SFD_CUDA(cudaStreamWaitEvent(C.slots[s]->stream, C.in_ready, 0));
  return status;
}

// Close the open buffer (Alg. 2 trigger, or a flush).
int close_buffer(Ctx& C) {
  const int m = C.pend_rows;
  if (m == 0) return SFD_OK;
  int status = SFD_OK;
  Slot& S = *C.slots[C.fill];
  memcpy(S.ptr_host, C.h_ptr.data(), (m + 1) * sizeof(int));
  SFD_CUDA(cudaMemcpyAsync(S.csr.ptr, S.ptr_host, (m + 1) * sizeof(int), cudaMemcpyHostToDevice,
                           S.stream));
  if (m >= C.ell && C.opt.mode == 0) {
    int64_t max_row = 0;
    for (int i = 0; i < m; ++i) max_row = std::max<int64_t>(max_row, C.h_ptr[i + 1] - C.h_ptr[i]);
    S.build(m, C.pend_nnz, max_row);
    const int q = q_for(C.opt, m);
    QControl qc;
    qc.q_fixed = q;
    if (C.opt.q_mode == 1 && C.has_qmodel) {
      qc.predict = true;
      qc.params = C.qparams;
      qc.margin = C.opt.q_margin;
    } else if (C.opt.q_mode == 2) {
      qc.features = true;
    }
    const int q_used = S.enqueue_attempt(m, q, C.seed, (uint64_t)C.b, 0,
                                         vs_steps(C.d, delta_br(C.opt.delta, C.b, 0)),
                                         C.opt.verify, &qc);
    C.fifo.push_back({C.fill, C.b, m, q_used, 0, q});
  } else {
    // too few rows for SparseShrink, or classical FrequentDirections (mode 1):
    // DenseShrink([B; A']) with A' dense
    status = drain(C);
    S.wait_freed();
    SFD_CUDA(cudaMemsetAsync(S.Bpt, 0, (size_t)C.d * S.ld * sizeof(float), S.stream));
    csr_to_dense_t(S.csr.ptr, S.csr.idx, S.csr.val, m, C.d, S.Bpt, S.ld, S.stream);
    SFD_CUDA(cudaEventRecord(S.done, S.stream));
    Merger& M = *C.merger;
    SFD_CUDA(cudaStreamWaitEvent(M.stream, S.done, 0));
    M.dense_shrink(S.Bpt, S.ld, m);
    SFD_CUDA(cudaEventRecord(S.freed, M.stream));
    S.freed_pending = true;
    C.st.buffers++;
  }
  C.b++;
  C.fill = -1;
  C.pend_rows = 0;
  C.pend_nnz = 0;
  C.h_ptr.assign(1, 0);
  return status;
}

int flush(Ctx& C) {
  int rc = close_buffer(C);
  int rc2 = drain(C);
  C.st.pending_rows = 0;
  C.st.pending_nnz = 0;
  return rc != SFD_OK ? rc : rc2;
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
  o->q_margin = 1.0f;
  o->q_tau = 1e-2f;
  o->autotune = 1;
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
  const int64_t cap_nnz = (int64_t)ell * d + d;
  if (cap_nnz > INT32_MAX - 1) return SFD_EINVAL;
  sfd_ctx* ctx = new (std::nothrow) sfd_ctx();
  if (!ctx) return SFD_ENOMEM;
  Ctx& C = ctx->c;
  if (opt) C.opt = *opt; else sfd_options_init(&C.opt);
  if (!(C.opt.delta > 0 && C.opt.delta < 1) || C.opt.c_q < 0 || C.opt.slots < 0 ||
      (C.opt.precision != 0 && C.opt.precision != 1) || C.opt.q_mode < 0 || C.opt.q_mode > 2 ||
      (C.opt.mode != 0 && C.opt.mode != 1) ||
      !(C.opt.q_tau >= 0.f && C.opt.q_tau < 1.f) || !(C.opt.q_margin > -64.f && C.opt.q_margin < 64.f)) {
    delete ctx;
    return SFD_EINVAL;
  }
  C.seed = seed;
  C.d = d;
  C.ell = ell;
  C.ld = ld_of(ell);
  C.inject_left = C.opt.inject_vs_fail;
  C.h_ptr.assign(1, 0);
  const int want = std::min(kMaxSlots, C.opt.slots > 0 ? C.opt.slots : kDefaultSlots);
  try {
    SFD_CUDA(cudaGetDevice(&C.dev));
    SFD_CUDA(cudaStreamCreateWithFlags(&C.in_stream, cudaStreamNonBlocking));
    SFD_CUDA(cudaEventCreateWithFlags(&C.in_ready, cudaEventDisableTiming));
    SFD_CUDA(cudaEventCreateWithFlags(&C.user_ev, cudaEventDisableTiming));
    C.chk_fro2 = C.stage_arena.alloc<double>(1032);
    C.chk_flags = C.stage_arena.alloc<int>(4);
    C.merger.reset(new Merger(d, ell));
    C.merger->mixed = C.opt.precision == 1;
    for (int i = 0; i < want; ++i) {
      try {
        C.slots.emplace_back(new Slot(d, ell, d, cap_nnz, nullptr));
        C.slots.back()->profile = C.opt.profile != 0;
        C.slots.back()->mixed = C.opt.precision == 1;
        C.slots.back()->autotune = C.opt.autotune != 0;
        C.slots.back()->choice = C.slots.front()->spmm_choice;
      } catch (const CudaError& e) {
        // fewer slots when memory is short; at least one is required
        if (e.err != cudaErrorMemoryAllocation || C.slots.empty()) throw;
        cudaGetLastError();
        break;
      }
    }
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

void sfd_destroy(sfd_ctx* ctx) { delete ctx; }

int sfd_append_rows(sfd_ctx* ctx, int64_t nrows, const int64_t* indptr, const int32_t* indices,
                    const float* values, int where) {
  if (!ctx) return SFD_EINVAL;
  Ctx& C = ctx->c;
  LaunchCount lc(C.st);
  if (nrows < 0 || (where != SFD_HOST && where != SFD_DEVICE))
    return fail(&C, SFD_EINVAL, "bad nrows/where");
  if (nrows == 0) return SFD_OK;
  if (!indptr) return fail(&C, SFD_EINVAL, "null indptr");
  try {
    SFD_CUDA(cudaSetDevice(C.dev));
    // 1. indptr on the host, checked
    std::vector<int64_t> ip(nrows + 1);
    if (where == SFD_DEVICE)
      SFD_CUDA(cudaMemcpy(ip.data(), indptr, (nrows + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    else
      memcpy(ip.data(), indptr, (nrows + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < nrows; ++i) {
      const int64_t c = ip[i + 1] - ip[i];
      if (c < 0 || c > C.d) return fail(&C, SFD_EINVAL, "indptr not non-decreasing or row longer than d");
    }
    const int64_t base = ip[0], total = ip[nrows] - ip[0];
    if (base < 0) return fail(&C, SFD_EINVAL, "negative indptr");
    if (total > 0 && (!indices || !values)) return fail(&C, SFD_EINVAL, "null indices/values");
    join_user_stream(C);
    // 2. the entries on the device (staged for host input), checked before any is used
    const int* didx;
    const float* dval;
    if (where == SFD_HOST) {
      if (total > C.stage_cap) {
        SFD_CUDA(cudaStreamSynchronize(C.in_stream));
        if (C.stage_idx) cudaFree(C.stage_idx);
        if (C.stage_val) cudaFree(C.stage_val);
        C.stage_idx = nullptr;
        C.stage_val = nullptr;
        C.stage_cap = 0;
        SFD_CUDA(cudaMalloc(&C.stage_idx, total * sizeof(int)));
        SFD_CUDA(cudaMalloc(&C.stage_val, total * sizeof(float)));
        C.stage_cap = total;
      }
      if (total > 0) {
        SFD_CUDA(cudaMemcpyAsync(C.stage_idx, indices + base, total * sizeof(int),
                                 cudaMemcpyHostToDevice, C.in_stream));
        SFD_CUDA(cudaMemcpyAsync(C.stage_val, values + base, total * sizeof(float),
                                 cudaMemcpyHostToDevice, C.in_stream));
      }
      didx = C.stage_idx;
      dval = C.stage_val;
    } else {
      didx = indices + base;
      dval = values + base;
    }
    if (total > 0) {
      SFD_CUDA(cudaMemsetAsync(C.chk_flags, 0, sizeof(int), C.in_stream));
      launch_check_entries(didx, dval, total, (int)C.d, nullptr, C.chk_fro2, C.chk_flags,
                           C.in_stream);
      int bad = 0;
      SFD_CUDA(cudaMemcpyAsync(&bad, C.chk_flags, sizeof(int), cudaMemcpyDeviceToHost, C.in_stream));
      SFD_CUDA(cudaStreamSynchronize(C.in_stream));
      if (bad) return fail(&C, SFD_EINVAL, "column index outside [0, d) or non-finite value");
    }
    SFD_CUDA(cudaEventRecord(C.in_ready, C.in_stream));
    // 3. Alg. 2: one row at a time; close the buffer when nnz >= l d or rows = d
    //    (classical FrequentDirections, mode 1: every l rows)
    const int64_t thresh = C.opt.mode == 1 ? INT64_MAX : (int64_t)C.ell * C.d;
    const int64_t row_cap = C.opt.mode == 1 ? C.ell : C.d;
    int status = SFD_OK;
    auto keep = [&status](int rc) {
      if (rc != SFD_OK) status = rc;
    };
    auto copy_rows = [&](int64_t r0, int64_t r1) {
      if (r1 <= r0) return;
      keep(acquire_fill_slot(C));
      Slot& S = *C.slots[C.fill];
      const int64_t e0 = ip[r0] - base, e1 = ip[r1] - base;
      if (e1 > e0) {
        SFD_CUDA(cudaMemcpyAsync(S.csr.idx + C.pend_nnz, didx + e0, (e1 - e0) * sizeof(int),
                                 cudaMemcpyDeviceToDevice, S.stream));
        SFD_CUDA(cudaMemcpyAsync(S.csr.val + C.pend_nnz, dval + e0, (e1 - e0) * sizeof(float),
                                 cudaMemcpyDeviceToDevice, S.stream));
      }
      for (int64_t r = r0; r < r1; ++r) {
        C.pend_nnz += ip[r + 1] - ip[r];
        C.pend_rows += 1;
        C.h_ptr.push_back((int)C.pend_nnz);
      }
    };
    int64_t seg_start = 0;
    int64_t rows_in_buf = C.pend_rows, nnz_in_buf = C.pend_nnz;
    for (int64_t i = 0; i < nrows; ++i) {
      rows_in_buf += 1;
      nnz_in_buf += ip[i + 1] - ip[i];
      if (nnz_in_buf >= thresh || rows_in_buf == row_cap) {
        copy_rows(seg_start, i + 1);
        seg_start = i + 1;
        keep(close_buffer(C));
        rows_in_buf = 0;
        nnz_in_buf = 0;
      }
    }
    copy_rows(seg_start, nrows);
    keep(drain(C));
    for (auto& s : C.slots) SFD_CUDA(cudaStreamSynchronize(s->stream));
    release_user_stream(C);
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

int sfd_sketch(sfd_ctx* ctx, float* B_out, int where) {
  if (!ctx || !B_out || (where != SFD_HOST && where != SFD_DEVICE)) return SFD_EINVAL;
  Ctx& C = ctx->c;
  LaunchCount lc(C.st);
  try {
    SFD_CUDA(cudaSetDevice(C.dev));
    join_user_stream(C);
    const int rc = flush(C);
    Merger& M = *C.merger;
    if (where == SFD_DEVICE) {
      transpose(M.B(), C.d, C.ell, M.ld, B_out, C.d, M.stream);
    } else {
      // the Merger's own l x d buffer: slot buffers are not scratch (their
      // padding columns must stay zero)
      transpose(M.B(), C.d, C.ell, M.ld, M.out, C.d, M.stream);
      SFD_CUDA(cudaMemcpyAsync(B_out, M.out, (size_t)C.ell * C.d * sizeof(float),
                               cudaMemcpyDeviceToHost, M.stream));
    }
    SFD_CUDA(cudaStreamSynchronize(M.stream));
    release_user_stream(C);
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
  if (D.d != S.d || D.ell != S.ell || D.dev != S.dev)
    return fail(&D, SFD_EINVAL, "shape/device mismatch");
  try {
    SFD_CUDA(cudaSetDevice(D.dev));
    join_user_stream(S);
    join_user_stream(D);
    const int rc1 = flush(S);
    const int rc2 = flush(D);
    Merger& MD = *D.merger;
    SFD_CUDA(cudaEventRecord(S.user_ev, S.merger->stream));
    SFD_CUDA(cudaStreamWaitEvent(MD.stream, S.user_ev, 0));
    MD.dense_shrink(S.merger->B(), S.merger->ld, D.ell, true);  // Sec. 3.1: DSh([B_dst; B_src])
    SFD_CUDA(cudaStreamSynchronize(MD.stream));
    release_user_stream(D);
    return rc1 != SFD_OK ? rc1 : rc2;
  } catch (const CudaError& e) {
    return from_cuda(&D, e);
  }
}

int sfd_get_stats(const sfd_ctx* ctx, sfd_stats* out) {
  if (!ctx || !out) return SFD_EINVAL;
  *out = ctx->c.st;
  out->spmm_launches = 0;
  out->spmm_ms = out->spmm_bytes = 0;
  for (auto& s : ctx->c.slots) {
    out->spmm_launches += s->prof_launches;
    out->spmm_ms += s->prof_ms;
    out->spmm_bytes += s->prof_bytes;
  }
  return SFD_OK;
}

int sfd_reset(sfd_ctx* ctx) {
  if (!ctx) return SFD_EINVAL;
  Ctx& C = ctx->c;
  try {
    SFD_CUDA(cudaSetDevice(C.dev));
    drain(C);
    for (auto& s : C.slots) {
      SFD_CUDA(cudaStreamSynchronize(s->stream));
      s->prof_launches = 0;
      s->prof_ms = s->prof_bytes = 0;
    }
    C.merger->zero();
    SFD_CUDA(cudaStreamSynchronize(C.merger->stream));
    C.fill = -1;
    C.next_slot = 0;
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

int sfd_set_q_model(sfd_ctx* ctx, const float* params) {
  if (!ctx) return SFD_EINVAL;
  Ctx& C = ctx->c;
  try {
    SFD_CUDA(cudaSetDevice(C.dev));
    if (!params) {
      C.has_qmodel = false;
      return SFD_OK;
    }
    for (int i = 0; i < kQParams; ++i)
      if (!std::isfinite(params[i])) return fail(&C, SFD_EINVAL, "non-finite model parameter");
    drain(C);
    if (!C.qparams) C.qparams = C.stage_arena.alloc<float>(kQParams);
    SFD_CUDA(cudaMemcpy(C.qparams, params, kQParams * sizeof(float), cudaMemcpyHostToDevice));
    C.has_qmodel = true;
    return SFD_OK;
  } catch (const CudaError& e) {
    return from_cuda(&C, e);
  }
}

int sfd_q_log(const sfd_ctx* ctx, int64_t cap, float* features, float* labels, int32_t* q_fixed,
              int64_t* n_out) {
  if (!ctx || !n_out || cap < 0) return SFD_EINVAL;
  const Ctx& C = ctx->c;
  const int64_t n = (int64_t)C.qlog_label.size();
  *n_out = n;
  const int64_t k = std::min(n, cap);
  if (k > 0 && (!features || !labels)) return SFD_EINVAL;
  for (int64_t i = 0; i < k; ++i) {
    memcpy(features + i * kQF, C.qlog_feat.data() + i * kQF, kQF * sizeof(float));
    labels[i] = C.qlog_label[i];
    if (q_fixed) q_fixed[i] = C.qlog_qfixed[i];
  }
  return SFD_OK;
}

}  // extern "C"
