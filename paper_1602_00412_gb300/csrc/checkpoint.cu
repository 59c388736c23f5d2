// Checkpoint and resume of an SFD stream (include/sfd.h: sfd_save, sfd_load).
//
// Between calls, the whole state of Alg. 2 is the sketch B (l x d), the open
// buffer A' (the rows appended since the last buffer closed) and the buffer
// counter b that keys every random draw (with the stream's seed and
// options). Every public call drains the pipeline before it returns, so no
// buffer is in flight when a checkpoint is taken, and restoring those three
// items gives a context whose future is the same bits as the original's: the
// next buffer closes at the same row, draws the same Philox G and x, and is
// folded into the same B.
//
// Blob layout (host byte order, little-endian on every supported host):
//   char[8]  magic "SFDCKPT1"
//   u32      SFD_ABI_VERSION, u32 header bytes (kHeaderBytes)
//   i64 d, i32 l, i32 has_qmodel, u64 seed, i64 b,
//   i64 pending rows, i64 pending entries, i32 inject_left, i32 mode,
//   options: f64 delta, i32 verify, f64 c_q, i32 q_override, i32 retry_cap,
//            i32 precision, i32 q_mode, i32 strict, f32 q_margin, f32 q_tau
//   stats: sfd_stats field by field (i64 / f64, 8 bytes each)
//   f32 B[l][d]                      the sketch, row-major
//   i32 ptr[pending rows + 1]        the open buffer (row pointer from 0)
//   i32 idx[pending entries], f32 val[pending entries]
//   f32 params[SFD_QPARAMS]          only when has_qmodel
//   u64 FNV-1a hash of every byte before it
#include <string.h>

#include <cmath>
#include <new>
#include <vector>

#include "context.cuh"

namespace sfd {
namespace {

constexpr char kMagic[8] = {'S', 'F', 'D', 'C', 'K', 'P', 'T', '1'};

struct Writer {
  std::vector<unsigned char>& out;
  template <typename T>
  void put(const T& v) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
    out.insert(out.end(), p, p + sizeof(T));
  }
  void bytes(const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    out.insert(out.end(), c, c + n);
  }
};

struct Reader {
  const unsigned char* p;
  size_t n, at = 0;
  bool ok = true;
  template <typename T>
  T get() {
    T v{};
    if (at + sizeof(T) > n) {
      ok = false;
      return v;
    }
    memcpy(&v, p + at, sizeof(T));
    at += sizeof(T);
    return v;
  }
  const unsigned char* take(size_t k) {
    if (at > n || k > n - at) {
      ok = false;
      return nullptr;
    }
    const unsigned char* q = p + at;
    at += k;
    return q;
  }
};

uint64_t fnv1a(const unsigned char* p, size_t n) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

void put_stats(Writer& w, const sfd_stats& s) {
  for (int64_t v : {s.rows_seen, s.nnz_seen, s.buffers, s.attempts, s.vs_rejects, s.unverified,
                    s.q_total, s.pending_rows, s.pending_nnz})
    w.put(v);
  for (double v : {s.last_delta, s.last_logsum, s.last_fro2}) w.put(v);
  w.put(s.kernel_launches);
  w.put(s.spmm_launches);
  w.put(s.spmm_ms);
  w.put(s.spmm_bytes);
}

void get_stats(Reader& r, sfd_stats& s) {
  for (int64_t* v : {&s.rows_seen, &s.nnz_seen, &s.buffers, &s.attempts, &s.vs_rejects,
                     &s.unverified, &s.q_total, &s.pending_rows, &s.pending_nnz})
    *v = r.get<int64_t>();
  for (double* v : {&s.last_delta, &s.last_logsum, &s.last_fro2}) *v = r.get<double>();
  s.kernel_launches = r.get<int64_t>();
  s.spmm_launches = r.get<int64_t>();
  s.spmm_ms = r.get<double>();
  s.spmm_bytes = r.get<double>();
}

constexpr uint32_t kHeaderBytes = 8 + 4 + 4 + 8 + 4 + 4 + 8 + 8 + 8 + 8 + 4 + 4 +
                                  (8 + 4 + 8 + 4 + 4 + 4 + 4 + 4 + 4 + 4) + 16 * 8;

std::vector<unsigned char> serialize(Ctx& C) {
  std::vector<unsigned char> buf;
  Writer w{buf};
  w.bytes(kMagic, 8);
  w.put<uint32_t>(SFD_ABI_VERSION);
  w.put<uint32_t>(kHeaderBytes);
  w.put<int64_t>(C.d);
  w.put<int32_t>(C.ell);
  w.put<int32_t>(C.has_qmodel ? 1 : 0);
  w.put<uint64_t>(C.seed);
  w.put<int64_t>(C.b);
  w.put<int64_t>(C.pend_rows);
  w.put<int64_t>(C.pend_nnz);
  w.put<int32_t>(C.inject_left);
  w.put<int32_t>(C.opt.mode);
  const sfd_options& o = C.opt;
  w.put<double>(o.delta);
  w.put<int32_t>(o.verify);
  w.put<double>(o.c_q);
  w.put<int32_t>(o.q_override);
  w.put<int32_t>(o.retry_cap);
  w.put<int32_t>(o.precision);
  w.put<int32_t>(o.q_mode);
  w.put<int32_t>(o.strict);
  w.put<float>(o.q_margin);
  w.put<float>(o.q_tau);
  put_stats(w, C.st);
  // the sketch: B^T (d x ld) on the device -> B (l x d) through the Merger's staging
  Merger& M = *C.merger;
  transpose(M.B(), C.d, C.ell, M.ld, M.out, C.d, M.stream);
  std::vector<float> B((size_t)C.ell * C.d);
  SFD_CUDA(cudaMemcpyAsync(B.data(), M.out, B.size() * sizeof(float), cudaMemcpyDeviceToHost,
                           M.stream));
  SFD_CUDA(cudaStreamSynchronize(M.stream));
  w.bytes(B.data(), B.size() * sizeof(float));
  // the open buffer
  w.bytes(C.h_ptr.data(), (size_t)(C.pend_rows + 1) * sizeof(int));
  if (C.pend_nnz > 0) {
    Slot& S = *C.slots[C.fill];
    SFD_CUDA(cudaStreamSynchronize(S.stream));
    std::vector<int> idx(C.pend_nnz);
    std::vector<float> val(C.pend_nnz);
    SFD_CUDA(cudaMemcpy(idx.data(), S.csr.idx, idx.size() * sizeof(int), cudaMemcpyDeviceToHost));
    SFD_CUDA(cudaMemcpy(val.data(), S.csr.val, val.size() * sizeof(float), cudaMemcpyDeviceToHost));
    w.bytes(idx.data(), idx.size() * sizeof(int));
    w.bytes(val.data(), val.size() * sizeof(float));
  }
  if (C.has_qmodel) {
    std::vector<float> prm(kQParams);
    SFD_CUDA(cudaMemcpy(prm.data(), C.qparams, kQParams * sizeof(float), cudaMemcpyDeviceToHost));
    w.bytes(prm.data(), prm.size() * sizeof(float));
  }
  w.put<uint64_t>(fnv1a(buf.data(), buf.size()));
  return buf;
}

}  // namespace
}  // namespace sfd

using namespace sfd;

extern "C" {

int sfd_save(sfd_ctx* ctx, void* buf, int64_t cap, int64_t* size_out) {
  if (!ctx || !size_out || cap < 0) return SFD_EINVAL;
  Ctx& C = ctx->c;
  try {
    SFD_CUDA(cudaSetDevice(C.dev));
    std::vector<unsigned char> blob = serialize(C);
    *size_out = (int64_t)blob.size();
    if (!buf) return SFD_OK;
    if (cap < (int64_t)blob.size()) {
      C.last_error = "checkpoint buffer too small";
      return SFD_EINVAL;
    }
    memcpy(buf, blob.data(), blob.size());
    return SFD_OK;
  } catch (const CudaError& e) {
    C.last_error = std::string(e.where) + ": " + cudaGetErrorString(e.err);
    return SFD_ECUDA;
  } catch (const std::bad_alloc&) {
    return SFD_ENOMEM;
  }
}

int sfd_load(const void* buf, int64_t size, const sfd_options* runtime, sfd_ctx** out) {
  if (!buf || !out || size < (int64_t)(kHeaderBytes + 8)) return SFD_EINVAL;
  *out = nullptr;
  if (runtime && runtime->abi_version != SFD_ABI_VERSION) return SFD_EINVAL;
  const unsigned char* p = static_cast<const unsigned char*>(buf);
  uint64_t stored = 0;
  memcpy(&stored, p + size - 8, 8);
  if (fnv1a(p, (size_t)size - 8) != stored) return SFD_EINVAL;
  Reader r{p, (size_t)size - 8};
  const unsigned char* magic = r.take(8);
  if (!magic || memcmp(magic, kMagic, 8) != 0) return SFD_EINVAL;
  if (r.get<uint32_t>() != SFD_ABI_VERSION || r.get<uint32_t>() != kHeaderBytes) return SFD_EINVAL;
  const int64_t d = r.get<int64_t>();
  const int32_t ell = r.get<int32_t>();
  const int32_t has_q = r.get<int32_t>();
  const uint64_t seed = r.get<uint64_t>();
  const int64_t b = r.get<int64_t>();
  const int64_t prow = r.get<int64_t>(), pnnz = r.get<int64_t>();
  const int32_t inject = r.get<int32_t>();
  const int32_t mode = r.get<int32_t>();
  sfd_options o;
  sfd_options_init(&o);
  o.mode = mode;
  o.delta = r.get<double>();
  o.verify = r.get<int32_t>();
  o.c_q = r.get<double>();
  o.q_override = r.get<int32_t>();
  o.retry_cap = r.get<int32_t>();
  o.precision = r.get<int32_t>();
  o.q_mode = r.get<int32_t>();
  o.strict = r.get<int32_t>();
  o.q_margin = r.get<float>();
  o.q_tau = r.get<float>();
  sfd_stats st{};
  get_stats(r, st);
  if (!r.ok || d < 1 || ell < 1 || ell > d || b < 0 || prow < 0 || pnnz < 0 || prow >= d ||
      pnnz > (int64_t)ell * d + d)
    return SFD_EINVAL;
  if (runtime) {  // how the resumed context runs; never what it computes
    o.cuda_stream = runtime->cuda_stream;
    o.slots = runtime->slots;
    o.profile = runtime->profile;
    o.autotune = runtime->autotune;
  }
  o.inject_vs_fail = 0;
  const float* Bh = reinterpret_cast<const float*>(r.take((size_t)ell * d * sizeof(float)));
  const int* ptr = reinterpret_cast<const int*>(r.take((size_t)(prow + 1) * sizeof(int)));
  const int* idx = reinterpret_cast<const int*>(r.take((size_t)pnnz * sizeof(int)));
  const float* val = reinterpret_cast<const float*>(r.take((size_t)pnnz * sizeof(float)));
  const float* prm =
      has_q ? reinterpret_cast<const float*>(r.take(kQParams * sizeof(float))) : nullptr;
  if (!r.ok || r.at != r.n || !Bh || !ptr || (pnnz > 0 && (!idx || !val)) || (has_q && !prm))
    return SFD_EINVAL;
  if (ptr[0] != 0 || ptr[prow] != pnnz) return SFD_EINVAL;
  for (int64_t i = 0; i < prow; ++i)
    if (ptr[i + 1] < ptr[i] || ptr[i + 1] - ptr[i] > d) return SFD_EINVAL;
  for (int64_t i = 0; i < pnnz; ++i)
    if (idx[i] < 0 || idx[i] >= d || !std::isfinite(val[i])) return SFD_EINVAL;
  sfd_ctx* ctx = nullptr;
  int rc = sfd_create(d, ell, seed, &o, &ctx);
  if (rc != SFD_OK) return rc;
  Ctx& C = ctx->c;
  try {
    if (has_q && (rc = sfd_set_q_model(ctx, prm)) != SFD_OK) {
      sfd_destroy(ctx);
      return rc;
    }
    Merger& M = *C.merger;
    SFD_CUDA(cudaMemcpyAsync(M.out, Bh, (size_t)ell * d * sizeof(float), cudaMemcpyHostToDevice,
                             M.stream));
    transpose(M.out, ell, (int)d, (int)d, M.B(), M.ld, M.stream);
    SFD_CUDA(cudaStreamSynchronize(M.stream));
    C.h_ptr.assign(ptr, ptr + prow + 1);
    C.pend_rows = (int)prow;
    C.pend_nnz = pnnz;
    if (prow > 0) {  // the open buffer goes to the first slot, as a fresh stream's would
      C.fill = 0;
      C.next_slot = 1 % (int)C.slots.size();
      Slot& S = *C.slots[0];
      if (pnnz > 0) {
        SFD_CUDA(cudaMemcpy(S.csr.idx, idx, pnnz * sizeof(int), cudaMemcpyHostToDevice));
        SFD_CUDA(cudaMemcpy(S.csr.val, val, pnnz * sizeof(float), cudaMemcpyHostToDevice));
      }
    }
    C.b = b;
    C.inject_left = inject;
    C.st = st;
    C.st.pending_rows = prow;
    C.st.pending_nnz = pnnz;
  } catch (const CudaError&) {
    sfd_destroy(ctx);
    return SFD_ECUDA;
  }
  *out = ctx;
  return SFD_OK;
}

}  // extern "C"
