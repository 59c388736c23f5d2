// Many SFD streams on one GPU (include/sfd.h, sfd_batch_*): independent
// stream contexts (Alg. 2 each), driven by worker threads so that their
// buffers' kernels overlap on the device, and a merge tree of DenseShrinks
// (Alg. 5; sketches are mergeable, Sec. 3.1) that folds them into one.
//
// Stream i is owned by worker i % workers, so the rows of one stream are
// processed in the order they were appended. Host arrays are copied when a
// call queues them; device arrays are read when the worker gets to them and
// must stay valid until sfd_batch_wait returns.
#include <string.h>

#include <algorithm>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "engine.cuh"

namespace {

struct Task {
  int stream = 0;
  int where = SFD_HOST;
  int64_t nrows = 0;
  std::vector<int64_t> ip;  // host copies
  std::vector<int32_t> ix;
  std::vector<float> v;
  const int64_t* dip = nullptr;  // device arrays (where == SFD_DEVICE)
  const int32_t* dix = nullptr;
  const float* dv = nullptr;
  // a merge task: ctx[stream] <- DenseShrink([ctx[stream]; ctx[src]])
  int merge_src = -1;
};

struct Worker {
  std::deque<Task> q;  // guarded by m
  std::mutex m;
  std::condition_variable cv;
  bool stop = false;   // guarded by m
  std::thread th;
};

}  // namespace

struct sfd_batch {
  std::vector<sfd_ctx*> ctx;
  std::vector<int64_t> d;
  std::vector<int32_t> ell;
  std::vector<Worker*> workers;
  std::mutex done_m;
  std::condition_variable done_cv;
  int64_t pending = 0;  // tasks queued and not finished (guarded by done_m)
  int error = SFD_OK;   // first error of a finished task (guarded by done_m)
  int dev = 0;
};

namespace {

void run_worker(sfd_batch* B, Worker* W) {
  cudaSetDevice(B->dev);
  for (;;) {
    Task t;
    {
      std::unique_lock<std::mutex> lk(W->m);
      W->cv.wait(lk, [&] { return W->stop || !W->q.empty(); });
      if (W->q.empty()) return;  // stopped and drained
      t = std::move(W->q.front());
      W->q.pop_front();
    }
    int rc;
    if (t.merge_src >= 0) {
      rc = sfd_merge(B->ctx[t.stream], B->ctx[t.merge_src]);
    } else if (t.where == SFD_HOST) {
      rc = sfd_append_rows(B->ctx[t.stream], t.nrows, t.ip.data(), t.ix.data(), t.v.data(),
                           SFD_HOST);
    } else {
      rc = sfd_append_rows(B->ctx[t.stream], t.nrows, t.dip, t.dix, t.dv, SFD_DEVICE);
    }
    {
      std::lock_guard<std::mutex> lk(B->done_m);
      if (rc != SFD_OK && B->error == SFD_OK) B->error = rc;
      B->pending--;
    }
    B->done_cv.notify_all();
  }
}

void enqueue(sfd_batch* B, int worker, Task&& t) {
  {
    std::lock_guard<std::mutex> lk(B->done_m);
    B->pending++;
  }
  Worker* W = B->workers[worker];
  {
    std::lock_guard<std::mutex> lk(W->m);
    W->q.push_back(std::move(t));
  }
  W->cv.notify_one();
}

// Wait until every queued task has finished; returns (and clears) the first error.
int wait_all(sfd_batch* B) {
  std::unique_lock<std::mutex> lk(B->done_m);
  B->done_cv.wait(lk, [&] { return B->pending == 0; });
  const int rc = B->error;
  B->error = SFD_OK;
  return rc;
}

void destroy(sfd_batch* B) {
  if (!B) return;
  for (Worker* W : B->workers) {
    {
      std::lock_guard<std::mutex> lk(W->m);
      W->stop = true;
    }
    W->cv.notify_all();
  }
  for (Worker* W : B->workers)
    if (W->th.joinable()) W->th.join();
  for (Worker* W : B->workers) delete W;
  for (sfd_ctx* c : B->ctx)
    if (c) sfd_destroy(c);
  delete B;
}

}  // namespace

extern "C" {

int sfd_batch_create(int32_t nstreams, const int64_t* d, const int32_t* ell, uint64_t seed,
                     const sfd_options* opt, int32_t workers, sfd_batch** out) {
  if (!out) return SFD_EINVAL;
  *out = nullptr;
  if (nstreams < 1 || !d || !ell || workers < 0) return SFD_EINVAL;
  sfd_options o;
  if (opt) o = *opt; else sfd_options_init(&o);
  if (o.abi_version != SFD_ABI_VERSION || o.cuda_stream) return SFD_EINVAL;
  if (o.slots == 0) o.slots = 1;  // many streams: one buffer in flight each by default
  sfd_batch* B = new (std::nothrow) sfd_batch();
  if (!B) return SFD_ENOMEM;
  cudaGetDevice(&B->dev);
  B->d.assign(d, d + nstreams);
  B->ell.assign(ell, ell + nstreams);
  B->ctx.assign(nstreams, nullptr);
  for (int i = 0; i < nstreams; ++i) {
    const int rc = sfd_create(d[i], ell[i], seed + (uint64_t)i, &o, &B->ctx[i]);
    if (rc != SFD_OK) {
      destroy(B);
      return rc;
    }
  }
  const int nw = workers > 0 ? std::min(workers, nstreams) : std::min(nstreams, 8);
  try {
    for (int w = 0; w < nw; ++w) {
      B->workers.push_back(new Worker());
      B->workers.back()->th = std::thread(run_worker, B, B->workers.back());
    }
  } catch (...) {
    destroy(B);
    return SFD_ENOMEM;
  }
  *out = B;
  return SFD_OK;
}

int sfd_batch_append(sfd_batch* B, int32_t stream, int64_t nrows, const int64_t* indptr,
                     const int32_t* indices, const float* values, int where) {
  if (!B || stream < 0 || stream >= (int32_t)B->ctx.size() || nrows < 0 ||
      (where != SFD_HOST && where != SFD_DEVICE) || (nrows > 0 && !indptr))
    return SFD_EINVAL;
  if (nrows == 0) return SFD_OK;
  Task t;
  t.stream = stream;
  t.where = where;
  t.nrows = nrows;
  if (where == SFD_HOST) {
    const int64_t base = indptr[0], total = indptr[nrows] - indptr[0];
    if (total < 0 || base < 0) return SFD_EINVAL;
    if (total > 0 && (!indices || !values)) return SFD_EINVAL;
    try {
      t.ip.resize(nrows + 1);
      for (int64_t i = 0; i <= nrows; ++i) t.ip[i] = indptr[i] - base;
      t.ix.assign(indices + (total > 0 ? base : 0), indices + (total > 0 ? base + total : 0));
      t.v.assign(values + (total > 0 ? base : 0), values + (total > 0 ? base + total : 0));
    } catch (const std::bad_alloc&) {
      return SFD_ENOMEM;
    }
  } else {
    t.dip = indptr;
    t.dix = indices;
    t.dv = values;
  }
  enqueue(B, stream % (int)B->workers.size(), std::move(t));
  return SFD_OK;
}

int sfd_batch_wait(sfd_batch* B) {
  if (!B) return SFD_EINVAL;
  return wait_all(B);
}

int sfd_batch_sketch(sfd_batch* B, int32_t stream, float* B_out, int where) {
  if (!B || stream < 0 || stream >= (int32_t)B->ctx.size()) return SFD_EINVAL;
  const int rc = wait_all(B);
  if (rc != SFD_OK) return rc;
  return sfd_sketch(B->ctx[stream], B_out, where);
}

int sfd_batch_merge_tree(sfd_batch* B, float* B_out, int where) {
  if (!B) return SFD_EINVAL;
  const int n = (int)B->ctx.size();
  for (int i = 1; i < n; ++i)
    if (B->d[i] != B->d[0] || B->ell[i] != B->ell[0]) return SFD_EINVAL;
  int rc = wait_all(B);
  if (rc != SFD_OK) return rc;
  for (int step = 1; step < n; step *= 2) {  // level: pairs (i, i + step), i a multiple of 2 step
    int k = 0;
    for (int i = 0; i + step < n; i += 2 * step, ++k) {
      Task t;
      t.stream = i;
      t.merge_src = i + step;
      enqueue(B, k % (int)B->workers.size(), std::move(t));
    }
    rc = wait_all(B);
    if (rc != SFD_OK) return rc;
  }
  return B_out ? sfd_sketch(B->ctx[0], B_out, where) : SFD_OK;
}

int sfd_batch_stats(const sfd_batch* B, int32_t stream, sfd_stats* out) {
  if (!B || !out || stream < 0 || stream >= (int32_t)B->ctx.size()) return SFD_EINVAL;
  return sfd_get_stats(B->ctx[stream], out);
}

void sfd_batch_destroy(sfd_batch* B) { destroy(B); }

}  // extern "C"
