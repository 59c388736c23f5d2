// State of an SFD stream context (internal; the C ABI sees sfd_ctx as an
// opaque handle). Shared by the stream driver (api.cu) and the checkpoint
// code (checkpoint.cu).
#pragma once

#include <deque>
#include <memory>
#include <string>
#include <vector>

#include "engine.cuh"

namespace sfd {

constexpr int kDefaultSlots = 6;
constexpr int kMaxSlots = 8;
// power counts tried when labelling a buffer for the learned form
constexpr int kLadder[] = {1, 2, 3, 4, 6, 8, 11, 16, 23, 32, 45, 64};

struct Ctx {
  sfd_options opt;
  uint64_t seed = 0;
  int64_t d = 0;
  int ell = 0, ld = 0, dev = 0;
  std::vector<std::unique_ptr<Slot>> slots;
  std::unique_ptr<Merger> merger;
  cudaStream_t in_stream = nullptr;   // input staging and validation
  cudaEvent_t in_ready = nullptr;
  cudaEvent_t user_ev = nullptr;
  DevArena stage_arena;
  int* stage_idx = nullptr;
  float* stage_val = nullptr;
  int64_t stage_cap = 0;
  double* chk_fro2 = nullptr;
  int* chk_flags = nullptr;
  // open buffer
  int fill = -1;
  int pend_rows = 0;
  int64_t pend_nnz = 0;
  std::vector<int> h_ptr;
  // closed buffers whose verdict has not been read
  struct Pend {
    int slot;
    int64_t b;
    int m;
    int q;        // power count of the attempt in flight
    int r;
    int q_fixed;  // the schedule's q (used by retries)
  };
  std::deque<Pend> fifo;
  int next_slot = 0;
  int64_t b = 0;
  int inject_left = 0;
  // learned power count: network parameters (device) and the label log
  float* qparams = nullptr;
  bool has_qmodel = false;
  std::vector<float> qlog_feat, qlog_label;
  std::vector<int> qlog_qfixed;
  sfd_stats st{};
  std::string last_error;

  ~Ctx() {
    if (merger) cudaStreamSynchronize(merger->stream);
    for (auto& s : slots)
      if (s) cudaStreamSynchronize(s->stream);
    slots.clear();
    merger.reset();
    stage_arena.release();
    if (stage_idx) cudaFree(stage_idx);
    if (stage_val) cudaFree(stage_val);
    if (in_ready) cudaEventDestroy(in_ready);
    if (user_ev) cudaEventDestroy(user_ev);
    if (in_stream) cudaStreamDestroy(in_stream);
  }
};

}  // namespace sfd

struct sfd_ctx {
  sfd::Ctx c;
};
