// Tensor-core (tcgen05, kind::tf32) forms of the two dense products of
// CholeskyQR inside SimultaneousIteration (Alg. 1): the Gram X^T X and the
// tall-skinny product X T, for blocks of at most 128 columns.
//
// Operands are staged by the CTA's threads into shared memory in the K-major
// canonical layout without swizzle: core matrices of 8 rows x 16 bytes
// (4 tf32 along K); element (r, k) of an R x K tile sits at byte
//   ((r / 8) * (K / 4) + k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4,
// so the descriptor's leading byte offset (next core along K) is 128 and its
// stride byte offset (next 8 rows) is K * 32. One thread issues the MMAs
// (M = 128, K = 8 each), the accumulator lives in tensor memory, and the
// epilogue reads it back with tcgen05.ld. Every mbarrier wait is bounded: on
// expiry the kernel sets flags[2], waits once more (bounded), frees its tensor
// memory and returns.
#include <algorithm>
#include <atomic>
#include <cstdint>

#include <cuda_fp16.h>

#include "sfd_internal.cuh"

namespace sfd {
namespace {

constexpr int kTcThreads = 128;
// A try_wait that finds its phase incomplete suspends the thread for about
// 3.9 us on GB300 (measured with k_wait_selftest), so 2^18 tries bound a
// wait at about one second; copies and MMAs complete within microseconds.
constexpr uint32_t kSpinLimit = 1u << 18;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version bits 46-48 = 0b001
  return d;
}

// Instruction descriptor: f32 accumulate, tf32 A and B, both K-major.
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ int core_off(int r, int k, int K) {  // in floats
  return (((r >> 3) * (K >> 2) + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4) >> 2;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_u32(mbar)));
}

// The first waits of every stage (a copy landed, an MMA done) take their
// iteration limit as a kernel argument (wl), kSpinLimit unless
// sfd_set_wait_limit changed it for tests (0: such a wait gives up at once).
// The waits that drain a failed stage (mbar_drain) keep kSpinLimit, so a CTA
// never releases shared or tensor memory with a copy or an MMA of its own
// still in flight.

__device__ __forceinline__ bool mbar_wait_n(uint64_t* mbar, uint32_t parity, uint32_t limit) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity));
  }
  return done != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t limit) {
  return mbar_wait_n(mbar, parity, limit);
}

__device__ __forceinline__ bool mbar_drain(uint64_t* mbar, uint32_t parity) {
  return mbar_wait_n(mbar, parity, kSpinLimit);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::);
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::);
}

__device__ __forceinline__ void tmem_free(uint32_t tmem, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

// Asynchronous global -> shared copies (cp.async): bytes beyond src_bytes are
// zero-filled, and src_bytes = 0 reads nothing.
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
               "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N));
}

// ------------------------------------------------------------------ Gram
// partial[chunk] (128 x 128 row-major; only the leading n x n block is
// written) = X[rows of chunk, 0:n]^T X[rows of chunk, 0:n]. Rows are staged
// 32 at a time (K = 32: four MMAs) through a ring of kGSt buffers filled by
// cp.async kGLook stages ahead of the MMAs. A buffer is refilled once the MMAs
// that read it have completed (its mbarrier); those were issued two stages
// earlier, so the wait rarely blocks. Element (m, k) of a stage is
// X[row k][column m], four consecutive rows per 16-byte core row.
constexpr int kGK = 32;             // rows per stage
constexpr int kGTile = 128 * kGK;   // floats per stage
constexpr int kGramChunks = 152;
// SPLIT (the fp32-accurate form): every value x is split into x_hi (x with
// the 13 low mantissa bits cleared, exactly a TF32 number) and x_lo = x - x_hi
// (exact in fp32), and X^T X is accumulated as hi^T hi + hi^T lo + lo^T hi:
// about 21 significant bits instead of TF32's 11.
template <bool SPLIT>
struct GramRing {
  static constexpr int St = SPLIT ? 4 : 6;  // stages in the ring
  static constexpr int Look = St - 2;       // stages loaded ahead of the MMAs
  static constexpr int Smem = St * kGTile * (SPLIT ? 2 : 1) * (int)sizeof(float);  // 128 / 96 KB
};

__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xffffe000u);
}

template <bool SPLIT>
__global__ void __launch_bounds__(kTcThreads)
    k_tc_gram(const float* __restrict__ X, int ldx, int n, int64_t rows, int64_t rows_per_chunk,
              float* __restrict__ partial, uint32_t wl, int* __restrict__ flags) {
  constexpr int kGSt = GramRing<SPLIT>::St;
  constexpr int kGLook = GramRing<SPLIT>::Look;
  extern __shared__ __align__(1024) float smem[];
  __shared__ __align__(8) uint64_t mbar[kGSt];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc(&tmem_slot, 128);
  if (tid == 0) {
    for (int b = 0; b < kGSt; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[b])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::);
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_tf32(128, 128);
  const int64_t r_beg = (int64_t)blockIdx.x * rows_per_chunk;
  const int64_t r_end = min(rows, r_beg + rows_per_chunk);
  const int nst = r_end > r_beg ? (int)((r_end - r_beg + kGK - 1) / kGK) : 0;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t lo_base = sbase + (uint32_t)(kGSt * kGTile) * 4u;  // SPLIT: the lo ring
  // thread tid copies column m = tid of the 32 rows of a stage
  const int m = tid;
  auto issue = [&](int st) {
    const int64_t r0 = r_beg + (int64_t)st * kGK;
    const uint32_t dst = sbase + (uint32_t)((st % kGSt) * kGTile) * 4u;
#pragma unroll
    for (int k = 0; k < kGK; ++k) {
      const int64_t g = r0 + k;
      const bool ok = g < r_end && m < n;
      cp_async4(dst + (uint32_t)core_off(m, k, kGK) * 4u, ok ? (const void*)(X + g * ldx + m) : X,
                ok ? 4u : 0u);
    }
  };
  uint32_t phase_bits = 0, used_bits = 0;
  bool ok = true;
#pragma unroll
  for (int st = 0; st < kGLook; ++st) {
    if (st < nst) issue(st);
    cp_async_commit();
  }
  for (int st = 0; st < nst; ++st) {
    const int ns = st + kGLook;
    if (ns < nst) {
      const int b = ns % kGSt;
      if (used_bits & (1u << b)) {  // the MMAs that read this buffer must be done
        const bool w = mbar_wait(&mbar[b], (phase_bits >> b) & 1u, wl);
        if (!__syncthreads_and(w)) { ok = false; break; }
        phase_bits ^= 1u << b;
        used_bits &= ~(1u << b);
      }
      issue(ns);
    }
    cp_async_commit();
    cp_async_wait<kGLook>();  // this thread's copies of stage st have landed
    const int b = st % kGSt;
    if (SPLIT) {  // split the elements this thread copied: hi in place, lo in the lo ring
      // (four consecutive k of a column are one 16-byte core row: float4)
      float* hi = smem + b * kGTile;
      float* lo = smem + (kGSt + b) * kGTile;
#pragma unroll
      for (int k = 0; k < kGK; k += 4) {
        const int o = core_off(m, k, kGK);
        const float4 x = *reinterpret_cast<const float4*>(hi + o);
        const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
        *reinterpret_cast<float4*>(hi + o) = h;
        *reinterpret_cast<float4*>(lo + o) = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::);
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::);
      const uint32_t base = sbase + (uint32_t)(b * kGTile) * 4u;
      const uint32_t lbase = lo_base + (uint32_t)(b * kGTile) * 4u;
#pragma unroll
      for (int kk = 0; kk < kGK / 8; ++kk) {
        const uint64_t da = smem_desc(base + kk * 256, 128, kGK * 32);
        mma_tf32(tmem, da, da, idesc, (st > 0 || kk > 0) ? 1u : 0u);
        if (SPLIT) {
          const uint64_t dl = smem_desc(lbase + kk * 256, 128, kGK * 32);
          mma_tf32(tmem, da, dl, idesc, 1u);
          mma_tf32(tmem, dl, da, idesc, 1u);
        }
      }
      mma_commit(&mbar[b]);
    }
    used_bits |= 1u << b;
  }
  cp_async_wait<0>();
  if (ok) {
    // every commit not yet waited for (one per buffer in use), so that no
    // mbarrier arrival can land after the CTA has released its shared memory
    bool all = true;
    for (int b = 0; b < kGSt; ++b)
      if (used_bits & (1u << b)) all = mbar_wait(&mbar[b], (phase_bits >> b) & 1u, wl) && all;
    ok = __syncthreads_and(all);
    if (ok) used_bits = 0;
  }
  if (!ok) {
    if (tid == 0) atomicOr(&flags[2], 1);
    for (int b = 0; b < kGSt; ++b)  // bounded: let MMAs in flight finish before freeing
      if (used_bits & (1u << b)) mbar_drain(&mbar[b], (phase_bits >> b) & 1u);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::);
  __syncthreads();
  float* out = partial + (int64_t)blockIdx.x * (128 * 128);
  const int row = warp * 32 + lane;
  const bool have = ok && nst > 0;
  for (int c0 = 0; c0 < n; c0 += 16) {
    float v[16];
    if (have) {
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = 0.f;
    }
    if (row < n) {
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        *reinterpret_cast<float4*>(&out[row * 128 + c0 + j]) =
            make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::);
  __syncthreads();
  if (warp == 0) tmem_free(tmem, 128);
}

// ------------------------------------------------------ Gram, bulk copies
// The same partial Grams as k_tc_gram for a block whose rows start on 16-byte
// boundaries (ldx % 4 == 0, X 16-byte aligned), so that the kGK rows of a
// stage are one contiguous run of memory: thread 0 moves each stage with a
// single bulk copy (the TMA engine, cp.async.bulk with an mbarrier completing
// on the byte count) into a ring of kBR raw stages, kept kBR - 1 stages
// ahead. Each thread then transposes its column of a landed stage into the
// K-major core layout of the MMA ring (two buffers, reused once the MMAs that
// read them have completed), so the per-element copies of k_tc_gram become
// one instruction per stage plus shared-memory moves.
constexpr int kBR = 6;  // raw stages in flight
constexpr int kGramThreads = 256;
template <bool SPLIT>
struct GramBulk {
  static constexpr int Raw = kGK * 128;                          // floats per raw stage (ldx <= 128)
  static constexpr int Core = kGTile * (SPLIT ? 2 : 1);          // floats per MMA buffer
  static constexpr int Smem = (kBR * Raw + 2 * Core) * (int)sizeof(float);  // 128 / 160 KB
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
               "r"(bytes));
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(smem_u32(mbar))
      : "memory");
}

template <bool SPLIT>
__global__ void __launch_bounds__(kGramThreads)
    k_tc_gram_bulk(const float* __restrict__ X, int ldx, int n, int64_t rows,
                   int64_t rows_per_chunk, float* __restrict__ partial, uint32_t wl, int* __restrict__ flags) {
  using G = GramBulk<SPLIT>;
  extern __shared__ __align__(1024) float smem[];
  float* raw = smem;                  // kBR x (kGK x ldx), row-major as in memory
  float* core = smem + kBR * G::Raw;  // 2 MMA buffers: hi (and lo)
  __shared__ __align__(8) uint64_t full[kBR];   // raw stage landed
  __shared__ __align__(8) uint64_t mmad[2];     // MMAs of a core buffer done
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc(&tmem_slot, 128);
  if (tid == 0) {
    for (int b = 0; b < kBR; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[b])), "r"(1));
    for (int b = 0; b < 2; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mmad[b])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::);
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_tf32(128, 128);
  const int64_t r_beg = (int64_t)blockIdx.x * rows_per_chunk;
  const int64_t r_end = min(rows, r_beg + rows_per_chunk);
  const int nst = r_end > r_beg ? (int)((r_end - r_beg + kGK - 1) / kGK) : 0;
  const uint32_t raw_s = smem_u32(raw), core_s = smem_u32(core);
  auto issue = [&](int st) {  // thread 0: stage st into raw buffer st % kBR
    const int64_t r0 = r_beg + (int64_t)st * kGK;
    const int nr = (int)min((int64_t)kGK, r_end - r0);
    const uint32_t bytes = (uint32_t)nr * (uint32_t)ldx * 4u;
    uint64_t* mb = &full[st % kBR];
    mbar_expect_tx(mb, bytes);
    bulk_g2s(raw_s + (uint32_t)((st % kBR) * G::Raw) * 4u, X + r0 * ldx, bytes, mb);
  };
  if (tid == 0)
    for (int st = 0; st < kBR - 1 && st < nst; ++st) issue(st);
  // stage s is use s / kBR of raw buffer s % kBR and commit s / 2 of MMA
  // buffer s % 2, so the parities of their mbarrier phases are known
  int st_fail = nst;
  // this thread's column, and which half of a stage's rows it transposes
  const int m = tid & 127, k_lo = (tid >> 7) * (kGK / 2);
  for (int st = 0; st < nst; ++st) {
    const int rb = st % kBR, cb = st & 1;
    const bool w1 = mbar_wait(&full[rb], (uint32_t)((st / kBR) & 1), wl);  // the raw stage landed
    // the MMAs of stage st - 2, which read this MMA buffer, are done
    const bool w2 = st < 2 || mbar_wait(&mmad[cb], (uint32_t)(((st - 2) >> 1) & 1), wl);
    if (!__syncthreads_and(w1 && w2)) { st_fail = st; break; }
    const int nr = (int)min((int64_t)kGK, r_end - (r_beg + (int64_t)st * kGK));
    const float* rs = raw + rb * G::Raw;
    float* hi = core + cb * G::Core;
    float* lo = hi + kGTile;
#pragma unroll
    for (int k = k_lo; k < k_lo + kGK / 2; k += 4) {
      float4 x;
      x.x = (k + 0 < nr && m < n) ? rs[(k + 0) * ldx + m] : 0.f;
      x.y = (k + 1 < nr && m < n) ? rs[(k + 1) * ldx + m] : 0.f;
      x.z = (k + 2 < nr && m < n) ? rs[(k + 2) * ldx + m] : 0.f;
      x.w = (k + 3 < nr && m < n) ? rs[(k + 3) * ldx + m] : 0.f;
      const int o = core_off(m, k, kGK);
      if (SPLIT) {
        const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
        *reinterpret_cast<float4*>(hi + o) = h;
        *reinterpret_cast<float4*>(lo + o) = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
      } else {
        *reinterpret_cast<float4*>(hi + o) = x;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::);
    __syncthreads();  // raw buffer rb is free, the MMA buffer is written
    if (tid == 0) {
      if (st + kBR - 1 < nst) issue(st + kBR - 1);  // into the buffer of stage st - 1
      asm volatile("tcgen05.fence::after_thread_sync;" ::);
      const uint32_t base = core_s + (uint32_t)(cb * G::Core) * 4u;
      const uint32_t lbase = base + (uint32_t)kGTile * 4u;
#pragma unroll
      for (int kk = 0; kk < kGK / 8; ++kk) {
        const uint64_t da = smem_desc(base + kk * 256, 128, kGK * 32);
        mma_tf32(tmem, da, da, idesc, (st > 0 || kk > 0) ? 1u : 0u);
        if (SPLIT) {
          const uint64_t dl = smem_desc(lbase + kk * 256, 128, kGK * 32);
          mma_tf32(tmem, da, dl, idesc, 1u);
          mma_tf32(tmem, dl, da, idesc, 1u);
        }
      }
      mma_commit(&mmad[cb]);
    }
  }
  bool ok = st_fail == nst;
  if (ok) {
    bool all = true;  // the last commit of each MMA buffer
    for (int s2 = max(0, nst - 2); s2 < nst; ++s2)
      all = mbar_wait(&mmad[s2 & 1], (uint32_t)((s2 >> 1) & 1), wl) && all;
    ok = __syncthreads_and(all);
  }
  if (!ok) {
    if (tid == 0) atomicOr(&flags[2], 1);
    // draining waits: the MMAs committed and the bulk copies issued finish
    // before the shared memory and tensor memory are released (every copy
    // up to stage nst - 1 has landed when the loop ran to the end)
    for (int s2 = max(0, st_fail - 2); s2 < st_fail; ++s2)
      mbar_drain(&mmad[s2 & 1], (uint32_t)((s2 >> 1) & 1));
    for (int s2 = st_fail; s2 < min(nst, st_fail + kBR - 1); ++s2)
      mbar_drain(&full[s2 % kBR], (uint32_t)((s2 / kBR) & 1));
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::);
  __syncthreads();
  float* out = partial + (int64_t)blockIdx.x * (128 * 128);
  // warps w and w + 4 read lane quarter w % 4 of tensor memory, each half of
  // the 16-column chunks
  const int q4 = warp & 3, row = q4 * 32 + lane;
  const int nch = (n + 15) >> 4, ch_mid = (nch + 1) >> 1;
  const bool have = ok && nst > 0;
  for (int c0 = (warp < 4 ? 0 : ch_mid) * 16; c0 < (warp < 4 ? ch_mid : nch) * 16; c0 += 16) {
    float v[16];
    if (have) {
      tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + c0, v);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = 0.f;
    }
    if (row < n) {
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        *reinterpret_cast<float4*>(&out[row * 128 + c0 + j]) =
            make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::);
  __syncthreads();
  if (warp == 0) tmem_free(tmem, 128);
}

// ------------------------------------------------------- wait self-test
// A wait that nothing ends: one CTA waits, with the given iteration limit, on
// an mbarrier that no thread and no copy ever arrives at. The wait gives up,
// the timeout flag is raised and the kernel returns; nothing is in flight, so
// the context stays usable. Tests use it to see the bound work and to time it.
__global__ void k_wait_selftest(uint32_t limit, int* __restrict__ flags) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::);
  }
  __syncthreads();
  const bool ok = mbar_wait_n(&mbar, 0u, limit);  // phase 0 never completes
  if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicOr(&flags[2], 1);
}

// ----------------------------------------------------------- cross Gram
// For two blocks X1 (rows x n1) and X2 (rows x n2) whose columns are known to
// be mutually orthogonal within each block (the rows of a sketch B, and of
// the B' of SparseShrink, are orthogonal by construction, Alg. 3 and Alg. 5),
// the Gram of [X1 X2] has diagonal diagonal blocks. This kernel forms the
// cross block X1^T X2 in the split TF32 form and the squared column norms
// of both blocks (the diagonals), per chunk of rows: partial[chunk] holds
// the 128 x 128 cross block, then 128 norms of X1, then 128 norms of X2.
// Rows are staged kXK = 16 at a time; a stage holds hi and lo of both tiles.
constexpr int kXK = 16;
constexpr int kXTile = 128 * kXK;  // floats per tile
constexpr int kXSt = 6;            // stages in the ring
constexpr int kXLook = kXSt - 2;
constexpr int kXSmem = kXSt * 4 * kXTile * (int)sizeof(float);  // 192 KB
constexpr int kXPartial = 128 * 128 + 256;                      // floats per chunk

__global__ void __launch_bounds__(kTcThreads)
    k_tc_cross(const float* __restrict__ X1, int ld1, int n1, const float* __restrict__ X2,
               int ld2, int n2, int64_t rows, int64_t rows_per_chunk, float* __restrict__ partial,
               uint32_t wl, int* __restrict__ flags) {
  extern __shared__ __align__(1024) float smem[];
  __shared__ __align__(8) uint64_t mbar[kXSt];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc(&tmem_slot, 128);
  if (tid == 0) {
    for (int b = 0; b < kXSt; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[b])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::);
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_tf32(128, 128);
  const int64_t r_beg = (int64_t)blockIdx.x * rows_per_chunk;
  const int64_t r_end = min(rows, r_beg + rows_per_chunk);
  const int nst = r_end > r_beg ? (int)((r_end - r_beg + kXK - 1) / kXK) : 0;
  const uint32_t sbase = smem_u32(smem);
  // stage b: tiles hi1, lo1, hi2, lo2 at b * 4 * kXTile + {0, 1, 2, 3} * kXTile
  const int m = tid;  // thread m copies (and splits) column m of both tiles
  auto issue = [&](int st) {
    const int64_t r0 = r_beg + (int64_t)st * kXK;
    const uint32_t dst = sbase + (uint32_t)((st % kXSt) * 4 * kXTile) * 4u;
#pragma unroll
    for (int k = 0; k < kXK; ++k) {
      const int64_t g = r0 + k;
      const bool in = g < r_end;
      const bool ok1 = in && m < n1, ok2 = in && m < n2;
      const uint32_t o = (uint32_t)core_off(m, k, kXK) * 4u;
      cp_async4(dst + o, ok1 ? (const void*)(X1 + g * ld1 + m) : X1, ok1 ? 4u : 0u);
      cp_async4(dst + (uint32_t)(2 * kXTile) * 4u + o, ok2 ? (const void*)(X2 + g * ld2 + m) : X2,
                ok2 ? 4u : 0u);
    }
  };
  float sq1 = 0.f, sq2 = 0.f;  // this thread's column norms, rows in order
  uint32_t phase_bits = 0, used_bits = 0;
  bool ok = true;
#pragma unroll
  for (int st = 0; st < kXLook; ++st) {
    if (st < nst) issue(st);
    cp_async_commit();
  }
  for (int st = 0; st < nst; ++st) {
    const int ns = st + kXLook;
    if (ns < nst) {
      const int b = ns % kXSt;
      if (used_bits & (1u << b)) {  // the MMAs that read this buffer must be done
        const bool w = mbar_wait(&mbar[b], (phase_bits >> b) & 1u, wl);
        if (!__syncthreads_and(w)) { ok = false; break; }
        phase_bits ^= 1u << b;
        used_bits &= ~(1u << b);
      }
      issue(ns);
    }
    cp_async_commit();
    cp_async_wait<kXLook>();  // this thread's copies of stage st have landed
    const int b = st % kXSt;
    float* t = smem + b * 4 * kXTile;
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {  // X1 then X2: hi in place, lo next to it
      float* hi = t + blk * 2 * kXTile;
      float* lo = hi + kXTile;
      float sq = 0.f;
#pragma unroll
      for (int k = 0; k < kXK; k += 4) {
        const int o = core_off(m, k, kXK);
        const float4 x = *reinterpret_cast<const float4*>(hi + o);
        sq = fmaf(x.x, x.x, sq);
        sq = fmaf(x.y, x.y, sq);
        sq = fmaf(x.z, x.z, sq);
        sq = fmaf(x.w, x.w, sq);
        const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
        *reinterpret_cast<float4*>(hi + o) = h;
        *reinterpret_cast<float4*>(lo + o) = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
      }
      if (blk == 0) sq1 += sq;
      else sq2 += sq;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::);
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::);
      const uint32_t base = sbase + (uint32_t)(b * 4 * kXTile) * 4u;
#pragma unroll
      for (int kk = 0; kk < kXK / 8; ++kk) {
        const uint64_t d1h = smem_desc(base + kk * 256, 128, kXK * 32);
        const uint64_t d1l = smem_desc(base + (uint32_t)kXTile * 4u + kk * 256, 128, kXK * 32);
        const uint64_t d2h = smem_desc(base + (uint32_t)(2 * kXTile) * 4u + kk * 256, 128, kXK * 32);
        const uint64_t d2l = smem_desc(base + (uint32_t)(3 * kXTile) * 4u + kk * 256, 128, kXK * 32);
        mma_tf32(tmem, d1h, d2h, idesc, (st > 0 || kk > 0) ? 1u : 0u);
        mma_tf32(tmem, d1h, d2l, idesc, 1u);
        mma_tf32(tmem, d1l, d2h, idesc, 1u);
      }
      mma_commit(&mbar[b]);
    }
    used_bits |= 1u << b;
  }
  cp_async_wait<0>();
  if (ok) {
    bool all = true;
    for (int b = 0; b < kXSt; ++b)
      if (used_bits & (1u << b)) all = mbar_wait(&mbar[b], (phase_bits >> b) & 1u, wl) && all;
    ok = __syncthreads_and(all);
    if (ok) used_bits = 0;
  }
  if (!ok) {
    if (tid == 0) atomicOr(&flags[2], 1);
    for (int b = 0; b < kXSt; ++b)  // bounded: let MMAs in flight finish before freeing
      if (used_bits & (1u << b)) mbar_drain(&mbar[b], (phase_bits >> b) & 1u);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::);
  __syncthreads();
  float* out = partial + (int64_t)blockIdx.x * kXPartial;
  const int row = warp * 32 + lane;
  const bool have = ok && nst > 0;
  for (int c0 = 0; c0 < n2; c0 += 16) {
    float v[16];
    if (have) {
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = 0.f;
    }
    if (row < n1) {
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        *reinterpret_cast<float4*>(&out[row * 128 + c0 + j]) =
            make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    }
  }
  out[128 * 128 + m] = have ? sq1 : 0.f;
  out[128 * 128 + 128 + m] = have ? sq2 : 0.f;
  asm volatile("tcgen05.fence::before_thread_sync;" ::);
  __syncthreads();
  if (warp == 0) tmem_free(tmem, 128);
}

// G ((n1 + n2) x (n1 + n2), row-major) from the chunk partials of k_tc_cross:
// one thread per entry of the first n1 rows (mirrored into the first n1
// columns) and per entry of the last n2 x n2 block; chunks summed in order.
__global__ void k_cross_reduce(const float* __restrict__ partial, int nchunks, int n1, int n2,
                               float* __restrict__ G) {
  const int N = n1 + n2;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t top = (int64_t)n1 * N;
  if (e >= top + (int64_t)n2 * n2) return;
  int i, j, off;
  bool zero = false;
  if (e < top) {
    i = (int)(e / N);
    j = (int)(e % N);
    if (j < n1) {
      zero = i != j;
      off = 128 * 128 + i;
    } else {
      off = i * 128 + (j - n1);
    }
  } else {
    const int64_t f = e - top;
    i = n1 + (int)(f / n2);
    j = n1 + (int)(f % n2);
    zero = i != j;
    off = 128 * 128 + 128 + (i - n1);
  }
  float s0 = 0.f, s1 = 0.f;
  if (!zero) {
    int ch = 0;
    for (; ch + 1 < nchunks; ch += 2) {
      s0 += partial[(int64_t)ch * kXPartial + off];
      s1 += partial[(int64_t)(ch + 1) * kXPartial + off];
    }
    if (ch < nchunks) s0 += partial[(int64_t)ch * kXPartial + off];
  }
  const float g = s0 + s1;
  G[(int64_t)i * N + j] = g;
  if (e < top && j >= n1) G[(int64_t)j * N + i] = g;
}

// ----------------------------------------------------------------- X * T
// Y[rows, 0:kout] = X[rows, 0:n] T (T: n x kout, row-major). T^T (Np x Kp,
// n padded to Kp = 8j, kout to Np = 16j) is staged once per CTA. Each CTA
// owns one contiguous range of rows_per_cta rows, cut into 128-row tiles
// that go through NB cp.async buffers: the first NB tiles are all requested
// before the first MMA (for 50,000 rows of l = 100 on 152 SMs,
// that is the CTA's whole range), and a buffer takes the tile NB further on
// once the MMAs that read it have completed. Each tile is multiplied (Kp / 8
// MMAs) and written back from tensor memory while the later tiles are still
// landing. Eight warps: the index arithmetic of the copies has no divisions,
// and in the write-back warps w and w + 4 share the 32 rows of tensor-memory
// lane quarter w % 4, each taking half of the columns. VEC: X rows start
// 16-byte aligned (ldx % 4 == 0), so each 16-byte core row is one copy;
// otherwise element by element. Rows past the range are zero-filled and not
// written.
constexpr int kGemmThreads = 256;
constexpr size_t kGemmSmemMax = 220 * 1024;  // dynamic shared memory of one k_tc_gemm CTA

template <bool VEC, int NB>
__global__ void __launch_bounds__(kGemmThreads)
    k_tc_gemm(const float* __restrict__ X, int ldx, int n, int64_t rows, int64_t rows_per_cta,
              const float* __restrict__ T, int kout, int Kp, int Np, float* __restrict__ Y,
              int ldy, __half* __restrict__ Yh, uint32_t wl, int* __restrict__ flags) {
  extern __shared__ __align__(1024) float smem[];
  float* Bs = smem;  // Np x Kp, then NB tiles of 128 x Kp
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kc_n = Kp >> 2;  // 16-byte chunks along K (at most 32)
  const uint32_t sB = smem_u32(Bs);
  const uint32_t sA0 = sB + (uint32_t)(Np * Kp) * 4u;
  const uint32_t tile_bytes = (uint32_t)(128 * Kp) * 4u;
  const int64_t r_beg = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = min(rows, r_beg + rows_per_cta);
  const int ntile = r_end > r_beg ? (int)((r_end - r_beg + 127) / 128) : 0;
  if (warp == 0) tmem_alloc(&tmem_slot, 128);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::);
  }
  auto issue = [&](int t) {  // tile t of this CTA into buffer t % NB
    const int64_t row0 = r_beg + (int64_t)t * 128;
    const uint32_t dst = sA0 + (uint32_t)(t % NB) * tile_bytes;
    if (VEC) {
      // thread: row tid % 8 of each core matrix, 16-byte chunk tid / 8 along
      // K; a warp moves 8 rows x 64 contiguous bytes into 4 core matrices
      const int r_lo = tid & 7, kc = tid >> 3;
      if (kc < kc_n) {
        const int nval = max(0, min(4, n - kc * 4));
        const float* src = X + (row0 + r_lo) * ldx + kc * 4;
        uint32_t d = dst + (uint32_t)(kc * 128 + r_lo * 16);
#pragma unroll 4
        for (int rg = 0; rg < 16; ++rg, src += 8 * (int64_t)ldx, d += (uint32_t)kc_n * 128u) {
          const bool in = row0 + rg * 8 + r_lo < r_end && nval > 0;
          cp_async16(d, in ? (const void*)src : X, in ? (uint32_t)nval * 4u : 0u);
        }
      }
    } else {
      for (int i = tid; i < 128 * Kp; i += kGemmThreads) {
        const int r = i / Kp, k = i % Kp;
        const int64_t g = row0 + r;
        const bool ok = g < r_end && k < n;
        cp_async4(dst + (uint32_t)core_off(r, k, Kp) * 4u, ok ? (const void*)(X + g * ldx + k) : X,
                  ok ? 4u : 0u);
      }
    }
  };
  // B(j, k) = T[k][j], zero past n and kout, by 4-byte asynchronous copies
  // (joining tile 0's group): thread takes columns 4 jq..4 jq + 3 of rows
  // k = tid / 32 + 8 i, so a warp reads 128 consecutive floats of a row
  {
    const int jq = tid & 31;
    if (jq * 4 < Np) {
      for (int k = tid >> 5; k < Kp; k += kGemmThreads / 32) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = jq * 4 + q;
          const bool in = k < n && j < kout;
          cp_async4(sB + (uint32_t)core_off(j, k, Kp) * 4u,
                    in ? (const void*)(T + (int64_t)k * kout + j) : T, in ? 4u : 0u);
        }
      }
    }
  }
  // one commit group per tile (empty past the last): before tile t's MMAs,
  // t + NB groups are committed, so waiting until at most NB - 1 are pending
  // means groups 0..t (and B) have landed
#pragma unroll
  for (int t = 0; t < NB; ++t) {
    if (t < ntile) issue(t);
    cp_async_commit();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::);
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_tf32(128, Np);
  const bool vec_out = (ldy & 3) == 0 && ((uintptr_t)Y & 15) == 0;
  const int nch = Np >> 4, ch_mid = (nch + 1) >> 1;
  const int ch_lo = warp < 4 ? 0 : ch_mid, ch_hi = warp < 4 ? ch_mid : nch;
  const int q4 = warp & 3;  // tensor-memory lane quarter of this warp
  uint32_t phase = 0;
  bool ok = true;
  for (int t = 0; t < ntile; ++t) {
    cp_async_wait<NB - 1>();
    asm volatile("fence.proxy.async.shared::cta;" ::);
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::);
      const uint32_t a0 = sA0 + (uint32_t)(t % NB) * tile_bytes;
      for (int kk = 0; kk < Kp / 8; ++kk) {
        const uint64_t da = smem_desc(a0 + kk * 256, 128, Kp * 32);
        const uint64_t db = smem_desc(sB + kk * 256, 128, Kp * 32);
        mma_tf32(tmem, da, db, idesc, kk > 0 ? 1u : 0u);
      }
      mma_commit(&mbar);
    }
    if (!__syncthreads_and(mbar_wait(&mbar, phase, wl))) {
      ok = false;
      break;
    }
    phase ^= 1u;
    // the MMAs that read buffer t % NB are done: it takes tile t + NB
    if (t + NB < ntile) issue(t + NB);
    cp_async_commit();
    asm volatile("tcgen05.fence::after_thread_sync;" ::);
    const int64_t g = r_beg + (int64_t)t * 128 + q4 * 32 + lane;
    for (int ch = ch_lo; ch < ch_hi; ++ch) {
      const int c0 = ch * 16;
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + c0, v);
      if (g < r_end && Yh) {  // fp16 copy only (|entries| <= 1: columns are orthonormal)
        __half* y = Yh + g * ldy + c0;
#pragma unroll
        for (int j = 0; j < 16; j += 8) {
          __half2 h[4];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            h[q] = __floats2half2_rn(c0 + j + 2 * q < kout ? v[j + 2 * q] : 0.f,
                                     c0 + j + 2 * q + 1 < kout ? v[j + 2 * q + 1] : 0.f);
          if (c0 + j + 8 <= ldy) *reinterpret_cast<uint4*>(&y[j]) = *reinterpret_cast<const uint4*>(h);
        }
      } else if (g < r_end) {
        float* y = Y + g * ldy + c0;
        if (vec_out && c0 + 16 <= kout) {
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            *reinterpret_cast<float4*>(&y[j]) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < kout) y[j] = v[j];
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::);
    __syncthreads();  // tensor memory is free for the next tile's MMAs
  }
  cp_async_wait<0>();
  if (!ok) {
    if (tid == 0) atomicOr(&flags[2], 1);
    mbar_drain(&mbar, phase);  // bounded: let an MMA in flight finish before freeing
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::);
  __syncthreads();
  if (warp == 0) tmem_free(tmem, 128);
}

// Y[rows, 0:kout] = X[rows, 0:n] T in the split form: X and T^T are split
// into TF32 hi and lo parts in shared memory and Y accumulates
// X_hi T_hi + X_hi T_lo + X_lo T_hi (about 21 significant bits). Each CTA owns
// one contiguous range of rows, in 128-row tiles. One A tile is staged at a
// time (hi and lo of both operands fill the shared memory), but the next
// tile's rows are requested as soon as the MMAs of the current one have
// completed, so they land while the current tile is written back from tensor
// memory. The splits are elementwise over whole buffers (the hi and lo
// buffers share one layout). Eight warps: warps w and w + 4 share tensor
// memory lane quarter w % 4, each writing half of the columns. accumulate:
// Y += X T, the old rows of Y requested while the MMAs run (Y rows 16-byte
// aligned, checked by the host).
// the split form's outputs are at most 112 wide: 7 chunks of 16 columns, at
// most 4 per warp half (the yold registers below)
constexpr int kGemm3MaxNp = 112;
static_assert((kGemm3MaxNp / 16 + 1) / 2 <= 4, "k_tc_gemm3: 4 chunks per warp half");

template <bool VEC>
__global__ void __launch_bounds__(kGemmThreads)
    k_tc_gemm3(const float* __restrict__ X, int ldx, int n, int64_t rows, int64_t rows_per_cta,
               const float* __restrict__ T, int kout, int Kp, int Np, float* __restrict__ Y,
               int ldy, bool accumulate, uint32_t wl, int* __restrict__ flags) {
  extern __shared__ __align__(1024) float smem[];
  float* Bh = smem;                  // Np x Kp
  float* Bl = Bh + Np * Kp;          // Np x Kp
  float* Ah = Bl + Np * Kp;          // 128 x Kp
  float* Al = Ah + 128 * Kp;         // 128 x Kp
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kc_n = Kp >> 2;  // 16-byte chunks along K (at most 28)
  const int64_t r_beg = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = min(rows, r_beg + rows_per_cta);
  const int ntile = r_end > r_beg ? (int)((r_end - r_beg + 127) / 128) : 0;
  if (warp == 0) tmem_alloc(&tmem_slot, 128);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::);
  }
  auto issue = [&](int t) {  // tile t of this CTA, raw, into Ah
    const int64_t row0 = r_beg + (int64_t)t * 128;
    const uint32_t dst = smem_u32(Ah);
    if (VEC) {
      const int r_lo = tid & 7, kc = tid >> 3;
      if (kc < kc_n) {
        const int nval = max(0, min(4, n - kc * 4));
        const float* src = X + (row0 + r_lo) * ldx + kc * 4;
        uint32_t d = dst + (uint32_t)(kc * 128 + r_lo * 16);
#pragma unroll 4
        for (int rg = 0; rg < 16; ++rg, src += 8 * (int64_t)ldx, d += (uint32_t)kc_n * 128u) {
          const bool in = row0 + rg * 8 + r_lo < r_end && nval > 0;
          cp_async16(d, in ? (const void*)src : X, in ? (uint32_t)nval * 4u : 0u);
        }
      }
    } else {
      for (int i = tid; i < 128 * Kp; i += kGemmThreads) {
        const int r = i / Kp, k = i % Kp;
        const int64_t g = row0 + r;
        const bool okk = g < r_end && k < n;
        cp_async4(dst + (uint32_t)core_off(r, k, Kp) * 4u, okk ? (const void*)(X + g * ldx + k) : X,
                  okk ? 4u : 0u);
      }
    }
  };
  {  // B(j, k) = T[k][j], zero past n and kout (a warp reads 128 floats of a row of T)
    const int jq = tid & 31;
    if (jq * 4 < Np) {
      for (int k = tid >> 5; k < Kp; k += kGemmThreads / 32) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = jq * 4 + q;
          const bool in = k < n && j < kout;
          cp_async4(smem_u32(Bh) + (uint32_t)core_off(j, k, Kp) * 4u,
                    in ? (const void*)(T + (int64_t)k * kout + j) : T, in ? 4u : 0u);
        }
      }
    }
  }
  if (ntile > 0) issue(0);
  cp_async_commit();
  asm volatile("tcgen05.fence::before_thread_sync;" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::);
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_tf32(128, Np);
  const bool vec_out = (ldy & 3) == 0 && ((uintptr_t)Y & 15) == 0;
  const int nch = Np >> 4, ch_mid = (nch + 1) >> 1;
  const int ch_lo = warp < 4 ? 0 : ch_mid, ch_hi = warp < 4 ? ch_mid : nch;
  const int q4 = warp & 3;
  uint32_t phase = 0;
  bool ok = true;
  for (int t = 0; t < ntile; ++t) {
    cp_async_wait<0>();  // this thread's copies of tile t (and, first, of B)
    __syncthreads();
    if (t == 0) {
      for (int i = tid; i < (Np * Kp) >> 2; i += kGemmThreads) {
        const float4 x = reinterpret_cast<const float4*>(Bh)[i];
        const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
        reinterpret_cast<float4*>(Bh)[i] = h;
        reinterpret_cast<float4*>(Bl)[i] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
      }
    }
    for (int i = tid; i < (128 * Kp) >> 2; i += kGemmThreads) {
      const float4 x = reinterpret_cast<const float4*>(Ah)[i];
      const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
      reinterpret_cast<float4*>(Ah)[i] = h;
      reinterpret_cast<float4*>(Al)[i] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::);
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::);
      const uint32_t ah = smem_u32(Ah), al = smem_u32(Al), bh = smem_u32(Bh), bl = smem_u32(Bl);
      for (int kk = 0; kk < Kp / 8; ++kk) {
        const uint64_t dah = smem_desc(ah + kk * 256, 128, Kp * 32);
        const uint64_t dal = smem_desc(al + kk * 256, 128, Kp * 32);
        const uint64_t dbh = smem_desc(bh + kk * 256, 128, Kp * 32);
        const uint64_t dbl = smem_desc(bl + kk * 256, 128, Kp * 32);
        mma_tf32(tmem, dah, dbh, idesc, kk > 0 ? 1u : 0u);
        mma_tf32(tmem, dah, dbl, idesc, 1u);
        mma_tf32(tmem, dal, dbh, idesc, 1u);
      }
      mma_commit(&mbar);
    }
    const int64_t g = r_beg + (int64_t)t * 128 + q4 * 32 + lane;
    float4 yold[16];  // this thread's old values, up to four 16-column chunks
    if (accumulate) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int c0 = (ch_lo + i) * 16;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          yold[4 * i + j] = g < r_end && ch_lo + i < ch_hi && c0 + 4 * j < kout
                                ? *reinterpret_cast<const float4*>(Y + g * ldy + c0 + 4 * j)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    if (!__syncthreads_and(mbar_wait(&mbar, phase, wl))) {
      ok = false;
      break;
    }
    phase ^= 1u;
    // the MMAs read A: its buffers take the next tile while this one is written back
    if (t + 1 < ntile) issue(t + 1);
    cp_async_commit();
    asm volatile("tcgen05.fence::after_thread_sync;" ::);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ch = ch_lo + i;
      if (ch >= ch_hi) break;
      const int c0 = ch * 16;
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + c0, v);
      if (g < r_end) {
        float* y = Y + g * ldy + c0;
        if (vec_out && c0 + 16 <= kout) {
#pragma unroll
          for (int j = 0; j < 16; j += 4) {
            float4 o = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            if (accumulate) {
              const float4 p = yold[4 * i + j / 4];
              o = make_float4(p.x + o.x, p.y + o.y, p.z + o.z, p.w + o.w);
            }
            *reinterpret_cast<float4*>(&y[j]) = o;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (c0 + j < kout) {
              float o = v[j];
              if (accumulate) {
                const float4 p = yold[4 * i + j / 4];
                o += (j & 3) == 0 ? p.x : (j & 3) == 1 ? p.y : (j & 3) == 2 ? p.z : p.w;
              }
              y[j] = o;
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::);
    __syncthreads();  // tensor memory is free for the next tile's MMAs
  }
  cp_async_wait<0>();
  if (!ok) {
    if (tid == 0) atomicOr(&flags[2], 1);
    mbar_drain(&mbar, phase);  // bounded: let an MMA in flight finish before freeing
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::);
  __syncthreads();
  if (warp == 0) tmem_free(tmem, 128);
}

}  // namespace

namespace {
// The first-wait limit every tensor-core launch of this process passes to its
// kernel (sfd_set_wait_limit).
std::atomic<uint32_t> g_host_wait_limit{kSpinLimit};
uint32_t wait_limit_arg() { return g_host_wait_limit.load(std::memory_order_relaxed); }
}  // namespace

void cross_gram_tc(const float* X1, int ld1, int n1, const float* X2, int ld2, int n2,
                   int64_t rows, float* G, Workspace& ws, cudaStream_t s) {
  if (n1 < 1 || n1 > 128 || n2 < 0 || n2 > 128)
    throw CudaError{cudaErrorInvalidValue, "cross_gram_tc: blocks of at most 128 columns"};
  static std::atomic<unsigned> attr{0};
  int dev = 0;
  SFD_CUDA(cudaGetDevice(&dev));
  if (dev < 32 && !(attr.load() & (1u << dev))) {
    SFD_CUDA(cudaFuncSetAttribute(k_tc_cross, cudaFuncAttributeMaxDynamicSharedMemorySize, kXSmem));
    attr.fetch_or(1u << dev);
  }
  int nchunks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + kXK - 1) / kXK, kGramChunks));
  int64_t rpc = (rows + nchunks - 1) / nchunks;
  rpc = ((rpc + kXK - 1) / kXK) * kXK;
  nchunks = (int)std::max<int64_t>(1, (rows + rpc - 1) / rpc);
  if ((int64_t)nchunks * kXPartial > (int64_t)320 * 128 * 128)
    throw CudaError{cudaErrorInvalidValue, "cross_gram_tc: partial buffer"};
  if (rows > 0) {
    k_tc_cross<<<nchunks, kTcThreads, kXSmem, s>>>(X1, ld1, n1, X2 ? X2 : X1, ld2, n2, rows, rpc,
                                                   ws.gram_partial, wait_limit_arg(), ws.flags);
    SFD_LAUNCH_CHECK();
  } else {
    nchunks = 0;
  }
  const int N = n1 + n2;
  const int64_t ne = (int64_t)n1 * N + (int64_t)n2 * n2;
  k_cross_reduce<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(ws.gram_partial, nchunks, n1, n2, G);
  SFD_LAUNCH_CHECK();
}

bool tc_supported(int n, int kout) { return n >= 1 && n <= 128 && kout >= 1 && kout <= 128; }

static size_t gemm3_smem(int n, int kout) {
  const int Kp = (n + 7) & ~7, Np = (kout + 15) & ~15;
  return (size_t)2 * (Np + 128) * Kp * sizeof(float);
}

bool tc_split_supported(int n, int kout) {
  return tc_supported(n, kout) && gemm3_smem(n, kout) <= 220 * 1024;
}

void gram_tc(const float* X, int ldx, ColMap map, int64_t rows, float* G, Workspace& ws,
             cudaStream_t s, bool split) {
  const int n = map.total();
  if (!tc_supported(n, n) || map.k1 != 0)
    throw CudaError{cudaErrorInvalidValue, "gram_tc: one block of at most 128 columns"};
  static std::atomic<unsigned> attr{0};
  int dev = 0;
  SFD_CUDA(cudaGetDevice(&dev));
  if (dev < 32 && !(attr.load() & (1u << dev))) {
    SFD_CUDA(cudaFuncSetAttribute(k_tc_gram<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  GramRing<false>::Smem));
    SFD_CUDA(cudaFuncSetAttribute(k_tc_gram<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  GramRing<true>::Smem));
    SFD_CUDA(cudaFuncSetAttribute(k_tc_gram_bulk<false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  GramBulk<false>::Smem));
    SFD_CUDA(cudaFuncSetAttribute(k_tc_gram_bulk<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  GramBulk<true>::Smem));
    attr.fetch_or(1u << dev);
  }
  int nchunks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + kGK - 1) / kGK, kGramChunks));
  int64_t rpc = (rows + nchunks - 1) / nchunks;
  rpc = ((rpc + kGK - 1) / kGK) * kGK;
  nchunks = (int)std::max<int64_t>(1, (rows + rpc - 1) / rpc);
  // rows on 16-byte boundaries and at most 128 floats long: one bulk copy per stage
  const bool bulk = (ldx & 3) == 0 && ldx <= 128 && ((uintptr_t)X & 15) == 0;
  if (rows > 0) {
    if (bulk && split)
      k_tc_gram_bulk<true><<<nchunks, kGramThreads, GramBulk<true>::Smem, s>>>(
          X, ldx, n, rows, rpc, ws.gram_partial, wait_limit_arg(), ws.flags);
    else if (bulk)
      k_tc_gram_bulk<false><<<nchunks, kGramThreads, GramBulk<false>::Smem, s>>>(
          X, ldx, n, rows, rpc, ws.gram_partial, wait_limit_arg(), ws.flags);
    else if (split)
      k_tc_gram<true><<<nchunks, kTcThreads, GramRing<true>::Smem, s>>>(
          X, ldx, n, rows, rpc, ws.gram_partial, wait_limit_arg(), ws.flags);
    else
      k_tc_gram<false><<<nchunks, kTcThreads, GramRing<false>::Smem, s>>>(
          X, ldx, n, rows, rpc, ws.gram_partial, wait_limit_arg(), ws.flags);
    SFD_LAUNCH_CHECK();
  } else {
    nchunks = 0;
  }
  gram_reduce_tiles(ws.gram_partial, nchunks, n, G, s);
}

void gemm_ts_tc(const float* X, int ldx, ColMap map, int64_t rows, const float* T, int kout,
                float* Y, int ldy, Workspace& ws, cudaStream_t s, __half* Yh, bool split,
                bool accumulate) {
  if (rows <= 0 || kout <= 0) return;
  const int n = map.total();
  if (accumulate && (!split || (ldy & 3) || ((uintptr_t)Y & 15)))
    throw CudaError{cudaErrorInvalidValue,
                    "gemm_ts_tc: accumulation in the split form, Y rows 16-byte aligned"};
  if (split) {
    if (!tc_split_supported(n, kout) || map.k1 != 0 || Yh)
      throw CudaError{cudaErrorInvalidValue, "gemm_ts_tc: split form needs n, kout <= 112"};
    static std::atomic<unsigned> attr3{0};
    int dv = 0;
    SFD_CUDA(cudaGetDevice(&dv));
    if (dv < 32 && !(attr3.load() & (1u << dv))) {
      SFD_CUDA(cudaFuncSetAttribute(k_tc_gemm3<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    220 * 1024));
      SFD_CUDA(cudaFuncSetAttribute(k_tc_gemm3<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    220 * 1024));
      attr3.fetch_or(1u << dv);
    }
    const int Kp = (n + 7) & ~7, Np = (kout + 15) & ~15;
    // one contiguous range of rows per CTA, at most one CTA per SM
    const int64_t ntiles = (rows + 127) / 128;
    const int grid = (int)std::min<int64_t>(ntiles, 152);
    const int64_t rpc = (rows + grid - 1) / grid;
    const bool vec = (ldx & 3) == 0 && ((uintptr_t)X & 15) == 0;
    if (vec)
      k_tc_gemm3<true><<<grid, kGemmThreads, gemm3_smem(n, kout), s>>>(
          X, ldx, n, rows, rpc, T, kout, Kp, Np, Y, ldy, accumulate, wait_limit_arg(),
          ws.flags);
    else
      k_tc_gemm3<false><<<grid, kGemmThreads, gemm3_smem(n, kout), s>>>(
          X, ldx, n, rows, rpc, T, kout, Kp, Np, Y, ldy, accumulate, wait_limit_arg(),
          ws.flags);
    SFD_LAUNCH_CHECK();
    return;
  }
  if (!tc_supported(n, kout) || map.k1 != 0)
    throw CudaError{cudaErrorInvalidValue, "gemm_ts_tc: one block, n and kout at most 128"};
  if (Yh && ((ldy & 7) != 0 || ((uintptr_t)Yh & 15) != 0 || ldy < kout))
    throw CudaError{cudaErrorInvalidValue, "gemm_ts_tc: fp16 output needs ld % 8 == 0, 16-byte rows"};
  const int Kp = (n + 7) & ~7;
  const int Np = (kout + 15) & ~15;
  // buffers of 128 x Kp: as many as fit beside T^T (2 to 4)
  const size_t b_bytes = (size_t)Np * Kp * sizeof(float), t_bytes = (size_t)128 * Kp * sizeof(float);
  const int nb = (int)std::min<size_t>(4, (kGemmSmemMax - b_bytes) / t_bytes);
  const size_t bytes = b_bytes + (size_t)nb * t_bytes;
  static std::atomic<unsigned> attr{0};
  int dev = 0;
  SFD_CUDA(cudaGetDevice(&dev));
  if (dev < 32 && !(attr.load() & (1u << dev))) {
    for (auto f : {k_tc_gemm<true, 2>, k_tc_gemm<true, 3>, k_tc_gemm<true, 4>, k_tc_gemm<false, 2>,
                   k_tc_gemm<false, 3>, k_tc_gemm<false, 4>})
      SFD_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmemMax));
    attr.fetch_or(1u << dev);
  }
  // one contiguous range of rows per CTA, at most one CTA per SM
  const int64_t ntiles = (rows + 127) / 128;
  const int grid = (int)std::min<int64_t>(ntiles, 152);
  const int64_t rpc = (rows + grid - 1) / grid;
  const bool vec = (ldx & 3) == 0 && ((uintptr_t)X & 15) == 0;
  auto k = vec ? (nb >= 4 ? k_tc_gemm<true, 4> : nb == 3 ? k_tc_gemm<true, 3> : k_tc_gemm<true, 2>)
               : (nb >= 4 ? k_tc_gemm<false, 4> : nb == 3 ? k_tc_gemm<false, 3> : k_tc_gemm<false, 2>);
  k<<<grid, kGemmThreads, bytes, s>>>(X, ldx, n, rows, rpc, T, kout, Kp, Np, Y, ldy, Yh,
                                      wait_limit_arg(), ws.flags);
  SFD_LAUNCH_CHECK();
}


void set_wait_limit(int64_t spins) {
  g_host_wait_limit.store(spins < 0 ? kSpinLimit : (uint32_t)std::min<int64_t>(spins, kSpinLimit));
}

int wait_selftest(int64_t spins, float* ms) {
  const uint32_t limit = spins < 0 ? kSpinLimit : (uint32_t)std::min<int64_t>(spins, kSpinLimit);
  int* flags = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int timed_out = 0;
  try {
    SFD_CUDA(cudaMalloc(&flags, 16 * sizeof(int)));
    SFD_CUDA(cudaMemset(flags, 0, 16 * sizeof(int)));
    SFD_CUDA(cudaEventCreate(&e0));
    SFD_CUDA(cudaEventCreate(&e1));
    SFD_CUDA(cudaEventRecord(e0, 0));
    k_wait_selftest<<<1, 128>>>(limit, flags);
    SFD_LAUNCH_CHECK();
    SFD_CUDA(cudaEventRecord(e1, 0));
    SFD_CUDA(cudaEventSynchronize(e1));
    if (ms) SFD_CUDA(cudaEventElapsedTime(ms, e0, e1));
    SFD_CUDA(cudaMemcpy(&timed_out, flags + 2, sizeof(int), cudaMemcpyDeviceToHost));
  } catch (...) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (flags) cudaFree(flags);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(flags);
  return timed_out;
}

}  // namespace sfd
