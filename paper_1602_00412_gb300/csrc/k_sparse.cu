// Sparse kernels of the SparseShrink hot path (Alg. 1-3 of Ghashami, Liberty,
// Phillips): buffer validation and ||A'||_F^2, the CSC copy of the buffer
// (stable LSD radix sort by column, so each column lists rows in ascending
// order and every result is deterministic), and the sparse x dense products
// A' X and A'^T Y of SimultaneousIteration / VerifySpectral.
//
// Both products run on one segmented kernel: the CSR copy (segments = rows)
// gives A' X, the CSC copy (segments = columns) gives A'^T Y. Work items cover
// at most kSplit entries, so the Zipf-heavy head columns of the CSC are cut
// into many items; their partial rows are summed in a fixed order by a second
// small kernel (no atomics, bit-reproducible).
#include <algorithm>

#include "sfd_internal.cuh"

namespace sfd {

namespace {

constexpr int kScanChunk = 4096;   // elements per block in the scans
constexpr int kRadixWarps = 16;
constexpr int kRadixItems = 8;     // per lane
constexpr int kRadixTile = kRadixWarps * 32 * kRadixItems;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ row ids
__global__ void k_row_ids(const int* __restrict__ ptr, int nseg, int* __restrict__ rows) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= nseg) return;
  int b = ptr[warp], e = ptr[warp + 1];
  for (int i = b + lane; i < e; i += 32) rows[i] = warp;
}

// ------------------------------------------------------------ check + norms
constexpr int kCheckBlocks = 1024;

__global__ void k_check_entries(const int* __restrict__ idx, const float* __restrict__ val,
                                int64_t nnz, int d, int* __restrict__ col_count,
                                double* __restrict__ block_fro2, int* __restrict__ flags) {
  float acc = 0.f;
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
       i += (int64_t)gridDim.x * blockDim.x) {
    int c = idx[i];
    float v = val[i];
    if (c < 0 || c >= d || !isfinite(v)) {
      bad = 1;
      continue;
    }
    if (col_count) atomicAdd(&col_count[c], 1);
    acc = fmaf(v, v, acc);
  }
  if (bad) atomicOr(&flags[0], 1);
  __shared__ float red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    v = warp_sum(v);
    if (threadIdx.x == 0) block_fro2[blockIdx.x] = (double)v;
  }
}

__global__ void k_sum_doubles(const double* __restrict__ in, int n, double* __restrict__ out) {
  // single block, fixed order: thread t sums t, t+bs, ...; then a tree in shared memory
  __shared__ double sh[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += in[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// every column index c in (keys[i-1], keys[i]] starts at position i
__global__ void k_colptr_from_sorted(const int* __restrict__ keys, int64_t n, int d,
                                     int* __restrict__ ptr) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i > n) return;
  const int prev = i == 0 ? -1 : keys[i - 1];
  const int cur = i == n ? d : keys[i];
  for (int c = prev + 1; c <= cur; ++c) ptr[c] = (int)i;
}

// -------------------------------------------------------------------- scans
__global__ void k_scan_block_sums(const int* __restrict__ in, int n, int* __restrict__ sums) {
  int base = blockIdx.x * kScanChunk;
  int a = 0;
  for (int i = threadIdx.x; i < kScanChunk; i += blockDim.x) {
    int g = base + i;
    if (g < n) a += in[g];
  }
  __shared__ int red[32];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) sums[blockIdx.x] = v;
  }
}

// Block-wide exclusive scan of one value per thread (blockDim a multiple of 32).
__device__ int block_exclusive_scan(int v, int* total) {
  __shared__ int ws[32];
  __shared__ int wtot;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
    int s = t;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s - t;
    if (lane == 31) wtot = s;
  }
  __syncthreads();
  int excl = ws[w] + x - v;
  if (total) *total = wtot;
  __syncthreads();
  return excl;
}

__global__ void __launch_bounds__(1024) k_scan_top(int* __restrict__ sums, int nb) {
  // exclusive scan of nb <= 1024 * 8 block sums in place
  int carry = 0;
  for (int base = 0; base < nb; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < nb ? sums[i] : 0;
    int tot;
    int e = block_exclusive_scan(v, &tot);
    if (i < nb) sums[i] = carry + e;
    carry += tot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) k_scan_final(const int* __restrict__ in, int n,
                                                     const int* __restrict__ sums,
                                                     int* __restrict__ out) {
  int base = blockIdx.x * kScanChunk;
  int carry = sums[blockIdx.x];
  constexpr int per = kScanChunk / 1024;
  int v[per];
  int loc = 0;
#pragma unroll
  for (int j = 0; j < per; ++j) {
    int g = base + threadIdx.x * per + j;
    v[j] = g < n ? in[g] : 0;
    loc += v[j];
  }
  int tot;
  int e = block_exclusive_scan(loc, &tot);
  int run = carry + e;
#pragma unroll
  for (int j = 0; j < per; ++j) {
    int g = base + threadIdx.x * per + j;
    if (g < n) out[g] = run;
    run += v[j];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = carry + tot;
}

// ------------------------------------------------------------- radix sort
__global__ void __launch_bounds__(kRadixWarps * 32)
    k_radix_hist(const int* __restrict__ key, int64_t n, int shift, int ntiles,
                 int* __restrict__ hist) {
  __shared__ int cnt[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kRadixTile;
  for (int i = threadIdx.x; i < kRadixTile; i += blockDim.x) {
    int64_t g = base + i;
    if (g < n) atomicAdd(&cnt[(key[g] >> shift) & 255], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i * ntiles + blockIdx.x] = cnt[i];
}

__global__ void __launch_bounds__(kRadixWarps * 32)
    k_radix_scatter(const int* __restrict__ key, const int* __restrict__ a,
                    const float* __restrict__ b, int64_t n, int shift, int ntiles,
                    const int* __restrict__ offs, int* __restrict__ key_o, int* __restrict__ a_o,
                    float* __restrict__ b_o) {
  __shared__ int wcount[kRadixWarps][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = lane; i < 256; i += 32) wcount[w][i] = 0;
  __syncwarp();
  int64_t base = (int64_t)blockIdx.x * kRadixTile + (int64_t)w * 32 * kRadixItems;
  int kk[kRadixItems], aa[kRadixItems], dg[kRadixItems], pos[kRadixItems];
  float bb[kRadixItems];
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int j = 0; j < kRadixItems; ++j) {
    int64_t g = base + j * 32 + lane;
    bool ok = g < n;
    kk[j] = ok ? key[g] : 0;
    aa[j] = ok ? a[g] : 0;
    bb[j] = ok ? b[g] : 0.f;
    int digit = ok ? ((kk[j] >> shift) & 255) : 256;
    dg[j] = digit;
    unsigned peers = __match_any_sync(0xffffffffu, digit);
    int rank = __popc(peers & lt);
    int leader = __ffs(peers) - 1;
    int basec = digit < 256 ? wcount[w][digit] : 0;
    pos[j] = basec + rank;
    __syncwarp();
    if (lane == leader && digit < 256) wcount[w][digit] = basec + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  if (threadIdx.x < 256) {
    int run = 0;
#pragma unroll
    for (int ww = 0; ww < kRadixWarps; ++ww) {
      int c = wcount[ww][threadIdx.x];
      wcount[ww][threadIdx.x] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kRadixItems; ++j) {
    if (dg[j] < 256) {
      int dst = offs[dg[j] * ntiles + blockIdx.x] + wcount[w][dg[j]] + pos[j];
      key_o[dst] = kk[j];
      a_o[dst] = aa[j];
      b_o[dst] = bb[j];
    }
  }
}

// ------------------------------------------------------------ work lists
__global__ void k_count_items(const int* __restrict__ ptr, int nseg, int* __restrict__ n_items,
                              int* __restrict__ n_slots, int* __restrict__ n_splitflag) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  int len = ptr[s + 1] - ptr[s];
  int k = len <= kSplit ? 1 : (len + kSplit - 1) / kSplit;
  n_items[s] = k;
  n_slots[s] = k > 1 ? k : 0;
  n_splitflag[s] = k > 1 ? 1 : 0;
}

__global__ void k_fill_items(const int* __restrict__ ptr, int nseg, const int* __restrict__ item_off,
                             const int* __restrict__ slot_off, const int* __restrict__ split_off,
                             int4* __restrict__ items, int* __restrict__ item_slot,
                             int* __restrict__ item_split, int* __restrict__ split_seg,
                             int* __restrict__ split_first, int* __restrict__ split_count) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  int b = ptr[s], e = ptr[s + 1];
  int k = item_off[s + 1] - item_off[s];
  int o = item_off[s];
  for (int t = 0; t < k; ++t) {
    items[o + t] = make_int4(s, b + t * kSplit, min(b + (t + 1) * kSplit, e), k > 1 ? slot_off[s] + t : -1);
    item_slot[o + t] = k > 1 ? slot_off[s] + t : -1;
    item_split[o + t] = k > 1 ? split_off[s] : -1;
  }
  if (k > 1) {
    int q = split_off[s];
    split_seg[q] = s;
    split_first[q] = slot_off[s];
    split_count[q] = k;
  }
}

// -------------------------------------------------------------- SpMM (k<=256)
// One warp per work item; lane l owns float4 columns l, l+32 (VPL of them).
// Entries are read 32 at a time (coalesced) and broadcast by shuffles; U
// gathers per lane are in flight at once.
// Two fp32 fused multiply-adds in one instruction (fma.rn.f32x2, sm_100 and
// later): each element is a*b + c rounded once, exactly as fmaf, so the packed
// form changes no result; it halves the multiply-add issue of the gathers.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

template <int VPL, int U>
__global__ void __launch_bounds__(256)
    k_spmm(const int* __restrict__ ptr, const int* __restrict__ idx, const float* __restrict__ val,
           const int4* __restrict__ items, const int* __restrict__ item_slot,
           const int* __restrict__ n_items_ptr, const float4* __restrict__ X, int ldx4, int nvec,
           float4* __restrict__ Y, int ldy4, float4* __restrict__ partial) {
  int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (item >= *n_items_ptr) return;
  const int4 it = items[item];
  const int seg = it.x, beg = it.y, end = it.z;
  float4 acc[VPL];
#pragma unroll
  for (int q = 0; q < VPL; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int p = beg; p < end; p += 32) {
    const int cnt = min(32, end - p);
    const int c_l = lane < cnt ? idx[p + lane] : 0;
    const float v_l = lane < cnt ? val[p + lane] : 0.f;
    for (int jj = 0; jj < cnt; jj += U) {
      int cu[U];
      float vu[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        // lanes past cnt carry value 0 and column 0: harmless multiply-adds
        cu[u] = __shfl_sync(0xffffffffu, c_l, (jj + u) & 31);
        vu[u] = jj + u < cnt ? __shfl_sync(0xffffffffu, v_l, (jj + u) & 31) : 0.f;
      }
#pragma unroll
      for (int q = 0; q < VPL; ++q) {
        const int vi = lane + 32 * q;
        if (vi < nvec) {
          float4 xs[U];
#pragma unroll
          for (int u = 0; u < U; ++u) xs[u] = __ldg(&X[(int64_t)cu[u] * ldx4 + vi]);
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const float2 vv = make_float2(vu[u], vu[u]);
            const float2 lo = ffma2(vv, make_float2(xs[u].x, xs[u].y), make_float2(acc[q].x, acc[q].y));
            const float2 hi = ffma2(vv, make_float2(xs[u].z, xs[u].w), make_float2(acc[q].z, acc[q].w));
            acc[q] = make_float4(lo.x, lo.y, hi.x, hi.y);
          }
        }
      }
    }
  }
  const int slot = it.w;
  float4* out = slot < 0 ? Y + (int64_t)seg * ldy4 : partial + (int64_t)slot * ldy4;
#pragma unroll
  for (int q = 0; q < VPL; ++q) {
    int vi = lane + 32 * q;
    if (vi < nvec) out[vi] = acc[q];
  }
}

// Y = A X with X in fp16 (k <= 128 columns, rows of ldx halves, ldx % 8 == 0):
// a warp takes one work item; its two half-warps take alternate entries, each
// lane loads 8 columns (16 bytes) of the gathered row, so the L2 gather moves
// half the bytes of the fp32 kernel. Sums are fp32; the two halves are added
// in a fixed order at the end.
template <int U>
__global__ void __launch_bounds__(256)
    k_spmm_h(const int* __restrict__ ptr, const int* __restrict__ idx, const float* __restrict__ val,
             const int4* __restrict__ items, const int* __restrict__ item_slot,
             const int* __restrict__ n_items_ptr, const uint4* __restrict__ X, int ldx8, int nv8,
             float4* __restrict__ Y, int ldy4, float4* __restrict__ partial) {
  const int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
  if (item >= *n_items_ptr) return;
  const int4 it = items[item];
  const int seg = it.x, beg = it.y, end = it.z;
  float acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.f;
  for (int p = beg; p < end; p += 32) {
    const int cnt = min(32, end - p);
    const int c_l = lane < cnt ? idx[p + lane] : 0;
    const float v_l = lane < cnt ? val[p + lane] : 0.f;
    for (int jj = 0; jj < cnt; jj += 2 * U) {
      int cu[U];
      float vu[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = jj + 2 * u + half;  // this half-warp's entry
        cu[u] = __shfl_sync(0xffffffffu, c_l, e & 31);
        const float vv = __shfl_sync(0xffffffffu, v_l, e & 31);
        vu[u] = e < cnt ? vv : 0.f;       // past cnt: column 0 times 0
      }
      if (hl < nv8) {
        uint4 xs[U];
#pragma unroll
        for (int u = 0; u < U; ++u) xs[u] = __ldg(&X[(int64_t)cu[u] * ldx8 + hl]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const __half2* h = reinterpret_cast<const __half2*>(&xs[u]);
          const float2 vv = make_float2(vu[u], vu[u]);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 a = ffma2(vv, __half22float2(h[q]), make_float2(acc[2 * q], acc[2 * q + 1]));
            acc[2 * q] = a.x;
            acc[2 * q + 1] = a.y;
          }
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], 16);
  if (half == 0 && hl < nv8) {
    const int slot = it.w;
    float4* out = slot < 0 ? Y + (int64_t)seg * ldy4 : partial + (int64_t)slot * ldy4;
    out[2 * hl] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    out[2 * hl + 1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
  }
}

// Sum of the partial rows of each split segment. One block per segment
// (grid-stride): warp g adds partials g, g+8, ..., and the 8 warp sums are
// combined in a fixed order. A hot column of the CSC copy has thousands of
// partials, so the sum is spread over the block instead of one warp's chain.
constexpr int kFixWarps = 8;

template <int VPL>
__global__ void __launch_bounds__(32 * kFixWarps)
    k_spmm_fixup(const int* __restrict__ split_seg, const int* __restrict__ split_first,
                 const int* __restrict__ split_count, const int* __restrict__ n_split_ptr,
                 const float4* __restrict__ partial, int ldy4, int nvec, float4* __restrict__ Y) {
  __shared__ float4 sums[kFixWarps][32 * VPL];
  const int lane = threadIdx.x & 31, wg = threadIdx.x >> 5;
  const int n_split = *n_split_ptr;
  for (int w = blockIdx.x; w < n_split; w += gridDim.x) {
    const int seg = split_seg[w], f = split_first[w], c = split_count[w];
#pragma unroll
    for (int q = 0; q < VPL; ++q) {
      const int vi = lane + 32 * q;
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
      if (vi < nvec) {
        // partials t = wg, wg + 8, ... in that order; kB loads are issued
        // before their adds (a head column has up to hundreds of partials)
        constexpr int kB = VPL == 1 ? 8 : 4;
        int t = wg;
        for (; t + (kB - 1) * kFixWarps < c; t += kB * kFixWarps) {
          float4 p[kB];
#pragma unroll
          for (int u = 0; u < kB; ++u) p[u] = partial[(int64_t)(f + t + u * kFixWarps) * ldy4 + vi];
#pragma unroll
          for (int u = 0; u < kB; ++u) {
            a.x += p[u].x; a.y += p[u].y; a.z += p[u].z; a.w += p[u].w;
          }
        }
        for (; t < c; t += kFixWarps) {
          const float4 p = partial[(int64_t)(f + t) * ldy4 + vi];
          a.x += p.x; a.y += p.y; a.z += p.z; a.w += p.w;
        }
      }
      sums[wg][vi] = a;
    }
    __syncthreads();
    for (int vi = threadIdx.x; vi < nvec; vi += blockDim.x) {
      float4 a = sums[0][vi];
#pragma unroll
      for (int g = 1; g < kFixWarps; ++g) {
        const float4 p = sums[g][vi];
        a.x += p.x; a.y += p.y; a.z += p.z; a.w += p.w;
      }
      Y[(int64_t)seg * ldy4 + vi] = a;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------- SpMV
// Eight lanes per work item (four items per warp): rows and columns of a
// buffer hold tens of entries, so a whole warp per item would idle. An item
// of a split segment stores its partial sum and takes a ticket on the
// segment's counter; the item whose ticket completes the segment adds the
// partials up (its eight lanes take every eighth partial, in order, then a
// fixed shuffle tree), writes y and resets the counter, so no second launch
// is needed and the sum does not depend on which item finishes last.
__global__ void __launch_bounds__(256)
    k_spmv(const int* __restrict__ ptr, const int* __restrict__ idx, const float* __restrict__ val,
           const int4* __restrict__ items, const int* __restrict__ item_slot,
           const int* __restrict__ item_split, const int* __restrict__ split_first,
           const int* __restrict__ split_count, unsigned* __restrict__ split_ticket,
           const int* __restrict__ n_items_ptr, const float* __restrict__ x, float* __restrict__ y,
           float* __restrict__ partial, const double* __restrict__ xscale) {
  const int n_items = *n_items_ptr;
  // x is used as x * xs (xs = (float)xscale[1], exactly the product a
  // separate scaling pass would store; 1 when xscale is null)
  const float xs = xscale ? (float)xscale[1] : 1.f;
  const int warp_first = (blockIdx.x * blockDim.x + (threadIdx.x & ~31)) >> 3;
  if (warp_first >= n_items) return;  // whole warp past the end
  const int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  const int gl = threadIdx.x & 7, lead = threadIdx.x & 31 & ~7;
  const bool live = item < n_items;
  float a = 0.f;
  int seg = 0, slot = -1;
  if (live) {
    const int4 it = items[item];
    seg = it.x;
    slot = it.w;
    const int end = it.z;
    // eight entries per lane at a time (an item of up to 64 entries, most rows
    // of a buffer, in one round), the last group predicated: their column
    // indices and values are loaded first, then the eight gathers of x are in
    // flight together; the products are added in the lane's entry order (the
    // same sum as one entry at a time)
    for (int p = it.y + gl; p < end; p += 64) {
      int c[8];
      float v[8], xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool in = p + 8 * u < end;
        c[u] = in ? idx[p + 8 * u] : 0;
        v[u] = in ? val[p + 8 * u] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) xv[u] = p + 8 * u < end ? __ldg(&x[c[u]]) : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (p + 8 * u < end) a = fmaf(v[u], xv[u] * xs, a);
    }
  }
  a += __shfl_xor_sync(0xffffffffu, a, 4);
  a += __shfl_xor_sync(0xffffffffu, a, 2);
  a += __shfl_xor_sync(0xffffffffu, a, 1);
  int q = -1;
  unsigned taken = 0;
  if (live && gl == 0) {
    if (slot < 0) {
      y[seg] = a;
    } else {
      partial[slot] = a;
      __threadfence();
      q = item_split[item];
      taken = atomicAdd(&split_ticket[q], 1u) + 1u;
    }
  }
  q = __shfl_sync(0xffffffffu, q, lead);
  taken = __shfl_sync(0xffffffffu, taken, lead);
  int f = 0, c = 0;
  if (q >= 0 && taken == (unsigned)split_count[q]) {  // this item completed the segment
    f = split_first[q];
    c = taken;
    __threadfence();
  }
  float b = 0.f;
  {  // partials gl, gl + 8, ... in that order, eight loads before their adds
    int t = gl;
    for (; t + 56 < c; t += 64) {
      float pv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) pv[u] = __ldcg(&partial[f + t + 8 * u]);
#pragma unroll
      for (int u = 0; u < 8; ++u) b += pv[u];
    }
    for (; t < c; t += 8) b += __ldcg(&partial[f + t]);
  }
  b += __shfl_xor_sync(0xffffffffu, b, 4);
  b += __shfl_xor_sync(0xffffffffu, b, 2);
  b += __shfl_xor_sync(0xffffffffu, b, 1);
  if (c > 0 && gl == 0) {
    y[seg] = b;
    split_ticket[q] = 0u;
  }
}

}  // namespace

// ======================================================================= API
void launch_row_ids(const int* ptr, int nseg, int* rows, cudaStream_t s) {
  if (nseg <= 0) return;
  int warps_per_block = 8;
  k_row_ids<<<(nseg + warps_per_block - 1) / warps_per_block, 256, 0, s>>>(ptr, nseg, rows);
  SFD_LAUNCH_CHECK();
}

void launch_check_entries(const int* idx, const float* val, int64_t nnz, int d, int* col_count,
                          double* fro2_out, int* flags, cudaStream_t s) {
  // fro2_out[0] receives the total; fro2_out[1..kCheckBlocks] hold block partials
  int nb = (int)std::min<int64_t>(kCheckBlocks, std::max<int64_t>(1, (nnz + 1023) / 1024));
  k_check_entries<<<nb, 256, 0, s>>>(idx, val, nnz, d, col_count, fro2_out + 1, flags);
  SFD_LAUNCH_CHECK();
  k_sum_doubles<<<1, 256, 0, s>>>(fro2_out + 1, nb, fro2_out);
  SFD_LAUNCH_CHECK();
}

void colptr_from_sorted(const int* keys, int64_t n, int d, int* ptr, cudaStream_t s) {
  k_colptr_from_sorted<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(keys, n, d, ptr);
  SFD_LAUNCH_CHECK();
}

void exclusive_scan(const int* in, int n, int* out, int* tmp, cudaStream_t s) {
  int nb = std::max(1, (n + kScanChunk - 1) / kScanChunk);
  k_scan_block_sums<<<nb, 1024, 0, s>>>(in, n, tmp);
  SFD_LAUNCH_CHECK();
  k_scan_top<<<1, 1024, 0, s>>>(tmp, nb);
  SFD_LAUNCH_CHECK();
  k_scan_final<<<nb, 1024, 0, s>>>(in, n, tmp, out);
  SFD_LAUNCH_CHECK();
}

void radix_sort_by_key(int* key, int* a, float* b, int* key_alt, int* a_alt, float* b_alt,
                       int64_t n, int bits, int* hist, int* scan_tmp, cudaStream_t s) {
  // Even number of 8-bit passes so the result lands back in (key, a, b).
  int passes = std::max(2, (bits + 7) / 8);
  if (passes & 1) ++passes;
  if (n <= 0) return;
  int ntiles = (int)((n + kRadixTile - 1) / kRadixTile);
  int* k0 = key; int* a0 = a; float* b0 = b;
  int* k1 = key_alt; int* a1 = a_alt; float* b1 = b_alt;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    if (shift >= 31) shift = 31;  // padding passes past the key width are no-ops (digit 0)
    k_radix_hist<<<ntiles, kRadixWarps * 32, 0, s>>>(k0, n, shift, ntiles, hist);
    SFD_LAUNCH_CHECK();
    exclusive_scan(hist, 256 * ntiles, hist + 256 * ntiles + 1, scan_tmp, s);
    k_radix_scatter<<<ntiles, kRadixWarps * 32, 0, s>>>(k0, a0, b0, n, shift, ntiles,
                                                       hist + 256 * ntiles + 1, k1, a1, b1);
    SFD_LAUNCH_CHECK();
    std::swap(k0, k1); std::swap(a0, a1); std::swap(b0, b1);
  }
}

void build_work(Csr& c, cudaStream_t s) {
  SegWork& w = c.work;
  int n = c.nseg;
  int* off = w.counters + 8;  // 3 * (n + 1) ints of offsets, then scan scratch
  int* item_off = off;
  int* slot_off = off + (n + 1);
  int* split_off = off + 2 * (n + 1);
  int* tmp = off + 3 * (n + 1);
  // the item and split counts live at fixed places (counters[0], [1]), not at
  // the end of offsets whose length follows the segment count: a CUDA graph
  // captured for one buffer keeps the pointer and is replayed for buffers of
  // other row counts
  w.d_n_items = w.counters;
  w.d_n_split = w.counters + 1;
  if (n <= 0) {
    SFD_CUDA(cudaMemsetAsync(w.counters, 0, 2 * sizeof(int), s));
    return;
  }
  // counts in split_seg/split_first/split_count scratch (filled after the scans)
  int* cnt_items = w.split_seg;
  int* cnt_slots = w.split_first;
  int* cnt_split = w.split_count;
  k_count_items<<<(n + 255) / 256, 256, 0, s>>>(c.ptr, n, cnt_items, cnt_slots, cnt_split);
  SFD_LAUNCH_CHECK();
  exclusive_scan(cnt_items, n, item_off, tmp, s);
  exclusive_scan(cnt_slots, n, slot_off, tmp, s);
  exclusive_scan(cnt_split, n, split_off, tmp, s);
  k_fill_items<<<(n + 255) / 256, 256, 0, s>>>(c.ptr, n, item_off, slot_off, split_off, w.items,
                                               w.item_slot, w.item_split, w.split_seg,
                                               w.split_first, w.split_count);
  SFD_LAUNCH_CHECK();
  SFD_CUDA(cudaMemcpyAsync(w.counters, item_off + n, sizeof(int), cudaMemcpyDeviceToDevice, s));
  SFD_CUDA(cudaMemcpyAsync(w.counters + 1, split_off + n, sizeof(int), cudaMemcpyDeviceToDevice,
                           s));
}

void spmm(const Csr& c, const float* X, int ldx, int k, float* Y, int ldy, float* partial,
          cudaStream_t s, int variant) {
  const SegWork& w = c.work;
  const int nvec = (k + 3) / 4;
  const int grid = (w.cap_items + 7) / 8;
  const float4* X4 = (const float4*)X;
  float4* Y4 = (float4*)Y;
  float4* P4 = (float4*)partial;
  if (nvec <= 32) {
    if (variant == 1)
      k_spmm<1, 4><<<grid, 256, 0, s>>>(c.ptr, c.idx, c.val, w.items, w.item_slot, w.d_n_items,
                                        X4, ldx / 4, nvec, Y4, ldy / 4, P4);
    else
      k_spmm<1, 8><<<grid, 256, 0, s>>>(c.ptr, c.idx, c.val, w.items, w.item_slot, w.d_n_items,
                                        X4, ldx / 4, nvec, Y4, ldy / 4, P4);
  } else {
    if (variant == 1)
      k_spmm<2, 2><<<grid, 256, 0, s>>>(c.ptr, c.idx, c.val, w.items, w.item_slot, w.d_n_items,
                                        X4, ldx / 4, nvec, Y4, ldy / 4, P4);
    else
      k_spmm<2, 4><<<grid, 256, 0, s>>>(c.ptr, c.idx, c.val, w.items, w.item_slot, w.d_n_items,
                                        X4, ldx / 4, nvec, Y4, ldy / 4, P4);
  }
  SFD_LAUNCH_CHECK();
  if (!c.may_split) return;  // every item covers its whole segment
  const int g2 = std::max(1, std::min(w.cap_split, 4 * 152));
  if (nvec <= 32)
    k_spmm_fixup<1><<<g2, 32 * kFixWarps, 0, s>>>(w.split_seg, w.split_first, w.split_count,
                                                  w.d_n_split, (const float4*)partial, ldy / 4,
                                                  nvec, (float4*)Y);
  else
    k_spmm_fixup<2><<<g2, 32 * kFixWarps, 0, s>>>(w.split_seg, w.split_first, w.split_count,
                                                  w.d_n_split, (const float4*)partial, ldy / 4,
                                                  nvec, (float4*)Y);
  SFD_LAUNCH_CHECK();
}

void spmm_h(const Csr& c, const __half* X, int ldx, int k, float* Y, int ldy, float* partial,
            cudaStream_t s, int variant) {
  if (k > 128 || (ldx & 7) || (ldy & 7))
    throw CudaError{cudaErrorInvalidValue, "spmm_h: k <= 128, ldx and ldy multiples of 8"};
  const SegWork& w = c.work;
  const int nv8 = (k + 7) / 8;
  const int grid = (w.cap_items + 7) / 8;
  const uint4* X8 = reinterpret_cast<const uint4*>(X);
  if (variant == 1)
    k_spmm_h<2><<<grid, 256, 0, s>>>(c.ptr, c.idx, c.val, w.items, w.item_slot, w.d_n_items, X8,
                                     ldx / 8, nv8, (float4*)Y, ldy / 4, (float4*)partial);
  else if (variant == 2)
    k_spmm_h<8><<<grid, 256, 0, s>>>(c.ptr, c.idx, c.val, w.items, w.item_slot, w.d_n_items, X8,
                                     ldx / 8, nv8, (float4*)Y, ldy / 4, (float4*)partial);
  else
    k_spmm_h<4><<<grid, 256, 0, s>>>(c.ptr, c.idx, c.val, w.items, w.item_slot, w.d_n_items, X8,
                                     ldx / 8, nv8, (float4*)Y, ldy / 4, (float4*)partial);
  SFD_LAUNCH_CHECK();
  const int nvec = 2 * nv8;  // float4 columns written per row
  if (!c.may_split) return;  // every item covers its whole segment
  const int g2 = std::max(1, std::min(w.cap_split, 4 * 152));
  if (nvec <= 32)
    k_spmm_fixup<1><<<g2, 32 * kFixWarps, 0, s>>>(w.split_seg, w.split_first, w.split_count,
                                                  w.d_n_split, (const float4*)partial, ldy / 4,
                                                  nvec, (float4*)Y);
  else
    k_spmm_fixup<2><<<g2, 32 * kFixWarps, 0, s>>>(w.split_seg, w.split_first, w.split_count,
                                                  w.d_n_split, (const float4*)partial, ldy / 4,
                                                  nvec, (float4*)Y);
  SFD_LAUNCH_CHECK();
}

void spmv(const Csr& c, const float* x, float* y, float* partial, cudaStream_t s,
          const double* xscale) {
  const SegWork& w = c.work;
  k_spmv<<<(w.cap_items + 31) / 32, 256, 0, s>>>(c.ptr, c.idx, c.val, w.items, w.item_slot,
                                                 w.item_split, w.split_first, w.split_count,
                                                 w.split_ticket, w.d_n_items, x, y, partial,
                                                 xscale);
  SFD_LAUNCH_CHECK();
}

}  // namespace sfd
