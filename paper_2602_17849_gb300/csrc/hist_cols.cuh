// hist_cols.cuh -- byte counting for the histogram kernels (Section 4: the
// symbol statistics every code is built from).
//
// Every lane owns one 32-bit counter per byte value, in a column of its
// warp's 256 x 32 table: value b of lane l is word 32 b + l, so the 32 lanes
// of a warp always update 32 different banks, whatever bytes they hold, and
// no two lanes ever touch the same word.  A byte costs a byte extract, an
// address and one shared reduction; a warp's 32 updates are one wavefront.
// Seven warps (224 KB of columns) run per SM.  Each lane keeps two batches of
// eight 16-byte loads in flight, and one thread of the CTA prefetches the
// CTA's batch three batches ahead into L2 with a bulk (TMA) prefetch, so the
// loads mostly wait on L2 rather than on HBM.
#pragma once

#include "qlc_common.cuh"

namespace qlc {

constexpr int kHcWarps = 7;                     // 7 x 32 KB of columns: one CTA per SM
constexpr int kHcThreads = kHcWarps * 32;
constexpr int kHcBatchWaves = 2;                // batch: two CTAs per SM over the launch
constexpr int kHcPrefetch = 3;                  // batches prefetched into L2 ahead of the loads
constexpr int kHcUnroll = 8;                    // 16-byte loads per lane per batch
constexpr uint32_t kHcColWords = 256 * 32;      // one warp's table
constexpr size_t kHcSmemBytes = (size_t)kHcWarps * kHcColWords * 4;  // the warps' tables

__device__ __forceinline__ void red_add_one(uint32_t saddr) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(saddr), "r"(1u) : "memory");
}

// Bulk prefetch of [p, p + bytes) into L2 (TMA; p and bytes multiples of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// Thread 0 prefetches the batch that starts at vector i (if any): at most
// U x T vectors, clipped to the span.
__device__ __forceinline__ void prefetch_batch(const uint4* v, uint64_t i, uint64_t nvec) {
  constexpr uint64_t B = (uint64_t)kHcUnroll * kHcThreads;
  if (i < nvec) prefetch_l2(v + i, (uint32_t)(min(B, nvec - i) * 16));
}

// col: shared address of this lane's column (value 0); value b is b * 128 bytes on.
__device__ __forceinline__ void count_word(uint32_t col, uint32_t w) {
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const uint32_t b = __byte_perm(w, 0, 0x4440 + j);
    if (QLC_GUARD(b < 256u, nullptr)) red_add_one(col + (b << 7));
  }
}
__device__ __forceinline__ void count_vec(uint32_t col, uint4 q) {
  count_word(col, q.x);
  count_word(col, q.y);
  count_word(col, q.z);
  count_word(col, q.w);
}

// Counts nvec 16-byte vectors at v; thread t of the CTA takes t, t + T, ...
// Loads of the next batch are issued before the current batch is counted.
__device__ __forceinline__ void count_span(const uint4* __restrict__ v, uint64_t nvec, uint32_t col, int tid) {
  constexpr int U = kHcUnroll;
  constexpr uint64_t T = kHcThreads;
  uint64_t i = (uint64_t)tid;
  if (kHcPrefetch > 0 && tid == 0)
    for (int k = 1; k <= kHcPrefetch; k++) prefetch_batch(v, k * U * T, nvec);
  if (i + (U - 1) * T < nvec) {
    uint4 a[U], b[U];
#pragma unroll
    for (int u = 0; u < U; u++) a[u] = ldg_nc_v4(v + i + u * T);
    i += U * T;
    while (true) {
      if (i + (U - 1) * T >= nvec) {
#pragma unroll
        for (int u = 0; u < U; u++) count_vec(col, a[u]);
        break;
      }
      if (kHcPrefetch > 0 && tid == 0) prefetch_batch(v, i + kHcPrefetch * U * T, nvec);
#pragma unroll
      for (int u = 0; u < U; u++) b[u] = ldg_nc_v4(v + i + u * T);
      i += U * T;
#pragma unroll
      for (int u = 0; u < U; u++) count_vec(col, a[u]);
      if (i + (U - 1) * T >= nvec) {
#pragma unroll
        for (int u = 0; u < U; u++) count_vec(col, b[u]);
        break;
      }
      if (kHcPrefetch > 0 && tid == 0) prefetch_batch(v, i + kHcPrefetch * U * T, nvec);
#pragma unroll
      for (int u = 0; u < U; u++) a[u] = ldg_nc_v4(v + i + u * T);
      i += U * T;
#pragma unroll
      for (int u = 0; u < U; u++) count_vec(col, b[u]);
    }
  }
  for (; i < nvec; i += T) count_vec(col, ldg_nc_v4(v + i));
  QLC_GUARD(i >= nvec && i - nvec < T, nullptr);  // the loop ended at the span's end
}

// Counts m single bytes at p (a ragged end), CTA-strided.
__device__ __forceinline__ void count_bytes(const uint8_t* __restrict__ p, uint64_t m, uint32_t col, int tid) {
  for (uint64_t i = (uint64_t)tid; i < m; i += kHcThreads) red_add_one(col + ((uint32_t)p[i] << 7));
}

// Zeroes this warp's table (the warp's lanes only; callers synchronise).
__device__ __forceinline__ void zero_cols(uint32_t* sm, int warp, int lane) {
  uint4* c4 = reinterpret_cast<uint4*>(sm + (size_t)warp * kHcColWords);
  for (uint32_t i = lane; i < kHcColWords / 4; i += 32) c4[i] = make_uint4(0u, 0u, 0u, 0u);
}

// Adds the CTA's counts to hist[0..255] and zeroes the tables.  Called by
// every thread of the CTA.  A warp sums each value's 32 lane counters with a
// rotated walk (lane l reads lane (k + l) mod 32's word: one bank per lane),
// the warps' sums meet in shared memory, and each value with a nonzero
// count costs one 64-bit global atomic.  A lane's counter stays below 2^32
// as long as a CTA counts fewer than 2^32 bytes between flushes, which the
// launches guarantee.
__device__ __forceinline__ void flush_cols(uint32_t* sm, unsigned long long* __restrict__ hist, int tid) {
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  uint32_t* cols = sm + (size_t)warp * kHcColWords;
  uint32_t s[8];
#pragma unroll
  for (int r = 0; r < 8; r++) {
    const uint32_t* row = cols + 32 * (lane + 32 * r);
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < 32; k++) acc += row[(k + lane) & 31];
    s[r] = acc;
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 8; r++) cols[lane + 32 * r] = s[r];  // the warp's sums: words 0..255 of its table
  __syncthreads();
  for (int b = tid; b < 256; b += kHcThreads) {
    unsigned long long t = 0;
#pragma unroll
    for (int w = 0; w < kHcWarps; w++) t += sm[(size_t)w * kHcColWords + b];
    if (t) atomicAdd(&hist[b], t);
  }
  __syncthreads();
  zero_cols(sm, warp, lane);
  __syncwarp();
}

// The column address of this lane.
__device__ __forceinline__ uint32_t lane_col(uint32_t* sm, int warp, int lane) {
  return (uint32_t)__cvta_generic_to_shared(sm + (size_t)warp * kHcColWords + lane);
}

// Kernels using the columns need kHcSmemBytes of dynamic shared memory;
// this raises the kernel's limit once per device.
template <typename Kernel>
inline bool hist_cols_smem_ok(Kernel k, int* done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return false;
  if (dev < 64 && done[dev]) return true;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHcSmemBytes) != cudaSuccess)
    return false;
  if (dev < 64) done[dev] = 1;
  return true;
}

}  // namespace qlc
