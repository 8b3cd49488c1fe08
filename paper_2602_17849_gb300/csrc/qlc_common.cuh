// qlc_common.cuh -- shared definitions of the libqlc CUDA kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/qlc.h"

namespace qlc {

constexpr uint32_t kGroupChunks = QLC_CHUNKS_PER_GROUP;  // chunks per group
constexpr uint32_t kIndexOff = QLC_INDEX_OFFSET;         // header 64 + dec 256
constexpr uint32_t kMaxCode = 11;                        // 3 + 8 suffix bits

__host__ __device__ __forceinline__ uint64_t align16(uint64_t v) {
  return (v + 15u) & ~uint64_t(15);
}
__host__ __device__ __forceinline__ uint64_t n_groups_of(uint64_t n_chunks) {
  return (n_chunks + kGroupChunks - 1) / kGroupChunks;
}
__host__ __device__ __forceinline__ uint64_t payload_start(uint64_t n_chunks) {
  return align16(kIndexOff + 8 * n_groups_of(n_chunks) + 2 * n_chunks);
}
__host__ __device__ __forceinline__ bool chunk_symbols_ok(uint64_t cs) {
  return cs >= QLC_MIN_CHUNK && cs <= QLC_MAX_CHUNK && cs % 128 == 0;
}

// Scheme validity (qlc.h): counts sum to 256, widths never decrease, an area
// with b < 8 bits is complete (2^b ranks), an 8-bit area holds 1..256 ranks.
__host__ __device__ inline bool scheme_ok(const uint16_t n[8], const uint8_t b[8]) {
  uint32_t total = 0;
  for (int i = 0; i < 8; i++) {
    if (b[i] > 8) return false;
    if (i > 0 && b[i] < b[i - 1]) return false;
    if (b[i] < 8) {
      if (n[i] != (1u << b[i])) return false;
    } else if (n[i] < 1 || n[i] > 256) {
      return false;
    }
    total += n[i];
  }
  return total == 256;
}

// Alignment of a caller's pointer to a bytes (a power of two); NULL counts as
// aligned, the entry points check NULL where it matters.
__host__ __device__ __forceinline__ bool aligned(const void* p, uintptr_t a) {
  return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0;
}

// First error wins.
__device__ __forceinline__ void set_status(uint32_t* st, uint32_t code) {
  if (st) atomicCAS(st, 0u, code);
}

// Checked build (-DQLC_CHECKED): QLC_GUARD(cond, status) is false when an
// index check fails; the caller then skips the access.  The first failure of
// each .cu file is recorded in that file's g_check_site (file number << 16 |
// line) and, where a status word is at hand, as QLC_ERR_CHECK.  In a normal
// build the guard is the constant true and compiles away.
#ifndef QLC_FILE_ID
#define QLC_FILE_ID 0
#endif
#ifdef QLC_CHECKED
static __device__ uint32_t g_check_site = 0;
#endif
__device__ __forceinline__ bool guard(bool ok, uint32_t* status, uint32_t site) {
#ifdef QLC_CHECKED
  if (!ok) {
    atomicCAS(&g_check_site, 0u, site);
    set_status(status, QLC_ERR_CHECK);
  }
  return ok;
#else
  (void)status;
  (void)site;
  return true;
#endif
}
#define QLC_GUARD(cond, status) (::qlc::guard((cond), (status), ((uint32_t)QLC_FILE_ID << 16) | __LINE__))

// Host side of the checked build: reads and clears this file's record.
// Each .cu file defines its own with QLC_DEFINE_CHECK_TAKE(name).
#ifdef QLC_CHECKED
#define QLC_DEFINE_CHECK_TAKE(name)                                       \
  uint32_t name() {                                                       \
    uint32_t v = 0, z = 0;                                                \
    if (cudaDeviceSynchronize() != cudaSuccess) return 0xFFFFFFFEu;       \
    if (cudaMemcpyFromSymbol(&v, g_check_site, 4) != cudaSuccess) return 0xFFFFFFFEu; \
    cudaMemcpyToSymbol(g_check_site, &z, 4);                              \
    return v;                                                             \
  }
#else
#define QLC_DEFINE_CHECK_TAKE(name) \
  uint32_t name() { return 0; }
#endif
uint32_t check_take_decode();
uint32_t check_take_encode();
uint32_t check_take_hist();
uint32_t check_take_batch();
uint32_t check_take_quant();

// Big-endian view of a little-endian 32-bit word: byte 0 becomes bits 31..24,
// so the first bit of the stream is the word's most significant bit.
__device__ __forceinline__ uint32_t bswap32(uint32_t w) { return __byte_perm(w, 0, 0x0123); }

__device__ __forceinline__ uint4 ldg_nc_v4(const uint4* p) {
  uint4 r;
  asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

__device__ __forceinline__ uint64_t ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The value of an e4m3 byte (Section 3, all-finite eXmY): its sign and
// magnitude bits placed at fp32 bits 31 and 26..20 read as (1 + m/8) 2^(e-127)
// for e >= 1 and m 2^-129 for e = 0 (an fp32 subnormal); one exact
// multiplication by 2^120 gives the value.
__device__ __forceinline__ float e4m3_to_f32(uint32_t c) {
  return __uint_as_float(((c & 0x80u) << 24) | ((c & 0x7Fu) << 20)) * 0x1p120f;
}
// The same bit pattern (value 2^-120 times) for byte j of w: the byte moved
// to the top (sign at bit 31), an arithmetic shift right by 4 (the
// magnitude to bits 26..20, the sign repeated above it), bits 30..27 cleared.
__device__ __forceinline__ uint32_t e4m3_scaled_bits(uint32_t w, int j) {
  const uint32_t t = __byte_perm(w, 0u, 0x0444u | ((uint32_t)j << 12));
  return (uint32_t)((int32_t)t >> 4) & 0x87F00000u;
}

// The shard holding work item t of a batch: the largest s < n_shards with
// item_base[s] <= t (item_base is non-decreasing and item_base[0] = 0, so
// shards without items are skipped).  Warp-wide: each round the 32 lanes
// probe 32 evenly spaced entries of the remaining range and the last lane
// whose entry is <= t narrows it, so 1152 shards take 3 rounds of loads
// instead of the 11 dependent loads of a binary search.  Every lane returns
// the same shard.
__device__ __forceinline__ int shard_of_warp(const unsigned long long* __restrict__ item_base, int n_shards,
                                             unsigned long long t, int lane) {
  int lo = 0, hi = n_shards;  // item_base[lo] <= t; the shard lies in [lo, hi)
  while (hi - lo > 1) {
    const int step = (hi - lo + 31) / 32;
    const int idx = lo + lane * step;
    const unsigned le = __ballot_sync(0xffffffffu, idx < hi && item_base[idx] <= t);
    lo += (31 - __clz(le)) * step;  // lane 0 always qualifies
    hi = min(lo + step, hi);
  }
  return lo;
}

// Number of SMs of the current device (cached per device).
int sm_count();

// A named NVTX range around a host entry point: profilers (nsys, ncu with
// --nvtx) show the kernels a call launches under the call's name.  Without a
// profiler attached a push or pop is a call through an empty slot.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ----------------------------------------------------------------- batches
// Batch workspace: 64 bytes of counters, item_base[n_shards + 1] (first work
// item of each shard; the last entry is the total), then one look-back word
// per encode work item.
struct BatchWs {
  unsigned int* ticket;                // shared by encode / decode / histogram
  unsigned long long* item_base;
  unsigned long long* gstat;
  unsigned long long gstat_cap;        // look-back words available
};
inline bool batch_ws_layout(void* ws, size_t bytes, int n_shards, BatchWs* w) {
  const size_t head = 64 + 8 * (size_t)(n_shards + 1);
  if (bytes < head) return false;
  uint8_t* p = static_cast<uint8_t*>(ws);
  w->ticket = reinterpret_cast<unsigned int*>(p);
  w->item_base = reinterpret_cast<unsigned long long*>(p + 64);
  w->gstat = reinterpret_cast<unsigned long long*>(p + head);
  w->gstat_cap = (bytes - head) / 8;
  return true;
}

enum PlanKind { kPlanHistogram = 0, kPlanEncode = 1, kPlanDecode = 2 };
constexpr int kPlanThreads = 1024;
constexpr uint64_t kHistItem = 256 * 1024;  // symbols per histogram work item

// One CTA: the number of work items of every shard (histogram: 256 KiB
// pieces; encode: groups of 32 chunks; decode: the container's groups),
// their exclusive prefix in item_base, and zeroed counters / look-back words.
// Shards that cannot be processed get no items and set *status.
__global__ void plan_kernel(int kind, const qlc_desc* descs, int n_shards, uint32_t cs, BatchWs w,
                            uint32_t* status);

}  // namespace qlc
