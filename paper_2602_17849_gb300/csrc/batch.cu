// batch.cu -- planning and histogram / LUT kernels for batches of shards.
//
// A batch is an array of qlc_desc in device memory (the paper's own workload
// is 1152 shards per tensor type, Section 3).  plan_kernel turns the shard
// sizes into work items (histogram: 256 KiB pieces; encode / decode: groups of
// 32 chunks) with a block-wide prefix sum; the persistent kernels then take
// items from a device counter, so shards of very different sizes share the
// GPU evenly and no host round trip is needed.
#define QLC_FILE_ID 4
#include "hist_cols.cuh"

namespace qlc {

__host__ __device__ inline uint64_t encoded_bound(uint64_t n, uint32_t cs) {
  const uint64_t n_chunks = (n + cs - 1) / cs;
  const uint64_t group_syms = (uint64_t)kGroupChunks * cs;
  const uint64_t full = n / group_syms, rest = n % group_syms;
  uint64_t total = payload_start(n_chunks);
  total += full * align16((group_syms * kMaxCode + 7) / 8);
  if (rest) total += align16((rest * kMaxCode + 7) / 8);
  return total;
}

__device__ __forceinline__ bool al16(const void* p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

// Work items of one shard; 0 (and a status) for a shard that cannot be run.
__device__ uint64_t item_count(int kind, const qlc_desc& d, uint32_t cs, uint32_t* status) {
  if (kind == kPlanHistogram) {
    if (d.in_bytes == 0) return 0;
    if (!d.in || !al16(d.in)) {
      set_status(status, QLC_ERR_ARG);
      return 0;
    }
    return (d.in_bytes + kHistItem - 1) / kHistItem;
  }
  if (kind == kPlanEncode) {
    const uint64_t n = d.in_bytes;
    const uint64_t n_chunks = (n + cs - 1) / cs;
    if (!d.out || !d.lut || !al16(d.out) || !al16(d.lut) || !aligned(d.out_bytes, 8) ||
        (n > 0 && (!d.in || !al16(d.in))) || n_chunks > 0xFFFFFFFFull) {
      set_status(status, QLC_ERR_ARG);
      return 0;
    }
    if (d.out_cap < encoded_bound(n, cs)) {
      set_status(status, QLC_ERR_CAPACITY);
      return 0;
    }
    return n == 0 ? 1 : n_groups_of(n_chunks);
  }
  // decode: the container's groups, from a header that at least parses
  if (!d.in || !al16(d.in) || !aligned(d.out_bytes, 8) || (d.out_cap > 0 && (!d.out || !al16(d.out)))) {
    set_status(status, QLC_ERR_ARG);
    return 0;
  }
  const uint8_t* c = static_cast<const uint8_t*>(d.in);
  if (d.in_bytes < kIndexOff || *reinterpret_cast<const uint32_t*>(c) != 0x31434C51u) {
    set_status(status, QLC_ERR_CORRUPT);
    return 0;
  }
  const uint64_t groups = n_groups_of(*reinterpret_cast<const uint32_t*>(c + 20));
  if (groups > d.in_bytes / 16) {  // every group takes at least 16 payload bytes
    set_status(status, QLC_ERR_CORRUPT);
    return 0;
  }
  return groups ? groups : 1;  // an empty container still gets its header checked
}

__global__ void __launch_bounds__(kPlanThreads)
plan_kernel(int kind, const qlc_desc* descs, int n_shards, uint32_t cs, BatchWs w, uint32_t* status) {
  __shared__ unsigned long long s_warp[kPlanThreads / 32];
  __shared__ unsigned long long s_carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < 16) w.ticket[tid] = 0;  // the 64 bytes of counters
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < n_shards; base += kPlanThreads) {
    const int s = base + tid;
    const unsigned long long cnt = s < n_shards ? item_count(kind, descs[s], cs, status) : 0ull;
    unsigned long long incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    unsigned long long wpre = 0, total = 0;
    for (int i = 0; i < kPlanThreads / 32; i++) {
      wpre += i < warp ? s_warp[i] : 0ull;
      total += s_warp[i];
    }
    if (s < n_shards) w.item_base[s] = s_carry + wpre + incl - cnt;
    __syncthreads();
    if (tid == 0) s_carry += total;
    __syncthreads();
  }
  unsigned long long total = s_carry;
  if (kind == kPlanEncode && total > w.gstat_cap) {
    if (tid == 0) set_status(status, QLC_ERR_CAPACITY);
    total = 0;
  }
  if (tid == 0) w.item_base[n_shards] = total;
  if (kind == kPlanEncode)
    for (unsigned long long i = tid; i < total; i += kPlanThreads) w.gstat[i] = 0;
}

// ------------------------------------------------------------- histograms

// Each CTA (seven warps, lane-private columns from hist_cols.cuh; two CTAs
// per SM over the launch, one resident at a time) takes a contiguous run of
// items.  Its items of one shard are one contiguous byte range, counted in a
// single streaming pass; the columns are flushed into a shard's histogram
// when the target histogram changes (never, for one shared histogram).  A
// run is 1 / (2 x SMs) of the batch's items, so a lane's counters stay below
// 2^32 for any batch smaller than 2^32 x 2 x SMs bytes, far above the
// device's memory.
__global__ void __launch_bounds__(kHcThreads, 1)
hist_batch_kernel(const qlc_desc* descs, int n_shards, const unsigned long long* item_base,
                  unsigned long long* hists, int shared) {
  extern __shared__ __align__(16) uint32_t hc_sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned long long total = item_base[n_shards];
  const unsigned long long per = (total + gridDim.x - 1) / gridDim.x;
  const unsigned long long t0 = (unsigned long long)blockIdx.x * per;
  const unsigned long long t1 = min(t0 + per, total);
  if (t0 >= t1) return;
  zero_cols(hc_sm, warp, lane);
  __syncwarp();
  const uint32_t col = lane_col(hc_sm, warp, lane);
  int s = 0;
  {
    int lo = 0, hi = n_shards - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (item_base[mid] <= t0) lo = mid; else hi = mid - 1;
    }
    s = lo;
  }
  int target = shared ? 0 : s;
  for (unsigned long long t = t0; t < t1;) {
    while (s + 1 < n_shards && item_base[s + 1] <= t) s++;
    const int tgt = shared ? 0 : s;
    if (tgt != target) {
      flush_cols(hc_sm, hists + (size_t)(QLC_GUARD(target < n_shards, nullptr) ? target : 0) * 256, tid);
      target = tgt;
    }
    const unsigned long long e = min(t1, item_base[s + 1]);  // this CTA's items of shard s end here
    const qlc_desc d = descs[s];
    const uint8_t* in = static_cast<const uint8_t*>(d.in);
    const uint64_t beg = (t - item_base[s]) * kHistItem;      // a multiple of 16
    const uint64_t end = min((uint64_t)((e - item_base[s]) * kHistItem), (uint64_t)d.in_bytes);
    const uint64_t vb = beg / 16, ve = end / 16;
    if (QLC_GUARD(s < n_shards && beg <= end, nullptr)) {
      count_span(reinterpret_cast<const uint4*>(in) + vb, ve - vb, col, tid);
      count_bytes(in + ve * 16, end - ve * 16, col, tid);
    }
    t = e;
  }
  flush_cols(hc_sm, hists + (size_t)target * 256, tid);
}

}  // namespace qlc

using namespace qlc;

extern "C" {

size_t qlc_batch_workspace_size(int n_shards, uint64_t total_symbols, uint32_t chunk_symbols) {
  if (n_shards < 1 || !chunk_symbols_ok(chunk_symbols)) return 0;
  const uint64_t group_syms = (uint64_t)kGroupChunks * chunk_symbols;
  const uint64_t items = (total_symbols + group_syms - 1) / group_syms + (uint64_t)n_shards;
  return (size_t)(64 + 8 * (uint64_t)(n_shards + 1) + 8 * items);
}

qlc_status qlc_histogram_batch(const qlc_desc* d_descs, int n_shards, uint64_t* d_hists, int shared,
                               void* d_ws, size_t ws_bytes, qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_histogram_batch");
  if (!d_descs || n_shards < 1 || !d_hists || !d_ws) return QLC_ERR_ARG;
  if (!aligned(d_ws, 16) || !aligned(d_descs, 16) || !aligned(d_hists, 8)) return QLC_ERR_ARG;
  BatchWs w;
  if (!batch_ws_layout(d_ws, ws_bytes, n_shards, &w)) return QLC_ERR_CAPACITY;
  static int smem_done[64] = {0};
  if (!hist_cols_smem_ok(hist_batch_kernel, smem_done)) return QLC_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t hist_bytes = (size_t)(shared ? 1 : n_shards) * 256 * sizeof(uint64_t);
  if (cudaMemsetAsync(d_hists, 0, hist_bytes, st) != cudaSuccess) return QLC_ERR_CUDA;
  // histogram errors (misaligned shards) have no status word: they are
  // reported as QLC_ERR_ARG by the encode plan of the same descriptors
  plan_kernel<<<1, kPlanThreads, 0, st>>>(kPlanHistogram, d_descs, n_shards, 0, w, nullptr);
  hist_batch_kernel<<<sm_count() * kHcBatchWaves, kHcThreads, kHcSmemBytes, st>>>(
      d_descs, n_shards, w.item_base, reinterpret_cast<unsigned long long*>(d_hists), shared ? 1 : 0);
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}

}  // extern "C"

namespace qlc {
QLC_DEFINE_CHECK_TAKE(check_take_batch)
}  // namespace qlc
