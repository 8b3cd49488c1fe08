// hist_lut.cu -- byte histogram (Section 4) and LUT construction (Section 7)
// kernels of libqlc, plus their C-ABI entry points.
#define QLC_FILE_ID 3
#include "hist_cols.cuh"
#include "../../include/qlc_testing.h"

#include <algorithm>
#include <atomic>
#include <functional>

namespace qlc {

// One CTA of seven warps per SM counts a contiguous slice of the tensor into
// lane-private columns (hist_cols.cuh); the last CTA also counts the bytes
// after the last whole 16-byte vector.
__global__ void __launch_bounds__(kHcThreads, 1)
hist_kernel(const uint8_t* __restrict__ in, uint64_t n, unsigned long long* __restrict__ hist) {
  extern __shared__ __align__(16) uint32_t hc_sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  zero_cols(hc_sm, warp, lane);
  __syncwarp();
  const uint32_t col = lane_col(hc_sm, warp, lane);
  const uint64_t nvec = n / 16;
  const uint64_t per = (nvec + gridDim.x - 1) / gridDim.x;
  const uint64_t beg = (uint64_t)blockIdx.x * per;
  const uint64_t end = min(beg + per, nvec);
  if (beg < end) count_span(reinterpret_cast<const uint4*>(in) + beg, end - beg, col, tid);
  if (blockIdx.x == gridDim.x - 1) count_bytes(in + nvec * 16, n - nvec * 16, col, tid);
  flush_cols(hc_sm, hist, tid);
}

// Rank of a symbol (Section 7): symbols with a larger count, or the same
// count and a smaller value, come first.  With key(t) = count(t) * 256 +
// (255 - t), which is unique and orders exactly that way (counts stay below
// 2^56), the rank of s is the number of keys above key(s): no sort, one
// comparison per key.  One thread per symbol; all threads read the same key
// at a time (a broadcast).
constexpr int kLutThreads = 256;

__device__ __forceinline__ void load_keys(const unsigned long long* __restrict__ hist, unsigned long long* key,
                                          int tid) {
  key[tid] = (hist[tid] << 8) | (unsigned long long)(255 - tid);
}

// The rank of symbol s.
__device__ __forceinline__ int rank_of(const unsigned long long* key, int s) {
  const unsigned long long k = key[s];
  int r = 0;
#pragma unroll 16
  for (int t = 0; t < 256; t++) r += key[t] > k;
  return r;
}

// Codeword of a rank under a scheme (Section 5): area code i, then the
// rank's position in area i in area_bits[i] bits; 8-bit areas store the rank.
__host__ __device__ inline uint32_t lut_entry(const qlc_scheme& sc, int r) {
  uint32_t base = 0;
  for (int i = 0; i < 8; i++) {
    const uint32_t n = sc.area_n[i];
    if ((uint32_t)r < base + n) {
      const uint32_t b = sc.area_bits[i];
      const uint32_t suffix = b == 8 ? (uint32_t)r : (uint32_t)r - base;
      const uint32_t code = ((uint32_t)i << b) | suffix;
      return (code << 4) | (3 + b);
    }
    base += n;
  }
  return 0;
}

__global__ void __launch_bounds__(kLutThreads)
lut_kernel(const unsigned long long* __restrict__ hist, qlc_scheme sc, qlc_lut* __restrict__ lut) {
  __shared__ unsigned long long key[256];
  const int tid = threadIdx.x;
  load_keys(hist, key, tid);
  __syncthreads();
  const int s = tid;
  const int r = rank_of(key, s);
  lut->enc[s] = (uint16_t)lut_entry(sc, r);
  lut->dec[r] = (uint8_t)s;
  if (tid < (int)(sizeof(qlc_scheme) / 4))
    reinterpret_cast<uint32_t*>(&lut->scheme)[tid] = reinterpret_cast<const uint32_t*>(&sc)[tid];
}

struct SchemeSet {
  qlc_scheme s[8];
  int count;
};

// Section 6: the scheme can be adapted to the distribution.  Each candidate
// is scored by its payload bits sum_s count[s] * len(rank[s]) and the
// smallest wins (ties: the earlier candidate).
// One CTA per histogram: CTA b builds luts[b] from hists[b * 256 ...].
__global__ void __launch_bounds__(kLutThreads)
lut_best_kernel(const unsigned long long* __restrict__ hists, SchemeSet set, qlc_lut* __restrict__ luts) {
  constexpr int kWarps = kLutThreads / 32;
  __shared__ unsigned long long key[256];
  __shared__ unsigned long long bits[8][kWarps];
  const unsigned long long* hist = hists + (size_t)blockIdx.x * 256;
  qlc_lut* lut = luts + blockIdx.x;
  const int tid = threadIdx.x;
  load_keys(hist, key, tid);
  __syncthreads();
  const int s = tid, warp = tid >> 5, lane = tid & 31;
  const int r = rank_of(key, s);
  const unsigned long long count = key[s] >> 8;
  for (int k = 0; k < set.count; k++) {
    unsigned long long v = count * (unsigned long long)(lut_entry(set.s[k], r) & 15u);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) bits[k][warp] = v;
  }
  __syncthreads();
  int best = 0;
  unsigned long long best_bits = ~0ull;
  for (int k = 0; k < set.count; k++) {
    unsigned long long t = 0;
    for (int w = 0; w < kWarps; w++) t += bits[k][w];
    if (t < best_bits) {
      best_bits = t;
      best = k;
    }
  }
  const qlc_scheme& sc = set.s[best];
  lut->enc[s] = (uint16_t)lut_entry(sc, r);
  lut->dec[r] = (uint8_t)s;
  if (tid < (int)(sizeof(qlc_scheme) / 4))
    reinterpret_cast<uint32_t*>(&lut->scheme)[tid] = reinterpret_cast<const uint32_t*>(&sc)[tid];
}

int sm_count() {
  // one atomic slot per device below 64 (any thread may fill it; all write
  // the same value); other devices ask the runtime each time
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 148;
  if (dev < 64) {
    const int c = cached[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
  if (dev < 64) cached[dev].store(v, std::memory_order_relaxed);
  return v;
}

}  // namespace qlc

using namespace qlc;

static const qlc_scheme kTable1 = {{8, 8, 8, 8, 8, 16, 32, 168}, {3, 3, 3, 3, 3, 4, 5, 8}, 1, {0}};
static const qlc_scheme kTable2 = {{2, 8, 8, 8, 8, 32, 32, 158}, {1, 3, 3, 3, 3, 5, 5, 8}, 2, {0}};

static bool scheme_valid(const qlc_scheme* s) {
  if (!s || !scheme_ok(s->area_n, s->area_bits)) return false;
  if (s->id == 1 || s->id == 2) {
    const qlc_scheme& t = s->id == 1 ? kTable1 : kTable2;
    for (int i = 0; i < 8; i++)
      if (t.area_n[i] != s->area_n[i] || t.area_bits[i] != s->area_bits[i]) return false;
  } else if (s->id != 0) {
    return false;
  }
  return true;
}

static qlc_scheme clean_scheme(const qlc_scheme* s) {
  qlc_scheme c = *s;
  for (int i = 0; i < 7; i++) c.reserved[i] = 0;
  return c;
}

extern "C" {

int qlc_version(void) { return QLC_VERSION; }

const char* qlc_status_string(qlc_status s) {
  switch (s) {
    case QLC_OK: return "ok";
    case QLC_ERR_ARG: return "invalid argument";
    case QLC_ERR_CAPACITY: return "buffer too small";
    case QLC_ERR_CORRUPT: return "corrupt container";
    case QLC_ERR_TIMEOUT: return "device wait timed out";
    case QLC_ERR_CUDA: return "CUDA error";
    case QLC_ERR_CHECK: return "index check failed";
  }
  return "unknown status";
}

qlc_status qlc_scheme_table(int id, qlc_scheme* out) {
  if (!out || (id != 1 && id != 2)) return QLC_ERR_ARG;
  *out = id == 1 ? kTable1 : kTable2;
  return QLC_OK;
}

int qlc_scheme_check(const qlc_scheme* s) { return scheme_valid(s) ? 1 : 0; }

qlc_status qlc_histogram(const uint8_t* d_in, size_t n, uint64_t* d_hist, int accumulate,
                         qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_histogram");
  if (!d_hist || (n > 0 && !d_in)) return QLC_ERR_ARG;
  if (!aligned(d_in, 16) || !aligned(d_hist, 8)) return QLC_ERR_ARG;
  static int smem_done[64] = {0};
  if (!hist_cols_smem_ok(hist_kernel, smem_done)) return QLC_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!accumulate && cudaMemsetAsync(d_hist, 0, 256 * sizeof(uint64_t), st) != cudaSuccess)
    return QLC_ERR_CUDA;
  if (n == 0) return QLC_OK;
  // one CTA per SM, at least 48 KiB each; a CTA counts under 2^31 bytes
  const uint64_t nvec = n / 16;
  uint64_t grid = (nvec + 3071) / 3072;
  const uint64_t cap = (uint64_t)sm_count();
  if (grid > cap) grid = cap;
  const uint64_t floor_grid = (nvec >> 27) + 1;
  if (grid < floor_grid) grid = floor_grid;
  if (grid > 0x7fffffffu) return QLC_ERR_ARG;
  hist_kernel<<<(int)grid, kHcThreads, kHcSmemBytes, st>>>(d_in, n, reinterpret_cast<unsigned long long*>(d_hist));
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}

qlc_status qlc_build_lut(const uint64_t* d_hist, const qlc_scheme* h_scheme, qlc_lut* d_lut,
                         qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_build_lut");
  if (!d_hist || !d_lut || !scheme_valid(h_scheme)) return QLC_ERR_ARG;
  if (!aligned(d_hist, 8) || !aligned(d_lut, 16)) return QLC_ERR_ARG;
  lut_kernel<<<1, kLutThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const unsigned long long*>(d_hist), clean_scheme(h_scheme), d_lut);
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}

qlc_status qlc_build_lut_best(const uint64_t* d_hist, const qlc_scheme* h_schemes, int n_schemes,
                              qlc_lut* d_lut, qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_build_lut_best");
  if (!d_hist || !d_lut || !h_schemes || n_schemes < 1 || n_schemes > 8) return QLC_ERR_ARG;
  if (!aligned(d_hist, 8) || !aligned(d_lut, 16)) return QLC_ERR_ARG;
  SchemeSet set;
  set.count = n_schemes;
  for (int k = 0; k < n_schemes; k++) {
    if (!scheme_valid(&h_schemes[k])) return QLC_ERR_ARG;
    set.s[k] = clean_scheme(&h_schemes[k]);
  }
  lut_best_kernel<<<1, kLutThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const unsigned long long*>(d_hist), set, d_lut);
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}

qlc_status qlc_build_lut_batch(const uint64_t* d_hists, int n_luts, const qlc_scheme* h_schemes,
                               int n_schemes, qlc_lut* d_luts, qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_build_lut_batch");
  if (!d_hists || !d_luts || !h_schemes || n_luts < 1 || n_schemes < 1 || n_schemes > 8)
    return QLC_ERR_ARG;
  if (!aligned(d_hists, 8) || !aligned(d_luts, 16)) return QLC_ERR_ARG;
  SchemeSet set;
  set.count = n_schemes;
  for (int k = 0; k < n_schemes; k++) {
    if (!scheme_valid(&h_schemes[k])) return QLC_ERR_ARG;
    set.s[k] = clean_scheme(&h_schemes[k]);
  }
  lut_best_kernel<<<n_luts, kLutThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const unsigned long long*>(d_hists), set, d_luts);
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}

qlc_status qlc_build_lut_host(const uint64_t* h_hist, const qlc_scheme* h_scheme, qlc_lut* h_lut) {
  if (!h_hist || !h_lut || !scheme_valid(h_scheme)) return QLC_ERR_ARG;
  h_lut->scheme = clean_scheme(h_scheme);
  for (int s = 0; s < 256; s++) {
    int r = 0;
    for (int t = 0; t < 256; t++) r += (h_hist[t] > h_hist[s]) || (h_hist[t] == h_hist[s] && t < s);
    h_lut->enc[s] = (uint16_t)lut_entry(h_lut->scheme, r);
    h_lut->dec[r] = (uint8_t)s;
  }
  return QLC_OK;
}

// Section 8 leaves the choice of areas, symbols per area and code lengths as
// future work.  Within the family this library codes (qlc_scheme), the best
// scheme for a histogram is found exhaustively: areas 1..7 are complete
// (2^b ranks, b non-decreasing in 0..7), area 8 takes the remaining ranks,
// either raw (8 bits) or complete when their number is a power of two.  Cost
// = sum over ranks of count * code length, counts taken in decreasing order.
qlc_status qlc_scheme_search(const uint64_t* h_hist, qlc_scheme* out, uint64_t* out_bits) {
  if (!h_hist || !out) return QLC_ERR_ARG;
  uint64_t c[256];
  for (int i = 0; i < 256; i++) c[i] = h_hist[i];
  std::sort(c, c + 256, std::greater<uint64_t>());
  uint64_t pre[257];
  pre[0] = 0;
  for (int i = 0; i < 256; i++) pre[i + 1] = pre[i] + c[i];
  uint64_t best = ~0ull;
  uint8_t best_b[8] = {0};
  uint16_t best_n[8] = {0};
  uint8_t b[8];
  // depth-first over b[0] <= b[1] <= ... <= b[6]
  struct Rec {
    static void go(int i, uint32_t base, uint64_t cost, uint8_t* b, const uint64_t* pre, uint64_t* best,
                   uint8_t* best_b, uint16_t* best_n) {
      if (i == 7) {
        const uint32_t rem = 256 - base;
        uint32_t last_bits = 8;
        if ((rem & (rem - 1)) == 0 && rem <= 128) {  // power of two: complete area
          uint32_t lb = 0;
          while ((1u << lb) < rem) lb++;
          if (lb >= b[6]) last_bits = lb;
        }
        const uint64_t total = cost + (3 + last_bits) * (pre[256] - pre[base]);
        if (total < *best) {
          *best = total;
          for (int k = 0; k < 7; k++) {
            best_b[k] = b[k];
            best_n[k] = (uint16_t)(1u << b[k]);
          }
          best_b[7] = (uint8_t)last_bits;
          best_n[7] = (uint16_t)rem;
        }
        return;
      }
      for (uint32_t bi = i ? b[i - 1] : 0; bi <= 7; bi++) {
        const uint32_t n = 1u << bi;
        if (base + n > 255) break;  // area 8 keeps at least one rank
        b[i] = (uint8_t)bi;
        go(i + 1, base + n, cost + (3 + bi) * (pre[base + n] - pre[base]), b, pre, best, best_b, best_n);
      }
    }
  };
  Rec::go(0, 0, 0, b, pre, &best, best_b, best_n);
  qlc_scheme sc = {};
  for (int i = 0; i < 8; i++) {
    sc.area_n[i] = best_n[i];
    sc.area_bits[i] = best_b[i];
  }
  sc.id = 0;
  for (int id = 1; id <= 2; id++) {
    const qlc_scheme& t = id == 1 ? kTable1 : kTable2;
    bool same = true;
    for (int i = 0; i < 8; i++) same = same && t.area_n[i] == sc.area_n[i] && t.area_bits[i] == sc.area_bits[i];
    if (same) sc.id = (uint8_t)id;
  }
  *out = sc;
  if (out_bits) *out_bits = best;
  return QLC_OK;
}

qlc_status qlc_peek_header(const void* h_hdr, size_t hdr_bytes, uint64_t* n, uint64_t* container_bytes) {
  if (!h_hdr || hdr_bytes < QLC_HEADER_BYTES) return QLC_ERR_ARG;
  const uint8_t* p = static_cast<const uint8_t*>(h_hdr);
  auto le = [&](int off, int bytes) {
    uint64_t v = 0;
    for (int i = 0; i < bytes; i++) v |= (uint64_t)p[off + i] << (8 * i);
    return v;
  };
  if (p[0] != 'Q' || p[1] != 'L' || p[2] != 'C' || p[3] != '1' || le(4, 2) != QLC_VERSION)
    return QLC_ERR_CORRUPT;
  const uint64_t nn = le(8, 8);
  const uint64_t n_chunks = le(20, 4);
  if (n) *n = nn;
  if (container_bytes) *container_bytes = payload_start(n_chunks) + le(48, 8);
  return QLC_OK;
}

}  // extern "C"

namespace qlc {
QLC_DEFINE_CHECK_TAKE(check_take_hist)
}  // namespace qlc

extern "C" uint32_t qlc_test_check_take(void) {
#ifdef QLC_CHECKED
  const uint32_t v[5] = {qlc::check_take_decode(), qlc::check_take_encode(), qlc::check_take_hist(),
                         qlc::check_take_batch(), qlc::check_take_quant()};
  for (uint32_t x : v)
    if (x) return x;
  return 0;
#else
  return 0xFFFFFFFFu;
#endif
}
