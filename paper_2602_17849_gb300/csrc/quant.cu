// quant.cu -- block-32 e4m3 quantisation fused with the byte histogram, and
// dequantisation (Section 3: the tensors are all-finite eXmY e4m3 with one
// scale per block of 32 elements; Section 4: the 256-bin histogram).
//
// Quantisation reads the wide input once and writes the codes and scales; the
// histogram the LUT needs (Section 7) is counted in the same pass, so the
// codes are not read again before encoding.  Rule per block of 32 (the last
// may be shorter): scale = absmax / 480 in fp32; code = the e4m3 byte nearest
// to x / scale (fp32 division), ties to the even code, saturating at 480, sign
// kept; a block whose scale is 0 (absmax 0, or absmax / 480 rounding to 0 in
// fp32) gets codes 0x00.
//
// A warp handles 1 KiB of input per step: 32 contiguous bytes per lane, 8
// fp32 (or 16 bf16) elements, so one block of 32 is 4 (or 2) lanes and its
// absmax is a 2 (or 1) step butterfly.  Codes leave as one 8- (or 16-) byte
// store per lane.
#include <cuda_bf16.h>

#include <atomic>

#define QLC_FILE_ID 5
#include "qlc_common.cuh"

namespace qlc {

constexpr int kQuantWarps = 8;
constexpr int kQuantThreads = kQuantWarps * 32;
constexpr int kQuantDepth = 4;  // input ring slots (warp steps) per warp
constexpr int kQuantVec = 2;    // 16-byte input vectors per lane and step

// The e4m3 byte nearest to v, ties to the even code, saturating (|v| finite).
// With k = max(exponent of |v|, -6), the grid of e4m3 values around |v| is
// (q / 8) 2^k for integer q (q in [8, 16] for normals, [0, 8] below 2^-6), so
// q = |v| 2^(3-k) rounded to nearest even (the scaling is exact) and the
// code is 8 k + 48 + q, which also carries q = 16 into the next exponent.
__device__ __forceinline__ uint32_t e4m3_rne(float v) {
  const uint32_t u = __float_as_uint(v);
  const int e = (int)((u >> 23) & 0xFFu) - 127;
  const int k = max(e, -6);
  const float t = fabsf(v) * __uint_as_float((uint32_t)(130 - k) << 23);
  const uint32_t code = (uint32_t)(8 * k + 48) + __float2uint_rn(t);
  return min(code, 0x7Fu) | ((u >> 24) & 0x80u);
}

// Codes of two products q = x * y, y within 2 ulp of 1 / scale, from the
// hardware conversion to e4m3 (round to nearest even).  Below 448 its grid is
// this format's grid (subnormals m 2^-9, normals (1 + m/8) 2^(e-7), sign bit
// 7), so the codes agree there; it saturates at 448 (0x7E), and this format
// goes on to 480 (0x7F), the code of every magnitude above the midpoint 464.
// The rule rounds the quotient x / scale once; q is within 2^-21.6 |q| of it
// (y's error and the product's rounding).  Each value is converted twice,
// moved up and down by 2^-20 of itself, which brackets the quotient: both
// codes equal (the code is monotone in the value) means the quotient has
// that code too.  Above 464 the code's low bit is set by a flag computed on
// the FMA pipe: (|v| - 464) 2^20 clamped to [0, 1] is 1.0 above 464 (the
// fp32 neighbours of 464 are 2^-15 away) and 0.0 up to it, and
// f0 + 256 f1 + 2^23 holds the two flags in its low bits, one per byte.
// Gives both sides' codes (qa | qb << 8): where a byte differs the caller
// takes the exact division for that element.
__device__ __forceinline__ uint32_t sat_flags(float a, float b) {
  const float fa = __saturatef(fmaf(fabsf(a), 0x1p20f, -464.0f * 0x1p20f));
  const float fb = __saturatef(fmaf(fabsf(b), 0x1p20f, -464.0f * 0x1p20f));
  return __float_as_uint(fmaf(fb, 256.0f, fa + 0x1p23f));
}
__device__ __forceinline__ void e4m3x2_bracket(float qa, float qb, uint32_t* up, uint32_t* lo) {
  constexpr float d = 0x1p-20f;
  const float ua = fmaf(qa, d, qa), ub = fmaf(qb, d, qb);  // the larger magnitudes
  const float la = fmaf(qa, -d, qa), lb = fmaf(qb, -d, qb);
  uint16_t cu, cl;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(cu) : "f"(ub), "f"(ua));
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(cl) : "f"(lb), "f"(la));
  *up = (uint32_t)cu | (sat_flags(ua, ub) & 0x0101u);  // 0x7E -> 0x7F above 464
  *lo = (uint32_t)cl | (sat_flags(la, lb) & 0x0101u);
}

// amax / 480 rounded to nearest.  For amax in [2^-100, FLT_MAX] a product
// with 1/480 (rounded) and one correction by its fused-multiply-add residual
// (Markstein's correction step) give the correctly rounded quotient; checked
// against the division for every float with an exponent in that range (the
// quotient's pattern repeats from binade to binade there).  Other values
// (zero, tiny, non-finite) take the division.
__device__ __forceinline__ float scale_of(float amax) {
  constexpr float c = 1.0f / 480.0f;
  if (amax >= 0x1p-100f && amax <= 3.40282347e38f) {
    const float q0 = amax * c;
    return fmaf(fmaf(-q0, 480.0f, amax), c, q0);
  }
  return amax / 480.0f;
}

// max(a, b) that returns NaN when either is NaN.
__device__ __forceinline__ float fmax_nan(float a, float b) {
  float r;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

template <int kDtype>
struct QuantIo;

template <>
struct QuantIo<QLC_DTYPE_F32> {
  static constexpr int kPerVec = 4;
  __device__ static void unpack(uint4 q, float* v) {
    v[0] = __uint_as_float(q.x), v[1] = __uint_as_float(q.y), v[2] = __uint_as_float(q.z),
    v[3] = __uint_as_float(q.w);
  }
  __device__ static void load_tail(const void* x, uint64_t i, uint64_t n, float* v) {
    const float* p = static_cast<const float*>(x);
    for (int j = 0; j < 4 * kQuantVec; j++) v[j] = i + j < n ? p[i + j] : 0.0f;
  }
};

template <>
struct QuantIo<QLC_DTYPE_BF16> {
  static constexpr int kPerVec = 8;
  __device__ static void unpack(uint4 q, float* v) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 4; j++) {
      v[2 * j] = __uint_as_float(w[j] << 16);
      v[2 * j + 1] = __uint_as_float(w[j] & 0xFFFF0000u);
    }
  }
  __device__ static void load_tail(const void* x, uint64_t i, uint64_t n, float* v) {
    const uint16_t* p = static_cast<const uint16_t*>(x);
    for (int j = 0; j < 8 * kQuantVec; j++) v[j] = i + j < n ? __uint_as_float((uint32_t)p[i + j] << 16) : 0.0f;
  }
};

__device__ __forceinline__ void q_cp_async16(uint32_t smem, const void* g, bool pred) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q cp.async.cg.shared.global [%0], [%1], 16;\n\t}" ::"r"(smem),
      "l"(g), "r"((uint32_t)pred)
      : "memory");
}
__device__ __forceinline__ void q_cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void q_cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Steps per launch: step indices and their products stay in 32 bits.
constexpr uint64_t kQuantMaxSteps = 1ull << 30;

// Scale and codes of one lane's E elements v (its block of 32 spans
// 32 / E lanes, whose absmax the shuffles combine).  Sets bad for NaN or
// infinity among v.  w receives the codes, 4 per word, element 4t + b in
// byte b of w[t].
template <int E>
__device__ __forceinline__ float lane_codes(const float (&v)[E], uint32_t (&w)[E / 4], bool& bad) {
  constexpr int kLanesPerBlock = 32 / E;
  constexpr int kWords = E / 4;
  float amax = 0.0f;
#pragma unroll
  for (int j = 0; j < E; j++) amax = fmax_nan(amax, fabsf(v[j]));
  bad |= !(amax <= 3.402823466e38f);  // NaN or infinity in this lane
#pragma unroll
  for (int o = 1; o < kLanesPerBlock; o <<= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  const float scale = scale_of(amax);
  // one reciprocal per lane and block, within 2 ulp for scale in
  // [2^-126, 2^126]; a scale below 2^-125 takes the exact division for
  // every element
  const float y = __fdividef(1.0f, scale);
  // dw: nonzero bytes mark the elements whose code the bracket leaves open
  // (all of them for a scale below 2^-125)
  uint32_t dw[kWords], open = 0u;
  const uint32_t all = scale >= 0x1p-125f ? 0u : ~0u;
#pragma unroll
  for (int t = 0; t < kWords; t++) {
    uint32_t u0, l0, u1, l1;
    e4m3x2_bracket(v[4 * t] * y, v[4 * t + 1] * y, &u0, &l0);
    e4m3x2_bracket(v[4 * t + 2] * y, v[4 * t + 3] * y, &u1, &l1);
    w[t] = __byte_perm(u0, u1, 0x5410);
    dw[t] = (w[t] ^ __byte_perm(l0, l1, 0x5410)) | all;
    open |= dw[t];
  }
  if (!(scale > 0.0f)) {
#pragma unroll
    for (int t = 0; t < kWords; t++) w[t] = 0u;
  } else if (open != 0u) {  // rare: the open elements alone take the exact division
#pragma unroll
    for (int t = 0; t < kWords; t++) {
      while (dw[t] != 0u) {
        const uint32_t sh = (uint32_t)(__ffs(dw[t]) - 1) & ~7u;  // bit 0 of the byte
        const uint32_t jb = sh >> 3;
        const float vj = jb == 0 ? v[4 * t] : jb == 1 ? v[4 * t + 1] : jb == 2 ? v[4 * t + 2] : v[4 * t + 3];
        w[t] = (w[t] & ~(0xFFu << sh)) | (e4m3_rne(vj / scale) << sh);
        dw[t] &= ~(0xFFu << sh);
      }
    }
  }
  return scale;
}

// Input pipeline: warp step s covers elements [s kStep, (s + 1) kStep),
// 1 KiB of input, 32 contiguous bytes per lane; warps take steps s = first,
// first + W, ... (W warps in the grid).  A warp keeps its next
// kQuantDepth - 1 steps in flight: its k-th step goes by cp.async into its
// 1 KiB of shared slot k mod kQuantDepth, each copy instruction 512
// contiguous bytes (one commit group per step; in a ragged last step only
// the 16-byte vectors wholly inside are copied).  About 100 bytes per thread
// are in flight without holding registers.  Lanes read bytes other lanes
// copied, so each step starts with the lane's wait on its own groups and a
// warp barrier; a slot is refilled after that barrier, when every lane has
// finished the step that read it.  Every step but a ragged last one takes
// the short path; there a lane whose 32 bytes are not wholly inside reads
// its elements with plain loads.
template <int kDtype>
__global__ void __launch_bounds__(kQuantThreads)
quantize_kernel(const void* __restrict__ x, uint64_t n, uint8_t* __restrict__ codes, float* __restrict__ scales,
                unsigned long long* __restrict__ hist, uint32_t* __restrict__ status) {
  constexpr int E = QuantIo<kDtype>::kPerVec * kQuantVec;  // elements per lane
  constexpr int kLanesPerBlock = 32 / E;
  constexpr uint32_t kStep = 32 * E;             // elements per warp step
  constexpr uint32_t kWords = E / 4;             // code words per lane
  constexpr uint32_t kSlot = kQuantWarps * kQuantVec * 512u;  // bytes of a ring slot
  __shared__ uint32_t sh[kQuantWarps][256];  // per-warp histograms
  __shared__ uint4 ring[kQuantDepth][kQuantWarps][kQuantVec * 32];
  if (hist) {
    for (int i = threadIdx.x; i < kQuantWarps * 256; i += kQuantThreads) (&sh[0][0])[i] = 0;
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* my = sh[warp];
  const uint32_t n_steps = (uint32_t)((n + kStep - 1) / kStep);  // <= kQuantMaxSteps
  const uint32_t warps = gridDim.x * kQuantWarps;
  const uint32_t first = blockIdx.x * kQuantWarps + warp;
  const uint32_t cnt = first < n_steps ? (n_steps - first + warps - 1) / warps : 0;  // this warp's steps
  // this warp's steps whose whole 1 KiB lies inside: all but a ragged last
  const uint32_t nfw = cnt > 0 && first + (cnt - 1) * warps == n_steps - 1 && (uint64_t)n_steps * kStep > n
                           ? cnt - 1 : cnt;
  const uint64_t n_bytes = n * (16 / QuantIo<kDtype>::kPerVec);
  uint8_t* c_lane = codes + lane * E;
  float* s_lane = scales + lane / kLanesPerBlock;
  const bool scale_lane = lane % kLanesPerBlock == 0;
  // copy instruction u of lane l: bytes [512 u + 16 l, + 16) of the step
  const uint8_t* x_copy = static_cast<const uint8_t*>(x) + lane * 16;
  const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(&ring[0][warp][lane]);
  auto fetch = [&](uint32_t k) {  // step k of this warp into slot k mod kQuantDepth
    const uint32_t d = ring_s + (k % kQuantDepth) * kSlot;
    const uint64_t b = (uint64_t)(first + k * warps) * (512u * kQuantVec);
    if (k < nfw) {
#pragma unroll
      for (int u = 0; u < kQuantVec; u++)
        q_cp_async16(d + 512u * u, x_copy + b + 512u * u,
                     QLC_GUARD(b + lane * 16 + 512u * u + 16 <= n_bytes, status));
    } else if (k < cnt) {  // the ragged last step: the vectors wholly inside
#pragma unroll
      for (int u = 0; u < kQuantVec; u++) {
        const bool in = b + lane * 16 + 512u * u + 16 <= n_bytes;
        q_cp_async16(d + 512u * u, in ? x_copy + b + 512u * u : x_copy, in);
      }
    }
    q_cp_async_commit();
  };
  auto count = [&](const uint32_t (&w)[kWords], int m) {  // the first m codes into the histogram
#pragma unroll
    for (int j = 0; j < E; j++) {
      if (j < m) {
        const uint32_t c = __byte_perm(w[j / 4], 0, 0x4440 + (j % 4));
        atomicAdd(&my[c], 1u);
      }
    }
  };
#pragma unroll
  for (uint32_t d = 0; d + 1 < kQuantDepth; d++) fetch(d);
  bool bad = false;
  uint32_t s = first, k = 0;
  for (; k < nfw; k++, s += warps) {
    // groups committed so far: kQuantDepth - 1 + k; step k's is complete
    // when at most kQuantDepth - 2 are pending
    q_cp_async_wait<kQuantDepth - 2>();
    __syncwarp();
    fetch(k + kQuantDepth - 1);  // into the slot step k - 1 was read from
    float v[E];
    const uint4* r = &ring[k % kQuantDepth][warp][lane * kQuantVec];
#pragma unroll
    for (int u = 0; u < kQuantVec; u++) QuantIo<kDtype>::unpack(r[u], v + u * QuantIo<kDtype>::kPerVec);
    uint32_t w[kWords];
    const float scale = lane_codes<E>(v, w, bad);
    if (scale_lane && QLC_GUARD((uint64_t)s * kStep + lane * E < n, status)) s_lane[(uint64_t)s * (kStep / 32)] = scale;
    if (QLC_GUARD((uint64_t)s * kStep + (lane + 1) * E <= n, status)) {
      if constexpr (kWords == 2)
        *reinterpret_cast<uint2*>(c_lane + (uint64_t)s * kStep) = make_uint2(w[0], w[1]);
      else
        *reinterpret_cast<uint4*>(c_lane + (uint64_t)s * kStep) = make_uint4(w[0], w[1], w[2], w[3]);
      if (hist) count(w, E);
    }
  }
  if (k < cnt) {  // the ragged last step
    q_cp_async_wait<0>();
    __syncwarp();
    const uint64_t i = (uint64_t)s * kStep + (uint64_t)lane * E;
    float v[E];
    if (i + E <= n) {
      const uint4* r = &ring[k % kQuantDepth][warp][lane * kQuantVec];
#pragma unroll
      for (int u = 0; u < kQuantVec; u++) QuantIo<kDtype>::unpack(r[u], v + u * QuantIo<kDtype>::kPerVec);
    } else {
      QuantIo<kDtype>::load_tail(x, i, n, v);  // zeros past the end
    }
    uint32_t w[kWords];
    const float scale = lane_codes<E>(v, w, bad);
    if (scale_lane && i < n && QLC_GUARD(i / 32 < (n + 31) / 32, status)) scales[i / 32] = scale;
    for (int j = 0; j < E; j++)
      if (i + j < n) codes[i + j] = (uint8_t)(w[j / 4] >> (8 * (j % 4)));
    if (hist && i < n) count(w, (int)(n - i < (uint64_t)E ? n - i : E));
  }
  q_cp_async_wait<0>();
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(status, QLC_ERR_ARG);
  if (hist) {
    for (int b = threadIdx.x; b < 256; b += kQuantThreads) {
      uint32_t t = 0;
#pragma unroll
      for (int w = 0; w < kQuantWarps; w++) t += sh[w][b];
      if (t) atomicAdd(&hist[b], (unsigned long long)t);
    }
  }
}

// out[i] = value(codes[i]) * scales[i / 32].  Warp step s covers codes
// [512 s, 512 s + 512); in part k (0..3) lane l takes codes
// [512 s + 128 k + 4 l, + 4), so each load and store instruction of the warp
// covers contiguous bytes (128 bytes of codes, 512 of fp32 or 256 of bf16).
template <int kDtype>
__global__ void __launch_bounds__(256)
dequantize_kernel(const uint8_t* __restrict__ codes, const float* __restrict__ scales, uint64_t n,
                  void* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint64_t n_steps = (n + 511) / 512;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  for (uint64_t s = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; s < n_steps; s += warps) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint64_t i = s * 512 + 128 * k + 4 * lane;
      if (i >= n) continue;
      const float sc = scales[i / 32];
      uint32_t w = 0;
      if (i + 4 <= n) {
        w = __ldg(reinterpret_cast<const unsigned int*>(codes + i));
      } else {
        for (int j = 0; j < 4; j++)
          if (i + j < n) w |= (uint32_t)codes[i + j] << (8 * j);
      }
      float y[4];
#pragma unroll
      for (int j = 0; j < 4; j++) y[j] = __uint_as_float(e4m3_scaled_bits(w, j)) * 0x1p120f * sc;
      if (kDtype == QLC_DTYPE_F32) {
        float* o = static_cast<float*>(out) + i;
        if (i + 4 <= n) {
          __stcs(reinterpret_cast<float4*>(o), make_float4(y[0], y[1], y[2], y[3]));
        } else {
          for (int j = 0; j < 4; j++)
            if (i + j < n) o[j] = y[j];
        }
      } else {
        __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out) + i;
        if (i + 4 <= n) {
          const __nv_bfloat162 h0 = __floats2bfloat162_rn(y[0], y[1]), h1 = __floats2bfloat162_rn(y[2], y[3]);
          __stcs(reinterpret_cast<uint2*>(o), make_uint2(*reinterpret_cast<const uint32_t*>(&h0),
                                                         *reinterpret_cast<const uint32_t*>(&h1)));
        } else {
          for (int j = 0; j < 4; j++)
            if (i + j < n) o[j] = __float2bfloat16_rn(y[j]);
        }
      }
    }
  }
}

}  // namespace qlc

namespace qlc {
// Resident quantiser CTAs per SM (the occupancy calculator's figure, cached
// per device below 64 and dtype; at least 1).
static int quant_ctas_per_sm(qlc_dtype dtype) {
  static std::atomic<int> cached[64][2];
  const int k = dtype == QLC_DTYPE_F32 ? 0 : 1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 64;
  if (dev < 64) {
    const int c = cached[dev][k].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int v = 0;
  const cudaError_t e =
      k == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, quantize_kernel<QLC_DTYPE_F32>, kQuantThreads, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, quantize_kernel<QLC_DTYPE_BF16>, kQuantThreads, 0);
  if (e != cudaSuccess || v <= 0) v = 1;
  if (dev < 64) cached[dev][k].store(v, std::memory_order_relaxed);
  return v;
}
}  // namespace qlc

using namespace qlc;

extern "C" qlc_status qlc_quantize_e4m3(const void* d_x, qlc_dtype dtype, size_t n, uint8_t* d_codes,
                                        float* d_scales, uint64_t* d_hist, int accumulate, uint32_t* d_status,
                                        qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_quantize_e4m3");
  if (dtype != QLC_DTYPE_F32 && dtype != QLC_DTYPE_BF16) return QLC_ERR_ARG;
  if (n > 0 && (!d_x || !d_codes || !d_scales)) return QLC_ERR_ARG;
  if (!aligned(d_x, 16) || !aligned(d_codes, 16) || !aligned(d_scales, 16) || !aligned(d_hist, 8) ||
      !aligned(d_status, 4))
    return QLC_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (d_hist && !accumulate && cudaMemsetAsync(d_hist, 0, 256 * sizeof(uint64_t), st) != cudaSuccess)
    return QLC_ERR_CUDA;
  if (n == 0) return QLC_OK;
  // one resident wave: each CTA loops over its steps with its copies in
  // flight; inputs above kQuantMaxSteps steps go in several launches (slices
  // of whole blocks, the histogram accumulating)
  const uint64_t step = (uint64_t)32 * kQuantVec * (dtype == QLC_DTYPE_F32 ? 4 : 8);  // elements per warp step
  const uint64_t elem = dtype == QLC_DTYPE_F32 ? 4 : 2;
  const uint64_t slice = kQuantMaxSteps * step;
  const uint64_t cap = (uint64_t)sm_count() * quant_ctas_per_sm(dtype);
  unsigned long long* h = reinterpret_cast<unsigned long long*>(d_hist);
  for (uint64_t off = 0; off < n; off += slice) {
    const uint64_t m = n - off < slice ? n - off : slice;
    const uint64_t want = (m + step * kQuantWarps - 1) / (step * kQuantWarps);
    const int grid = (int)(want < cap ? want : cap);
    const void* xs = static_cast<const uint8_t*>(d_x) + off * elem;
    if (dtype == QLC_DTYPE_F32)
      quantize_kernel<QLC_DTYPE_F32><<<grid, kQuantThreads, 0, st>>>(xs, m, d_codes + off, d_scales + off / 32, h,
                                                                     d_status);
    else
      quantize_kernel<QLC_DTYPE_BF16><<<grid, kQuantThreads, 0, st>>>(xs, m, d_codes + off, d_scales + off / 32, h,
                                                                      d_status);
  }
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}

extern "C" qlc_status qlc_dequantize_e4m3(const uint8_t* d_codes, const float* d_scales, size_t n, void* d_out,
                                          qlc_dtype dtype, qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_dequantize_e4m3");
  if (dtype != QLC_DTYPE_F32 && dtype != QLC_DTYPE_BF16) return QLC_ERR_ARG;
  if (n > 0 && (!d_codes || !d_scales || !d_out)) return QLC_ERR_ARG;
  if (!aligned(d_codes, 16) || !aligned(d_out, 16) || !aligned(d_scales, 4)) return QLC_ERR_ARG;
  if (n == 0) return QLC_OK;
  const uint64_t want = ((n + 511) / 512 + 7) / 8;  // warp steps of 512 codes, 8 warps per CTA
  const uint64_t cap = (uint64_t)sm_count() * 8;
  const int grid = (int)(want < cap ? want : cap);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (dtype == QLC_DTYPE_F32)
    dequantize_kernel<QLC_DTYPE_F32><<<grid, 256, 0, st>>>(d_codes, d_scales, n, d_out);
  else
    dequantize_kernel<QLC_DTYPE_BF16><<<grid, 256, 0, st>>>(d_codes, d_scales, n, d_out);
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}

namespace qlc {
QLC_DEFINE_CHECK_TAKE(check_take_quant)
}  // namespace qlc
