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
// A warp handles 32 x 16 bytes of input per step: 4 fp32 (or 8 bf16) elements
// per lane, so one block of 32 is 8 (or 4) lanes and its absmax is a 3 (or 2)
// step butterfly.  Codes leave as one 4- (or 8-) byte store per lane.
#include <cuda_bf16.h>

#define QLC_FILE_ID 5
#include "qlc_common.cuh"

namespace qlc {

constexpr int kQuantWarps = 8;
constexpr int kQuantThreads = kQuantWarps * 32;
constexpr int kQuantUnroll = 2;

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

// The same rounding of q0 = x * (1 / scale), which is not the quotient the
// rule names (x / scale, rounded once) but lies within 2^-23 |x / scale| of
// it: both 1 / scale and the product are rounded to nearest.  The code is a
// step function of the value whose steps sit at the midpoints between
// neighbouring e4m3 magnitudes, exact fp32 numbers, so q0 and the rounded
// quotient get the same code unless one of them lies within 2^-22 |q0| of a
// midpoint.  In grid units (t = |q0| 2^(3-k), |q0| < 2^(k+1)) that margin is
// under 2^-18 of a step; *near is set when t lies within 2^-17 of a midpoint,
// and the caller then takes the exact division.  Outside the margin the code
// is the rule's, so the result is exact either way.
__device__ __forceinline__ uint32_t e4m3_rne_or_near(float q0, bool* near) {
  const uint32_t u = __float_as_uint(q0);
  const int e = (int)((u >> 23) & 0xFFu) - 127;
  const int k = max(e, -6);
  const float t = fabsf(q0) * __uint_as_float((uint32_t)(130 - k) << 23);
  const float rt = rintf(t);
  *near = fabsf(t - rt) > 0.5f - 0x1p-17f;  // t - rt is exact
  const uint32_t code = (uint32_t)(8 * k + 48) + (uint32_t)rt;
  return min(code, 0x7Fu) | ((u >> 24) & 0x80u);
}

template <int kDtype>
struct QuantIo;

template <>
struct QuantIo<QLC_DTYPE_F32> {
  static constexpr int kPerLane = 4;
  __device__ static void load(const void* x, uint64_t i, uint64_t n, float* v) {
    const float* p = static_cast<const float*>(x) + i;
    if (i + 4 <= n) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(p));
      v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
    } else {
      for (int j = 0; j < 4; j++) v[j] = i + j < n ? p[j] : 0.0f;
    }
  }
};

template <>
struct QuantIo<QLC_DTYPE_BF16> {
  static constexpr int kPerLane = 8;
  __device__ static void load(const void* x, uint64_t i, uint64_t n, float* v) {
    const uint16_t* p = static_cast<const uint16_t*>(x) + i;
    if (i + 8 <= n) {
      const uint4 q = ldg_nc_v4(reinterpret_cast<const uint4*>(p));
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int j = 0; j < 4; j++) {
        v[2 * j] = __uint_as_float(w[j] << 16);
        v[2 * j + 1] = __uint_as_float(w[j] & 0xFFFF0000u);
      }
    } else {
      for (int j = 0; j < 8; j++) v[j] = i + j < n ? __uint_as_float((uint32_t)p[j] << 16) : 0.0f;
    }
  }
};

template <int kDtype>
__global__ void __launch_bounds__(kQuantThreads)
quantize_kernel(const void* __restrict__ x, uint64_t n, uint8_t* __restrict__ codes, float* __restrict__ scales,
                unsigned long long* __restrict__ hist, uint32_t* __restrict__ status) {
  constexpr int E = QuantIo<kDtype>::kPerLane;  // elements per lane
  constexpr int kLanesPerBlock = 32 / E;
  constexpr uint64_t kStep = 32 * E;             // elements per warp step
  __shared__ uint32_t sh[kQuantWarps][257];
  if (hist) {
    for (int i = threadIdx.x; i < kQuantWarps * 257; i += kQuantThreads) (&sh[0][0])[i] = 0;
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* my = sh[warp];
  const uint64_t n_steps = (n + kStep - 1) / kStep;
  const uint64_t warps = (uint64_t)gridDim.x * kQuantWarps;
  bool bad = false;
  for (uint64_t s0 = (uint64_t)blockIdx.x * kQuantWarps + warp; s0 < n_steps; s0 += warps * kQuantUnroll) {
    float v[kQuantUnroll][E];
#pragma unroll
    for (int u = 0; u < kQuantUnroll; u++) {
      const uint64_t s = s0 + u * warps;
      const uint64_t i = s * kStep + (uint64_t)lane * E;
      if (s < n_steps && i < n) {
        QuantIo<kDtype>::load(x, i, n, v[u]);
      } else {
#pragma unroll
        for (int j = 0; j < E; j++) v[u][j] = 0.0f;
      }
    }
#pragma unroll
    for (int u = 0; u < kQuantUnroll; u++) {
      const uint64_t s = s0 + u * warps;
      if (s >= n_steps) break;  // warp-uniform
      const uint64_t i = s * kStep + (uint64_t)lane * E;
      float amax = 0.0f;
#pragma unroll
      for (int j = 0; j < E; j++) {
        bad |= !isfinite(v[u][j]);
        amax = fmaxf(amax, fabsf(v[u][j]));
      }
#pragma unroll
      for (int o = 1; o < kLanesPerBlock; o <<= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      const float scale = amax / 480.0f;
      // one reciprocal per lane and block; a scale below 2^-125 (whose
      // reciprocal could overflow) takes the exact division for every element
      const float y = 1.0f / scale;
      const bool by_product = scale >= 0x1p-125f;
      uint32_t c[E];
      bool exact = !by_product;
#pragma unroll
      for (int j = 0; j < E; j++) {
        bool near;
        c[j] = e4m3_rne_or_near(v[u][j] * y, &near);
        exact |= near;
      }
      if (!(scale > 0.0f)) {
#pragma unroll
        for (int j = 0; j < E; j++) c[j] = 0u;
      } else if (exact) {  // rare: one branch per lane and block
#pragma unroll
        for (int j = 0; j < E; j++) c[j] = e4m3_rne(v[u][j] / scale);
      }
      if (i < n && (lane % kLanesPerBlock) == 0 && QLC_GUARD(i / 32 < (n + 31) / 32, status)) scales[i / 32] = scale;
      if (i + E <= n) {
        if (E == 4) {
          *reinterpret_cast<uint32_t*>(codes + i) = c[0] | c[1] << 8 | c[2] << 16 | c[3] << 24;
        } else {
          *reinterpret_cast<uint2*>(codes + i) =
              make_uint2(c[0] | c[1] << 8 | c[2] << 16 | c[3] << 24, c[4] | c[5] << 8 | c[6] << 16 | c[7] << 24);
        }
        if (hist) {
#pragma unroll
          for (int j = 0; j < E; j++)
            if (QLC_GUARD(c[j] < 256u, status)) atomicAdd(&my[c[j] + (c[j] >> 7)], 1u);
        }
      } else {
        for (int j = 0; j < E; j++) {
          if (i + j < n) {
            codes[i + j] = (uint8_t)c[j];
            if (hist && QLC_GUARD(c[j] < 256u, status)) atomicAdd(&my[c[j] + (c[j] >> 7)], 1u);
          }
        }
      }
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(status, QLC_ERR_ARG);
  if (hist) {
    for (int b = threadIdx.x; b < 256; b += kQuantThreads) {
      uint32_t t = 0;
#pragma unroll
      for (int w = 0; w < kQuantWarps; w++) t += sh[w][b + (b >> 7)];
      if (t) atomicAdd(&hist[b], (unsigned long long)t);
    }
  }
}

// out[i] = value(codes[i]) * scales[i / 32]; 16 codes per lane per step.
template <int kDtype>
__global__ void __launch_bounds__(256)
dequantize_kernel(const uint8_t* __restrict__ codes, const float* __restrict__ scales, uint64_t n,
                  void* __restrict__ out) {
  const uint64_t n16 = (n + 15) / 16;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n16; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = t * 16;
    const float sc = scales[i / 32];
    uint32_t w[4];
    if (i + 16 <= n) {
      const uint4 q = ldg_nc_v4(reinterpret_cast<const uint4*>(codes + i));
      w[0] = q.x, w[1] = q.y, w[2] = q.z, w[3] = q.w;
    } else {
      w[0] = w[1] = w[2] = w[3] = 0;
#pragma unroll
      for (int j = 0; j < 16; j++)
        if (i + j < n) w[j >> 2] |= (uint32_t)codes[i + j] << (8 * (j & 3));
    }
    float y[16];
#pragma unroll
    for (int j = 0; j < 16; j++) y[j] = e4m3_to_f32((w[j >> 2] >> (8 * (j & 3))) & 0xFFu) * sc;
    if (kDtype == QLC_DTYPE_F32) {
      float* o = static_cast<float*>(out) + i;
      if (i + 16 <= n) {
#pragma unroll
        for (int k = 0; k < 4; k++)
          __stcs(reinterpret_cast<float4*>(o) + k, make_float4(y[4 * k], y[4 * k + 1], y[4 * k + 2], y[4 * k + 3]));
      } else {
#pragma unroll
        for (int j = 0; j < 16; j++)
          if (i + j < n) o[j] = y[j];
      }
    } else {
      __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out) + i;
      if (i + 16 <= n) {
        uint32_t p[8];
#pragma unroll
        for (int k = 0; k < 8; k++) {
          const __nv_bfloat162 h = __floats2bfloat162_rn(y[2 * k], y[2 * k + 1]);
          p[k] = *reinterpret_cast<const uint32_t*>(&h);
        }
        __stcs(reinterpret_cast<uint4*>(o), make_uint4(p[0], p[1], p[2], p[3]));
        __stcs(reinterpret_cast<uint4*>(o) + 1, make_uint4(p[4], p[5], p[6], p[7]));
      } else {
#pragma unroll
        for (int j = 0; j < 16; j++)
          if (i + j < n) o[j] = __float2bfloat16_rn(y[j]);
      }
    }
  }
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
  const uint64_t per_cta = (uint64_t)kQuantThreads * (dtype == QLC_DTYPE_F32 ? 4 : 8) * kQuantUnroll;
  const uint64_t want = (n + per_cta - 1) / per_cta;
  const uint64_t cap = (uint64_t)sm_count() * 8;
  const int grid = (int)(want < cap ? want : cap);
  unsigned long long* h = reinterpret_cast<unsigned long long*>(d_hist);
  if (dtype == QLC_DTYPE_F32)
    quantize_kernel<QLC_DTYPE_F32><<<grid, kQuantThreads, 0, st>>>(d_x, n, d_codes, d_scales, h, d_status);
  else
    quantize_kernel<QLC_DTYPE_BF16><<<grid, kQuantThreads, 0, st>>>(d_x, n, d_codes, d_scales, h, d_status);
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}

extern "C" qlc_status qlc_dequantize_e4m3(const uint8_t* d_codes, const float* d_scales, size_t n, void* d_out,
                                          qlc_dtype dtype, qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_dequantize_e4m3");
  if (dtype != QLC_DTYPE_F32 && dtype != QLC_DTYPE_BF16) return QLC_ERR_ARG;
  if (n > 0 && (!d_codes || !d_scales || !d_out)) return QLC_ERR_ARG;
  if (!aligned(d_codes, 16) || !aligned(d_out, 16) || !aligned(d_scales, 4)) return QLC_ERR_ARG;
  if (n == 0) return QLC_OK;
  const uint64_t want = ((n + 15) / 16 + 255) / 256;
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
