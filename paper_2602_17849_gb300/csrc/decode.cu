// decode.cu -- QLC decoder (Section 7) for container v1.
//
// One warp per group of 32 chunks, one lane per chunk: the codes are not
// self-synchronising, so each lane starts at its chunk's bit offset (group
// offset + exclusive scan of the group's chunk_bits) and decodes its chunk
// serially.  Per symbol: the top 3 bits of a 64-bit bit buffer are the area
// code; the code length 3 + bits[area] comes from a byte permute of two
// registers (no memory access on the serial path); the whole codeword (area
// code and suffix, right-aligned) indexes a 2048-entry code -> symbol table in
// shared memory built from the LUT and the area table.  The rank is never
// formed explicitly: for every code of every area the table holds
// dec[offset + suffix] (offset 0 for 8-bit areas), exactly the paper's rule.
// Input: each lane's chunk bytes stream through a 128-byte shared-memory ring
// filled by cp.async; the buffer is refilled one word per two symbols under
// predication, so lanes never diverge.  Output: 16 symbols per shared store
// into a swizzled 32 x 32-byte tile; every 32 symbols the warp writes the tile
// out, one 32-byte segment per chunk.
#include <cuda_bf16.h>

#include "qlc_common.cuh"

namespace qlc {

constexpr int kDecCtasPerSm = 26;  // 26 x (7.4 KB + 1 KB reserved) fits in 228 KB

struct DecHeader {
  uint64_t n, payload_bytes, P, n_chunks, n_groups;
  uint32_t cs;
  uint32_t len_lo, len_hi;  // code length of areas 0-3 / 4-7, one byte each
};

__constant__ uint16_t c_table_n[2][8] = {{8, 8, 8, 8, 8, 16, 32, 168}, {2, 8, 8, 8, 8, 32, 32, 158}};
__constant__ uint8_t c_table_b[2][8] = {{3, 3, 3, 3, 3, 4, 5, 8}, {1, 3, 3, 3, 3, 5, 5, 8}};

// Parses and validates the header (all lanes, redundantly); same checks, in
// the same order of kinds, as the container rules: 0 = ok, else a status.
__device__ uint32_t parse_header(const uint8_t* in, uint64_t in_bytes, uint64_t out_cap,
                                 DecHeader* h, uint32_t* s_seen, int lane) {
  if (in_bytes < kIndexOff) return QLC_ERR_CORRUPT;
  const uint32_t w0 = *reinterpret_cast<const uint32_t*>(in);
  const uint32_t w1 = *reinterpret_cast<const uint32_t*>(in + 4);
  const unsigned long long reserved = *reinterpret_cast<const unsigned long long*>(in + 56);
  bool ok = w0 == 0x31434C51u && (w1 & 0xFFFFu) == QLC_VERSION && (w1 >> 24) == 0 && reserved == 0;
  const uint32_t id = (w1 >> 16) & 0xFFu;
  uint16_t an[8];
  uint8_t ab[8];
  for (int i = 0; i < 8; i++) {
    an[i] = *reinterpret_cast<const uint16_t*>(in + 24 + 2 * i);
    ab[i] = in[40 + i];
  }
  ok = ok && scheme_ok(an, ab);
  if (id == 1 || id == 2) {
    for (int i = 0; i < 8; i++) ok = ok && an[i] == c_table_n[id - 1][i] && ab[i] == c_table_b[id - 1][i];
  } else {
    ok = ok && id == 0;
  }
  h->n = *reinterpret_cast<const unsigned long long*>(in + 8);
  h->cs = *reinterpret_cast<const uint32_t*>(in + 16);
  h->n_chunks = *reinterpret_cast<const uint32_t*>(in + 20);
  ok = ok && chunk_symbols_ok(h->cs) && h->n_chunks == (h->n + h->cs - 1) / h->cs;
  // dec must be a permutation of 0..255
  if (lane < 8) s_seen[lane] = 0;
  __syncwarp();
  for (int i = lane; i < 256; i += 32) {
    const uint32_t s = in[64 + i];
    atomicOr(&s_seen[s >> 5], 1u << (s & 31));
  }
  __syncwarp();
  uint32_t seen = 0;
  for (int i = 0; i < 8; i++) seen += __popc(s_seen[i]);
  ok = ok && seen == 256;
  h->n_groups = n_groups_of(h->n_chunks);
  h->P = payload_start(h->n_chunks);
  h->payload_bytes = *reinterpret_cast<const unsigned long long*>(in + 48);
  ok = ok && h->P <= in_bytes && h->payload_bytes <= in_bytes - h->P;
  if (!ok) return QLC_ERR_CORRUPT;
  if (out_cap < h->n) return QLC_ERR_CAPACITY;
  h->len_lo = h->len_hi = 0;
  for (int i = 0; i < 4; i++) {
    h->len_lo |= (3u + ab[i]) << (8 * i);
    h->len_hi |= (3u + ab[i + 4]) << (8 * i);
  }
  return 0;
}

// cp.async (global -> shared, 16 bytes, bypassing L1) and its groups.
__device__ __forceinline__ void cp_async16(uint32_t smem, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

constexpr uint32_t kBlk = 32;       // symbols per lane between output flushes
constexpr uint32_t kRingVec = 8;    // 16-byte vectors in each lane's input ring (128 B)

// (hi * 8) >> 32 + c, i.e. (hi >> 29) + c, on the multiply-add pipe.
__device__ __forceinline__ uint32_t mad_hi(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
// prmt.b32 in its default mode; a selector nibble with bit 3 set yields the
// sign of the selected byte replicated (0x00 for bytes below 0x80).
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}
__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
// 0x80000000 >> s with PTX semantics (0 for s >= 32).
__device__ __forceinline__ uint32_t top_bit_shr(uint32_t s) {
  uint32_t d;
  asm("shr.b32 %0, %1, %2;" : "=r"(d) : "r"(0x80000000u), "r"(s));
  return d;
}
__device__ __forceinline__ uint32_t ld_shared_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}


// Per-lane decoder state.  Input: the lane's chunk bytes are copied 16 bytes
// at a time (cp.async) into a 128-byte ring in shared memory, ahead of use.
// Bits: a 64-bit buffer (hi:lo) of valid bits, most significant first, with
// nb1 = (valid bits - 1).  Two symbols (at most 2 x 11 bits) are decoded per
// round with no branch; then one 32-bit word is inserted, under predication,
// when at most 32 bits are left, which keeps at least 32 valid bits at the
// start of every round.
struct LaneDec {
  uint32_t hi, lo;
  uint32_t nb1;
  uint32_t rpb;  // byte offset (group-relative) of the next word to insert
  uint32_t nxt;  // that word, already read from the ring
  uint32_t fv;   // next 16-byte vector to fetch (group-relative)
  uint32_t vend; // vectors in the group
  const uint4* gp;
  uint32_t ring_s;  // shared address of this lane's ring (128-byte aligned)

  // Fetch vectors up to the ring's capacity past the read position, never
  // past the group end, and commit them as one cp.async group.
  __device__ __forceinline__ void fetch() {
    const uint32_t want = min((rpb >> 4) + kRingVec, vend);
    for (; fv < want; fv++) cp_async16(ring_s + (fv % kRingVec) * 16, gp + fv);
    cp_async_commit();
  }
  // The same top-up between blocks, as three predicated copies with no
  // branch: a block of kBlk symbols consumes at most kBlk * 11 bits = 44
  // bytes, so the read position, and with it `want`, moves by at most three
  // 16-byte vectors per block.
  __device__ __forceinline__ void fetch3() {
    const uint32_t want = min((rpb >> 4) + kRingVec, vend);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const uint32_t p = fv < want;
      asm volatile(
          "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q cp.async.cg.shared.global [%0], [%1], 16;\n\t}" ::"r"(
              ring_s + (fv % kRingVec) * 16),
          "l"(gp + fv), "r"(p)
          : "memory");
      fv += p;
    }
    cp_async_commit();
  }
  __device__ __forceinline__ uint32_t ring_word(uint32_t byte_off) const {
    // ring_s is 128-byte aligned, so OR places the offset inside the ring
    return bswap32(ld_shared_u32(ring_s | (byte_off & (kRingVec * 16 - 1))));
  }
  // Code length of the codeword at the top of x (Section 7: the area code,
  // i.e. the top 3 bits, fixes it): a byte permute of two registers; the
  // selector's sign-mode nibbles make bytes 1-3 zero.
  __device__ __forceinline__ static uint32_t code_len(uint32_t x, uint32_t len_lo, uint32_t len_hi) {
    return prmt(len_lo, len_hi, mad_hi(x, 8u, 0x8880u));
  }
  // Insert the next word below the valid bits when at most 32 remain:
  // q = 2^(32 - valid), or 0 when no word is due, so the insertion is two
  // multiply-adds with no select.
  __device__ __forceinline__ void refill() {
    const uint32_t q = top_bit_shr(nb1);
    hi = mad_hi(nxt, q, hi);  // nxt >> valid
    lo = mad_lo(nxt, q, lo);  // nxt << (32 - valid)
    if (nb1 < 32) {
      nb1 += 32;
      rpb += 4;
      nxt = ring_word(rpb);
    }
  }
  // Two symbols (at most 22 bits) from the top of the buffer, packed as
  // s0 | s1 << 8; the buffer advances once by both lengths.
  __device__ __forceinline__ uint32_t round2(const uint8_t* T, uint32_t len_lo, uint32_t len_hi) {
    const uint32_t la = code_len(hi, len_lo, len_hi);
    const uint32_t a = T[__funnelshift_l(hi, 0u, la)];
    const uint32_t h1 = __funnelshift_l(lo, hi, la);
    const uint32_t lb = code_len(h1, len_lo, len_hi);
    const uint32_t b = T[__funnelshift_l(h1, 0u, lb)];
    const uint32_t lab = la + lb;
    hi = __funnelshift_l(lo, hi, lab);
    lo <<= lab;
    nb1 -= lab;
    refill();
    return mad_lo(b, 256u, a);
  }
  // One symbol with a refill (ragged chunk ends only).
  __device__ __forceinline__ uint32_t round1(const uint8_t* T, uint32_t len_lo, uint32_t len_hi) {
    const uint32_t la = code_len(hi, len_lo, len_hi);
    const uint32_t a = T[__funnelshift_l(hi, 0u, la)];
    hi = __funnelshift_l(lo, hi, la);
    lo <<= la;
    nb1 -= la;
    refill();
    return a;
  }
};

struct DecShared {
  uint8_t T[2048];
  __align__(128) uint4 ring[32 * kRingVec];
  __align__(16) uint4 tile[32 * (kBlk / 16)];
  __align__(16) uint8_t dec[256];
  uint32_t seen[8];
};

// code -> symbol table: every code (i << bits[i]) | s of every area i maps to
// dec[offset_i + s] (offset 0 for 8-bit areas); dec is staged in shared.
__device__ void build_table(const uint8_t* in, DecShared& sm, int lane) {
  reinterpret_cast<uint32_t*>(sm.dec)[lane] = reinterpret_cast<const uint32_t*>(in + 64)[lane];
  reinterpret_cast<uint32_t*>(sm.dec)[lane + 32] = reinterpret_cast<const uint32_t*>(in + 64)[lane + 32];
  __syncwarp();
  uint32_t base = 0;
  for (int i = 0; i < 8; i++) {
    const uint32_t b = in[40 + i];
    for (uint32_t s = lane; s < (1u << b); s += 32) sm.T[(i << b) | s] = sm.dec[b == 8 ? s : base + s];
    base += *reinterpret_cast<const uint16_t*>(in + 24 + 2 * i);
  }
  __syncwarp();
}

// Output of the decoder: the symbols themselves (kOutCodes), or their
// block-32 dequantised values (value(code) * scale, fp32 or rounded to bf16).
constexpr int kOutCodes = -1;

// Streaming 16-byte store of decoded symbols when pred (a predicated store).
__device__ __forceinline__ void put16_if(uint8_t* dst, uint4 v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t@q st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};\n\t}" ::"l"(dst),
      "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"((uint32_t)pred)
      : "memory");
}

// Sixteen decoded symbols v of one chunk, starting at symbol index i of the
// tensor (a multiple of 16), to their destination.
template <int kOut>
__device__ __forceinline__ void put16(void* out, const float* scales, uint64_t i, uint4 v) {
  if (kOut == kOutCodes) {
    // streaming store: the output is written once
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(static_cast<uint8_t*>(out) + i), "r"(v.x),
                 "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
  } else {
    const float sc = scales[i / 32];
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    float y[16];
#pragma unroll
    for (int j = 0; j < 16; j++) y[j] = e4m3_to_f32((w[j >> 2] >> (8 * (j & 3))) & 0xFFu) * sc;
    if (kOut == QLC_DTYPE_F32) {
      float4* o = reinterpret_cast<float4*>(static_cast<float*>(out) + i);
#pragma unroll
      for (int k = 0; k < 4; k++) __stcs(o + k, make_float4(y[4 * k], y[4 * k + 1], y[4 * k + 2], y[4 * k + 3]));
    } else {
      uint32_t p[8];
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const __nv_bfloat162 hb = __floats2bfloat162_rn(y[2 * k], y[2 * k + 1]);
        p[k] = *reinterpret_cast<const uint32_t*>(&hb);
      }
      uint4* o = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out) + i);
      __stcs(o, make_uint4(p[0], p[1], p[2], p[3]));
      __stcs(o + 1, make_uint4(p[4], p[5], p[6], p[7]));
    }
  }
}

// Fewer than 16 symbols (a tensor's ragged end).
template <int kOut>
__device__ __forceinline__ void put_tail(void* out, const float* scales, uint64_t i, const uint8_t* sb,
                                         uint32_t cnt) {
  for (uint32_t b = 0; b < cnt; b++) {
    if (kOut == kOutCodes) {
      static_cast<uint8_t*>(out)[i + b] = sb[b];
    } else {
      const float y = e4m3_to_f32(sb[b]) * scales[(i + b) / 32];
      if (kOut == QLC_DTYPE_F32)
        static_cast<float*>(out)[i + b] = y;
      else
        static_cast<__nv_bfloat16*>(out)[i + b] = __float2bfloat16_rn(y);
    }
  }
}

// Decodes group g of a validated container (one warp; lane = chunk).
template <int kOut>
__device__ void decode_group(const DecHeader& h, const uint8_t* __restrict__ in, void* __restrict__ out,
                             const float* __restrict__ scales, uint64_t g, DecShared& sm, LaneDec& d,
                             uint32_t* status, int lane) {
  const unsigned long long* group_off = reinterpret_cast<const unsigned long long*>(in + kIndexOff);
  const uint16_t* chunk_bits = reinterpret_cast<const uint16_t*>(in + kIndexOff + 8 * h.n_groups);
  const uint4* vbase = reinterpret_cast<const uint4*>(in + h.P);
  const uint32_t cs = h.cs;
  const uint32_t len_lo = h.len_lo, len_hi = h.len_hi;
  const uint8_t* s_T = sm.T;
  uint4* s_tile = sm.tile;
  do {
    const uint64_t c = g * kGroupChunks + lane;
    const bool exists = c < h.n_chunks;
    const uint32_t nsym = exists ? (uint32_t)min((uint64_t)cs, h.n - c * cs) : 0u;
    const uint32_t bits = exists ? chunk_bits[c] : 0u;
    uint32_t incl = bits;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const uint32_t gbits = __shfl_sync(0xffffffffu, incl, 31);
    const uint64_t goff = group_off[g];
    const uint64_t gnext = g + 1 < h.n_groups ? group_off[g + 1] : h.payload_bytes;
    const bool group_ok = (g != 0 || goff == 0) && (goff & 15u) == 0 && goff <= gnext &&
                          gnext <= h.payload_bytes && gnext - goff == align16((gbits + 7u) / 8u);
    if (!group_ok) {
      if (lane == 0) set_status(status, QLC_ERR_CORRUPT);
      break;
    }
    // lane start bit (group-relative), ring fill, buffer fill
    const uint32_t S = incl - bits;
    d.gp = vbase + goff / 16;
    d.vend = (uint32_t)((gnext - goff) / 16);
    d.fv = S >> 7;
    d.rpb = (S >> 5) * 4;
    d.fetch();
    cp_async_wait<0>();
    d.hi = d.ring_word(d.rpb);
    d.lo = d.ring_word(d.rpb + 4);
    d.rpb += 8;
    d.nxt = d.ring_word(d.rpb);
    {
      const uint32_t o = S & 31u;
      d.hi = __funnelshift_l(d.lo, d.hi, o);
      d.lo <<= o;
      d.nb1 = 63u - o;
    }

    // the two 16-symbol pieces of each block this lane writes out: piece q of
    // rows r = lane / 2 and 16 + lane / 2 (their chunks' lengths and first
    // symbol indices are fixed for the group)
    const int q = lane & 1;
    uint32_t row_n[2];
    uint64_t row_i[2];
#pragma unroll
    for (int t = 0; t < 2; t++) {
      const uint64_t rc = g * kGroupChunks + 16 * t + (lane >> 1);
      row_n[t] = rc < h.n_chunks ? (uint32_t)min((uint64_t)cs, h.n - rc * cs) : 0u;
      row_i[t] = rc * cs + 16 * q;
    }
    const uint32_t nmax = __reduce_max_sync(0xffffffffu, nsym);
    for (uint32_t i0 = 0; i0 < nmax; i0 += kBlk) {
      d.fetch3();
      cp_async_wait<1>();
      const uint32_t cnt = nsym > i0 ? min(kBlk, nsym - i0) : 0u;
      if (cnt == kBlk) {
#pragma unroll
        for (int k = 0; k < (int)(kBlk / 16); k++) {
          uint32_t w[4];
#pragma unroll
          for (int j = 0; j < 4; j++) {
            const uint32_t p0 = d.round2(s_T, len_lo, len_hi);
            const uint32_t p1 = d.round2(s_T, len_lo, len_hi);
            w[j] = __byte_perm(p0, p1, 0x5410);
          }
          s_tile[lane * 2 + (k ^ ((lane >> 2) & 1))] = make_uint4(w[0], w[1], w[2], w[3]);
        }
      } else if (cnt > 0) {
        for (int k = 0; k < (int)(kBlk / 16); k++) {
          uint32_t w[4];
#pragma unroll
          for (int j = 0; j < 4; j++) {
            uint32_t v = 0;
#pragma unroll
            for (int q = 0; q < 4; q++)
              if (16 * k + 4 * j + q < (int)cnt) v |= d.round1(s_T, len_lo, len_hi) << (8 * q);
            w[j] = v;
          }
          s_tile[lane * 2 + (k ^ ((lane >> 2) & 1))] = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
      __syncwarp();
      // the tile's row r is lane r's 32 output bytes: two 16-byte pieces per row
      const bool ragged = __any_sync(0xffffffffu, i0 + kBlk > row_n[0] || i0 + kBlk > row_n[1]);
      if (kOut == kOutCodes && !ragged) {
        // every piece is whole: predicated streaming stores, no branch
#pragma unroll
        for (int t = 0; t < 2; t++) {
          const int r = 16 * t + (lane >> 1);
          const uint4 v = s_tile[r * 2 + (q ^ ((r >> 2) & 1))];
          put16_if(static_cast<uint8_t*>(out) + row_i[t] + i0, v, i0 + 16 * q < row_n[t]);
        }
      } else {
#pragma unroll
        for (int t = 0; t < 2; t++) {
          const int r = 16 * t + (lane >> 1);
          const uint32_t off = i0 + 16 * q;
          if (off < row_n[t]) {
            const uint4* src = &s_tile[r * 2 + (q ^ ((r >> 2) & 1))];
            if (off + 16 <= row_n[t])
              put16<kOut>(out, scales, row_i[t] + i0, *src);
            else
              put_tail<kOut>(out, scales, row_i[t] + i0, reinterpret_cast<const uint8_t*>(src), row_n[t] - off);
          }
        }
      }
      __syncwarp();
    }
    cp_async_wait<0>();
    if (exists) {
      // bits taken into the buffer minus bits still in it = bits consumed
      const uint64_t consumed = (uint64_t)(d.rpb / 4 - (S >> 5)) * 32 - (d.nb1 + 1) - (S & 31u);
      if (consumed != bits) set_status(status, QLC_ERR_CORRUPT);
    }
  } while (false);
}

// One container: every CTA (one warp) validates the header, builds its table
// and decodes groups blockIdx.x, blockIdx.x + gridDim.x, ...
template <int kOut>
__global__ void __launch_bounds__(32, kDecCtasPerSm)
decode_kernel(const uint8_t* __restrict__ in, uint64_t in_bytes, void* __restrict__ out,
              const float* __restrict__ scales, uint64_t out_cap, unsigned long long* __restrict__ n_out,
              uint32_t* __restrict__ status) {
  __shared__ DecShared sm;
  const int lane = threadIdx.x;
  DecHeader h;
  const uint32_t err = parse_header(in, in_bytes, out_cap, &h, sm.seen, lane);
  if (err) {
    if (blockIdx.x == 0 && lane == 0) {
      if (err == QLC_ERR_CAPACITY) *n_out = h.n;
      set_status(status, err);
    }
    return;
  }
  if (blockIdx.x == 0 && lane == 0) *n_out = h.n;
  if (blockIdx.x >= h.n_groups) return;
  if (__cvta_generic_to_shared(sm.ring) & 127u) {  // the ring addressing relies on it
    if (lane == 0) set_status(status, QLC_ERR_CUDA);
    return;
  }
  build_table(in, sm, lane);
  LaneDec d;
  d.ring_s = (uint32_t)__cvta_generic_to_shared(&sm.ring[lane * kRingVec]);
  for (uint64_t g = blockIdx.x; g < h.n_groups; g += gridDim.x)
    decode_group<kOut>(h, in, out, scales, g, sm, d, status, lane);
}

// A batch: warps take (shard, group) items from a device counter; a warp
// re-reads the header and rebuilds its table when its shard changes.
__global__ void __launch_bounds__(32, kDecCtasPerSm)
decode_batch_kernel(const qlc_desc* __restrict__ descs, int n_shards,
                    const unsigned long long* __restrict__ item_base, unsigned int* __restrict__ ticket,
                    uint32_t* __restrict__ status) {
  __shared__ DecShared sm;
  const int lane = threadIdx.x;
  if (__cvta_generic_to_shared(sm.ring) & 127u) {
    if (lane == 0) set_status(status, QLC_ERR_CUDA);
    return;
  }
  const unsigned long long total = item_base[n_shards];
  LaneDec d;
  d.ring_s = (uint32_t)__cvta_generic_to_shared(&sm.ring[lane * kRingVec]);
  int cur = -1, bad = -1;
  DecHeader h;
  while (true) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(ticket, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= total) break;
    const int sh = shard_of_warp(item_base, n_shards, t, lane);
    if (sh == bad) continue;
    const qlc_desc dd = descs[sh];
    const uint8_t* in = static_cast<const uint8_t*>(dd.in);
    const uint64_t g = t - item_base[sh];
    if (sh != cur) {
      const uint32_t err = parse_header(in, dd.in_bytes, dd.out_cap, &h, sm.seen, lane);
      if (err) {
        if (lane == 0) {
          if (err == QLC_ERR_CAPACITY && dd.out_bytes) *dd.out_bytes = h.n;
          set_status(status, err);
        }
        bad = sh;
        cur = -1;
        continue;
      }
      build_table(in, sm, lane);
      cur = sh;
    }
    if (g == 0 && lane == 0 && dd.out_bytes) *dd.out_bytes = h.n;
    if (g < h.n_groups) decode_group<kOutCodes>(h, in, dd.out, nullptr, g, sm, d, status, lane);
  }
}

}  // namespace qlc

using namespace qlc;

static int decode_grid(uint64_t out_cap) {
  const uint64_t max_groups = (out_cap + kGroupChunks * QLC_MIN_CHUNK - 1) / (kGroupChunks * QLC_MIN_CHUNK);
  const uint64_t cap = (uint64_t)sm_count() * kDecCtasPerSm;
  return (int)(max_groups < 1 ? 1 : (max_groups < cap ? max_groups : cap));
}

extern "C" qlc_status qlc_decode(const uint8_t* d_in, size_t in_bytes, uint8_t* d_out, size_t out_cap,
                                 uint64_t* d_n_out, uint32_t* d_status, qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_decode");
  if (!d_in || !d_n_out || (out_cap > 0 && !d_out)) return QLC_ERR_ARG;
  if (!aligned(d_in, 16) || !aligned(d_out, 16) || !aligned(d_n_out, 8) || !aligned(d_status, 4))
    return QLC_ERR_ARG;
  decode_kernel<kOutCodes><<<decode_grid(out_cap), 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      d_in, in_bytes, d_out, nullptr, out_cap, reinterpret_cast<unsigned long long*>(d_n_out), d_status);
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}

extern "C" qlc_status qlc_decode_dequantize(const uint8_t* d_in, size_t in_bytes, const float* d_scales,
                                            void* d_out, qlc_dtype dtype, size_t out_cap, uint64_t* d_n_out,
                                            uint32_t* d_status, qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_decode_dequantize");
  if (dtype != QLC_DTYPE_F32 && dtype != QLC_DTYPE_BF16) return QLC_ERR_ARG;
  if (!d_in || !d_n_out || (out_cap > 0 && (!d_out || !d_scales))) return QLC_ERR_ARG;
  if (!aligned(d_in, 16) || !aligned(d_out, 16) || !aligned(d_scales, 4) || !aligned(d_n_out, 8) ||
      !aligned(d_status, 4))
    return QLC_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* no = reinterpret_cast<unsigned long long*>(d_n_out);
  if (dtype == QLC_DTYPE_F32)
    decode_kernel<QLC_DTYPE_F32><<<decode_grid(out_cap), 32, 0, st>>>(d_in, in_bytes, d_out, d_scales, out_cap, no,
                                                                     d_status);
  else
    decode_kernel<QLC_DTYPE_BF16><<<decode_grid(out_cap), 32, 0, st>>>(d_in, in_bytes, d_out, d_scales, out_cap,
                                                                      no, d_status);
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}

extern "C" qlc_status qlc_decode_batch(const qlc_desc* d_descs, int n_shards, void* d_ws, size_t ws_bytes,
                                       uint32_t* d_status, const qlc_launch* h_launch, qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_decode_batch");
  if (!d_descs || n_shards < 1 || !d_ws) return QLC_ERR_ARG;
  if (!aligned(d_ws, 16) || !aligned(d_descs, 16) || !aligned(d_status, 4)) return QLC_ERR_ARG;
  BatchWs w;
  if (!batch_ws_layout(d_ws, ws_bytes, n_shards, &w)) return QLC_ERR_CAPACITY;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  plan_kernel<<<1, kPlanThreads, 0, st>>>(kPlanDecode, d_descs, n_shards, 0, w, d_status);
  if (cudaGetLastError() != cudaSuccess) return QLC_ERR_CUDA;
  int per_sm = kDecCtasPerSm;
  if (h_launch && h_launch->decode_ctas_per_sm > 0 && h_launch->decode_ctas_per_sm < kDecCtasPerSm)
    per_sm = h_launch->decode_ctas_per_sm;
  decode_batch_kernel<<<sm_count() * per_sm, 32, 0, st>>>(d_descs, n_shards, w.item_base, w.ticket, d_status);
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}
