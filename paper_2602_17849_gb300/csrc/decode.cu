// decode.cu -- QLC decoder (Section 7) for container v1.
//
// One warp per group of 32 chunks, one lane per chunk: the codes are not
// self-synchronising, so each lane starts at its chunk's bit offset (group
// offset + exclusive scan of the group's chunk_bits) and decodes its chunk
// serially.  Per symbol: the top 3 bits of a 32-bit window are the area code;
// the code length 3 + bits[area] comes from a byte permute of two registers
// (no memory access); the whole codeword (area code and suffix, right-aligned)
// indexes a 2048-entry code -> symbol table in shared memory built from the
// LUT and the area table.  The rank is never formed explicitly: for every code
// of every area the table holds dec[offset + suffix] (offset 0 for 8-bit
// areas), exactly the paper's rule.
// Input: each lane's bytes arrive by cp.async in 16-byte vectors into a
// staging ring, and once per block of 32 symbols the lane moves the vectors it
// will need next, byte-swapped, into its column of a word ring (word k of lane
// l in bank l, so the lanes' reads never collide).  The lane decodes from a
// 64-bit register buffer: two symbols per round from the 32-bit window at its
// bit position (one funnel shift); when the position crosses a word the
// buffer moves up and the next word comes from the ring, read one word ahead
// of its use so that no memory access lies on the round-to-round chain.
// Output: each lane writes its 32 symbols of a block with one 32-byte
// streaming store.
#include <cuda_bf16.h>

#define QLC_FILE_ID 1
#include "qlc_common.cuh"

namespace qlc {

constexpr int kDecCtasPerSm = 20;  // 20 x (8.3 KB + 1 KB reserved); at 24 the register cap (80) spills

struct DecHeader {
  uint64_t n, payload_bytes, P, n_chunks, n_groups;
  uint64_t in_bytes, out_cap;  // the caller's buffers (bounds of the checked build)
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
  h->in_bytes = in_bytes;
  h->out_cap = out_cap;
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

constexpr uint32_t kBlk = 32;       // symbols per lane per block
constexpr uint32_t kStageVec = 8;   // 16-byte vectors staged per lane (128 B of its stream)
constexpr uint32_t kColRows = 16;   // words in each lane's column ring

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

// Shared memory of one decoding warp (one CTA): the lanes' staging ring and
// column ring, and the code table.
struct DecShared {
  uint32_t col[kColRows][32];  // word k of lane l at col[k % 16][l]
  uint4 stage[kStageVec][32];  // vector v of lane l at stage[v % 8][l]
  uint8_t T[2048];                // code -> symbol
  __align__(16) uint8_t dec[256];
  uint32_t seen[8];
};

// A lane's bit stream, positions group-relative.  The stream's words j and
// j + 1 sit in a 64-bit buffer (hi:lo, most significant bit first) and word
// j + 2 in nxt, where j = p / 32; the window at bit p is one funnel shift of
// the buffer.  When a round crosses into the next word the buffer moves up
// by one word and word j + 3 is read from the column ring, so no memory
// access lies on the chain from one round to the next.
struct LaneDec {
  uint32_t p;      // bit position of the next codeword
  uint32_t hi, lo, nxt;
  uint32_t tv;     // next vector to move from the staging ring to the column ring
  uint32_t fv;     // next vector to fetch
  uint32_t vend;   // vectors of this stream in the group
  uint64_t vlim;   // vectors from the group's start to the end of the container (checked build)
  const uint4* gp; // the group's payload
  uint32_t lane4;      // byte offset of col[0][lane] in the column ring
  uint32_t col_s;      // shared address of col[0][lane]
  uint32_t stage_s;    // shared address of stage[0][lane]

  // Fetches (cp.async, 16 bytes each) vector fv into its staging slot when
  // fv < want, k times, with no branch; the caller commits the group.
  template <int k>
  __device__ __forceinline__ void fetch(uint32_t want) {
#pragma unroll
    for (int i = 0; i < k; i++) {
      const uint32_t q = fv < want && QLC_GUARD(fv < vlim, nullptr);
      asm volatile(
          "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q cp.async.cg.shared.global [%0], [%1], 16;\n\t}" ::"r"(
              stage_s + (fv % kStageVec) * 512),
          "l"(gp + fv), "r"(q)
          : "memory");
      fv += q;
    }
  }
  // Moves vector tv from the staging ring to the column ring (byte-swapped,
  // so each word reads most significant bit first) when its first word is
  // at most `need` and it exists.
  __device__ __forceinline__ void move(uint32_t need) {
    const uint32_t q = (tv * 4 <= need) & (tv < vend);
    const uint32_t src = stage_s + (tv % kStageVec) * 512;
    const uint32_t dst = col_s + (tv % 4) * 512;
      asm volatile(
          "{\n\t.reg .pred q;\n\t.reg .b32 a, b, c, d;\n\t"
          "setp.ne.u32 q, %2, 0;\n\t"
          "@q ld.shared.v4.u32 {a, b, c, d}, [%0];\n\t"
          "prmt.b32 a, a, 0, 0x0123;\n\t"
          "prmt.b32 b, b, 0, 0x0123;\n\t"
          "prmt.b32 c, c, 0, 0x0123;\n\t"
          "prmt.b32 d, d, 0, 0x0123;\n\t"
          "@q st.shared.u32 [%1], a;\n\t"
          "@q st.shared.u32 [%1+128], b;\n\t"
          "@q st.shared.u32 [%1+256], c;\n\t"
          "@q st.shared.u32 [%1+384], d;\n\t"
          "}" ::"r"(src),
          "r"(dst), "r"(q)
          : "memory");
    tv += q;
  }
  __device__ __forceinline__ uint32_t ring(const DecShared& sm, uint32_t k) const {
    return *reinterpret_cast<const uint32_t*>(reinterpret_cast<const uint8_t*>(sm.col) + (((k << 7) & 0x780u) | lane4));
  }
  // Set-up at bit S of the group: fill the staging ring, wait for it, move
  // the words the first block can read, load the buffer, refill.  Words
  // j .. j + 2 (at most two vectors) go to the buffer before the rest is
  // moved: the ring holds 16 words, and word j + 16 shares word j's row.
  __device__ __forceinline__ void start(const DecShared& sm, uint32_t S) {
    p = S;
    tv = fv = min(S >> 7, vend);
    fetch<kStageVec>(min(tv + kStageVec, vend));
    cp_async_commit();
    cp_async_wait<0>();
    const uint32_t j = S >> 5;
    move(j + 2);
    move(j + 2);
    hi = ring(sm, j);
    lo = ring(sm, j + 1);
    nxt = ring(sm, j + 2);
#pragma unroll
    for (int i = 0; i < 3; i++) move(j + 13);
    fetch<5>(min(tv + kStageVec, vend));
    cp_async_commit();
  }
  // Before each block of at most 32 symbols (at most 352 bits, so the ring
  // is read up to word p/32 + 13): move up to three vectors (the position
  // moved at most 11 words since the last block) and refetch as many.
  // Vectors moved now were fetched two blocks ago at the latest, so waiting
  // for all but the latest cp.async group suffices.
  __device__ __forceinline__ void advance() {
    cp_async_wait<1>();
    const uint32_t need = (p >> 5) + 13;
#pragma unroll
    for (int i = 0; i < 3; i++) move(need);
    fetch<3>(min(tv + kStageVec, vend));
    cp_async_commit();
  }
  // Code length of the codeword at the top of x (Section 7: the area code,
  // i.e. the top 3 bits, fixes it): a byte permute of two registers; the
  // selector's sign-mode nibbles make bytes 1-3 zero.
  __device__ __forceinline__ static uint32_t code_len(uint32_t x, uint32_t len_lo, uint32_t len_hi) {
    return prmt(len_lo, len_hi, mad_hi(x, 8u, 0x8880u));
  }
  // Advances the position to pn (less than 32 bits on): when it crosses into
  // the next word the buffer moves up a word and the word after nxt is read.
  __device__ __forceinline__ void step_to(const DecShared& sm, uint32_t pn) {
    if ((pn ^ p) & 32u) {
      hi = lo;
      lo = nxt;
      nxt = ring(sm, (pn >> 5) + 2);
    }
    p = pn;
  }
  // Two symbols (at most 22 bits) from the window, packed as s0 | s1 << 8.
  __device__ __forceinline__ uint32_t round2(const DecShared& sm, uint32_t len_lo, uint32_t len_hi) {
    const uint32_t x = __funnelshift_l(lo, hi, p);
    const uint32_t la = code_len(x, len_lo, len_hi);
    const uint32_t ia = __funnelshift_l(x, 0u, la);
    const uint32_t a = QLC_GUARD(ia < 2048u, nullptr) ? sm.T[ia] : 0u;
    const uint32_t x2 = x << la;
    const uint32_t lb = code_len(x2, len_lo, len_hi);
    const uint32_t ib = __funnelshift_l(x2, 0u, lb);
    const uint32_t b = QLC_GUARD(ib < 2048u, nullptr) ? sm.T[ib] : 0u;
    step_to(sm, p + la + lb);
    return mad_lo(b, 256u, a);
  }
  // One symbol (ragged chunk ends only).
  __device__ __forceinline__ uint32_t round1(const DecShared& sm, uint32_t len_lo, uint32_t len_hi) {
    const uint32_t x = __funnelshift_l(lo, hi, p);
    const uint32_t la = code_len(x, len_lo, len_hi);
    const uint32_t ia = __funnelshift_l(x, 0u, la);
    const uint32_t a = QLC_GUARD(ia < 2048u, nullptr) ? sm.T[ia] : 0u;
    step_to(sm, p + la);
    return a;
  }
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
    for (uint32_t s = lane; s < (1u << b); s += 32)
      if (QLC_GUARD(((i << b) | s) < 2048u && (b == 8 ? s : base + s) < 256u, nullptr))
        sm.T[(i << b) | s] = sm.dec[b == 8 ? s : base + s];
    base += *reinterpret_cast<const uint16_t*>(in + 24 + 2 * i);
  }
  __syncwarp();
}

// Output of the decoder: the symbols themselves (kOutCodes), or their
// block-32 dequantised values (value(code) * scale, fp32 or rounded to bf16).
constexpr int kOutCodes = -1;

// Streaming 32-byte store (dst 32-byte aligned) or two 16-byte stores.
__device__ __forceinline__ void st_cs_32(uint8_t* dst, const uint32_t w[8], bool aligned32) {
  if (aligned32) {
    asm volatile("st.global.cs.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(dst), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
  } else {
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(dst), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
                 : "memory");
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(dst + 16), "r"(w[4]), "r"(w[5]), "r"(w[6]),
                 "r"(w[7])
                 : "memory");
  }
}

// Single symbols (ragged chunk ends).
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

// Thirty-two decoded symbols w of one chunk, starting at symbol index i of
// the tensor (a multiple of 32), to their destination; sc is their block's
// scale (dequantising outputs).
template <int kOut>
__device__ __forceinline__ void put32(void* out, float sc, uint64_t i, const uint32_t w[8], bool aligned32) {
  if (kOut == kOutCodes) {
    st_cs_32(static_cast<uint8_t*>(out) + i, w, aligned32);
  } else {
    // the block's 32 values share one scale (i is a multiple of 32); they go
    // out in whole 32-byte sectors: 4 stores of 8 fp32, or 2 of 16 bf16
    uint32_t v[kOut == QLC_DTYPE_F32 ? 32 : 16];
#pragma unroll
    for (int j = 0; j < 32; j++) {
      const float y = __uint_as_float(e4m3_scaled_bits(w[j >> 2], j & 3)) * 0x1p120f * sc;
      if (kOut == QLC_DTYPE_F32) {
        v[j] = __float_as_uint(y);
      } else if (j & 1) {
        const __nv_bfloat162 hb = __floats2bfloat162_rn(__uint_as_float(v[j >> 1]), y);
        v[j >> 1] = *reinterpret_cast<const uint32_t*>(&hb);
      } else {
        v[j >> 1] = __float_as_uint(y);
      }
    }
    constexpr int kVec = kOut == QLC_DTYPE_F32 ? 4 : 2;  // 32-byte pieces
    uint8_t* dst = static_cast<uint8_t*>(out) + i * (kOut == QLC_DTYPE_F32 ? 4 : 2);
#pragma unroll
    for (int k = 0; k < kVec; k++) st_cs_32(dst + 32 * k, v + 8 * k, aligned32);
  }
}

// One decoded symbol s at index i of the tensor (ragged chunk ends).
template <int kOut>
__device__ __forceinline__ void put1(void* out, const float* scales, uint64_t i, uint32_t s) {
  const uint8_t b = (uint8_t)s;
  put_tail<kOut>(out, scales, i, &b, 1);
}

// Decodes group g of a validated container (one warp; lane = chunk).  With
// out_slot the output pointer is read from that shared word at each block
// instead of out: a pointer that is not a kernel parameter would otherwise
// hold two registers across the decoding loop, which then issued about 10 %
// more instructions (the batch decoder, 124.3 M against 112.8 M on 256 MiB).
template <int kOut>
__device__ __forceinline__ void decode_group(const DecHeader& h, const uint8_t* __restrict__ in, void* __restrict__ out,
                             const float* __restrict__ scales, uint64_t g, DecShared& sm, LaneDec& d,
                             uint32_t* status, int lane, bool aligned32, bool sc_vec = false,
                             void* const volatile* out_slot = nullptr) {
  const unsigned long long* group_off = reinterpret_cast<const unsigned long long*>(in + kIndexOff);
  const uint16_t* chunk_bits = reinterpret_cast<const uint16_t*>(in + kIndexOff + 8 * h.n_groups);
  const uint4* vbase = reinterpret_cast<const uint4*>(in + h.P);
  const uint32_t cs = h.cs;
  const uint32_t len_lo = h.len_lo, len_hi = h.len_hi;
  const uint64_t c = g * kGroupChunks + lane;
  const bool exists = c < h.n_chunks;
  const uint32_t nsym = exists ? (uint32_t)min((uint64_t)cs, h.n - c * cs) : 0u;
  const uint32_t bits =
      exists && QLC_GUARD(kIndexOff + 8 * h.n_groups + 2 * (c + 1) <= h.in_bytes, status) ? chunk_bits[c] : 0u;
  uint32_t incl = bits;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  const uint32_t gbits = __shfl_sync(0xffffffffu, incl, 31);
  const uint64_t goff = QLC_GUARD(kIndexOff + 8 * (g + 1) <= h.in_bytes, status) ? group_off[g] : 0ull;
  const uint64_t gnext = g + 1 < h.n_groups
                             ? (QLC_GUARD(kIndexOff + 8 * (g + 2) <= h.in_bytes, status) ? group_off[g + 1] : 0ull)
                             : h.payload_bytes;
  const bool group_ok = (g != 0 || goff == 0) && (goff & 15u) == 0 && goff <= gnext &&
                        gnext <= h.payload_bytes && gnext - goff == align16((gbits + 7u) / 8u);
  if (!group_ok) {
    if (lane == 0) set_status(status, QLC_ERR_CORRUPT);
    return;
  }
  // lane start bit (group-relative) and ring set-up
  const uint32_t S = incl - bits;
  d.gp = vbase + goff / 16;
  d.vend = (uint32_t)((gnext - goff) / 16);
  d.vlim = (h.in_bytes - h.P - goff) / 16;  // goff <= payload_bytes <= in_bytes - P (validated)
  d.start(sm, S);
  const uint64_t i_chunk = c * cs;  // the chunk's first symbol
  const uint32_t nmax = __reduce_max_sync(0xffffffffu, nsym);
  // dequantising outputs: the scales of the chunk's whole blocks, four per
  // 16-byte load (a lane's loads hit lines of their own, so four scales per
  // load cut the load traffic of the L1 data pipe fourfold), each four
  // loaded four blocks before their use
  const uint32_t nfull = nsym / kBlk;
  const float* sc_chunk = kOut != kOutCodes ? scales + i_chunk / 32 : nullptr;
  auto scales4 = [&](uint32_t q) {  // scales of whole blocks 4q .. 4q + 3 (0 past the last)
    float4 r = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (kOut == kOutCodes) return r;
    if (4 * q + 4 <= nfull && sc_vec) return __ldg(reinterpret_cast<const float4*>(sc_chunk + 4 * q));
    if (4 * q < nfull) r.x = sc_chunk[4 * q];
    if (4 * q + 1 < nfull) r.y = sc_chunk[4 * q + 1];
    if (4 * q + 2 < nfull) r.z = sc_chunk[4 * q + 2];
    if (4 * q + 3 < nfull) r.w = sc_chunk[4 * q + 3];
    return r;
  };
  float4 sc_cur = make_float4(0.0f, 0.0f, 0.0f, 0.0f), sc_nxt = scales4(0);
  for (uint32_t i0 = 0; i0 < nmax; i0 += kBlk) {
    d.advance();
    const uint32_t b = i0 / kBlk;  // the same block index in every lane
    if (kOut != kOutCodes && (b & 3u) == 0) {
      sc_cur = sc_nxt;
      sc_nxt = scales4(b / 4 + 1);
    }
    const float sc = (b & 3u) == 0 ? sc_cur.x : (b & 3u) == 1 ? sc_cur.y : (b & 3u) == 2 ? sc_cur.z : sc_cur.w;
    const uint32_t cnt = nsym > i0 ? min(kBlk, nsym - i0) : 0u;
    void* o = out_slot ? *out_slot : out;
    if (cnt == kBlk) {
      uint32_t w[8];
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const uint32_t p0 = d.round2(sm, len_lo, len_hi);
        const uint32_t p1 = d.round2(sm, len_lo, len_hi);
        w[j] = __byte_perm(p0, p1, 0x5410);
      }
      if (QLC_GUARD(i_chunk + i0 + kBlk <= h.out_cap, status)) put32<kOut>(o, sc, i_chunk + i0, w, aligned32);
    } else {
      for (uint32_t k = 0; k < cnt; k++) {
        const uint32_t sym = d.round1(sm, len_lo, len_hi);
        if (QLC_GUARD(i_chunk + i0 + k < h.out_cap, status)) put1<kOut>(o, scales, i_chunk + i0 + k, sym);
      }
    }
  }
  cp_async_wait<0>();
  if (exists && d.p - S != bits) set_status(status, QLC_ERR_CORRUPT);
}

// Lane set-up shared by the kernels; 0 if the ring is not placed as its
// addressing requires.
__device__ __forceinline__ bool lane_init(DecShared& sm, LaneDec& d, int lane) {
  d.lane4 = 4u * lane;
  d.col_s = (uint32_t)__cvta_generic_to_shared(&sm.col[0][lane]);
  d.stage_s = (uint32_t)__cvta_generic_to_shared(&sm.stage[0][lane]);
  return (__cvta_generic_to_shared(sm.stage) & 15u) == 0;
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
  LaneDec d;
  if (!lane_init(sm, d, lane)) {
    if (lane == 0) set_status(status, QLC_ERR_CUDA);
    return;
  }
  build_table(in, sm, lane);
  const bool aligned32 = (reinterpret_cast<uintptr_t>(out) & 31u) == 0;
  const bool sc_vec = (reinterpret_cast<uintptr_t>(scales) & 15u) == 0;  // scales read four at a time
  for (uint64_t g = blockIdx.x; g < h.n_groups; g += gridDim.x)
    decode_group<kOut>(h, in, out, scales, g, sm, d, status, lane, aligned32, sc_vec);
}

// A batch: warps take (shard, group) items from a device counter; a warp
// re-reads the header and rebuilds its table when its shard changes.
__global__ void __launch_bounds__(32, kDecCtasPerSm)
decode_batch_kernel(const qlc_desc* __restrict__ descs, int n_shards,
                    const unsigned long long* __restrict__ item_base, unsigned int* __restrict__ ticket,
                    uint32_t* __restrict__ status) {
  __shared__ DecShared sm;
  const int lane = threadIdx.x;
  LaneDec d;
  if (!lane_init(sm, d, lane)) {
    if (lane == 0) set_status(status, QLC_ERR_CUDA);
    return;
  }
  const unsigned long long total = item_base[n_shards];
  int cur = -1, bad = -1;
  DecHeader h;
  __shared__ void* volatile s_out;  // the current item's output
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
    const bool aligned32 = (reinterpret_cast<uintptr_t>(dd.out) & 31u) == 0;
    __syncwarp();  // every lane is done with the previous item's output
    if (lane == 0) s_out = dd.out;
    __syncwarp();
    if (g < h.n_groups)
      decode_group<kOutCodes>(h, in, nullptr, nullptr, g, sm, d, status, lane, aligned32, false, &s_out);
  }
}

}  // namespace qlc

using namespace qlc;

// One CTA (warp) per group where the container's groups are few enough, up
// to kDecCtasPerSm per SM.  The host knows out_cap, not the chunk size: a
// container of out_cap symbols has between min_groups (chunks of
// QLC_MAX_CHUNK) and max_groups (chunks of QLC_MIN_CHUNK) groups.  A grid
// much larger than the groups lets the block scheduler put up to 16 of the
// working CTAs on some SMs and 13 on others (measured with 2048 groups: a
// grid of 2048 or 2128 CTAs gives every SM 13 or 14 working CTAs, grids of
// 2432 or 3040 up to 16, and decode runs 4 % slower).  So a container large
// enough to fill the GPU at the largest chunk gets min_groups CTAs: every CTA
// works at that chunk, and at smaller chunks each CTA takes several groups.
static int decode_grid(uint64_t out_cap) {
  const uint64_t per_group_min = (uint64_t)kGroupChunks * QLC_MIN_CHUNK;
  const uint64_t per_group_max = (uint64_t)kGroupChunks * QLC_MAX_CHUNK;
  const uint64_t max_groups = (out_cap + per_group_min - 1) / per_group_min;
  const uint64_t min_groups = (out_cap + per_group_max - 1) / per_group_max;
  const uint64_t sms = (uint64_t)sm_count(), cap = sms * kDecCtasPerSm;
  const uint64_t want = min_groups >= 2 * sms ? min_groups : max_groups;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
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

namespace qlc {
QLC_DEFINE_CHECK_TAKE(check_take_decode)
}  // namespace qlc
