// decode.cu -- QLC decoder (Section 7) for container v1.
//
// One warp per group of 32 chunks, one lane per chunk: the codes are not
// self-synchronising, so each lane starts at its chunk's bit offset (group
// offset + exclusive scan of the group's chunk_bits) and decodes its chunk
// serially.  Per symbol: a 32-bit window at the bit offset; its top 3 bits are
// the area code; the code length 3 + bits[area] comes from a byte permute of
// two registers (no memory access on the serial path); the whole codeword
// (area code and suffix, right-aligned) indexes a 2048-entry code -> symbol
// table in shared memory built from the LUT and the area table.  The rank is
// never formed explicitly: for every code of every area the table holds
// dec[offset + suffix] (offset 0 for 8-bit areas), exactly the paper's rule.
// Input: 16-byte vector loads per lane, two vectors of prefetch.  Output:
// 16 symbols per shared-memory store into a swizzled 32 x 128-byte tile; every
// 128 symbols the warp writes the tile out as 128-byte row segments.
#include "qlc_common.cuh"

namespace qlc {

constexpr int kDecCtasPerSm = 16;

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

// Per-lane bit reader over a group's payload: a 64-bit window (w0:w1) with
// bit offset o into w0, the rest of the current 16-byte vector (a, b, c) and
// two prefetched vectors.
struct Reader {
  uint32_t w0, w1, o;
  uint32_t a, b, c;
  int left;  // words of the current vector not yet moved into the window
  uint4 n1, n2;
  const uint4* vp;
  const uint4* vend;
  uint32_t shifted;  // words shifted out of the window so far

  __device__ __forceinline__ uint4 fetch() {
    uint4 r = make_uint4(0, 0, 0, 0);
    if (vp < vend) r = ldg_nc_v4(vp);
    vp++;
    return r;
  }
  __device__ __forceinline__ uint32_t pop() {
    uint32_t r;
    if (left == 0) {
      r = bswap32(n1.x);
      a = bswap32(n1.y);
      b = bswap32(n1.z);
      c = bswap32(n1.w);
      left = 3;
      n1 = n2;
      n2 = fetch();
    } else {
      r = a;
      a = b;
      b = c;
      left--;
    }
    return r;
  }
  __device__ __forceinline__ void init(const uint4* vbase, uint64_t S, uint64_t vend_idx) {
    vend = vbase + vend_idx;
    vp = vbase + (S >> 7);
    left = 0;
    n1 = fetch();
    n2 = fetch();
    const int skip = (int)((S >> 5) & 3);
    for (int k = 0; k < skip; k++) pop();
    w0 = pop();
    w1 = pop();
    o = (uint32_t)(S & 31);
    shifted = 0;
  }
  // One symbol (Section 7): area code -> code length; codeword -> symbol.
  __device__ __forceinline__ uint32_t next(const uint8_t* T, uint32_t len_lo, uint32_t len_hi) {
    const uint32_t x = __funnelshift_l(w1, w0, o);
    const uint32_t len = __byte_perm(len_lo, len_hi, x >> 29) & 0xFFu;
    const uint32_t code = __funnelshift_l(x, 0u, len);
    const uint32_t sym = T[code];
    o += len;
    if (o >= 32) {
      o -= 32;
      w0 = w1;
      w1 = pop();
      shifted++;
    }
    return sym;
  }
};

__global__ void __launch_bounds__(32, kDecCtasPerSm)
decode_kernel(const uint8_t* __restrict__ in, uint64_t in_bytes, uint8_t* __restrict__ out,
              uint64_t out_cap, unsigned long long* __restrict__ n_out, uint32_t* __restrict__ status) {
  __shared__ __align__(16) uint8_t s_T[2048];
  __shared__ __align__(16) uint4 s_rows[32 * 8];
  __shared__ uint32_t s_seen[8];
  const int lane = threadIdx.x;

  DecHeader h;
  const uint32_t err = parse_header(in, in_bytes, out_cap, &h, s_seen, lane);
  if (err) {
    if (blockIdx.x == 0 && lane == 0) {
      if (err == QLC_ERR_CAPACITY) *n_out = h.n;
      set_status(status, err);
    }
    return;
  }
  if (blockIdx.x == 0 && lane == 0) *n_out = h.n;
  if (blockIdx.x >= h.n_groups) return;

  // code -> symbol table: every code (i << bits[i]) | s of every area i
  {
    uint32_t base = 0;
    for (int i = 0; i < 8; i++) {
      const uint32_t b = in[40 + i];
      for (uint32_t s = lane; s < (1u << b); s += 32) {
        const uint32_t rank = b == 8 ? s : base + s;
        s_T[(i << b) | s] = in[64 + rank];
      }
      base += *reinterpret_cast<const uint16_t*>(in + 24 + 2 * i);
    }
  }
  __syncwarp();

  const unsigned long long* group_off = reinterpret_cast<const unsigned long long*>(in + kIndexOff);
  const uint16_t* chunk_bits = reinterpret_cast<const uint16_t*>(in + kIndexOff + 8 * h.n_groups);
  const uint4* vbase = reinterpret_cast<const uint4*>(in + h.P);
  const uint32_t cs = h.cs;

  for (uint64_t g = blockIdx.x; g < h.n_groups; g += gridDim.x) {
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
      continue;
    }
    const uint64_t S = goff * 8 + (incl - bits);
    Reader rd;
    rd.init(vbase, S, gnext / 16);
    const uint32_t nmax = __reduce_max_sync(0xffffffffu, nsym);

    for (uint32_t i0 = 0; i0 < nmax; i0 += 128) {
      const uint32_t cnt = nsym > i0 ? min(128u, nsym - i0) : 0u;
      if (cnt == 128) {
#pragma unroll 1
        for (int k = 0; k < 8; k++) {
          uint32_t w[4];
#pragma unroll
          for (int j = 0; j < 4; j++) {
            uint32_t v = rd.next(s_T, h.len_lo, h.len_hi);
            v |= rd.next(s_T, h.len_lo, h.len_hi) << 8;
            v |= rd.next(s_T, h.len_lo, h.len_hi) << 16;
            v |= rd.next(s_T, h.len_lo, h.len_hi) << 24;
            w[j] = v;
          }
          s_rows[lane * 8 + (k ^ (lane & 7))] = make_uint4(w[0], w[1], w[2], w[3]);
        }
      } else if (cnt > 0) {
        for (int k = 0; k < 8; k++) {
          uint32_t w[4];
#pragma unroll
          for (int j = 0; j < 4; j++) {
            uint32_t v = 0;
#pragma unroll
            for (int q = 0; q < 4; q++) {
              const uint32_t idx = 16 * k + 4 * j + q;
              if (idx < cnt) v |= rd.next(s_T, h.len_lo, h.len_hi) << (8 * q);
            }
            w[j] = v;
          }
          s_rows[lane * 8 + (k ^ (lane & 7))] = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 8; t++) {
        const int r = 4 * t + (lane >> 3), q = lane & 7;
        const uint64_t rc = g * kGroupChunks + r;
        const uint32_t rn = rc < h.n_chunks ? (uint32_t)min((uint64_t)cs, h.n - rc * cs) : 0u;
        const uint32_t off = i0 + 16 * q;
        if (off < rn) {
          const uint4 val = s_rows[r * 8 + (q ^ (r & 7))];
          uint8_t* dst = out + rc * cs + off;
          if (off + 16 <= rn) {
            *reinterpret_cast<uint4*>(dst) = val;
          } else {
            const uint8_t* src = reinterpret_cast<const uint8_t*>(&s_rows[r * 8 + (q ^ (r & 7))]);
            for (uint32_t b = 0; b < rn - off; b++) dst[b] = src[b];
          }
        }
      }
      __syncwarp();
    }
    if (exists) {
      const uint64_t consumed = (uint64_t)rd.shifted * 32 + rd.o - (S & 31);
      if (consumed != bits) set_status(status, QLC_ERR_CORRUPT);
    }
  }
}

}  // namespace qlc

using namespace qlc;

extern "C" qlc_status qlc_decode(const uint8_t* d_in, size_t in_bytes, uint8_t* d_out, size_t out_cap,
                                 uint64_t* d_n_out, uint32_t* d_status, qlc_stream_t stream) {
  if (!d_in || !d_n_out || (out_cap > 0 && !d_out)) return QLC_ERR_ARG;
  if (((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out)) & 15u) != 0)
    return QLC_ERR_ARG;
  const uint64_t max_groups = (out_cap + kGroupChunks * QLC_MIN_CHUNK - 1) / (kGroupChunks * QLC_MIN_CHUNK);
  const uint64_t cap = (uint64_t)sm_count() * kDecCtasPerSm;
  const int grid = (int)(max_groups < 1 ? 1 : (max_groups < cap ? max_groups : cap));
  decode_kernel<<<grid, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      d_in, in_bytes, d_out, out_cap, reinterpret_cast<unsigned long long*>(d_n_out), d_status);
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}
