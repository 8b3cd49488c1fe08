// encode.cu -- QLC encoder (Sections 5 and 7) writing container v1.
//
// One persistent kernel.  CTAs take groups (32 chunks) in ticket order; the
// LUT is staged in shared memory once per tensor, one copy per lane, so every
// lookup is free of bank conflicts.
//   pass 1  each warp sums the code lengths of its chunks (w, w+8, ...) ->
//           chunk_bits;
//   look-back  warp 0 scans the 32 chunk sizes, publishes the group's padded
//           byte size and finds the sum of all earlier groups' sizes
//           (decoupled look-back, bounded waits);
//   pass 2  each warp re-reads its chunks (from L2: at most three groups per
//           SM are in flight) and packs them, 512 symbols per step: codeword
//           pairs, a warp scan of the lanes' bit counts, per-lane word
//           accumulation into a per-warp staging window (completed words are
//           plain stores, a lane's partial last word one shared OR), and
//           16-byte streaming stores of every completed 16-byte block; blocks
//           shared by neighbouring chunks are merged once per group.
// HBM traffic is one read of the input and one write of the container.
#include <cuda.h>

#include <mutex>
#include <unordered_map>
#include <utility>

#define QLC_FILE_ID 2
#include "qlc_common.cuh"
#include "../../include/qlc_testing.h"

namespace qlc {

constexpr int kEncThreads = 256;
constexpr int kEncWarps = kEncThreads / 32;
constexpr int kEncCtasPerSm = 3;
constexpr int kSub = 32 * 16;  // symbols a warp packs per step (16 per lane)
// per-warp staging buffer: 4 guard words, 4 carry words, one step's words, 4 spare
constexpr int kWStage = 4 + 4 + (kSub * kMaxCode + 31) / 32 + 4;
constexpr int kPass1Unroll = 8;

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr unsigned long long kFlagError = 3ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s per look-back wait

// Streaming (evict-first) 16-byte store: the container is written once and
// should not push the input, which pass 2 re-reads, out of L2.
__device__ __forceinline__ void st_cs_v4(uint4* p, uint4 v) {
  asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

// OR v into a shared word.
__device__ __forceinline__ void red_or(uint32_t saddr, uint32_t v) {
  asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(saddr), "r"(v) : "memory");
}

// When the accumulator's first word is complete (nb >= 32): store it to the
// shared word at wa, move the spill word lo up, advance wa and nb by one word.
// One predicate drives all of it, with no branch.
__device__ __forceinline__ void emit_if_full(uint32_t& hi, uint32_t& wa, uint32_t& nb, uint32_t lo) {
  asm volatile(
      "{\n\t.reg .pred q;\n\t"
      "setp.ge.u32 q, %2, 32;\n\t"
      "@q st.shared.u32 [%1], %0;\n\t"
      "selp.b32 %0, %3, %0, q;\n\t"
      "@q add.u32 %1, %1, 4;\n\t"
      "@q sub.u32 %2, %2, 32;\n\t"
      "}"
      : "+r"(hi), "+r"(wa), "+r"(nb)
      : "r"(lo)
      : "memory");
}

__device__ __forceinline__ uint32_t ld_shared_u32(uint32_t saddr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(saddr) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The encoder table holds one copy per lane (entry s of lane l at word
// 32 s + l), so the 32 lanes of a lookup always hit 32 different banks.
// tab points at this lane's copy.
__device__ __forceinline__ uint32_t enc_entry(const uint32_t* tab, uint32_t s) { return tab[s << 5]; }

// Sum of the encoder entries of 16 symbols.  An entry is
// codeword << (32 - len) | len with len <= 11, so its bits below 21 are the
// length alone, and the low 21 bits of a sum of entries are the sum of the
// lengths as long as that stays below 2^21.
__device__ __forceinline__ uint32_t entry_sum16(const uint32_t* tab, uint4 q) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < 4; k++)
#pragma unroll
    for (int j = 0; j < 4; j++) s += enc_entry(tab, __byte_perm(w[k], 0, 0x4440 + j));
  return s;
}

// Decoupled look-back over groups (warp-wide).  Publishes this group's size,
// returns the byte offset of the group (sum of all earlier groups' sizes).
// Every wait is bounded; on timeout *err is set and an error flag is
// published so that later groups stop waiting too.
__device__ unsigned long long lookback(unsigned long long* gstat, uint64_t g, uint64_t first,
                                       uint64_t gbytes, int lane, bool* err) {
  *err = false;
  if (g == first) {
    if (lane == 0) st_release_u64(&gstat[g], kFlagPrefix | gbytes);
    return 0;
  }
  if (lane == 0) st_release_u64(&gstat[g], kFlagAgg | gbytes);
  unsigned long long excl = 0;
  int64_t idx = (int64_t)g - 1 - lane;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    unsigned long long v = kFlagPrefix;  // before the shard's first group: prefix 0
    if (idx >= (int64_t)first) {
      while (true) {
        v = ld_acquire_u64(&gstat[idx]);
        if (v >> 62) break;
        if (globaltimer_ns() - t0 > kWaitLimitNs) {
          v = kFlagError;
          break;
        }
        __nanosleep(64);
      }
    }
    const unsigned flag = (unsigned)(v >> 62);
    const unsigned stop = __ballot_sync(0xffffffffu, flag >= 2);
    if (stop) {
      const int k = __ffs(stop) - 1;  // nearest earlier group with a full prefix
      const unsigned bad = __ballot_sync(0xffffffffu, flag == 3 && lane <= k);
      excl += warp_sum_u64(lane <= k ? (v & kValMask) : 0ull);
      *err = bad != 0;
      break;
    }
    excl += warp_sum_u64(v & kValMask);
    idx -= 32;
  }
  if (lane == 0) st_release_u64(&gstat[g], (*err ? kFlagError : kFlagPrefix) | (excl + gbytes));
  return excl;
}

__device__ void write_header(uint8_t* out, uint64_t n, uint32_t cs, uint64_t n_chunks,
                             const qlc_lut* lut, int tid) {
  if (tid == 0) {
    *reinterpret_cast<uint32_t*>(out + 0) = 0x31434C51u;  // "QLC1"
    *reinterpret_cast<uint16_t*>(out + 4) = QLC_VERSION;
    out[6] = lut->scheme.id;
    out[7] = 0;
    *reinterpret_cast<unsigned long long*>(out + 8) = n;
    *reinterpret_cast<uint32_t*>(out + 16) = cs;
    *reinterpret_cast<uint32_t*>(out + 20) = (uint32_t)n_chunks;
    *reinterpret_cast<unsigned long long*>(out + 56) = 0;
  }
  if (tid < 8) {
    *reinterpret_cast<uint16_t*>(out + 24 + 2 * tid) = lut->scheme.area_n[tid];
    out[40 + tid] = lut->scheme.area_bits[tid];
  }
  if (tid < 256) out[64 + tid] = lut->dec[tid];
  const uint64_t idx_end = kIndexOff + 8 * n_groups_of(n_chunks) + 2 * n_chunks;
  const uint64_t P = payload_start(n_chunks);
  if (idx_end + tid < P) out[idx_end + tid] = 0;
}

// Work source of the encode kernel: one tensor (descs == nullptr), or the
// shards of a batch, whose groups are numbered consecutively shard after
// shard (item_base[s] = first item of shard s, item_base[n_shards] = total).
struct EncArgs {
  const uint8_t* in;
  uint64_t n;
  const qlc_lut* lut;
  uint8_t* out;
  unsigned long long* out_bytes;
  uint64_t n_items;  // one tensor: its groups
  const qlc_desc* descs;
  const unsigned long long* item_base;
  int n_shards;
  uint32_t cs;
  unsigned int* ticket;
  unsigned long long* gstat;
  uint32_t* status;
  uint64_t out_cap;    // one tensor: bytes at out (batches: each descriptor's)
  uint64_t gstat_cap;  // look-back words at gstat
};

// Packing state of one warp within one chunk.  The warp appends 512
// symbols per step (16 per lane, in lane order) to the chunk's bit stream in a
// per-warp staging window; completed 16-byte blocks go to the payload, except
// the chunk's first block when it is shared with the previous chunk, which
// goes to the chunk's seam slot.
struct Packer {
  const uint32_t* tab;   // this lane's copy of the encoder table
  uint32_t* stage;       // the warp's two staging buffers
  uint32_t stage_s;      // their shared address
  uint4* dst;            // the group's payload
  uint32_t seam_s;       // shared address of the chunk's seam slot [0]
  uint32_t seam_idx_s;   // and of its block index
  uint32_t seam_blk;     // block shared with the previous chunk, ~0u if none
  uint32_t blk_lim;      // 16-byte blocks available at dst (checked build)
  uint32_t base_bit;     // group-relative bit of the step's first symbol
  uint32_t win;          // group-relative word held at stage word 4 (a multiple of 4)
  uint32_t cur;          // staging buffer in use
  int lane;

  // Moves block b (< nblk) of the current buffer out and zeroes it; branch-free.
  __device__ __forceinline__ void put_block(uint32_t b, uint32_t nblk, const uint32_t* sb) const {
    const uint32_t blk = win / 4 + b;
    if (!QLC_GUARD(b >= nblk || blk < blk_lim, nullptr)) nblk = 0;
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(sb) + 16u * b;
    asm volatile(
        "{\n\t"
        ".reg .pred p, s, g;\n\t"
        ".reg .b32 a0, a1, a2, a3, z;\n\t"
        "mov.b32 z, 0;\n\t"
        "setp.lt.u32 p, %0, %1;\n\t"
        "setp.eq.and.u32 s, %2, %3, p;\n\t"
        "setp.ne.and.u32 g, %2, %3, p;\n\t"
        "@p ld.shared.v4.u32 {a0, a1, a2, a3}, [%4];\n\t"
        "@p st.shared.v4.u32 [%4], {z, z, z, z};\n\t"
        "prmt.b32 a0, a0, 0, 0x0123;\n\t"
        "prmt.b32 a1, a1, 0, 0x0123;\n\t"
        "prmt.b32 a2, a2, 0, 0x0123;\n\t"
        "prmt.b32 a3, a3, 0, 0x0123;\n\t"
        "@g st.global.cs.v4.u32 [%5], {a0, a1, a2, a3};\n\t"
        "@s st.shared.v4.u32 [%6], {a0, a1, a2, a3};\n\t"
        "@s st.shared.u32 [%7], %2;\n\t"
        "}" ::"r"(b),
        "r"(nblk), "r"(blk), "r"(seam_blk), "r"(sa), "l"(dst + blk), "r"(seam_s), "r"(seam_idx_s)
        : "memory");
  }

  template <bool kRagged>
  __device__ __forceinline__ void step(uint4 q, int cnt) {
    // 16 codewords -> 8 pairs: MSB-aligned (at most 22 bits), lengths in L8.
    // An entry is codeword << (32 - len) | len, so e & 31 == len.
    const uint32_t qw[4] = {q.x, q.y, q.z, q.w};
    uint32_t e[16];
#pragma unroll
    for (int j = 0; j < 16; j++) {
      e[j] = enc_entry(tab, __byte_perm(qw[j >> 2], 0, 0x4440 + (j & 3)));
      if (kRagged) e[j] = j < cnt ? e[j] : 0u;
    }
    uint32_t P[8], L8[8];
    uint32_t L = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const uint32_t e0 = e[2 * k], e1 = e[2 * k + 1];
      // second code right after the first: e1 >> len0 also moves e1's length
      // field down to bits 0..3-len0, which the mask clears with e0's (the pair
      // itself, at most 22 bits, sits at bits 31..10)
      P[k] = (e0 | __funnelshift_r(e1, 0u, e0)) & ~31u;
      L8[k] = (e0 + e1) & 31u;  // the two lengths; code bits sit above bit 20
      L += L8[k];
    }
    uint32_t incl = L;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    // Each lane packs its pairs into a two-word accumulator (hi:lo, hi
    // first) that starts at the lane's bit offset within its first word,
    // preloaded with that word (the bits carried from the previous step, in
    // lane 0; zero elsewhere).  Every completed word is stored whole: a lane's
    // first word also holds the previous lane's last bits, which that lane
    // ORs in afterwards with its partial last word.  Stores precede the ORs
    // in program order, and no two lanes store the same word.
    const uint32_t p = base_bit + incl - L + 32u * (4u - win);  // bit relative to stage word 0
    if (QLC_GUARD(((p + L) >> 5) < (uint32_t)kWStage, nullptr)) {
      uint32_t wa = stage_s + cur * kWStage * 4 + (p >> 5) * 4;
      uint32_t nb = p & 31u;  // bits in hi
      uint32_t hi = ld_shared_u32(wa);
#pragma unroll
      for (int k = 0; k < 8; k++) {
        hi |= P[k] >> nb;
        const uint32_t lo = __funnelshift_rc(0u, P[k], nb);  // P << (32 - nb), 0 when nb == 0
        nb += L8[k];                                         // at most 31 + 22
        emit_if_full(hi, wa, nb, lo);
      }
      red_or(wa, hi);  // the partial last word (0 adds nothing)
    }
    __syncwarp();
    // completed 16-byte blocks go out (at most 45 per step: 128 carried +
    // 512 * 11 new bits); the partial last block moves to the other buffer
    const uint32_t end_bit = base_bit + total;
    const uint32_t nblk = ((end_bit >> 5) - win) / 4;
    uint32_t* sb = stage + cur * kWStage + 4;
    put_block(lane, nblk, sb);
    if (nblk > 32) put_block(lane + 32, nblk, sb);
    if (lane < 4) {
      stage[(cur ^ 1) * kWStage + 4 + lane] = sb[4 * nblk + lane];
      sb[4 * nblk + lane] = 0;
    }
    seam_blk = ~0u;  // only a chunk's first step can complete its first block
    win += 4 * nblk;
    base_bit = end_bit;
    cur ^= 1;
    __syncwarp();
  }
};

__global__ void __launch_bounds__(kEncThreads, kEncCtasPerSm)
encode_kernel(EncArgs A) {
  __shared__ __align__(16) uint32_t s_enc[256 * 32];  // codeword << (32 - len) | len, one copy per lane
  __shared__ __align__(16) uint32_t s_stage[kEncWarps][2][kWStage];  // per-warp ping-pong
  __shared__ uint32_t s_chunk_bits[kGroupChunks];
  __shared__ uint32_t s_chunk_start[kGroupChunks + 1];  // group-relative bit of each chunk
  __shared__ __align__(16) uint4 s_seam[kGroupChunks][2];  // a chunk's first / last 16-byte block
  __shared__ uint32_t s_seam_idx[kGroupChunks][2];         // their block index, ~0u if none
  __shared__ unsigned long long s_item, s_first, s_excl;
  __shared__ const uint8_t* s_in;
  __shared__ uint64_t s_n;
  __shared__ const qlc_lut* s_lut;
  __shared__ uint8_t* s_out;
  __shared__ uint64_t s_cap;
  __shared__ unsigned long long* s_ob;
  __shared__ int s_err;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t cs = A.cs;
  const uint64_t group_syms = (uint64_t)kGroupChunks * cs;
  const uint32_t stage_s = (uint32_t)__cvta_generic_to_shared(&s_stage[warp][0][0]);
  const uint32_t* tab = &s_enc[lane];
  const uint64_t n_items = A.descs ? A.item_base[A.n_shards] : A.n_items;
  const qlc_lut* cur_lut = nullptr;
  for (int i = tid; i < kEncWarps * 2 * kWStage; i += kEncThreads) (&s_stage[0][0][0])[i] = 0;

  while (true) {
    __syncthreads();
    if (warp == 0) {  // the next group and, in a batch, its shard
      unsigned long long t = 0;
      if (lane == 0) t = atomicAdd(A.ticket, 1u);
      t = __shfl_sync(0xffffffffu, t, 0);
      const int sh = A.descs && t < n_items ? shard_of_warp(A.item_base, A.n_shards, t, lane) : 0;
      if (lane == 0) {
        s_item = t;
        if (t < n_items) {
          if (A.descs) {
            const qlc_desc d = A.descs[sh];
            s_first = A.item_base[sh];
            s_in = static_cast<const uint8_t*>(d.in);
            s_n = d.in_bytes;
            s_lut = d.lut;
            s_out = static_cast<uint8_t*>(d.out);
            s_cap = d.out_cap;
            s_ob = reinterpret_cast<unsigned long long*>(d.out_bytes);
          } else {
            s_first = 0;
            s_in = A.in;
            s_n = A.n;
            s_lut = A.lut;
            s_out = A.out;
            s_cap = A.out_cap;
            s_ob = A.out_bytes;
          }
        }
      }
    }
    __syncthreads();
    const unsigned long long item = s_item;
    if (item >= n_items) break;
    const uint64_t g = item - s_first;  // group within its tensor
    const uint8_t* in = s_in;
    const uint64_t n = s_n;
    uint8_t* out = s_out;
    const qlc_lut* lut = s_lut;
    if (lut != cur_lut) {
      // A LUT entry must be a codeword of 3..11 bits; anything else (a LUT
      // not made by qlc_build_lut*) would overrun the staging window and the
      // output bound, so the tensor is refused.
      const uint32_t e = lut->enc[tid];
      const uint32_t len = e & 15u, code = e >> 4;
      const bool bad = len < 3 || len > kMaxCode || (code >> len) != 0;
      if (__syncthreads_or(bad)) {
        if (tid == 0) {
          set_status(A.status, QLC_ERR_ARG);
          st_release_u64(&A.gstat[item], kFlagError);
        }
        cur_lut = nullptr;
        continue;
      }
      {
        const uint32_t v = (code << (32 - len)) | len;
        uint4* row = reinterpret_cast<uint4*>(&s_enc[32 * tid]);
#pragma unroll
        for (int k = 0; k < 8; k++) row[k] = make_uint4(v, v, v, v);
      }
      cur_lut = lut;
      __syncthreads();
    }
    const uint64_t n_chunks = (n + cs - 1) / cs;
    const uint64_t n_groups = n_groups_of(n_chunks);
    const uint64_t P = payload_start(n_chunks);
    if (n == 0) {  // an empty shard of a batch: header-only container
      write_header(out, 0, cs, 0, lut, tid);
      if (tid == 0) {
        *reinterpret_cast<unsigned long long*>(out + 48) = 0;
        if (s_ob) *s_ob = P;
      }
      continue;
    }
    uint8_t* payload = out + P;
    unsigned long long* group_off = reinterpret_cast<unsigned long long*>(out + kIndexOff);
    uint16_t* chunk_bits = reinterpret_cast<uint16_t*>(out + kIndexOff + 8 * n_groups);
    const uint64_t gbeg = g * group_syms;
    const uint64_t gend = min(gbeg + group_syms, n);
    if (g == 0) write_header(out, n, cs, n_chunks, lut, tid);

    // ---- pass 1: bits of each chunk; warp w takes chunks w, w+8, ...
    for (uint32_t c = warp; c < kGroupChunks; c += kEncWarps) {
      const uint64_t cbeg = gbeg + (uint64_t)c * cs;
      uint32_t bits = 0;
      if (cbeg < gend) {
        const uint32_t m = (uint32_t)(min(cbeg + cs, gend) - cbeg);
        const uint32_t nv = m / 16;
        const uint4* v = reinterpret_cast<const uint4*>(in + cbeg);
        uint32_t k = lane;
        for (; k + (kPass1Unroll - 1) * 32 < nv; k += kPass1Unroll * 32) {
          uint4 q[kPass1Unroll];
#pragma unroll
          for (int u = 0; u < kPass1Unroll; u++) q[u] = ldg_nc_v4(v + k + 32 * u);
#pragma unroll
          for (int u = 0; u < kPass1Unroll; u++) bits += entry_sum16(tab, q[u]);
        }
        for (; k < nv; k += 32) bits += entry_sum16(tab, ldg_nc_v4(v + k));
        for (uint32_t t = nv * 16 + lane; t < m; t += 32) bits += enc_entry(tab, in[cbeg + t]);
        bits &= (1u << 21) - 1;  // a lane sums at most 4096 lengths of <= 11 bits
        bits = warp_sum_u32(bits);
        if (lane == 0 && QLC_GUARD(g * kGroupChunks + c < n_chunks, A.status))
          chunk_bits[g * kGroupChunks + c] = (uint16_t)bits;
      }
      if (lane == 0) s_chunk_bits[c] = bits;
    }
    __syncthreads();

    // ---- look-back: this group's byte offset in the payload
    if (warp == 0) {
      const uint32_t cb = s_chunk_bits[lane];
      uint32_t incl = cb;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      s_chunk_start[lane] = incl - cb;
      if (lane == 31) s_chunk_start[32] = incl;
      s_seam_idx[lane][0] = s_seam_idx[lane][1] = ~0u;
      const uint32_t gbits = __shfl_sync(0xffffffffu, incl, 31);
      const uint64_t gbytes = align16((gbits + 7) / 8);
      bool err = !QLC_GUARD(item < A.gstat_cap, A.status);
      const unsigned long long excl = err ? 0ull : lookback(A.gstat, item, s_first, gbytes, lane, &err);
      if (lane == 0) {
        s_excl = excl;
        s_err = err;
        if (err) {
          set_status(A.status, QLC_ERR_TIMEOUT);
        } else {
          if (QLC_GUARD(g < n_groups, A.status)) group_off[g] = excl;
          if (g == n_groups - 1) {
            *reinterpret_cast<unsigned long long*>(out + 48) = excl + gbytes;
            if (s_ob) *s_ob = P + excl + gbytes;
          }
        }
      }
    }
    __syncthreads();
    if (s_err) continue;
    uint4* dst = reinterpret_cast<uint4*>(payload + s_excl);

    // ---- pass 2: each warp packs its own chunks (w, w+8, w+16, w+24), 512
    // symbols per step, with warp scans only: a chunk's start bit is known
    // from pass 1.  Completed 16-byte blocks go straight out, except the 16-
    // byte blocks a chunk shares with its neighbours, which wait in s_seam.
    for (uint32_t c = warp; c < kGroupChunks; c += kEncWarps) {
      const uint64_t cbeg = gbeg + (uint64_t)c * cs;
      if (cbeg >= gend) break;
      const uint32_t m = (uint32_t)(min(cbeg + cs, gend) - cbeg);
      if (!QLC_GUARD(cbeg + m <= n, A.status)) break;
      const uint32_t S = s_chunk_start[c];
      Packer pk;
      pk.tab = tab;
      pk.stage = &s_stage[warp][0][0];
      pk.stage_s = stage_s;
      pk.dst = dst;
      pk.blk_lim = (uint32_t)min((uint64_t)((s_cap - P - s_excl) / 16), (uint64_t)0xFFFFFFFFu);
      pk.seam_s = (uint32_t)__cvta_generic_to_shared(&s_seam[c][0]);
      pk.seam_idx_s = (uint32_t)__cvta_generic_to_shared(&s_seam_idx[c][0]);
      pk.seam_blk = (S & 127u) ? (S >> 7) : ~0u;
      pk.base_bit = S;
      pk.win = (S >> 5) & ~3u;
      pk.cur = 0;
      pk.lane = lane;
      // full steps, with the input of the next two steps in flight
      const uint32_t n_full = m / kSub;
      const uint4* src = reinterpret_cast<const uint4*>(in + cbeg) + lane;
      uint4 q0 = make_uint4(0, 0, 0, 0), q1 = q0;
      if (n_full > 0) q0 = ldg_nc_v4(src);
      if (n_full > 1) q1 = ldg_nc_v4(src + 32);
      for (uint32_t i = 0; i < n_full; i++) {
        const uint4 q = q0;
        q0 = q1;
        if (i + 2 < n_full) q1 = ldg_nc_v4(src + 32 * (i + 2));
        pk.step<false>(q, 16);
      }
      // the ragged end of a tensor's last chunk: lane l takes symbols 16 l ...
      if (m % kSub) {
        const uint32_t off = n_full * kSub + 16u * lane;
        const int cnt = off < m ? (int)min(16u, m - off) : 0;
        uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < 16; j++)
          if (j < cnt) w[j >> 2] |= (uint32_t)in[cbeg + off + j] << (8 * (j & 3));
        pk.step<true>(make_uint4(w[0], w[1], w[2], w[3]), cnt);
      }
      // the chunk's partial last block (shared with the next chunk, or the
      // group's zero-padded end) goes to the seam; the buffer is left zeroed
      if (lane == 0) {
        const uint32_t E = s_chunk_start[c + 1];
        uint32_t* cb = pk.stage + pk.cur * kWStage + 4;
        if (E & 127u) {
          s_seam[c][1] = make_uint4(bswap32(cb[0]), bswap32(cb[1]), bswap32(cb[2]), bswap32(cb[3]));
          s_seam_idx[c][1] = E >> 7;
        }
        cb[0] = cb[1] = cb[2] = cb[3] = 0;
      }
      __syncwarp();
    }
    __syncthreads();
    // Seams: lane l writes the block holding chunk l's end, OR-ed with the
    // blocks of chunk l+1 that fall in the same 16 bytes.  A chunk shorter
    // than a block (only the last chunk of a tensor) is merged by the lane of
    // the chunk before it.
    if (warp == 0) {
      const uint32_t i1 = s_seam_idx[lane][1];
      const bool mine = i1 != ~0u && !(lane > 0 && s_seam_idx[lane - 1][1] == i1);
      if (mine) {
        uint4 v = s_seam[lane][1];
        if (lane + 1 < kGroupChunks) {
          for (int k = 0; k < 2; k++) {
            if (s_seam_idx[lane + 1][k] == i1) {
              const uint4 u = s_seam[lane + 1][k];
              v.x |= u.x;
              v.y |= u.y;
              v.z |= u.z;
              v.w |= u.w;
            }
          }
        }
        if (QLC_GUARD((uint64_t)i1 < (s_cap - P - s_excl) / 16, A.status)) st_cs_v4(&dst[i1], v);
      }
    }
  }
}

// n = 0: a header-only container.
__global__ void header_only_kernel(uint8_t* out, uint32_t cs, const qlc_lut* lut,
                                   unsigned long long* out_bytes) {
  const int tid = threadIdx.x;
  write_header(out, 0, cs, 0, lut, tid);
  if (tid == 0) {
    *reinterpret_cast<unsigned long long*>(out + 48) = 0;
    *out_bytes = payload_start(0);
  }
}

}  // namespace qlc

using namespace qlc;

extern "C" {

size_t qlc_encoded_size(size_t n, uint32_t chunk_symbols) {
  if (!chunk_symbols_ok(chunk_symbols)) return 0;
  const uint64_t n_chunks = (n + chunk_symbols - 1) / chunk_symbols;
  const uint64_t group_syms = (uint64_t)kGroupChunks * chunk_symbols;
  const uint64_t full = n / group_syms, rest = n % group_syms;
  uint64_t total = payload_start(n_chunks);
  total += full * align16((group_syms * kMaxCode + 7) / 8);
  if (rest) total += align16((rest * kMaxCode + 7) / 8);
  return (size_t)total;
}

size_t qlc_encode_workspace_size(size_t n, uint32_t chunk_symbols) {
  if (!chunk_symbols_ok(chunk_symbols)) return 0;
  const uint64_t n_chunks = (n + chunk_symbols - 1) / chunk_symbols;
  return (size_t)(16 + 8 * n_groups_of(n_chunks));
}

static int enc_grid(uint64_t items, const qlc_launch* launch) {
  int per_sm = kEncCtasPerSm;
  if (launch && launch->encode_ctas_per_sm > 0 && launch->encode_ctas_per_sm < kEncCtasPerSm)
    per_sm = launch->encode_ctas_per_sm;
  const uint64_t cap = (uint64_t)sm_count() * per_sm;
  return (int)(items < 1 ? 1 : (items < cap ? items : cap));
}

qlc_status qlc_encode(const uint8_t* d_in, size_t n, const qlc_lut* d_lut, uint32_t chunk_symbols,
                      uint8_t* d_out, size_t out_cap, void* d_ws, size_t ws_bytes,
                      uint64_t* d_out_bytes, uint32_t* d_status, qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_encode");
  if (!d_lut || !d_out || !d_out_bytes || (n > 0 && (!d_in || !d_ws))) return QLC_ERR_ARG;
  if (!chunk_symbols_ok(chunk_symbols)) return QLC_ERR_ARG;
  if (!aligned(d_in, 16) || !aligned(d_out, 16) || !aligned(d_lut, 16) || !aligned(d_ws, 16) ||
      !aligned(d_out_bytes, 8) || !aligned(d_status, 4))
    return QLC_ERR_ARG;
  const uint64_t n_chunks = (n + chunk_symbols - 1) / chunk_symbols;
  if (n_chunks > 0xFFFFFFFFull) return QLC_ERR_ARG;
  if (out_cap < qlc_encoded_size(n, chunk_symbols)) return QLC_ERR_CAPACITY;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) {
    header_only_kernel<<<1, 256, 0, st>>>(d_out, chunk_symbols, d_lut,
                                          reinterpret_cast<unsigned long long*>(d_out_bytes));
    return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
  }
  const size_t ws_need = qlc_encode_workspace_size(n, chunk_symbols);
  if (ws_bytes < ws_need) return QLC_ERR_CAPACITY;
  if (cudaMemsetAsync(d_ws, 0, ws_need, st) != cudaSuccess) return QLC_ERR_CUDA;
  EncArgs A = {};
  A.in = d_in;
  A.n = n;
  A.lut = d_lut;
  A.out = d_out;
  A.out_bytes = reinterpret_cast<unsigned long long*>(d_out_bytes);
  A.n_items = n_groups_of(n_chunks);
  A.cs = chunk_symbols;
  A.ticket = static_cast<unsigned int*>(d_ws);
  A.gstat = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(d_ws) + 16);
  A.status = d_status;
  A.out_cap = out_cap;
  A.gstat_cap = (ws_bytes - 16) / 8;
  encode_kernel<<<enc_grid(A.n_items, nullptr), kEncThreads, 0, st>>>(A);
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}

qlc_status qlc_test_encode_stalled_lookback(const uint8_t* d_in, size_t n, const qlc_lut* d_lut,
                                            uint32_t chunk_symbols, uint8_t* d_out, size_t out_cap,
                                            void* d_ws, size_t ws_bytes, uint64_t* d_out_bytes,
                                            uint32_t* d_status, qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_test_encode_stalled_lookback");
  if (!d_in || !d_lut || !d_out || !d_ws || !chunk_symbols_ok(chunk_symbols)) return QLC_ERR_ARG;
  if (!aligned(d_in, 16) || !aligned(d_out, 16) || !aligned(d_lut, 16) || !aligned(d_ws, 16) ||
      !aligned(d_out_bytes, 8) || !aligned(d_status, 4))
    return QLC_ERR_ARG;
  const uint64_t n_chunks = (n + chunk_symbols - 1) / chunk_symbols;
  if (n_groups_of(n_chunks) < 2) return QLC_ERR_ARG;
  if (out_cap < qlc_encoded_size(n, chunk_symbols)) return QLC_ERR_CAPACITY;
  const size_t ws_need = qlc_encode_workspace_size(n, chunk_symbols);
  if (ws_bytes < ws_need) return QLC_ERR_CAPACITY;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_ws, 0, ws_need, st) != cudaSuccess) return QLC_ERR_CUDA;
  if (cudaMemsetAsync(d_ws, 1, 1, st) != cudaSuccess) return QLC_ERR_CUDA;  // group counter = 1
  EncArgs A = {};
  A.in = d_in;
  A.n = n;
  A.lut = d_lut;
  A.out = d_out;
  A.out_bytes = reinterpret_cast<unsigned long long*>(d_out_bytes);
  A.n_items = n_groups_of(n_chunks);
  A.cs = chunk_symbols;
  A.ticket = static_cast<unsigned int*>(d_ws);
  A.gstat = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(d_ws) + 16);
  A.status = d_status;
  A.out_cap = out_cap;
  A.gstat_cap = (ws_bytes - 16) / 8;
  encode_kernel<<<enc_grid(A.n_items, nullptr), kEncThreads, 0, st>>>(A);
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}

qlc_status qlc_encode_batch(const qlc_desc* d_descs, int n_shards, uint32_t chunk_symbols, void* d_ws,
                            size_t ws_bytes, uint32_t* d_status, const qlc_launch* h_launch,
                            qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_encode_batch");
  if (!d_descs || n_shards < 1 || !d_ws || !chunk_symbols_ok(chunk_symbols)) return QLC_ERR_ARG;
  if (!aligned(d_ws, 16) || !aligned(d_descs, 16) || !aligned(d_status, 4)) return QLC_ERR_ARG;
  BatchWs w;
  if (!batch_ws_layout(d_ws, ws_bytes, n_shards, &w)) return QLC_ERR_CAPACITY;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  plan_kernel<<<1, kPlanThreads, 0, st>>>(kPlanEncode, d_descs, n_shards, chunk_symbols, w, d_status);
  if (cudaGetLastError() != cudaSuccess) return QLC_ERR_CUDA;
  EncArgs A = {};
  A.descs = d_descs;
  A.item_base = w.item_base;
  A.n_shards = n_shards;
  A.cs = chunk_symbols;
  A.ticket = w.ticket;
  A.gstat = w.gstat;
  A.status = d_status;
  A.gstat_cap = w.gstat_cap;
  // the item count is only known on the device: launch the full resident grid
  encode_kernel<<<enc_grid(~0ull, h_launch), kEncThreads, 0, st>>>(A);
  return cudaGetLastError() == cudaSuccess ? QLC_OK : QLC_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Encoding without any device allocation by the caller or the library.
//
// Some callers cannot allocate device memory: a plugin running inside a host
// framework whose allocator owns all of the GPU's memory, or a request path
// that must not call cudaMalloc (which can synchronise the device).  For them
// the look-back state that qlc_encode keeps in a caller-provided workspace
// lives instead in this file-scope device array, sized for up to
// kNoAllocMaxGroups groups of 32 chunks.  Every GPU that loads the library
// holds these bytes until the process exits.
namespace qlc {
constexpr uint64_t kNoAllocMaxGroups = 65536;
constexpr size_t kNoAllocScratchBytes = 16 + 8 * kNoAllocMaxGroups;  // 512 KiB + 16 B
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Unique id of the calling thread's current CUDA context, 0 if there is none
// or the driver cannot report it.  The driver entry points come through the
// runtime, so the library needs no link to the driver library.
static unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of g_noalloc_scratch in the current device's context (the
// host-side symbol is not a device address).  It is looked up with the
// device current on the first call, and again whenever the device's context
// has changed since (a reset destroys the old context, and the array moves
// with the new one); without a context id from the driver it is looked up
// on every call.  The cache is shared by all host threads and guarded by a
// mutex.
static void* noalloc_scratch_ptr(qlc_status* err) {
  static std::mutex mu;
  static std::unordered_map<int, std::pair<unsigned long long, void*>> cache;  // device -> (context id, address)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    *err = QLC_ERR_CUDA;
    return nullptr;
  }
  const unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> lock(mu);
  const auto it = cache.find(dev);
  if (it != cache.end() && id != 0 && it->second.first == id) return it->second.second;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
    *err = QLC_ERR_CUDA;
    return nullptr;
  }
  // the lookup makes the device's primary context current if none was
  cache[dev] = {current_context_id(), p};
  return p;
}
}  // namespace qlc

extern "C" qlc_status qlc_encode_noalloc(const uint8_t* d_in, size_t n, const qlc_lut* d_lut,
                                          uint32_t chunk_symbols, uint8_t* d_out, size_t out_cap,
                                          uint64_t* d_out_bytes, uint32_t* d_status,
                                          qlc_stream_t stream) {
  NvtxRange nvtx_range("qlc_encode_noalloc");
  if (!chunk_symbols_ok(chunk_symbols)) return QLC_ERR_ARG;
  const uint64_t n_chunks = (n + chunk_symbols - 1) / chunk_symbols;
  if (n_groups_of(n_chunks) > kNoAllocMaxGroups) return QLC_ERR_CAPACITY;
  qlc_status err = QLC_OK;
  void* ws = noalloc_scratch_ptr(&err);
  if (!ws) return err;
  // qlc_encode clears the part of the array it uses before its kernel runs.
  return qlc_encode(d_in, n, d_lut, chunk_symbols, d_out, out_cap, ws, kNoAllocScratchBytes,
                    d_out_bytes, d_status, stream);
}

namespace qlc {
QLC_DEFINE_CHECK_TAKE(check_take_encode)
}  // namespace qlc
