/*
 * qlc_oracle.c -- plain, slow, bit-serial CPU oracle for Quad Length Codes
 * (arXiv 2602.17849).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this file.  It
 * shares no source with the CUDA library and includes none of its headers.
 *
 * What the paper fixes, and where:
 *   - Section 5, Table 1: 256 symbols in 8 areas, a 3-bit area code, then a
 *     suffix of 3,3,3,3,3,4,5,8 bits for 8,8,8,8,8,16,32,168 symbols.
 *   - Section 6, Table 2: 1,3,3,3,3,5,5,8 bits for 2,8,8,8,8,32,32,158.
 *   - Section 7: ranks come from sorting symbols by decreasing frequency; the
 *     encoder looks a symbol's code up in a 256-entry table (Table 3); the
 *     decoder reads the area code, then that area's suffix bits, adds the
 *     area's offset and looks the rank up in a 256-entry table (Table 4).
 *   - Section 4: entropy and compressibility = (8 - bits per symbol) / 8.
 *   - Section 3: the tensors are e4m3 in the all-finite eXmY variant, with a
 *     scale per block of 32 elements.
 *
 * Readings where the paper is silent or ambiguous:
 *   R1 Last area (8 suffix bits): Table 3 prints ranks 253..255 as
 *      111_11111101..111_11111111, i.e. the suffix is the raw 8-bit rank and
 *      that area's offset is 0.  Any area with 8 suffix bits is coded this
 *      way; a suffix below the area's first rank is still decoded as that
 *      rank (the paper's decoding rule is total), the encoder never emits it.
 *   R2 Equal counts: the smaller symbol value gets the smaller rank.
 *   R3 Bits are written most significant first; the first bit of a stream is
 *      bit 7 of its first byte.
 *   R5 Block-32 quantisation (Section 3 names the format and block size
 *      only): scale = absmax / 480 in fp32, code = the nearest e4m3 value to
 *      x / scale (fp32 division), ties to the even code, saturating at 480,
 *      sign kept; a block whose scale is 0 (absmax 0, or absmax / 480 below
 *      the smallest fp32 subnormal) has codes 0x00.  The codec
 *      itself never depends on this; only the fused quantise / dequantise
 *      entry points and the input generator do.
 *   R4 Scheme family: areas with fewer than 8 suffix bits hold exactly
 *      2^bits ranks; areas with 8 suffix bits hold 1..256; the counts sum to
 *      256 and suffix widths never decrease from area to area.
 *
 * Container v1 (not in the paper; all integers little-endian):
 *     0  char[4]  magic "QLC1"
 *     4  u16      version = 1
 *     6  u8       scheme id (1 = Table 1, 2 = Table 2, 0 = other)
 *     7  u8       flags = 0
 *     8  u64      n, number of symbols
 *    16  u32      chunk_symbols, multiple of 128 in [128, 4096]
 *    20  u32      n_chunks = ceil(n / chunk_symbols)
 *    24  u16[8]   symbols per area
 *    40  u8[8]    suffix bits per area
 *    48  u64      payload bytes
 *    56  u64      reserved = 0
 *    64  u8[256]  decoder LUT: rank -> symbol (Table 4)
 *   320  u64[G]   group_off: payload byte offset of each group of 32 chunks
 *        u16[n_chunks] chunk_bits: bits of each chunk's codewords
 *        zero pad to a multiple of 16 bytes; the payload starts there (P)
 *     P  payload: group g holds chunks 32g..32g+31, their codewords back to
 *        back (bit-contiguous across chunk borders), zero-padded to a
 *        multiple of 16 bytes.  group_off[0] = 0 and each next group starts
 *        where the padded previous one ends; payload bytes = their sum.
 *
 * Parity status: every function here is pinned by tests under tests/ (see
 * the file headers there); the paper's own compressibility figures (13.9%,
 * 15.9%, 16.3%, ...) are measured on tensors that are not available, so the
 * values themselves are parity unpinned and only their ordering is checked.
 */
#include "qlc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define HDR_BYTES 64u
#define LUT_OFF 64u
#define INDEX_OFF 320u
#define CHUNKS_PER_GROUP 32u

/* Table 1 (Section 5) and Table 2 (Section 6). */
static const uint16_t TABLE1_N[8] = {8, 8, 8, 8, 8, 16, 32, 168};
static const uint8_t TABLE1_BITS[8] = {3, 3, 3, 3, 3, 4, 5, 8};
static const uint16_t TABLE2_N[8] = {2, 8, 8, 8, 8, 32, 32, 158};
static const uint8_t TABLE2_BITS[8] = {1, 3, 3, 3, 3, 5, 5, 8};

int oracle_scheme(int id, uint16_t area_n[8], uint8_t area_bits[8]) {
  const uint16_t *n;
  const uint8_t *b;
  if (id == 1) {
    n = TABLE1_N;
    b = TABLE1_BITS;
  } else if (id == 2) {
    n = TABLE2_N;
    b = TABLE2_BITS;
  } else {
    return ORACLE_ERR_ARG;
  }
  for (int i = 0; i < 8; i++) {
    area_n[i] = n[i];
    area_bits[i] = b[i];
  }
  return ORACLE_OK;
}

int oracle_scheme_valid(const uint16_t area_n[8], const uint8_t area_bits[8]) {
  unsigned total = 0;
  for (int i = 0; i < 8; i++) {
    if (area_bits[i] > 8) return 0;
    if (i > 0 && area_bits[i] < area_bits[i - 1]) return 0;
    if (area_bits[i] < 8) {
      if (area_n[i] != (1u << area_bits[i])) return 0;
    } else {
      if (area_n[i] < 1 || area_n[i] > 256) return 0;
    }
    total += area_n[i];
  }
  return total == 256;
}

void oracle_histogram(const uint8_t *x, uint64_t n, uint64_t hist[256]) {
  for (int s = 0; s < 256; s++) hist[s] = 0;
  for (uint64_t i = 0; i < n; i++) hist[x[i]]++;
}

/* "comes before" in the Section 7 sort: larger count first, then R2. */
static int before(const uint64_t hist[256], int a, int b) {
  if (hist[a] != hist[b]) return hist[a] > hist[b];
  return a < b;
}

void oracle_rank(const uint64_t hist[256], uint8_t sym_of_rank[256],
                 uint8_t rank_of_sym[256]) {
  int order[256];
  for (int s = 0; s < 256; s++) order[s] = s;
  /* insertion sort, plain and stable */
  for (int i = 1; i < 256; i++) {
    int s = order[i];
    int j = i - 1;
    while (j >= 0 && before(hist, s, order[j])) {
      order[j + 1] = order[j];
      j--;
    }
    order[j + 1] = s;
  }
  for (int r = 0; r < 256; r++) {
    sym_of_rank[r] = (uint8_t)order[r];
    rank_of_sym[order[r]] = (uint8_t)r;
  }
}

/* First rank of each area: the sum of the counts of the areas before it. */
static void area_bases(const uint16_t area_n[8], unsigned base[8]) {
  unsigned b = 0;
  for (int i = 0; i < 8; i++) {
    base[i] = b;
    b += area_n[i];
  }
}

int oracle_codeword(const uint16_t area_n[8], const uint8_t area_bits[8],
                    int rank, uint32_t *code) {
  unsigned base[8];
  if (rank < 0 || rank > 255) return 0;
  area_bases(area_n, base);
  for (int i = 0; i < 8; i++) {
    if ((unsigned)rank >= base[i] && (unsigned)rank < base[i] + area_n[i]) {
      /* Section 5: area code i (3 bits) followed by the symbol's position
       * in the area; R1: with 8 suffix bits the position is the raw rank. */
      unsigned suffix = area_bits[i] == 8 ? (unsigned)rank : (unsigned)rank - base[i];
      *code = ((uint32_t)i << area_bits[i]) | suffix;
      return 3 + area_bits[i];
    }
  }
  return 0;
}

int oracle_decode_codeword(const uint16_t area_n[8], const uint8_t area_bits[8],
                           uint32_t code, int len) {
  unsigned base[8];
  area_bases(area_n, base);
  if (len < 3 || len > 11) return -1;
  unsigned area = (code >> (len - 3)) & 7u;
  if (3 + area_bits[area] != len) return -1;
  unsigned suffix = code & ((1u << area_bits[area]) - 1u);
  /* Section 7: rank = area offset + suffix; R1: offset 0 for 8 bits. */
  return area_bits[area] == 8 ? (int)suffix : (int)(base[area] + suffix);
}

/* ---------------------------------------------------------------- bits */

static void put_bit(uint8_t *buf, uint64_t pos, int bit) {
  uint8_t mask = (uint8_t)(0x80u >> (pos & 7u));
  if (bit)
    buf[pos >> 3] |= mask;
  else
    buf[pos >> 3] &= (uint8_t)~mask;
}

/* Reads bit `pos` of buf[0..nbytes); bits past the end read as 0. */
static int get_bit(const uint8_t *buf, uint64_t nbytes, uint64_t pos) {
  if ((pos >> 3) >= nbytes) return 0;
  return (buf[pos >> 3] >> (7u - (pos & 7u))) & 1;
}

static void put_le(uint8_t *p, uint64_t v, int bytes) {
  for (int i = 0; i < bytes; i++) p[i] = (uint8_t)(v >> (8 * i));
}

static uint64_t get_le(const uint8_t *p, int bytes) {
  uint64_t v = 0;
  for (int i = 0; i < bytes; i++) v |= (uint64_t)p[i] << (8 * i);
  return v;
}

static uint64_t align16(uint64_t v) { return (v + 15u) & ~(uint64_t)15u; }

static int chunk_symbols_ok(uint32_t cs) {
  return cs >= 128 && cs <= 4096 && cs % 128 == 0;
}

static uint64_t payload_start(uint64_t n_chunks) {
  uint64_t n_groups = (n_chunks + CHUNKS_PER_GROUP - 1) / CHUNKS_PER_GROUP;
  return align16(INDEX_OFF + 8 * n_groups + 2 * n_chunks);
}

uint64_t oracle_container_bound(uint64_t n, uint32_t chunk_symbols) {
  if (!chunk_symbols_ok(chunk_symbols)) return 0;
  uint64_t n_chunks = (n + chunk_symbols - 1) / chunk_symbols;
  uint64_t total = payload_start(n_chunks);
  uint64_t group_syms = (uint64_t)CHUNKS_PER_GROUP * chunk_symbols;
  for (uint64_t first = 0; first < n; first += group_syms) {
    uint64_t syms = n - first < group_syms ? n - first : group_syms;
    total += align16((syms * 11 + 7) / 8);
  }
  return total;
}

static int is_permutation(const uint8_t t[256]) {
  int seen[256] = {0};
  for (int i = 0; i < 256; i++) {
    if (seen[t[i]]) return 0;
    seen[t[i]] = 1;
  }
  return 1;
}

static int scheme_id_ok(int id, const uint16_t area_n[8], const uint8_t area_bits[8]) {
  uint16_t n[8];
  uint8_t b[8];
  if (id == 0) return 1;
  if (oracle_scheme(id, n, b) != ORACLE_OK) return 0;
  for (int i = 0; i < 8; i++)
    if (n[i] != area_n[i] || b[i] != area_bits[i]) return 0;
  return 1;
}

int oracle_encode(const uint8_t *x, uint64_t n, const uint16_t area_n[8],
                  const uint8_t area_bits[8], int scheme_id,
                  const uint8_t sym_of_rank[256], uint32_t chunk_symbols,
                  uint8_t *out, uint64_t cap, uint64_t *out_bytes) {
  if (!chunk_symbols_ok(chunk_symbols)) return ORACLE_ERR_ARG;
  if (!oracle_scheme_valid(area_n, area_bits)) return ORACLE_ERR_ARG;
  if (!scheme_id_ok(scheme_id, area_n, area_bits)) return ORACLE_ERR_ARG;
  if (!is_permutation(sym_of_rank)) return ORACLE_ERR_ARG;
  if (cap < oracle_container_bound(n, chunk_symbols)) return ORACLE_ERR_CAPACITY;

  uint8_t rank_of_sym[256];
  for (int r = 0; r < 256; r++) rank_of_sym[sym_of_rank[r]] = (uint8_t)r;
  /* Table 3: the encoder LUT, indexed by input symbol. */
  uint32_t enc_code[256];
  int enc_len[256];
  for (int s = 0; s < 256; s++)
    enc_len[s] = oracle_codeword(area_n, area_bits, rank_of_sym[s], &enc_code[s]);

  uint64_t n_chunks = (n + chunk_symbols - 1) / chunk_symbols;
  if (n_chunks > 0xFFFFFFFFu) return ORACLE_ERR_ARG;
  uint64_t n_groups = (n_chunks + CHUNKS_PER_GROUP - 1) / CHUNKS_PER_GROUP;
  uint64_t P = payload_start(n_chunks);
  memset(out, 0, P);

  uint8_t *payload = out + P;
  uint64_t pos = 0; /* bit position in the payload */
  for (uint64_t g = 0; g < n_groups; g++) {
    put_le(out + INDEX_OFF + 8 * g, pos / 8, 8);
    for (uint64_t c = g * CHUNKS_PER_GROUP;
         c < n_chunks && c < (g + 1) * CHUNKS_PER_GROUP; c++) {
      uint64_t start = pos;
      uint64_t first = c * chunk_symbols;
      uint64_t last = first + chunk_symbols < n ? first + chunk_symbols : n;
      for (uint64_t i = first; i < last; i++) {
        uint32_t code = enc_code[x[i]];
        int len = enc_len[x[i]];
        for (int k = len - 1; k >= 0; k--) put_bit(payload, pos++, (code >> k) & 1u);
      }
      put_le(out + INDEX_OFF + 8 * n_groups + 2 * c, pos - start, 2);
    }
    while (pos % 128 != 0) put_bit(payload, pos++, 0);
  }

  memcpy(out, "QLC1", 4);
  put_le(out + 4, 1, 2);
  out[6] = (uint8_t)scheme_id;
  out[7] = 0;
  put_le(out + 8, n, 8);
  put_le(out + 16, chunk_symbols, 4);
  put_le(out + 20, n_chunks, 4);
  for (int i = 0; i < 8; i++) {
    put_le(out + 24 + 2 * i, area_n[i], 2);
    out[40 + i] = area_bits[i];
  }
  put_le(out + 48, pos / 8, 8);
  put_le(out + 56, 0, 8);
  memcpy(out + LUT_OFF, sym_of_rank, 256);
  *out_bytes = P + pos / 8;
  return ORACLE_OK;
}

int oracle_decode(const uint8_t *c, uint64_t c_bytes, uint8_t *out,
                  uint64_t cap, uint64_t *n_out) {
  if (c_bytes < INDEX_OFF) return ORACLE_ERR_CORRUPT;
  if (memcmp(c, "QLC1", 4) != 0) return ORACLE_ERR_CORRUPT;
  if (get_le(c + 4, 2) != 1 || c[7] != 0 || get_le(c + 56, 8) != 0)
    return ORACLE_ERR_CORRUPT;
  uint16_t area_n[8];
  uint8_t area_bits[8];
  for (int i = 0; i < 8; i++) {
    area_n[i] = (uint16_t)get_le(c + 24 + 2 * i, 2);
    area_bits[i] = c[40 + i];
  }
  if (!oracle_scheme_valid(area_n, area_bits)) return ORACLE_ERR_CORRUPT;
  if (!scheme_id_ok(c[6], area_n, area_bits)) return ORACLE_ERR_CORRUPT;
  uint64_t n = get_le(c + 8, 8);
  uint32_t cs = (uint32_t)get_le(c + 16, 4);
  uint64_t n_chunks = get_le(c + 20, 4);
  if (!chunk_symbols_ok(cs)) return ORACLE_ERR_CORRUPT;
  if (n_chunks != (n + cs - 1) / cs) return ORACLE_ERR_CORRUPT;
  const uint8_t *dec = c + LUT_OFF;
  if (!is_permutation(dec)) return ORACLE_ERR_CORRUPT;
  uint64_t n_groups = (n_chunks + CHUNKS_PER_GROUP - 1) / CHUNKS_PER_GROUP;
  uint64_t P = payload_start(n_chunks);
  uint64_t payload_bytes = get_le(c + 48, 8);
  if (P > c_bytes || payload_bytes > c_bytes - P) return ORACLE_ERR_CORRUPT;
  *n_out = n;
  if (cap < n) return ORACLE_ERR_CAPACITY;

  unsigned base[8];
  area_bases(area_n, base);
  const uint8_t *payload = c + P;
  uint64_t expect_off = 0;
  for (uint64_t g = 0; g < n_groups; g++) {
    uint64_t goff = get_le(c + INDEX_OFF + 8 * g, 8);
    if (goff != expect_off) return ORACLE_ERR_CORRUPT;
    uint64_t pos = goff * 8;
    for (uint64_t ch = g * CHUNKS_PER_GROUP;
         ch < n_chunks && ch < (g + 1) * CHUNKS_PER_GROUP; ch++) {
      uint64_t cbits = get_le(c + INDEX_OFF + 8 * n_groups + 2 * ch, 2);
      uint64_t start = pos;
      uint64_t first = ch * cs;
      uint64_t last = first + cs < n ? first + cs : n;
      for (uint64_t i = first; i < last; i++) {
        /* Section 7: the area code gives the suffix length ... */
        unsigned area = 0;
        for (int k = 0; k < 3; k++) area = (area << 1) | (unsigned)get_bit(payload, payload_bytes, pos++);
        unsigned suffix = 0;
        for (int k = 0; k < area_bits[area]; k++)
          suffix = (suffix << 1) | (unsigned)get_bit(payload, payload_bytes, pos++);
        /* ... then the area offset is added (R1: 0 for 8 suffix bits) and
         * the decoder LUT maps the rank back to the symbol. */
        unsigned rank = area_bits[area] == 8 ? suffix : base[area] + suffix;
        out[i] = dec[rank];
      }
      if (pos - start != cbits) return ORACLE_ERR_CORRUPT;
    }
    expect_off = align16((pos + 7) / 8);
  }
  if (expect_off != payload_bytes) return ORACLE_ERR_CORRUPT;
  return ORACLE_OK;
}

/* ------------------------------------------------------------- Huffman */

void oracle_huffman_lengths(const uint64_t hist[256], uint8_t len[256]) {
  /* nodes 0..255 are the symbols, 256.. are merged nodes */
  uint64_t weight[511];
  int parent[511];
  int alive[511];
  int n_nodes = 256, n_alive = 0;
  for (int s = 0; s < 256; s++) {
    weight[s] = hist[s];
    parent[s] = -1;
    alive[s] = hist[s] > 0;
    n_alive += alive[s];
    len[s] = 0;
  }
  if (n_alive == 0) return;
  if (n_alive == 1) {
    for (int s = 0; s < 256; s++)
      if (hist[s] > 0) len[s] = 1;
    return;
  }
  while (n_alive > 1) {
    /* the two lightest live nodes; equal weights: the smaller node id */
    int a = -1, b = -1;
    for (int i = 0; i < n_nodes; i++) {
      if (!alive[i]) continue;
      if (a < 0 || weight[i] < weight[a]) {
        b = a;
        a = i;
      } else if (b < 0 || weight[i] < weight[b]) {
        b = i;
      }
    }
    int m = n_nodes++;
    weight[m] = weight[a] + weight[b];
    parent[m] = -1;
    alive[m] = 1;
    alive[a] = alive[b] = 0;
    parent[a] = parent[b] = m;
    n_alive--;
  }
  for (int s = 0; s < 256; s++) {
    if (hist[s] == 0) continue;
    int d = 0;
    for (int v = s; parent[v] >= 0; v = parent[v]) d++;
    len[s] = (uint8_t)d;
  }
}

double oracle_entropy(const uint64_t hist[256]) {
  double total = 0.0, h = 0.0;
  for (int s = 0; s < 256; s++) total += (double)hist[s];
  if (total == 0.0) return 0.0;
  for (int s = 0; s < 256; s++) {
    if (hist[s] == 0) continue;
    double p = (double)hist[s] / total;
    h -= p * log2(p);
  }
  return h;
}

uint64_t oracle_code_bits(const uint64_t hist[256], const uint16_t area_n[8],
                          const uint8_t area_bits[8]) {
  uint8_t sym_of_rank[256], rank_of_sym[256];
  oracle_rank(hist, sym_of_rank, rank_of_sym);
  uint64_t bits = 0;
  for (int s = 0; s < 256; s++) {
    uint32_t code;
    int len = oracle_codeword(area_n, area_bits, rank_of_sym[s], &code);
    bits += hist[s] * (uint64_t)len;
  }
  return bits;
}

/* Canonical code from lengths: codes assigned in order of (length, symbol). */
static void canonical_codes(const uint8_t len[256], uint64_t code[256]) {
  uint64_t next = 0;
  int prev_len = 0;
  for (int l = 1; l <= 64; l++) {
    for (int s = 0; s < 256; s++) {
      if (len[s] != l) continue;
      next <<= (l - prev_len);
      prev_len = l;
      code[s] = next++;
    }
  }
}

uint64_t oracle_huffman_roundtrip(const uint8_t *x, uint64_t n,
                                  const uint64_t hist[256]) {
  uint8_t len[256];
  uint64_t code[256];
  oracle_huffman_lengths(hist, len);
  for (int s = 0; s < 256; s++) code[s] = 0;
  canonical_codes(len, code);
  uint64_t total = 0;
  for (uint64_t i = 0; i < n; i++) total += len[x[i]];
  uint8_t *buf = (uint8_t *)calloc((size_t)(total / 8 + 1), 1);
  if (!buf) return UINT64_MAX;
  uint64_t pos = 0;
  for (uint64_t i = 0; i < n; i++)
    for (int k = len[x[i]] - 1; k >= 0; k--) put_bit(buf, pos++, (int)((code[x[i]] >> k) & 1u));
  /* bit-serial decode: extend the code one bit at a time until it matches */
  uint64_t rpos = 0;
  for (uint64_t i = 0; i < n; i++) {
    uint64_t v = 0;
    int l = 0, found = -1;
    while (found < 0 && l < 64) {
      v = (v << 1) | (uint64_t)get_bit(buf, total / 8 + 1, rpos++);
      l++;
      for (int s = 0; s < 256; s++)
        if (len[s] == l && code[s] == v) {
          found = s;
          break;
        }
    }
    if (found != x[i]) {
      free(buf);
      return UINT64_MAX;
    }
  }
  free(buf);
  return rpos == total ? total : UINT64_MAX;
}

/* ---- Block-32 e4m3 quantisation (Section 3: eXmY e4m3, block size 32) ---- */

double oracle_e4m3_value(uint8_t c) {
  const int s = c >> 7, e = (c >> 3) & 15, m = c & 7;
  const double mag = e == 0 ? m * ldexp(1.0, -9) : (1.0 + m / 8.0) * ldexp(1.0, e - 7);
  return s ? -mag : mag;
}

uint8_t oracle_e4m3_nearest(float v) {
  const double a = fabs((double)v); /* exact */
  int best;
  if (a >= 480.0) {
    best = 127; /* nothing lies above 480: saturate */
  } else {
    /* lo = the largest magnitude code with value <= a; a lies in
     * [value(lo), value(lo + 1)) and the nearer end wins, the even code on a
     * tie.  The midpoint of two neighbours is exact in double. */
    int lo = 0;
    for (int c = 1; c < 128; c++)
      if (oracle_e4m3_value((uint8_t)c) <= a) lo = c;
    const double mid = (oracle_e4m3_value((uint8_t)lo) + oracle_e4m3_value((uint8_t)(lo + 1))) / 2;
    if (a < mid)
      best = lo;
    else if (a > mid)
      best = lo + 1;
    else
      best = (lo & 1) ? lo + 1 : lo;
  }
  return (uint8_t)(best | (signbit(v) ? 0x80 : 0));
}

int oracle_quantize_block32(const float *x, uint64_t n, uint8_t *codes, float *scales) {
  int st = ORACLE_OK;
  for (uint64_t b0 = 0; b0 < n; b0 += 32) {
    const uint64_t b1 = b0 + 32 < n ? b0 + 32 : n;
    float amax = 0.0f;
    for (uint64_t i = b0; i < b1; i++) {
      if (!isfinite(x[i])) st = ORACLE_ERR_ARG;
      const float a = fabsf(x[i]);
      if (a > amax) amax = a;
    }
    const float scale = amax / 480.0f;
    scales[b0 / 32] = scale;
    for (uint64_t i = b0; i < b1; i++) codes[i] = scale > 0.0f ? oracle_e4m3_nearest(x[i] / scale) : 0;
  }
  return st;
}

void oracle_dequantize_block32(const uint8_t *codes, const float *scales, uint64_t n, float *out) {
  for (uint64_t i = 0; i < n; i++) out[i] = (float)oracle_e4m3_value(codes[i]) * scales[i / 32];
}

void oracle_bf16_to_f32(const uint16_t *x, uint64_t n, float *out) {
  for (uint64_t i = 0; i < n; i++) {
    const uint32_t u = (uint32_t)x[i] << 16;
    memcpy(&out[i], &u, 4);
  }
}

void oracle_f32_to_bf16(const float *x, uint64_t n, uint16_t *out) {
  for (uint64_t i = 0; i < n; i++) {
    /* the two bf16 neighbours of x[i] and the one nearer (ties: even) */
    uint32_t u;
    memcpy(&u, &x[i], 4);
    const uint32_t lo = u & 0xFFFF0000u, hi = lo + 0x10000u;
    const uint32_t rest = u & 0xFFFFu;
    uint32_t pick = lo;
    if (rest > 0x8000u || (rest == 0x8000u && ((lo >> 16) & 1u))) pick = hi;
    out[i] = (uint16_t)(pick >> 16);
  }
}
