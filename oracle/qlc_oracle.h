/*
 * qlc_oracle.h -- plain, slow, bit-serial CPU oracle for Quad Length Codes.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  The
 * product path (the CUDA library under paper_2602_17849_gb300/) never links,
 * imports or runs it, and shares no source with it.
 *
 * Every function follows the paper (arXiv 2602.17849, "Quad Length Codes for
 * Lossless Compression of e4m3") and, for the byte layout the paper leaves
 * open, the container-v1 layout written out in the header comment of
 * qlc_oracle.c.  Parity status of each function is stated there too.
 */
#ifndef QLC_ORACLE_H
#define QLC_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORACLE_OK = 0,
  ORACLE_ERR_ARG = 1,
  ORACLE_ERR_CAPACITY = 2,
  ORACLE_ERR_CORRUPT = 3
};

/* Table 1 (Section 5) for id 1, Table 2 (Section 6) for id 2. */
int oracle_scheme(int id, uint16_t area_n[8], uint8_t area_bits[8]);
/* 1 if the 8-area table is one this code family can express, else 0. */
int oracle_scheme_valid(const uint16_t area_n[8], const uint8_t area_bits[8]);

/* Section 4: 8-bit symbols, 256 bins. */
void oracle_histogram(const uint8_t *x, uint64_t n, uint64_t hist[256]);

/* Section 7: symbols sorted by decreasing frequency are mapped to ranks
 * 0..255.  Equal counts: the smaller symbol value gets the smaller rank. */
void oracle_rank(const uint64_t hist[256], uint8_t sym_of_rank[256],
                 uint8_t rank_of_sym[256]);

/* Section 5 / Table 3: the codeword (area code then suffix, MSB first) of a
 * rank.  Returns the length in bits, 0 on a bad argument. */
int oracle_codeword(const uint16_t area_n[8], const uint8_t area_bits[8],
                    int rank, uint32_t *code);

/* Section 7 decoding rule on a codeword given as an integer of `len` bits:
 * returns the rank, or -1 if the bits are not a codeword of that length. */
int oracle_decode_codeword(const uint16_t area_n[8], const uint8_t area_bits[8],
                           uint32_t code, int len);

/* Container v1: bytes needed in the worst case (11 bits per symbol). */
uint64_t oracle_container_bound(uint64_t n, uint32_t chunk_symbols);

/* Encode x[0..n) into a container.  sym_of_rank is the decoder LUT
 * (Table 4); it must be a permutation of 0..255. */
int oracle_encode(const uint8_t *x, uint64_t n, const uint16_t area_n[8],
                  const uint8_t area_bits[8], int scheme_id,
                  const uint8_t sym_of_rank[256], uint32_t chunk_symbols,
                  uint8_t *out, uint64_t cap, uint64_t *out_bytes);

/* Decode a container.  Writes n_symbols to *n_out even on error when the
 * header could be read. */
int oracle_decode(const uint8_t *c, uint64_t c_bytes, uint8_t *out,
                  uint64_t cap, uint64_t *n_out);

/* Huffman code lengths (Section 1 / Section 4 comparison code): 0 for
 * symbols that never occur, 1 when a single symbol occurs. */
void oracle_huffman_lengths(const uint64_t hist[256], uint8_t len[256]);

/* Shannon entropy in bits per symbol (Section 4). */
double oracle_entropy(const uint64_t hist[256]);

/* Sum over symbols of count * QLC code length, with ranks from the same
 * histogram (the payload size in bits, Section 5). */
uint64_t oracle_code_bits(const uint64_t hist[256], const uint16_t area_n[8],
                          const uint8_t area_bits[8]);

/* Bit-serial round trip of a Huffman code built from hist, as a self-check
 * of oracle_huffman_lengths: returns total bits, or UINT64_MAX on mismatch. */
uint64_t oracle_huffman_roundtrip(const uint8_t *x, uint64_t n,
                                  const uint64_t hist[256]);

/* ---- Block-32 e4m3 quantisation (Section 3) -- the f4 fusion's oracle ----
 * e4m3 here is the all-finite eXmY format: sign = bit 7, exponent = bits
 * 6..3 with bias 7, mantissa = bits 2..0; exponent 0 is subnormal
 * (m * 2^-9), otherwise (1 + m/8) * 2^(e-7); the largest value is 480. */

/* Value of an e4m3 byte. */
double oracle_e4m3_value(uint8_t c);

/* The e4m3 byte nearest to v (ties: the even code): |v| is placed between
 * two neighbouring magnitudes by scanning all 128 and compared with their
 * midpoint; values of 480 and beyond give 480; the sign of v is kept (so -0
 * and tiny negatives give 0x80). */
uint8_t oracle_e4m3_nearest(float v);

/* Blocks of 32 consecutive elements (the last may be shorter): scale =
 * absmax / 480 in fp32, code = nearest(x / scale) with the division in fp32;
 * a block whose scale is 0 (absmax 0, or absmax / 480 rounding to 0) gets
 * codes 0x00.  Returns
 * ORACLE_ERR_ARG if any element is not finite. */
int oracle_quantize_block32(const float *x, uint64_t n, uint8_t *codes, float *scales);

/* out[i] = float(value(codes[i])) * scales[i / 32], the product in fp32. */
void oracle_dequantize_block32(const uint8_t *codes, const float *scales, uint64_t n, float *out);

/* bf16 <-> fp32: widening is exact; narrowing rounds to nearest, ties to
 * the even bf16 (finite values only). */
void oracle_bf16_to_f32(const uint16_t *x, uint64_t n, float *out);
void oracle_f32_to_bf16(const float *x, uint64_t n, uint16_t *out);

#ifdef __cplusplus
}
#endif
#endif
