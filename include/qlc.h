/*
 * qlc.h -- C ABI of libqlc, a GB300 (sm_103a) CUDA implementation of Quad
 * Length Codes (QLC), arXiv 2602.17849, "Quad Length Codes for Lossless
 * Compression of e4m3".
 *
 * The code: a symbol is a byte.  Symbols are ranked 0..255 by decreasing
 * frequency (Section 7).  The 256 ranks are split into 8 areas; a codeword is
 * the 3-bit area code followed by the rank's position inside its area in that
 * area's number of suffix bits, most significant bit first (Section 5,
 * Table 1; Section 6, Table 2).  An area with 8 suffix bits stores the rank
 * itself (Table 3 prints rank 253 as 111_11111101).  Decoding reads 3 bits,
 * then the area's suffix bits, adds the area's offset and maps the rank back
 * to the symbol with a 256-entry table (Section 7, Table 4).
 *
 * Container v1 (the paper defines no byte layout; little-endian integers):
 *     0  "QLC1", u16 version = 1, u8 scheme id, u8 flags = 0,
 *     8  u64 n (symbols), u32 chunk_symbols, u32 n_chunks = ceil(n/chunk),
 *    24  u16 area_n[8], u8 area_bits[8], u64 payload_bytes, u64 reserved = 0
 *    64  u8 dec[256]            rank -> symbol
 *   320  u64 group_off[G]       G = ceil(n_chunks / 32); payload byte offset
 *        u16 chunk_bits[n_chunks]
 *        zero pad to 16 bytes; payload starts at P = align16(320 + 8G + 2 n_chunks)
 *     P  for each group of 32 chunks: the chunks' codewords back to back, MSB
 *        first, zero-padded to a multiple of 16 bytes.  group_off[0] = 0;
 *        each group starts where the previous padded group ends.
 * A chunk is chunk_symbols consecutive symbols (the last one may be short).
 * Chunks are the unit of parallel decoding: the codes are not
 * self-synchronising, so each chunk's start is found from the index.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are device pointers, h_* host pointers.  The caller
 *     owns every buffer; the library allocates no device memory.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; 0 = legacy default
 *     stream) and do not synchronise the host.
 *   - The return value reports argument and launch errors found on the host.
 *     Errors found on the device (a corrupt container, a capacity shortfall
 *     only the device can see, a wait that timed out) are written to
 *     *d_status with an atomic compare-and-swap from 0, so the first error
 *     is kept: set *d_status to 0 before a sequence of calls and read it after.
 *   - Device pointers must be aligned (cudaMalloc and PyTorch allocations
 *     are): byte buffers (inputs, outputs, containers, workspaces, value
 *     arrays), qlc_lut and qlc_desc arrays to 16 bytes; histograms and
 *     64-bit results (d_out_bytes, d_n_out) to 8; status words and scales to
 *     4.  A misaligned pointer returns QLC_ERR_ARG before anything is
 *     launched; in a batch, a descriptor with a misaligned pointer sets
 *     *d_status to QLC_ERR_ARG and its shard is skipped.
 */
#ifndef QLC_H
#define QLC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *qlc_stream_t; /* same type as cudaStream_t */

typedef enum {
  QLC_OK = 0,
  QLC_ERR_ARG = 1,      /* bad argument (host check) */
  QLC_ERR_CAPACITY = 2, /* an output or workspace buffer is too small */
  QLC_ERR_CORRUPT = 3,  /* container fails validation (device check) */
  QLC_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up */
  QLC_ERR_CUDA = 5,     /* a CUDA runtime call or launch failed */
  QLC_ERR_CHECK = 6     /* an index check failed (only the checked build checks) */
} qlc_status;

#define QLC_VERSION 1
#define QLC_CHUNKS_PER_GROUP 32
#define QLC_HEADER_BYTES 64
#define QLC_INDEX_OFFSET 320
#define QLC_MIN_CHUNK 128
#define QLC_MAX_CHUNK 4096

/* An 8-area scheme (Table 1 / Table 2 of the paper, or another member of the
 * same family).  Valid when the counts sum to 256, suffix widths never
 * decrease, an area with b < 8 suffix bits holds exactly 2^b ranks and an
 * area with 8 bits holds 1..256 ranks (coded as the raw rank).  32 bytes. */
typedef struct qlc_scheme {
  uint16_t area_n[8];  /* ranks per area */
  uint8_t area_bits[8];/* suffix bits per area; code length = 3 + bits */
  uint8_t id;          /* 1 = Table 1, 2 = Table 2, 0 = other */
  uint8_t reserved[7];
} qlc_scheme;

/* Encoder and decoder tables of one tensor (Section 7, Tables 3 and 4).
 * 800 bytes; lives in device memory for qlc_encode. */
typedef struct qlc_lut {
  qlc_scheme scheme;
  uint16_t enc[256]; /* symbol -> (codeword << 4) | code length  (Table 3) */
  uint8_t dec[256];  /* rank -> symbol                            (Table 4) */
} qlc_lut;

/* Library version (QLC_VERSION) and the container version it writes. */
int qlc_version(void);

/* Human-readable name of a status code; never NULL. */
const char *qlc_status_string(qlc_status s);

/* Fills *out with Table 1 (id 1, Section 5) or Table 2 (id 2, Section 6).
 * Host only.  QLC_ERR_ARG for another id or a NULL pointer. */
qlc_status qlc_scheme_table(int id, qlc_scheme *out);

/* 1 if *s is a valid scheme (see qlc_scheme), else 0.  Host only. */
int qlc_scheme_check(const qlc_scheme *s);

/* 256-bin byte histogram (Section 4: 8-bit symbols).
 * d_in: n bytes, 16-byte aligned.  d_hist: 256 uint64 counts on the device.
 * accumulate = 0 overwrites d_hist, 1 adds to it (aggregate histograms over
 * shards, as the paper's PMFs are averaged over shards).  Async on stream.
 * The kernel holds 224 KB of shared memory per block (one block per SM); the
 * first call on a device raises the kernel's shared-memory limit once (a
 * function attribute, allowed inside stream capture), and QLC_ERR_CUDA
 * reports a device that cannot provide it. */
qlc_status qlc_histogram(const uint8_t *d_in, size_t n, uint64_t *d_hist,
                         int accumulate, qlc_stream_t stream);

/* Builds the LUT of a histogram on the device (Section 7): ranks by
 * decreasing count, equal counts broken by smaller symbol first; codes from
 * *h_scheme.  d_hist: 256 uint64 on the device; h_scheme: host pointer to a
 * valid scheme (else QLC_ERR_ARG); d_lut: device qlc_lut written. */
qlc_status qlc_build_lut(const uint64_t *d_hist, const qlc_scheme *h_scheme,
                         qlc_lut *d_lut, qlc_stream_t stream);

/* Same as qlc_build_lut on host memory, synchronously (a CPU twin for
 * callers that build LUTs ahead of time, e.g. one per tensor type). */
qlc_status qlc_build_lut_host(const uint64_t *h_hist, const qlc_scheme *h_scheme,
                              qlc_lut *h_lut);

/* Picks, on the device, the scheme among h_schemes[0..n_schemes) with the
 * fewest payload bits for this histogram (ties: the earlier one) and builds
 * its LUT, as Section 6 adapts the scheme to the distribution.
 * 1 <= n_schemes <= 8.  Async on stream. */
qlc_status qlc_build_lut_best(const uint64_t *d_hist, const qlc_scheme *h_schemes,
                              int n_schemes, qlc_lut *d_lut, qlc_stream_t stream);

/* Section 8 (future work: tuning the areas, symbols per area and code
 * lengths): the scheme of the qlc_scheme family with the fewest payload bits
 * for a histogram, found exhaustively (areas 1..7 complete with
 * non-decreasing widths, area 8 the remaining ranks, raw or complete).
 * h_hist: 256 counts (host).  *out receives the scheme (id 1 / 2 when it is
 * Table 1 / Table 2, else 0); *out_bits (may be NULL) its payload bits.
 * Host only, synchronous. */
qlc_status qlc_scheme_search(const uint64_t *h_hist, qlc_scheme *out, uint64_t *out_bits);

/* Worst-case container bytes for n symbols (every code 11 bits); 0 if
 * chunk_symbols is not a multiple of 128 in [128, 4096]. */
size_t qlc_encoded_size(size_t n, uint32_t chunk_symbols);

/* Device workspace bytes qlc_encode needs (look-back state, one uint64 per
 * group of 32 chunks, plus a counter); 0 for a bad chunk_symbols. */
size_t qlc_encode_workspace_size(size_t n, uint32_t chunk_symbols);

/* Encodes d_in[0..n) into a container at d_out (Sections 5 and 7).
 * d_lut: device LUT from qlc_build_lut*.  chunk_symbols: multiple of 128 in
 * [128, 4096].  out_cap >= qlc_encoded_size(n, chunk_symbols), else
 * QLC_ERR_CAPACITY.  d_ws: ws_bytes >= qlc_encode_workspace_size() of device
 * scratch, overwritten (not preserved between calls).  *d_out_bytes receives
 * the container size.  Device errors go to *d_status: QLC_ERR_TIMEOUT when a
 * look-back wait exceeded its time bound, QLC_ERR_ARG when a LUT entry is not
 * a codeword of 3..11 bits (a LUT not made by qlc_build_lut*).  Async on
 * stream; d_in, d_out 16-byte aligned. */
qlc_status qlc_encode(const uint8_t *d_in, size_t n, const qlc_lut *d_lut,
                      uint32_t chunk_symbols, uint8_t *d_out, size_t out_cap,
                      void *d_ws, size_t ws_bytes, uint64_t *d_out_bytes,
                      uint32_t *d_status, qlc_stream_t stream);

/* Same result as qlc_encode, for callers that cannot allocate device memory
 * (for example a plugin whose host framework's allocator owns the GPU's
 * memory, or a request path that must not call cudaMalloc).  The paper has no
 * counterpart; this is a library convenience.  Instead of a caller workspace
 * it uses scratch space built into the library: one array per GPU of
 * 16 + 8 * 65536 bytes, held until the process exits, which bounds n to at
 * most 65536 groups of 32 chunks (65536 * 32 * chunk_symbols symbols; e.g.
 * 8 GiB at chunk 4096); larger n returns QLC_ERR_CAPACITY.  The first call on
 * each device looks up that device's array address (with the device
 * current), and so does the first call after the device's context changed
 * (a device reset), so make those calls before any stream capture.  The
 * address cache is safe to use from several host threads.  All calls share
 * the one array and each call clears it on `stream` before use: calls that
 * may run at the same time on the GPU (different streams without ordering
 * between them, or calls from several host threads on one stream, whose
 * clears and kernels may interleave) race and must not be issued.  Other
 * arguments, errors and alignment rules as for qlc_encode. */
qlc_status qlc_encode_noalloc(const uint8_t *d_in, size_t n, const qlc_lut *d_lut,
                              uint32_t chunk_symbols, uint8_t *d_out, size_t out_cap,
                              uint64_t *d_out_bytes, uint32_t *d_status,
                              qlc_stream_t stream);

/* Decodes a container (Section 7).  d_in: in_bytes of container, 16-byte
 * aligned.  d_out: out_cap bytes, 16-byte aligned; the decoder writes
 * n = the header's symbol count bytes.  *d_n_out receives n.  The container
 * is validated on the device (header fields, scheme, that dec is a
 * permutation, the group layout and that every chunk ends exactly at its
 * recorded bit count); a failure sets *d_status to QLC_ERR_CORRUPT and leaves
 * d_out partly written; out_cap < n sets QLC_ERR_CAPACITY.  Async on stream.
 * Not every bit string is checked: the decoding rule is total, so a
 * codeword of an area with 8 suffix bits whose suffix lies below that
 * area's first rank (0..87 under Table 1, 0..97 under Table 2; no encoder
 * writes one) decodes without error, as the rank equal to its suffix.  A
 * corruption that only produces such codewords and keeps every chunk's bit
 * count is therefore not detected. */
qlc_status qlc_decode(const uint8_t *d_in, size_t in_bytes, uint8_t *d_out,
                      size_t out_cap, uint64_t *d_n_out, uint32_t *d_status,
                      qlc_stream_t stream);

/* ------------------------------------------------------------------ batches
 * Many tensors ("shards", e.g. the 18 layers x 64 devices = 1152 shards per
 * tensor type of Section 3) in one launch per step.  A batch is an array of
 * descriptors in device memory.  Work is split into items of one group of 32
 * chunks; persistent CTAs take items from a device-side counter, so shards of
 * very different sizes share the GPU evenly.  Per-shard errors go to
 * *d_status; other shards are unaffected. */
typedef struct qlc_desc {
  const void *in;      /* encode / histogram: the shard's symbols; decode: its container */
  uint64_t in_bytes;   /* encode / histogram: n symbols; decode: container bytes */
  void *out;           /* encode: container buffer; decode: decoded symbols */
  uint64_t out_cap;    /* bytes available at out */
  const qlc_lut *lut;  /* encode: this shard's LUT (shards may share one) */
  uint64_t *out_bytes; /* encode: container size; decode: n (device pointer or NULL) */
} qlc_desc;            /* 48 bytes */

/* Launch shape knobs (an autotuner picks them); 0 = library default. */
typedef struct qlc_launch {
  uint16_t encode_ctas_per_sm; /* resident encode CTAs (256 threads) per SM, 1..3 */
  uint16_t decode_ctas_per_sm; /* resident decode warps per SM, 1..20 (larger: 20) */
  uint32_t reserved;
} qlc_launch;

/* Device workspace for the batch calls below, for n_shards shards holding
 * total_symbols symbols, encoded with chunk_symbols (decode batches of
 * containers with that chunk size or larger also fit). */
size_t qlc_batch_workspace_size(int n_shards, uint64_t total_symbols, uint32_t chunk_symbols);

/* Histograms of the shards (Section 4).  shared = 0: d_hists holds
 * n_shards x 256 counts, one histogram per shard; shared = 1: one histogram
 * over all shards (an a-priori LUT per tensor type, Section 7).  Overwrites
 * d_hists.  Uses d_ws.  Async on stream.  Shared memory as qlc_histogram. */
qlc_status qlc_histogram_batch(const qlc_desc *d_descs, int n_shards, uint64_t *d_hists, int shared,
                               void *d_ws, size_t ws_bytes, qlc_stream_t stream);

/* One LUT per histogram (Section 7), each with the scheme among
 * h_schemes[0..n_schemes) that gives it the fewest payload bits (Section 6).
 * d_hists: n_luts x 256; d_luts: n_luts qlc_lut.  Async on stream. */
qlc_status qlc_build_lut_batch(const uint64_t *d_hists, int n_luts, const qlc_scheme *h_schemes,
                               int n_schemes, qlc_lut *d_luts, qlc_stream_t stream);

/* Encodes every shard into its container (as qlc_encode); desc.out_bytes
 * receives each container's size.  Async on stream. */
qlc_status qlc_encode_batch(const qlc_desc *d_descs, int n_shards, uint32_t chunk_symbols,
                            void *d_ws, size_t ws_bytes, uint32_t *d_status,
                            const qlc_launch *h_launch, qlc_stream_t stream);

/* Decodes every shard's container (as qlc_decode); desc.out_bytes receives
 * each n.  Async on stream. */
qlc_status qlc_decode_batch(const qlc_desc *d_descs, int n_shards, void *d_ws, size_t ws_bytes,
                            uint32_t *d_status, const qlc_launch *h_launch, qlc_stream_t stream);

/* Reads n and the total container size from a host copy of the first
 * QLC_HEADER_BYTES bytes of a container (for sizing buffers).  Host only;
 * QLC_ERR_CORRUPT for a bad magic/version, QLC_ERR_ARG for NULL or
 * hdr_bytes < QLC_HEADER_BYTES. */
qlc_status qlc_peek_header(const void *h_hdr, size_t hdr_bytes, uint64_t *n,
                           uint64_t *container_bytes);

/* ---- Block-32 e4m3 quantisation fused with the codec (Section 3) ----
 * The paper's tensors are e4m3 (the all-finite eXmY variant) with one scale
 * per block of 32 consecutive elements.  These calls fuse that quantisation
 * into the pass that counts the histogram (Section 4), and the
 * dequantisation into the decoder's output (Section 7), so the e4m3 codes
 * make one trip less through HBM on each side.
 * Rule per block (the last block may be shorter): scale = absmax / 480 in
 * fp32; code = the e4m3 byte nearest to x / scale (fp32 division), ties to
 * the even code, saturating at 480, sign kept; a block whose scale is 0
 * (absmax 0, or absmax / 480 rounding to 0) gets codes 0x00.
 * Value of a code: sign * m 2^-9 for exponent field 0, else
 * sign * (1 + m/8) 2^(e-7). */
typedef enum { QLC_DTYPE_F32 = 0, QLC_DTYPE_BF16 = 1 } qlc_dtype;

/* Quantises n elements of d_x (dtype) into e4m3 codes d_codes[n] and scales
 * d_scales[ceil(n/32)] (fp32), and, when d_hist is not NULL, counts the codes
 * into d_hist[256] (added when accumulate != 0, else overwritten) in the same
 * pass, ready for qlc_build_lut.  d_x, d_codes and d_scales 16-byte aligned.
 * A non-finite element sets *d_status to QLC_ERR_ARG (its block's codes are
 * then unspecified).  Async on stream. */
qlc_status qlc_quantize_e4m3(const void *d_x, qlc_dtype dtype, size_t n, uint8_t *d_codes,
                             float *d_scales, uint64_t *d_hist, int accumulate,
                             uint32_t *d_status, qlc_stream_t stream);

/* d_out[i] = value(d_codes[i]) * d_scales[i / 32] with the product in fp32
 * (for QLC_DTYPE_BF16 then rounded to nearest even).  d_codes and d_out
 * 16-byte aligned.  Async on stream. */
qlc_status qlc_dequantize_e4m3(const uint8_t *d_codes, const float *d_scales, size_t n,
                               void *d_out, qlc_dtype dtype, qlc_stream_t stream);

/* qlc_decode and qlc_dequantize_e4m3 in one pass: each chunk's decoded codes
 * become values (d_scales: one per 32 symbols of the tensor) before they
 * leave the chip.  d_out: out_cap elements of dtype, 16-byte aligned;
 * *d_n_out receives n.  Validation and errors as qlc_decode (out_cap counts
 * elements).  Async on stream. */
qlc_status qlc_decode_dequantize(const uint8_t *d_in, size_t in_bytes, const float *d_scales,
                                 void *d_out, qlc_dtype dtype, size_t out_cap, uint64_t *d_n_out,
                                 uint32_t *d_status, qlc_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* QLC_H */
