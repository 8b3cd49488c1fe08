/*
 * qlc_testing.h -- test hooks of libqlc (not part of the codec's API).
 *
 * The paper has no counterpart to these; they exist so that tests can drive
 * the library's failure paths on a GPU without faulting, trapping or hanging
 * it.
 */
#ifndef QLC_TESTING_H
#define QLC_TESTING_H

#include "qlc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Runs qlc_encode's kernel with its group counter starting at 1 instead of 0,
 * so group 0 is never encoded and group 1's look-back waits for a value that
 * nobody writes.  Every device-side wait is bounded (about 1 s); the call
 * must end with QLC_ERR_TIMEOUT in *d_status, later groups giving up at once
 * through the propagated error flag, and leave the GPU usable.  Arguments as
 * for qlc_encode; n must span at least two groups of 32 chunks. */
qlc_status qlc_test_encode_stalled_lookback(const uint8_t *d_in, size_t n, const qlc_lut *d_lut,
                                            uint32_t chunk_symbols, uint8_t *d_out, size_t out_cap,
                                            void *d_ws, size_t ws_bytes, uint64_t *d_out_bytes,
                                            uint32_t *d_status, qlc_stream_t stream);

/* The checked build of the library (compiled with -DQLC_CHECKED) guards every
 * index into global and shared memory that its kernels compute from data: an
 * index out of its range skips the access, sets *d_status to QLC_ERR_CHECK
 * where the call has a status word, and records where it happened.  This
 * returns that record for the first failed check since the last call
 * (file number << 16 | source line; 0 if no check failed) and clears it.
 * Synchronises the device.  In a normal build it returns 0xFFFFFFFF. */
uint32_t qlc_test_check_take(void);

#ifdef __cplusplus
}
#endif
#endif /* QLC_TESTING_H */
