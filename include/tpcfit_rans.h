/* rANS entropy coding of int16 codes on the GPU (the track-model compression
 * residuals of tpcfit_result.res_y / res_z).
 *
 * The paper's TPC data go through rANS entropy coding after the track-model
 * compression (Sec. 5; the asynchronous reconstruction times the TPC rANS
 * decoding, Table 2); it gives no format.  The container written here:
 *
 *   symbols   code c in [-255, 255] -> symbol c + 255; any other code is the
 *             escape symbol 511 and its raw int16 goes to an escape list
 *   model     one static table: counts normalised to frequencies summing to
 *             2^12 (f = max(1, n_s 2^12 / N) for present symbols, the excess
 *             taken from / given to the most frequent symbol, lowest first)
 *   coder     range ANS (Duda 2013), 32-bit states in [2^16, 2^32), 16-bit
 *             renormalisation words
 *   layout    segments of `segment_symbols` symbols (a multiple of 32); in a
 *             segment symbol i is coded by lane i mod 32 at step i / 32 (32
 *             interleaved states); words in the order a forward decoder
 *             consumes them; payload per segment = 32 final states + words
 *   container 64-byte header ("TPR1", version 1, n, segment symbols,
 *             segments, scale bits 12, alphabet 512, escapes, payload bytes),
 *             frequency table (512 x uint16), segment payload byte offsets and
 *             escape offsets ((segments + 1) x uint64 each), payload, escapes
 *             (int16); little endian.
 *
 * All buffers are DEVICE memory, at least 8-byte aligned; `stream` is a
 * cudaStream_t as void* (NULL = the handle's stream).  Both calls block until
 * done.  Scratch comes from the handle (about 4 bytes per code while
 * encoding).  Errors: TPCFIT_E_INVAL for bad arguments, an output capacity
 * below the container's size (nothing useful is written), or a stream that is
 * malformed or damaged (decode); TPCFIT_E_NOMEM, TPCFIT_E_CUDA.
 */
#ifndef TPCFIT_RANS_H
#define TPCFIT_RANS_H

#include <stdint.h>

#include "tpcfit.h"

#ifdef __cplusplus
extern "C" {
#endif

#define TPCFIT_RANS_SEGMENT_DEFAULT 16384

/* Largest container size for n codes in segments of segment_symbols (0 =
 * TPCFIT_RANS_SEGMENT_DEFAULT); -1 on bad arguments. */
int64_t tpcfit_rans_bound(int64_t n, int32_t segment_symbols);

/* Encode n codes into out (capacity out_cap bytes); *out_size = container size. */
int tpcfit_rans_encode(tpcfit_handle *h, const int16_t *codes, int64_t n, int32_t segment_symbols, uint8_t *out,
                       int64_t out_cap, int64_t *out_size, void *stream);

/* Decode a container of in_size bytes into n codes; n must equal the
 * container's symbol count. */
int tpcfit_rans_decode(tpcfit_handle *h, const uint8_t *in, int64_t in_size, int16_t *codes, int64_t n,
                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TPCFIT_RANS_H */
