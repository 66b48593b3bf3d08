/*
 * Allocation-free variant of the tpcfit frame fit.  The paper has no
 * counterpart: this is a service for callers of the library.
 *
 * Who needs it: callers that cannot call cudaMalloc while they run, for
 * example an application whose device memory is already reserved by another
 * allocator (a framework's caching pool that owns the HBM, so an extra
 * cudaMalloc fails or fragments it), or an online processing loop that
 * forbids allocation in steady state to keep its latency predictable.
 */
#ifndef TPCFIT_NOALLOC_H
#define TPCFIT_NOALLOC_H

#include "tpcfit.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest frame tpcfit_fit_noalloc accepts.  The scratch for this many tracks
 * (about 1.6 MB: seeds, sort permutation and histogram, work counter, error
 * word, pad-row table) is a static device array.  A device holds it from the
 * moment the library's device code is loaded there until the process exits;
 * with the CUDA runtime's lazy module loading (the default) that is the first
 * call on that device. */
#define TPCFIT_NOALLOC_MAX_TRACKS 65536

/* Fit one DEVICE frame into DEVICE results, like tpcfit_fit, without creating
 * a handle and without allocating any memory (no cudaMalloc, no cudaFree, no
 * allocating library routine).  The caller passes the frame and result
 * buffers; `cfg` (NULL = tpcfit_default_config) gives the fit parameters and
 * cfg->device the GPU; `stream` is a cudaStream_t passed as void* (NULL = the
 * default stream).  The call enqueues the fit on `stream` and waits for it.
 *
 * Set-up: the first call on each device looks up the device address of the
 * static scratch array; make that first call before any stream capture.
 * That first call is also where the CUDA driver, loading the library's
 * device code on the device, places the static array (and the kernels): a
 * driver-side allocation of about 1.6 MB plus code, which can fail if another
 * allocator has already taken all of the device memory (the kernels, too,
 * are loaded on their first launch).  A caller that must not allocate at
 * all in its steady state makes one call on each device during its set-up,
 * before that state begins, with a small frame and the configuration (and
 * residual outputs) it will use; later calls allocate nothing.
 *
 * Device: the call makes cfg->device current while it runs and gives the
 * calling thread its previous current device back before it returns.
 *
 * Residual codes: when res->res_y or res->res_z is set, they are written as
 * by tpcfit_fit (steps cfg->res_step_y_cm, cfg->res_step_z_cm), by one more
 * kernel that needs no scratch.
 *
 * Sharing: all calls on a device share the one scratch array, which keeps the
 * last call's contents; every call clears what must start at zero.  Calls that
 * overlap on the GPU (two in flight at the same time, from any threads or
 * streams) race on the array and give wrong results: serialise them.
 *
 * Returns TPCFIT_OK, TPCFIT_E_INVAL (NULL pointers, host memory, a frame with
 * more than TPCFIT_NOALLOC_MAX_TRACKS tracks, parameters out of range, or
 * malformed offsets), TPCFIT_E_NODEV (device cannot be selected) or
 * TPCFIT_E_CUDA (a launch, copy or wait failed), with the detail in
 * tpcfit_last_error_message().  Per-track results and statuses are as for
 * tpcfit_fit. */
int tpcfit_fit_noalloc(const tpcfit_config *cfg, const tpcfit_frame *frame, tpcfit_result *res, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TPCFIT_NOALLOC_H */
