/*
 * tpcfit: batched Kalman-filter fit of TPC tracks on one GB300 (sm_103a).
 *
 * The paper (Eulisse & Rohr, "The O2 software framework and GPU usage in ALICE
 * online and offline reconstruction in Run 3") identifies TPC tracking as the
 * step that dominates synchronous processing (Sec. 5, Table 1: TPC processing
 * 99.37 %) and asynchronous processing (Table 2: 61.41 %), and runs it on GPUs
 * (Sec. 6).  It does not write the fit out; this library implements the
 * textbook Kalman track fit (state y, z, sinphi, tanlambda, q/pT on pad-row
 * planes of a sector, exact helix in a uniform Bz field, chi2-gated cluster
 * updates, Highland multiple scattering, an outward then an inward pass).
 *
 * Conventions for every entry point:
 *  - return TPCFIT_OK (0) or a negative TPCFIT_E_* code; tpcfit_strerror()
 *    names it and tpcfit_last_error_message() gives detail for the calling
 *    thread;
 *  - the caller owns every frame and result buffer; the library owns its
 *    handle, device scratch pools, streams and events;
 *  - numerical failures of one track never fail a call: they are reported in
 *    that track's status (TPCFIT_TRACK_*);
 *  - one handle is driven by one caller thread at a time.
 *
 * Data layout (structure of arrays, one frame = one time frame or event batch):
 *  clusters of track t are indices [track_offsets[t], track_offsets[t+1]) of
 *  x, y, z, sy2, sz2 (float32, cm and cm^2) and row (uint8 pad-row index,
 *  strictly ascending within a track); track_offsets is int64[n_tracks+1]
 *  with track_offsets[0] == 0 and track_offsets[n_tracks] == n_clusters.
 *  Results: state float32[n_tracks*5] = (y, z, sinphi, tanlambda, q/pT) at
 *  x_ref (the innermost cluster's x); cov float32[n_tracks*15] packed lower
 *  triangle (00,10,11,20,21,22,30,...,44); chi2 float64 (inward pass); ndf
 *  int32 = 2*accepted_inward - 5; status int32; accept uint8[n_clusters]
 *  (bit0 accepted in the outward pass, bit1 in the inward pass).
 */
#ifndef TPCFIT_H
#define TPCFIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TPCFIT_OK 0
#define TPCFIT_E_INVAL (-1)    /* bad argument or malformed frame (offsets) */
#define TPCFIT_E_NOMEM (-2)    /* device allocation failed, or a frame larger than the HBM budget */
#define TPCFIT_E_CUDA (-3)     /* a CUDA runtime call failed */
#define TPCFIT_E_TIMEOUT (-4)  /* a bounded wait expired */
#define TPCFIT_E_BUSY (-5)     /* no free serving slot and the queue is full */
#define TPCFIT_E_NOTFOUND (-6) /* unknown ticket */
#define TPCFIT_E_NODEV (-7)    /* no CUDA device, or not an sm_103 device */

#define TPCFIT_MEM_HOST 0      /* pointers are host memory (pinned gives overlapped copies) */
#define TPCFIT_MEM_DEVICE 1    /* pointers are device memory of the handle's device */

/* per-track status */
#define TPCFIT_TRACK_OK 0
#define TPCFIT_TRACK_TOO_FEW 1    /* fewer than max(min_clusters, 3) clusters */
#define TPCFIT_TRACK_SNP_LIMIT 2  /* |sinphi| reached snp_max */
#define TPCFIT_TRACK_NOT_PD 3     /* innovation matrix not positive definite */
#define TPCFIT_TRACK_NONFINITE 4  /* non-finite cluster value, or non-finite fitted state */
#define TPCFIT_TRACK_BAD_INPUT 5  /* rows not ascending, row >= n_rows, variance <= 0, bad offsets */
#define TPCFIT_TRACK_STOPPED 6    /* energy loss: one row would change p^2 by more than 50 % */
#define TPCFIT_TRACK_DERAILED 7   /* the fit completed, but its inward pass accepted fewer than 80 % of
                                     the track's clusters: it lost the track for a stretch, and its state
                                     and covariance (written as for OK) do not describe it */

/* ticket states for tpcfit_poll */
#define TPCFIT_PENDING 0
#define TPCFIT_DONE 1
#define TPCFIT_FAILED 2

typedef struct tpcfit_handle tpcfit_handle; /* opaque, library-owned */

/* Fit and runtime parameters.  The fit parameters are readings of the method
 * (the paper gives none): see tpcfit_default_config for the values used. */
typedef struct tpcfit_config {
  float bz_tesla;         /* solenoid field (0.5 T) */
  float chi2_max;         /* gate on the 2-dof chi2 of one cluster; equality accepts (16) */
  float xx0_per_row;      /* radiation length fraction per crossed pad row (5e-4; 0 disables scattering) */
  float mass_gev;         /* particle mass for beta in the Highland formula (pion, 0.13957) */
  float snp_max;          /* |sinphi| limit (0.999) */
  float seed_cov[5];      /* seed covariance diagonal (1, 1, 0.01, 0.01, 1) */
  float restart_scale;    /* inward restart covariance: diag(min(scale*C_out, seed_cov)) (100) */
  int32_t min_clusters;   /* tracks with fewer clusters are not fitted (10) */
  int32_t n_rows;         /* pad rows (152, at most 256) */
  float row_x0_cm;        /* x of pad row 0 (85 cm) */
  float row_pitch_cm;     /* row spacing (162/151 cm); row r lies at float(x0 + r*pitch) */
  uint64_t hbm_budget_bytes; /* serving: device bytes that resident frames may use (120 GB) */
  int32_t max_slots;      /* serving: frames resident at once (8) */
  int32_t device;         /* CUDA device ordinal (0) */
  int32_t block_threads;  /* fit kernel block size: 128 or 256 (0 = 128) */
  int32_t blocks_per_sm;  /* fit kernel resident blocks per SM; 0 = tuned default (640 threads per SM for the
                             plain fit in blocks of 128, else 512; the variant and the serving engine run
                             at most 4 blocks of 128 per SM) */
  int32_t sort_tracks;    /* 1: fit tracks longest-first (default); 0: in frame order */
  float res_step_y_cm;    /* residual code step in y (0.01 cm), see tpcfit_result.res_y */
  float res_step_z_cm;    /* residual code step in z (0.01 cm) */
  /* Mean ionisation energy loss (Bethe formula without density effect, |charge| 1,
   * particle of mass mass_gev) in a thin layer at every crossed pad row, of
   * x*rho = xrho_per_row g/cm^2 along the row normal.  The layer of row r is
   * crossed right after the row-r cluster in outward motion: the outward pass
   * subtracts its loss after the update at row r, the inward pass adds it back
   * before the update.  q/pT scales by p/p' and row/column 4 of the covariance
   * with it; no straggling.  A row that would change p^2 by more than 50 %
   * ends the fit with TPCFIT_TRACK_STOPPED. */
  float xrho_per_row;     /* g/cm^2 per crossed row (0 = no energy loss, the default) */
  float eloss_z_over_a;   /* Z/A of the layer material (0 = neon, 0.49555) */
  float eloss_i_ev;       /* mean excitation energy of the material in eV (0 = neon, 137) */
  /* Seed iteration: after the inward pass, the fitted state at the innermost
   * cluster seeds another outward pass (with seed_cov), restart and inward
   * pass, fit_iterations times (0-16; 0 = none, the default).  Outputs, accept
   * flags and ndf are the last pass's; a failing pass ends the fit with its
   * status.  Each iteration costs about one more fit. */
  int32_t fit_iterations;
  /* Inward re-seed: when the outward pass accepted fewer than reseed_pct %
   * of a track's clusters, the inward pass starts from a fresh three-point
   * seed at the outermost cluster (circle through the last, middle and first
   * cluster, reversed) with seed_cov, instead of from the outward state with
   * the inflated restart covariance.  0-100; the default is 50. */
  int32_t reseed_pct;
  int64_t host_chunk_clusters; /* host frames: chunk scale C (16M clusters); chunks shrink from up to 4C at the
                                 start of the frame to C/4 at its end (two device staging buffers of the
                                 largest chunk); serving splits frames into parts of about C */
} tpcfit_config;

/* One time frame in SoA layout: the clusters of track t are
 * [track_offsets[t], track_offsets[t+1]), rows strictly ascending.  Device
 * arrays must come from a CUDA allocator (cudaMalloc, a memory pool, a
 * framework's caching allocator): the fit reads each track's row bytes as the
 * aligned 32-bit words that hold them, which lie inside such allocations. */
typedef struct tpcfit_frame {
  int64_t n_tracks, n_clusters;
  const int64_t *track_offsets; /* n_tracks+1 */
  /* n_clusters each.  In a host frame (tpcfit_fit, tpcfit_submit) x may be
   * NULL: the clusters then lie on their pad-row planes, x = the row table's
   * float(row_x0 + row * row_pitch), derived on the device from `row` (4 B per
   * cluster less to copy); device frames must carry x. */
  const float *x, *y, *z, *sy2, *sz2;
  const uint8_t *row;             /* n_clusters */
  const uint8_t *sector;          /* n_tracks, may be NULL (informational only) */
  int32_t mem;                    /* TPCFIT_MEM_HOST or TPCFIT_MEM_DEVICE */
} tpcfit_frame;

typedef struct tpcfit_result {
  float *state;   /* n_tracks*5 */
  float *cov;     /* n_tracks*15 */
  float *x_ref;   /* n_tracks */
  double *chi2;   /* n_tracks */
  int32_t *ndf;   /* n_tracks */
  int32_t *status;/* n_tracks */
  uint8_t *accept;/* n_clusters */
  int32_t mem;    /* TPCFIT_MEM_HOST or TPCFIT_MEM_DEVICE */
  /* optional per-cluster chi2 of the outward and inward pass (NaN where the
   * pass did not reach the cluster); NULL = not written.  Device results of
   * tpcfit_fit / tpcfit_fit_async only (a host frame with these set is
   * TPCFIT_E_INVAL; serving ignores them). */
  double *chi2_out_cluster; /* n_clusters */
  double *chi2_in_cluster;  /* n_clusters */
  /* optional: state (y, z, sinphi, tanlambda, q/pT) the inward pass restarted
   * from, at the outermost cluster; NULL = not written (same rules as above) */
  float *restart_state;     /* n_tracks*5 */
  /* optional track-model compression residuals (Sec. 5: the TPC data are
   * stored as cluster-to-track residuals instead of absolute coordinates):
   * for the clusters of a track with status OK, round-half-even((y_c - y_t) /
   * res_step_y_cm) and likewise in z, where (y_t, z_t) is the fitted helix
   * (state at x_ref, no scattering) evaluated at the cluster's x; clipped to
   * +-32767.  -32768 marks a cluster that is not encoded (track not OK, or a
   * helix that does not reach the cluster).  A decoder holding the fitted
   * state, x_ref and the clusters' x restores y, z to within half a step.
   * NULL = not written.  Written by tpcfit_fit (device and host frames),
   * tpcfit_fit_async, batches and serving; not by tpcfit_fit_noalloc. */
  int16_t *res_y;           /* n_clusters */
  int16_t *res_z;           /* n_clusters */
  /* optional: the two-filter smoother (a fit variant).  When both are set,
   * the fit runs as a smoother: the outward pass is the forward filter; the
   * backward filter starts as the inward pass does (restart from the outward
   * state, or the reversed seed) but adds each row's scattering before the
   * row's update (the kink follows the measurement in outward motion); at
   * every cluster the two independent estimates of the state arriving there
   * are combined.  smoothed_state[5k..5k+4] = (y, z, sinphi, tanlambda, q/pT)
   * at cluster k's x, smoothed_cov[15k..15k+14] its packed covariance (NaN
   * where the fit did not complete).  The track outputs above are then the
   * smoothed state and covariance at x_ref (cluster 0), with chi2, ndf, the
   * inward accept bit and the status of the backward filter.  Device frames
   * and results of tpcfit_fit, tpcfit_fit_async and batches only (a host
   * frame is TPCFIT_E_INVAL; serving ignores them); not with energy loss or
   * seed iteration (TPCFIT_E_INVAL).  NULL = the plain fit. */
  float *smoothed_state;    /* n_clusters*5 */
  float *smoothed_cov;      /* n_clusters*15 */
} tpcfit_result;

/* Kernel timings of the last completed fit on a handle (CUDA events on the
 * stream the kernels ran on), in milliseconds. */
typedef struct tpcfit_timing {
  float prepare_ms, sort_ms, fit_ms, total_ms; /* last completed timed call */
  int32_t kernel_launches;  /* kernels launched by the last call */
  int32_t fit_grid, fit_block;
  int32_t fit_regs;         /* registers per thread of the fit kernel */
  int64_t n_timed;          /* timed calls accumulated since tpcfit_reset_timing */
  double prepare_ms_sum, sort_ms_sum, fit_ms_sum, total_ms_sum;
} tpcfit_timing;

/* Fill *cfg with the defaults listed above.  Never fails. */
void tpcfit_default_config(tpcfit_config *cfg);

/* Create a handle on cfg->device (cfg NULL = defaults).  Fails with
 * TPCFIT_E_NODEV if the device is missing or not compute capability 10.3,
 * TPCFIT_E_INVAL on out-of-range parameters.  *out is set only on success. */
int tpcfit_create(const tpcfit_config *cfg, tpcfit_handle **out);

/* Fit one frame and block until the results are in *res (Sec. 5/6: the TPC
 * track fit of one time frame).  Host frames are copied to device scratch in
 * chunks overlapped with the fit; device frames are read in place.  Returns
 * TPCFIT_E_INVAL for malformed offsets (results undefined), TPCFIT_E_NOMEM if
 * scratch cannot be allocated. */
int tpcfit_fit(tpcfit_handle *h, const tpcfit_frame *frame, tpcfit_result *res);

/* Enqueue the fit of a DEVICE frame into DEVICE results on a caller stream
 * (a cudaStream_t passed as void*, NULL = the handle's stream) and return
 * without waiting.  The caller keeps the buffers alive until the stream
 * reaches this point.  Offsets are checked on the device: a malformed frame
 * marks its tracks BAD_INPUT and is reported by the next tpcfit_sync. */
int tpcfit_fit_async(tpcfit_handle *h, const tpcfit_frame *frame, tpcfit_result *res, void *stream);

/* Wait (bounded by timeout_s; < 0 = no bound) for the handle's enqueued work
 * and report a malformed-frame error seen since the last sync. */
int tpcfit_sync(tpcfit_handle *h, double timeout_s);

/* Batched events (Sec. 5: a frame holds many collisions; Sec. 4: a fixed
 * pipeline replayed per input): the tracks of many events of uneven
 * multiplicity are concatenated into one DEVICE frame, each event a
 * contiguous range of tracks, and fitted by one launch sequence (offset
 * check and seed, sort, persistent fit kernel) captured once into a CUDA
 * graph; every tpcfit_batch_launch replays it with no host work per event.
 * Results land in the DEVICE result buffers given at creation, track by
 * track, so an event's results are the same index range.  The frame's and
 * the results' buffers and the handle must outlive the batch; their contents
 * may change between replays, their sizes may not.  The batch owns its
 * scratch (not the handle's), so it may replay while the handle fits other
 * frames on other streams.  Replays of one batch run one after another
 * (CUDA orders launches of one graph), whatever streams they are given. */
typedef struct tpcfit_batch tpcfit_batch;

/* Capture the launch sequence of `frame` -> `res` into a graph.  Both must be
 * device memory; the frame's offsets are checked on the device at every
 * replay (a malformed frame is reported by tpcfit_batch_sync). */
int tpcfit_batch_create(tpcfit_handle *h, const tpcfit_frame *frame, tpcfit_result *res, tpcfit_batch **out);

/* Replay the captured graph on `stream` (a cudaStream_t as void*, NULL = the
 * batch's own stream); returns without waiting. */
int tpcfit_batch_launch(tpcfit_batch *b, void *stream);

/* Wait for the batch's replays (bounded by timeout_s; < 0 = no bound) and
 * report a malformed frame seen by the last replay. */
int tpcfit_batch_sync(tpcfit_batch *b, double timeout_s);

/* Release the graph and the batch's scratch (waits for replays first). */
int tpcfit_batch_destroy(tpcfit_batch *b);

/* Serving (Sec. 4 horizontal parallelism, Sec. 7 rate limiting by frames in
 * flight): copy a host frame into a library-owned resident slot when the HBM
 * budget and a slot allow, fit it together with the frames already on the
 * device (one engine launch over all of them, see tpcfit_get_serve_stats), and
 * copy the results into *res (host memory).  Returns at once with
 * a ticket; a frame larger than the whole budget fails with TPCFIT_E_NOMEM.
 * *frame's and *res's buffers must stay valid until the ticket is DONE or
 * FAILED. */
int tpcfit_submit(tpcfit_handle *h, const tpcfit_frame *frame, tpcfit_result *res, uint64_t *ticket);

/* State of a ticket: TPCFIT_PENDING, TPCFIT_DONE or TPCFIT_FAILED, and when
 * done the completion time in seconds on the library's monotonic clock
 * (tpcfit_now).  A finished ticket is forgotten after it is reported. */
int tpcfit_poll(tpcfit_handle *h, uint64_t ticket, int *state, double *t_done_s);

/* Counters of the serving engine since serving started on the handle (all
 * zero before the first tpcfit_submit).  The engine fits every part of the
 * resident frames that is ready (copied in, checked, seeded and sorted) in
 * one persistent launch, whose warps take (part, 32-track group) descriptors
 * from a device table; a part's results are copied back as soon as its last
 * group is fitted.  launches: engine launches; parts: parts they fitted;
 * max_parts_per_launch: the most parts one launch fitted. */
typedef struct tpcfit_serve_stats {
  int64_t launches, parts, max_parts_per_launch;
} tpcfit_serve_stats;

/* Fill *out (TPCFIT_E_INVAL if h or out is NULL). */
int tpcfit_get_serve_stats(tpcfit_handle *h, tpcfit_serve_stats *out);

/* Block until a ticket finishes (bounded by timeout_s; < 0 = no bound). */
int tpcfit_wait(tpcfit_handle *h, uint64_t ticket, double timeout_s, int *state, double *t_done_s);

/* Library monotonic clock, seconds. */
double tpcfit_now(void);

/* Timings of the last completed device-frame fit (tpcfit_fit, or
 * tpcfit_fit_async after the work completed) and sums over every timed call
 * since tpcfit_reset_timing.  Waits for the handle's timed work to finish.
 * TPCFIT_E_INVAL if nothing was timed yet. */
int tpcfit_last_timing(tpcfit_handle *h, tpcfit_timing *out);

/* Clear the accumulated timing sums. */
int tpcfit_reset_timing(tpcfit_handle *h);

/* Wait for all work, release every device resource and the handle. */
int tpcfit_destroy(tpcfit_handle *h);

/* Static description of an error code; never NULL. */
const char *tpcfit_strerror(int code);

/* Detail of the last error on the calling thread; never NULL. */
const char *tpcfit_last_error_message(void);

#ifdef __cplusplus
}
#endif
#endif /* TPCFIT_H */
