/* Track following on the GPU: the tracking step in front of the fit.
 *
 * The paper runs the full TPC tracking on the GPU (Sec. 5: TPC tracking is
 * the dominant step; Sec. 6: it runs per time frame on each GPU) and
 * describes no algorithm.  Reading implemented here: every seed (a state at
 * the plane of one pad row, in one sector, with a diagonal covariance) is
 * carried outward row by row with the fit's propagation, scattering and gated
 * FP64 update; at each row the clusters of its sector and row with
 * |y_c - y| <= k sqrt(C_yy + v) and |z_c - z| <= k sqrt(C_zz + v) are the
 * candidates (k = window_sigma, v = nominal_v), and the one with the smallest
 * chi2 (its own variances; ties: lowest cluster index) is attached if it
 * passes the gate.  Following ends at the last row, at the sector edge
 * (|y| > x tan_edge) or |z| > z_max (END), after max_miss consecutive rows
 * without a cluster (MISSES), or on a numerical failure (the fit's statuses).
 *
 * The clusters are bucketed into cells (sector, row, z bin, y bin) by a
 * counting sort in the handle's scratch; then one thread per seed follows.
 * All buffers are DEVICE memory; `stream` is a cudaStream_t as void* (NULL =
 * the handle's stream).
 */
#ifndef TPCFIT_FOLLOW_H
#define TPCFIT_FOLLOW_H

#include <stdint.h>

#include "tpcfit.h"

#ifdef __cplusplus
extern "C" {
#endif

/* following statuses (besides the fit's TPCFIT_TRACK_SNP_LIMIT, _NOT_PD, _BAD_INPUT) */
#define TPCFIT_FOLLOW_END 0    /* last row, sector edge or |z| limit reached */
#define TPCFIT_FOLLOW_MISSES 1 /* max_miss consecutive rows without a cluster */

typedef struct tpcfit_follow_config {
  float window_sigma; /* half-width of the search window in sigma (4) */
  float nominal_v;    /* cluster variance used for the window (0.01 cm^2) */
  int32_t max_miss;   /* rows without a cluster that end a track (4) */
  float tan_edge;     /* sector edge: |y| <= x tan_edge (tan 10 deg) */
  float z_max;        /* |z| limit (250 cm) */
  float seed_cov[5];  /* diagonal seed covariance (0.01, 0.01, 1e-4, 1e-4, 0.01) */
  int32_t n_sectors;  /* sectors 0 .. n_sectors-1 (36: 18 per z side); clusters of other sectors are ignored */
  int32_t n_ybins;    /* y bins per (sector, row) cell row (32) */
  int32_t n_zbins;    /* z bins over [-z_max, z_max] (50) */
  int32_t reserved[4];
} tpcfit_follow_config;

typedef struct tpcfit_hits {
  int64_t n_clusters;
  const float *x, *y, *z, *sy2, *sz2; /* n_clusters; x is used by tpcfit_gather_tracks only */
  const uint8_t *row;                 /* n_clusters */
  const uint8_t *sector;              /* n_clusters */
} tpcfit_hits;

typedef struct tpcfit_seeds {
  int64_t n_seeds;
  const float *state;   /* n_seeds*5: y, z, sinphi, tanlambda, q/pT at the plane of `row` */
  const uint8_t *row;   /* n_seeds */
  const uint8_t *sector;/* n_seeds */
} tpcfit_seeds;

typedef struct tpcfit_tracks {
  int32_t *att;      /* n_seeds * n_rows: cluster attached at each row, -1 = none */
  int32_t *n_att;    /* n_seeds */
  int32_t *status;   /* n_seeds */
  float *state;      /* n_seeds*5: state where following ended; may be NULL */
} tpcfit_tracks;

void tpcfit_follow_default_config(tpcfit_follow_config *c);

/* Follow every seed through the clusters (asynchronous on `stream`; the
 * fit parameters -- field, gate, scattering, rows -- are the handle's). */
int tpcfit_follow(tpcfit_handle *h, const tpcfit_follow_config *fc, const tpcfit_hits *hits,
                  const tpcfit_seeds *seeds, tpcfit_tracks *tracks, void *stream);

/* Gather the attached clusters of each followed track, in row order, into a
 * frame that tpcfit_fit takes: offsets (n_seeds+1) and the cluster arrays
 * (capacity `cap` clusters).  Blocks; *n_out = clusters gathered;
 * TPCFIT_E_INVAL if they exceed cap. */
int tpcfit_gather_tracks(tpcfit_handle *h, const tpcfit_hits *hits, const tpcfit_tracks *tracks, int64_t n_seeds,
                         int64_t *offsets, float *x, float *y, float *z, float *sy2, float *sz2, uint8_t *row,
                         int64_t cap, int64_t *n_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TPCFIT_FOLLOW_H */
