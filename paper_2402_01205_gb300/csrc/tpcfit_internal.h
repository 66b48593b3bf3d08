// Internal interface between the C-ABI runtime and the CUDA kernels.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "tpcfit.h"

namespace tpcfit {

constexpr int kMaxRows = 256;        // row index is uint8
constexpr int kKeyBins = kMaxRows + 1; // sort key: cluster count clamped to [0, 256]

// Everything one fit launch sequence needs; passed by value to the kernels.
struct FitArgs {
  // frame (device pointers); cluster arrays start at the frame's first cluster
  int64_t n_tracks, n_clusters;
  const int64_t *off;      // n_tracks+1 offsets
  int64_t off_base;        // value subtracted from every offset (chunked host frames)
  const float *x, *y, *z, *sy2, *sz2;
  const uint8_t *row;
  // results (device pointers, same indexing as the frame)
  float *state, *cov, *x_ref;
  double *chi2;
  int32_t *ndf, *status;
  uint8_t *accept;
  double *chi2_out_c, *chi2_in_c;  // optional per-cluster chi2 (nullptr: not written)
  float *restart_state;            // optional inward restart state (nullptr: not written)
  float *sm_state, *sm_cov;        // smoother variant: per-cluster smoothed state / packed covariance (nullptr: fit)
  float *sm_pred;                  // smoother variant: the forward predictions, smooth_pred_bytes() of scratch
  int16_t *res_y, *res_z;          // optional residual codes (nullptr: not written)
  float res_inv_step_y, res_inv_step_z;
  // scratch (device)
  float *seed;                   // n_tracks*5
  int32_t *perm;                 // n_tracks (sorted order), or nullptr for frame order
  uint32_t *hist;                // kKeyBins histogram, then bin cursors
  unsigned long long *work;      // persistent-kernel work counter
  int32_t *frame_error;          // bit0: malformed offsets
  const float *row_x;            // kMaxRows pad-row plane positions
  // fit parameters
  float b;                       // -kB * Bz: d(curvature)/d(q/pT)
  float chi2_max;
  double chi2_max_d;
  float xx0, mass2, snp_max, restart_scale;
  float xrho;                    // energy-loss layer per row (g/cm^2); 0 = none
  float el_kza, el_a, el_ratio;  // K Z/A (GeV cm^2/g), 2 m_e / I, m_e / M
  int32_t n_iter;                // seed iterations: refits seeded from the fitted state
  int32_t reseed_pct;            // inward re-seed below this outward acceptance (percent)
  float seed_cov[5];
  int32_t min_clusters, n_rows;
  int32_t stage_vec;             // set by launch_fit: cluster arrays share their 16-byte phase
};

// Host-to-device copies of the clusters [c0, c1) of a host frame into staging
// arrays that hold c1 - c0 + 2 * kCopyPad elements each.  Each array's copy is
// widened so that it starts and ends on a 256-byte boundary of its host
// address, where the array allows it (never before its element 0 or past
// n_clusters): copies off those boundaries run well below the link rate (on
// GB300: a 4 GB frame in 12 chunks took 20.8 ms unaligned against 19.4 ms
// aligned; one copy: 19.2 ms).  `view` receives the staging arrays advanced to
// cluster c0 (n_clusters = c1 - c0); each 4-byte array's copy lands up to 3
// elements further into its staging array, so that cluster c0 of every one of
// them sits at the start of a 16-byte line (the fit then stages whole chunks
// as 16-byte copies).  Returns the first failing CUDA error.
// Elements: a 256-byte boundary lies within 256 elements of any address, and
// 3 more align the 4-byte arrays.
constexpr int64_t kCopyPad = 260;

struct ClusterArrays {
  float *x, *y, *z, *sy2, *sz2;
  uint8_t *row;
};

cudaError_t launch_x_from_rows(const uint8_t *row, int64_t n, const float *row_x, float *x, cudaStream_t st);

// A NULL x in the host frame: the clusters lie on their pad-row planes, and
// the staged x is filled on the device from the staged rows and the row table
// `row_x` (device memory), over the row array's staged range: on `st` right
// after the copies, or, when `fill` is given, by the caller (who launches
// launch_x_from_rows(fill->row, fill->n, row_x, fill->x, ...) on a stream that
// waits for the copies, so that the copy stream stays busy with copies).
struct XFill {
  const uint8_t *row = nullptr;
  int64_t n = 0;
  float *x = nullptr;
};

inline cudaError_t copy_clusters_in(const tpcfit_frame &f, int64_t c0, int64_t c1, const ClusterArrays &stage,
                                    const float *row_x, tpcfit_frame &view, cudaStream_t st,
                                    XFill *fill = nullptr) {
  cudaError_t err = cudaSuccess;
  int64_t row_a0 = c0, row_n = 0;
  // elements to skip at the start of a 4-byte staging array so that cluster c0 lands on a 16-byte line
  auto shift4 = [&](int64_t first) -> int64_t { return (4 - ((c0 - first) & 3)) & 3; };
  auto one = [&](const void *src, void *dst, size_t elem) -> const void * {
    const uintptr_t base = reinterpret_cast<uintptr_t>(src);
    int64_t a0 = c0 - (int64_t)(((base + (uintptr_t)c0 * elem) & 255u) / elem);
    if (a0 < 0) a0 = 0;
    int64_t a1 = c1 + (int64_t)(((256u - ((base + (uintptr_t)c1 * elem) & 255u)) & 255u) / elem);
    if (a1 > f.n_clusters) a1 = f.n_clusters;
    char *d = static_cast<char *>(dst) + (elem == 4 ? shift4(a0) * 4 : 0);
    if (c1 > c0 && err == cudaSuccess)
      err = cudaMemcpyAsync(d, static_cast<const char *>(src) + a0 * (int64_t)elem, (size_t)(a1 - a0) * elem,
                            cudaMemcpyHostToDevice, st);
    if (elem == 1) {
      row_a0 = a0;
      row_n = a1 - a0;
    }
    return d + (c0 - a0) * (int64_t)elem;
  };
  view.row = static_cast<const uint8_t *>(one(f.row, stage.row, 1));
  if (f.x) {
    view.x = static_cast<const float *>(one(f.x, stage.x, 4));
  } else {
    const int64_t n_fill = c1 > c0 ? row_n : 0;
    float *xd = stage.x + shift4(row_a0);  // x[k] beside row[k] of the staged rows
    if (fill) {
      fill->row = stage.row;
      fill->n = n_fill;
      fill->x = xd;
    } else if (n_fill > 0 && err == cudaSuccess) {
      err = launch_x_from_rows(stage.row, n_fill, row_x, xd, st);
    }
    view.x = xd + (c0 - row_a0);
  }
  view.y = static_cast<const float *>(one(f.y, stage.y, 4));
  view.z = static_cast<const float *>(one(f.z, stage.z, 4));
  view.sy2 = static_cast<const float *>(one(f.sy2, stage.sy2, 4));
  view.sz2 = static_cast<const float *>(one(f.sz2, stage.sz2, 4));
  view.n_clusters = c1 - c0;
  return err;
}

// Chunk schedule of a host frame (tpcfit_api.cu): cut points in track indices;
// -1, or the track at which the offsets decrease or leave [0, nc_all].
int64_t chunk_cuts(const int64_t *off, int64_t nt, int64_t nc_all, int64_t C, std::vector<int64_t> &cuts);

// The fit parameters of FitArgs from a configuration (both entry points).
inline void fit_params(FitArgs &a, const tpcfit_config &c) {
  a.b = (float)(-0.299792458e-2 * (double)c.bz_tesla);
  a.chi2_max = c.chi2_max;
  a.chi2_max_d = (double)c.chi2_max;
  a.xx0 = c.xx0_per_row;
  a.mass2 = c.mass_gev * c.mass_gev;
  a.snp_max = c.snp_max;
  a.restart_scale = c.restart_scale;
  const double za = c.eloss_z_over_a > 0.0f ? c.eloss_z_over_a : 0.49555;  // neon: 10 / 20.1797
  const double iev = c.eloss_i_ev > 0.0f ? c.eloss_i_ev : 137.0;            // neon
  const double me = 0.51099895e-3;                                           // electron mass, GeV
  a.xrho = c.xrho_per_row;
  a.el_kza = (float)(0.307075e-3 * za);  // K = 0.307075 MeV cm^2 / mol
  a.el_a = (float)(2.0 * me / (iev * 1e-9));
  a.el_ratio = c.mass_gev > 0.0f ? (float)(me / (double)c.mass_gev) : 0.0f;
  a.n_iter = c.fit_iterations;
  a.reseed_pct = c.reseed_pct;
  for (int i = 0; i < 5; ++i) a.seed_cov[i] = c.seed_cov[i];
  a.min_clusters = c.min_clusters;
  a.n_rows = c.n_rows;
}

// NULL, or why the variant parameters (energy loss, seed iteration) of a configuration are invalid.
inline const char *check_variant_params(const tpcfit_config &c) {
  if (!(c.xrho_per_row >= 0.0f) || !(c.eloss_z_over_a >= 0.0f) || !(c.eloss_i_ev >= 0.0f))
    return "energy-loss parameters must be >= 0";
  if (c.xrho_per_row > 0.0f && !(c.mass_gev > 0.0f)) return "energy loss needs mass_gev > 0";
  if (c.fit_iterations < 0 || c.fit_iterations > 16) return "fit_iterations must be in [0, 16]";
  if (c.reseed_pct < 0 || c.reseed_pct > 100) return "reseed_pct must be in [0, 100]";
  return nullptr;
}

// Track following (tpcfit_follow.cu builds the cell grid; the kernel lives
// with the fit's device code).  Cell of a cluster: ((sector * n_rows + row) *
// nz + iz) * ny + iy, iz from z over [-z_max, z_max], iy from y over
// [-ymax_r, ymax_r] with ymax_r = row_x[row] * tan_edge * 1.02.
struct FollowArgs {
  int32_t n_sectors, n_rows, ny, nz;
  float z_max, tan_edge;
  const uint32_t *cell_start;             // n_cells + 1
  const float4 *crec;                     // clusters in cell order: (y, z, sy2, sz2)
  const int32_t *cidx;                    // their indices in the caller's arrays
  int64_t n_seeds;
  const float *seed_state;                // n_seeds * 5
  const uint8_t *seed_row, *seed_sector;
  float seed_cov[5];
  int32_t *att, *n_att, *status;          // att: n_seeds * n_rows (pre-set to -1)
  float *state_out;                       // n_seeds * 5, may be null
  const float *row_x;
  float b, chi2_max;
  double chi2_max_d;
  float xx0, mass2, snp_max;
  float window_sigma, nominal_v;
  int32_t max_miss;
};

__host__ __device__ inline int follow_ybin(float y, float xr, float tan_edge, int ny) {
  const float ym = xr * tan_edge * 1.02f;
  int i = (int)floorf((y + ym) * ((float)ny / (2.0f * ym)));
  return i < 0 ? 0 : (i >= ny ? ny - 1 : i);
}
__host__ __device__ inline int follow_zbin(float z, float z_max, int nz) {
  int i = (int)floorf((z + z_max) * ((float)nz / (2.0f * z_max)));
  return i < 0 ? 0 : (i >= nz ? nz - 1 : i);
}

cudaError_t launch_follow(const FollowArgs &a, cudaStream_t stream);

// Record `msg` as the calling thread's tpcfit_last_error_message; returns code.
int set_error_message(int code, const char *msg);

// Launch helpers (all asynchronous on `stream`); each returns the CUDA error
// of its launch.
cudaError_t launch_prepare(const FitArgs &a, cudaStream_t stream);
cudaError_t launch_sort(const FitArgs &a, cudaStream_t stream, int *launches);
// The fit kernel on `grid` persistent blocks of `block` threads (128 or 256).
cudaError_t launch_fit(const FitArgs &a, int grid, int block, cudaStream_t stream);
// Set the shared-memory attribute of the instantiation launch_fit takes for
// these arguments (before a stream capture: no such call inside it).
cudaError_t fit_set_attributes(const FitArgs &a, int block);

// One fit launch over the prepared parts of several resident frames (the
// serving engine, tpcfit_serve.cu): `parts` is a device table of their
// arguments (as from fit_args_for_launch, after k_prepare and the sort ran for
// each), `prefix` their track-group offsets (32 tracks per group; part p owns
// groups [prefix[p], prefix[p+1])), `cursor` a zeroed group counter,
// `remaining` each part's group count, and `done_flag` one host-mapped word
// per part that the launch sets to 1 once that part's results are complete and
// visible to the host and to copies.
struct PartsArgs {
  const FitArgs *parts;
  const unsigned long long *prefix;
  unsigned long long *cursor;
  unsigned *remaining;
  volatile int32_t *done_flag;
  int n_parts;
};
cudaError_t launch_fit_parts(const PartsArgs &p, bool variant, int grid, int block, cudaStream_t stream);
// the arguments with the launch-time fields (cluster staging mode) filled in
FitArgs fit_args_for_launch(const FitArgs &a);
// the two-filter smoother variant in place of the fit (a.sm_state, a.sm_cov set),
// on a persistent grid of smooth_grid() blocks (0 if the device cannot be queried)
int smooth_grid();
// device scratch the smoother needs on that grid for frames of n_rows pad rows
size_t smooth_pred_bytes(int grid, int n_rows);
cudaError_t launch_smooth(const FitArgs &a, int grid, cudaStream_t stream);
// track-model compression residual codes (nothing when a.res_y and a.res_z are null)
cudaError_t launch_residuals(const FitArgs &a, cudaStream_t stream);
// Occupancy-derived resident blocks per SM for the fit kernel at `block` threads.
int fit_blocks_per_sm(int block);
// tuned default residency (blocks per SM) for a block size
int fit_default_blocks_per_sm(int block, bool variant);
// registers per thread of the instantiation a handle launches for frames of
// more tracks than 4 blocks of 128 per SM hold (smaller frames run the
// 4-block instantiation)
int fit_regs_per_thread(int block, bool variant, int blocks_per_sm);

}  // namespace tpcfit
