// Kernels that run after or beside the fit: track-model compression residual
// codes (k_residuals) and track following (k_follow), on the fit's device
// code (fit_device.cuh).

#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>

#include "fit_device.cuh"
#include "tpcfit_internal.h"

namespace tpcfit {

// ---------------------------------------------------------------------------
// k_residuals: track-model compression residual codes, after k_fit.  One warp
// per track (grid-stride); the lanes take the track's clusters 32 at a time,
// so the loads of x, y, z and the stores of the codes are coalesced.  Input:
// the fitted state and x_ref that k_fit wrote.
// ---------------------------------------------------------------------------
constexpr int kResChunks = 5;  // 160 clusters: a whole track of 152 pad rows in one sweep

__global__ void __launch_bounds__(256) k_residuals(FitArgs A) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < A.n_tracks; t += warps) {
    const int64_t a = A.off[t] - A.off_base, e = A.off[t + 1] - A.off_base;
    if (a < 0 || e < a || e > A.n_clusters) continue;  // malformed offsets: k_prepare reported the frame
    const bool ok = A.status[t] == ST_OK;
    float y0 = 0.f, z0 = 0.f, s0 = 0.f, tl = 0.f, w = 0.f, x0 = 0.f;
    if (ok) {
      const float *p = A.state + 5 * t;
      y0 = p[0]; z0 = p[1]; s0 = p[2]; tl = p[3]; w = p[4];
      x0 = A.x_ref[t];
    }
    const float C = A.b * w;
    // up to 32 * kResChunks clusters per sweep: every load of the sweep is
    // issued before the first residual is formed (one memory latency per track)
    for (int64_t base = a; base < e; base += 32 * kResChunks) {
      float xs[kResChunks], ys[kResChunks], zs[kResChunks];
#pragma unroll
      for (int q = 0; q < kResChunks; ++q) {
        const int64_t k = base + q * 32 + lane;
        xs[q] = ys[q] = zs[q] = 0.f;
        if (k < e) {
          xs[q] = A.x[k];
          ys[q] = A.y[k];
          zs[q] = A.z[k];
        }
      }
#pragma unroll
      for (int q = 0; q < kResChunks; ++q) {
        const int64_t k = base + q * 32 + lane;
        if (k >= e) break;
        int16_t cy = -32768, cz = -32768;
        float yt, zt;
        if (ok && helix_at(y0, z0, s0, tl, C, xs[q] - x0, yt, zt)) {
          cy = res_code(ys[q] - yt, A.res_inv_step_y);
          cz = res_code(zs[q] - zt, A.res_inv_step_z);
        }
        if (A.res_y) A.res_y[k] = cy;
        if (A.res_z) A.res_z[k] = cz;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// k_follow: track following, one thread per seed.  The seed is carried row by
// row with the fit's propagation, update and scattering; at each row the
// clusters of the seed's sector and row inside the +-k sigma window are read
// from the cells the window overlaps, and the one with the smallest chi2
// (FP32; ties: lowest cluster index) goes through the fit's gated update.
// ---------------------------------------------------------------------------
enum { FL_END = 0, FL_MISSES = 1 };
constexpr int kFollowBatch = 4;  // cluster records loaded together in the candidate search

__global__ void __launch_bounds__(256) k_follow(FollowArgs A) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= A.n_seeds) return;
  const float *sd = A.seed_state + 5 * s;
  Trk T;
  T.ya = sd[0];
  T.za = sd[1];
  T.dy = T.dz = 0.f;
  T.sp = sd[2];
  T.spl = 0.f;
  T.tl0 = sd[3];
  T.dtl = 0.f;
  T.w0 = sd[4];
  T.dw = 0.f;
#pragma unroll
  for (int i = 0; i < 15; ++i) T.c[i] = 0.f;
  T.c[0] = A.seed_cov[0];
  T.c[2] = A.seed_cov[1];
  T.c[5] = A.seed_cov[2];
  T.c[9] = A.seed_cov[3];
  T.c[14] = A.seed_cov[4];
  T.clear_comp();
  const Gate gate = make_gate(A.chi2_max, A.chi2_max_d);
  const int r0 = A.seed_row[s], sec = A.seed_sector[s];
  int status = FL_END, misses = 0, n = 0;
  int32_t *att = A.att + s * A.n_rows;
  float xcur = A.row_x[r0 < A.n_rows ? r0 : 0];
  if (sec >= A.n_sectors || r0 >= A.n_rows) status = ST_BAD_INPUT;
  for (int r = r0; status == FL_END && r < A.n_rows; ++r) {
    const float xr = A.row_x[r];
    if (r > r0) {
      if (!propagate(T, xr - xcur, A.b, A.snp_max)) { status = ST_SNP_LIMIT; break; }
      xcur = xr;
    }
    const float yp = T.ya + T.dy, zp = T.za + T.dz;
    if (fabsf(yp) > xr * A.tan_edge || fabsf(zp) > A.z_max) break;  // END
    const float wy = A.window_sigma * sqrtf(T.c[0] + A.nominal_v);
    const float wz = A.window_sigma * sqrtf(T.c[2] + A.nominal_v);
    const int iy0 = follow_ybin(yp - wy, xr, A.tan_edge, A.ny), iy1 = follow_ybin(yp + wy, xr, A.tan_edge, A.ny);
    const int iz0 = follow_zbin(zp - wz, A.z_max, A.nz), iz1 = follow_zbin(zp + wz, A.z_max, A.nz);
    const int64_t base = ((int64_t)sec * A.n_rows + r) * A.nz;
    // best candidate: its position bq in cell order; its cluster index bk is
    // read only to break an exact tie (ties: lowest index), else once after
    // the search, while the update runs
    int64_t bq = -1;
    int32_t bk = -1;
    float bchi = INFINITY;
    float4 bc = make_float4(0.f, 0.f, 0.f, 0.f);
    const float S01 = T.c[1];
    for (int iz = iz0; iz <= iz1; ++iz) {
      const int64_t row0 = (base + iz) * A.ny;
      const uint32_t q0 = A.cell_start[row0 + iy0], q1 = A.cell_start[row0 + iy1 + 1];
      // records in batches of kFollowBatch, all loads of a batch in flight
      // together (a window holds a few clusters: about one memory latency per
      // z bin instead of one per candidate); tested in cell order
      for (uint32_t qb = q0; qb < q1; qb += kFollowBatch) {
        float4 cb[kFollowBatch];
#pragma unroll
        for (int u = 0; u < kFollowBatch; ++u)
          cb[u] = (qb + u < q1) ? A.crec[qb + u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < kFollowBatch; ++u) {
          const uint32_t q = qb + u;
          if (q >= q1) break;
          const float4 c = cb[u];
          const float r0v = (c.x - T.ya) - T.dy, r1v = (c.y - T.za) - T.dz;
          if (fabsf(r0v) > wy || fabsf(r1v) > wz) continue;
          const float S00 = T.c[0] + c.z, S11 = T.c[2] + c.w;
          const float det = fmaf(S00, S11, -S01 * S01);
          // ranking only (the gated update recomputes chi2 with its FP64 island)
          const float chi = __fdividef(r0v * fmaf(S11, r0v, -S01 * r1v) + r1v * fmaf(S00, r1v, -S01 * r0v), det);
          if (chi < bchi) {
            bchi = chi;
            bq = q;
            bk = -1;
            bc = c;
          } else if (chi == bchi && bq >= 0) {
            if (bk < 0) bk = A.cidx[bq];
            const int32_t k = A.cidx[q];
            if (k < bk) {
              bq = q;
              bk = k;
              bc = c;
            }
          }
        }
      }
    }
    const int32_t best = bq < 0 ? -1 : (bk >= 0 ? bk : A.cidx[bq]);
    bool acc = false;
    if (best >= 0) {
      double chi2;
      const int ust = update(T, bc.x, bc.y, bc.z, bc.w, gate, false, acc, chi2);
      if (ust != ST_OK) { status = ust; break; }
    }
    if (acc) {
      att[r] = best;
      ++n;
      misses = 0;
    } else if (++misses > A.max_miss) {
      status = FL_MISSES;
      break;
    }
    if (A.xx0 > 0.f) ms_noise(T, A.xx0, A.mass2);
  }
  A.n_att[s] = n;
  A.status[s] = status;
  if (A.state_out) {
    float *po = A.state_out + 5 * s;
    po[0] = T.ya + T.dy;
    po[1] = T.za + T.dz;
    po[2] = T.snp();
    po[3] = T.tl();
    po[4] = T.w();
  }
}

cudaError_t launch_follow(const FollowArgs &a, cudaStream_t stream) {
  if (a.n_seeds <= 0) return cudaSuccess;
  k_follow<<<(unsigned)((a.n_seeds + 255) / 256), 256, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_residuals(const FitArgs &a, cudaStream_t stream) {
  if (a.n_tracks <= 0 || (!a.res_y && !a.res_z)) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (a.n_tracks + 7) / 8;  // 8 warps (tracks) per block in flight
  const int64_t cap = (int64_t)sms * 8;
  k_residuals<<<(unsigned)(want < cap ? want : cap), 256, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace tpcfit
