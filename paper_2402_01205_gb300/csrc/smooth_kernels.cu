// Two-filter smoother of the track fit (a fit variant): the state and
// covariance at every cluster of a track from all of its clusters.
//
// The paper's TPC chain stores clusters as residuals to their track (Sec. 5,
// track-model compression) and names no smoothing method; the smoother here
// is the textbook two-filter form (Fraser and Potter 1969; Fruhwirth 1987 for
// track fitting), in the scattering model of the fit's outward pass: the
// particle moves outward and, at each crossed pad row, is first measured (if
// the row has a cluster) and then scattered.
//
//  1. forward filter = the fit's outward pass.  Before its update at cluster
//     k the predicted state (p-, C-) (clusters 0..k-1 and the seed prior) is
//     stored in the prediction scratch;
//  2. backward filter = the inward pass, started as the fit starts it (the
//     outward state with the inflated diagonal restart covariance, or the
//     reversed three-point seed), except that at each crossed row it adds the
//     row's scattering before the row's update (the kink follows the
//     measurement in outward motion);
//  3. after its update at cluster k it holds (p+, C+) from clusters k..n-1
//     and combines them with the stored prediction of the same state:
//       S = C- + C+,  K = C- S^-1,  p = p- + K (p+ - p-),  C = K C+,
//     and writes the smoothed state into the caller's slots of cluster k.  When
//     the forward filter lost the track (it accepted fewer than reseed_pct %
//     of the clusters, so that the backward filter re-seeds) its predictions
//     carry no valid information: the smoothed state is the backward
//     filter's.
//
// The track outputs are the smoothed state and covariance at cluster 0; chi2,
// ndf, the inward accept bit and the status come from the backward filter as
// in the fit.
//
// Precision: the filters are the fit's (FP32 with the FP64 innovation island).
// The 5x5 combination is FP32: S is scaled to unit diagonal (its correlation
// matrix) before a Cholesky factorisation, and C = K C+ is formed as a
// product, not as the difference C- - K C-, which cancels wherever one filter
// knows far more than the other (near the ends of the track).
//
// One thread per track on the persistent grid of the fit (same sort, same
// work counter); both filters read the clusters through the fit's staging
// ring (stage_device.cuh).  The 20 floats of a prediction are kept in scratch
// owned by the warp as five 16-byte vectors laid out [row step of the
// track][vector][lane]: the tracks of a warp cross as many rows and step
// through them together, so a warp-wide vector access is one contiguous
// 512-byte run (scalar accesses to the caller's per-cluster slots took 20
// requests per lane).  The backward filter loads the next cluster's
// prediction right after the combination at the current one, so the load
// overlaps a whole step; the smoothed outputs are written with the widest
// vector stores their alignment allows.

#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>

#include "fit_device.cuh"
#include "stage_device.cuh"
#include "tpcfit_internal.h"

namespace tpcfit {

namespace {

constexpr int kSmoothBlock = 128;
constexpr int kSmoothDerailPct = 80;  // as the fit: DERAILED below 80 % inward acceptance
constexpr int kSmoothBitWords = kMaxRows / 32;  // forward accept bits of one track (<= 256 clusters)

// absolute state of a track
__device__ __forceinline__ void state_of(const Trk &T, float p[5]) {
  p[0] = T.ya + T.dy;
  p[1] = T.za + T.dz;
  p[2] = T.snp();
  p[3] = T.tl();
  p[4] = T.w();
}

// packed covariance with the compensation terms added in
__device__ __forceinline__ void cov_of(const Trk &T, float c[15]) {
#pragma unroll
  for (int i = 0; i < 15; ++i) c[i] = T.c[i];
  c[3] += T.c3l;
  c[5] += T.c5l;
  c[9] += T.c9l;
  c[12] += T.c12l;
  c[14] += T.c14l;
}

__device__ __forceinline__ int pk(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

// Two-filter combination of the prediction (pm, cm) with the filtered state
// (pp, cp) of the same plane (packed covariances).  Returns false when S is
// not positive definite (the outputs are then unchanged).
__device__ __forceinline__ bool combine(const float pm[5], const float cm[15], const float pp[5], const float cp[15],
                                        float ps[5], float cs[15]) {
  float S[15], d[5];
#pragma unroll
  for (int i = 0; i < 15; ++i) S[i] = cm[i] + cp[i];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float v = S[pk(i, i)];
    if (!(v > 0.0f)) return false;
    d[i] = rsqrtf(v);
  }
  // L L^T = D S D (unit diagonal), lower triangle packed in place; rl[j] =
  // 1 / L_jj (the substitutions multiply by it instead of dividing)
  float L[15], rl[5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) L[pk(i, j)] = S[pk(i, j)] * d[i] * d[j];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    float s = L[pk(j, j)];
#pragma unroll
    for (int m = 0; m < j; ++m) s = fmaf(-L[pk(j, m)], L[pk(j, m)], s);
    if (!(s > 0.0f)) return false;
    const float r = rsqrtf(s);
    L[pk(j, j)] = s * r;  // sqrt(s)
    rl[j] = r;
#pragma unroll
    for (int i = j + 1; i < 5; ++i) {
      float t = L[pk(i, j)];
#pragma unroll
      for (int m = 0; m < j; ++m) t = fmaf(-L[pk(i, m)], L[pk(j, m)], t);
      L[pk(i, j)] = t * r;
    }
  }
  // X = S^-1 C- = D (L L^T)^-1 D C-, column by column; K = C- S^-1 = X^T
  float X[5][5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    float v[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) v[i] = d[i] * cm[pk(i, c)];
#pragma unroll
    for (int i = 0; i < 5; ++i) {  // L y = v
      float t = v[i];
#pragma unroll
      for (int m = 0; m < i; ++m) t = fmaf(-L[pk(i, m)], v[m], t);
      v[i] = t * rl[i];
    }
#pragma unroll
    for (int i = 4; i >= 0; --i) {  // L^T x = y
      float t = v[i];
#pragma unroll
      for (int m = i + 1; m < 5; ++m) t = fmaf(-L[pk(m, i)], v[m], t);
      v[i] = t * rl[i];
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) X[i][c] = d[i] * v[i];
  }
  // p = p- + K (p+ - p-), K[i][m] = X[m][i]
  float dp[5];
#pragma unroll
  for (int m = 0; m < 5; ++m) dp[m] = pp[m] - pm[m];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    float t = pm[i];
#pragma unroll
    for (int m = 0; m < 5; ++m) t = fmaf(X[m][i], dp[m], t);
    ps[i] = t;
  }
  // C = K C+ (symmetric in exact arithmetic: averaged with its transpose)
  float KC[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      float t = 0.0f;
#pragma unroll
      for (int m = 0; m < 5; ++m) t = fmaf(X[m][i], cp[pk(m, j)], t);
      KC[i][j] = t;
    }
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) cs[pk(i, j)] = 0.5f * (KC[i][j] + KC[j][i]);
  return true;
}

__device__ __forceinline__ void store5(float *dst, const float v[5]) {
#pragma unroll
  for (int i = 0; i < 5; ++i) dst[i] = v[i];
}
__device__ __forceinline__ void store15(float *dst, const float v[15]) {
#pragma unroll
  for (int i = 0; i < 15; ++i) dst[i] = v[i];
}

__device__ void seed_cov_of(const FitArgs &A, Trk &T) {
#pragma unroll
  for (int i = 0; i < 15; ++i) T.c[i] = 0.f;
  T.c[0] = A.seed_cov[0];
  T.c[2] = A.seed_cov[1];
  T.c[5] = A.seed_cov[2];
  T.c[9] = A.seed_cov[3];
  T.c[14] = A.seed_cov[4];
  T.clear_comp();
}

constexpr int kPredVec = 5;  // 16-byte vectors of one prediction (20 floats)

// Vector q of the prediction at row step j (row of the track's first
// cluster + j) of the lane's track in the warp's scratch, laid out [row step
// j][vector q][lane] (`pred` = the warp's base + the lane's 16-byte column):
// the lanes' q-th vectors of one row step are one contiguous 512-byte run.
// The tracks of a warp cross as many rows and step through them together, so
// the lanes that have a cluster on the step's row write that run at once and
// read it back at once (rows without a cluster leave their lane's entries
// unused).
__device__ __forceinline__ float4 *pred_vec(float *pred, int j, int q) {
  return reinterpret_cast<float4 *>(pred + (j * kPredVec + q) * (32 * 4));
}

// N floats to a 4-byte aligned address whose first H floats lie before a
// 16-byte boundary: scalar / 8-byte head, 16-byte body, 8-byte / scalar tail.
template <int N, int H> __device__ __forceinline__ void store_from(float *dst, const float *v) {
  int i = 0;
  if (H & 1) {
    dst[0] = v[0];
    i = 1;
  }
  if (H & 2) {
    *reinterpret_cast<float2 *>(dst + i) = make_float2(v[i], v[i + 1]);
    i += 2;
  }
#pragma unroll
  for (int q = 0; q < (N - H) / 4; ++q, i += 4)
    *reinterpret_cast<float4 *>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
  if ((N - H) & 2) {
    *reinterpret_cast<float2 *>(dst + i) = make_float2(v[i], v[i + 1]);
    i += 2;
  }
  if ((N - H) & 1) dst[i] = v[i];
}
// N floats with the widest aligned vector stores (fewer store instructions and
// memory requests per lane than N scalar stores).
template <int N> __device__ __forceinline__ void store_vec(float *dst, const float (&v)[N]) {
  switch ((reinterpret_cast<uintptr_t>(dst) >> 2) & 3u) {  // floats past a 16-byte boundary
    case 0: store_from<N, 0>(dst, v); break;
    case 1: store_from<N, 3>(dst, v); break;
    case 2: store_from<N, 2>(dst, v); break;
    default: store_from<N, 1>(dst, v); break;
  }
}

// The forward prediction (state and packed covariance) at row step j of the
// lane's track.
__device__ __forceinline__ void store_pred(float *pred, int j, const float pm[5], const float cm[15]) {
  *pred_vec(pred, j, 0) = make_float4(pm[0], pm[1], pm[2], pm[3]);
  *pred_vec(pred, j, 1) = make_float4(pm[4], cm[0], cm[1], cm[2]);
  *pred_vec(pred, j, 2) = make_float4(cm[3], cm[4], cm[5], cm[6]);
  *pred_vec(pred, j, 3) = make_float4(cm[7], cm[8], cm[9], cm[10]);
  *pred_vec(pred, j, 4) = make_float4(cm[11], cm[12], cm[13], cm[14]);
}
__device__ __forceinline__ void load_pred(const float *pred, int j, float pm[5], float cm[15]) {
  float *pw = const_cast<float *>(pred);
  const float4 s0 = *pred_vec(pw, j, 0), s1 = *pred_vec(pw, j, 1), s2 = *pred_vec(pw, j, 2), s3 = *pred_vec(pw, j, 3),
               s4 = *pred_vec(pw, j, 4);
  pm[0] = s0.x; pm[1] = s0.y; pm[2] = s0.z; pm[3] = s0.w; pm[4] = s1.x;
  cm[0] = s1.y; cm[1] = s1.z; cm[2] = s1.w;
  cm[3] = s2.x; cm[4] = s2.y; cm[5] = s2.z; cm[6] = s2.w;
  cm[7] = s3.x; cm[8] = s3.y; cm[9] = s3.z; cm[10] = s3.w;
  cm[11] = s4.x; cm[12] = s4.y; cm[13] = s4.z; cm[14] = s4.w;
}

// Smoothing of track t by one lane.  Clusters are staged as in the fit (the
// lane's column of the block's staging ring: `f4`, `wrow`; copies issued and
// waited for at warp-uniform steps every kChunk rows of a pass), the pad-row
// table is `s_rowx`, `bits` the lane's column of forward accept bits (word w
// at bits[w * kSmoothBlock]), so that the backward filter writes each accept
// byte once instead of reading back the forward filter's, and `pred` the
// lane's column of the warp's prediction scratch.  The backward filter loads the next cluster's
// prediction as soon as the combination of the current one has used its
// registers, a whole step ahead of its use.
__device__ void smooth_track(const FitArgs &A, int64_t t, const float *s_rowx, float *f4, uint32_t *wrow,
                             uint32_t *bits, float *pred) {
  const int64_t a = A.off[t] - A.off_base, e = A.off[t + 1] - A.off_base;
  const int st0 = A.status[t];
  const float *sd = A.seed + 5 * t;
  const float qnan = __int_as_float(0x7fc00000);
  Trk T;
  T.sp = sd[2];
  T.spl = 0.f;
  T.tl0 = sd[3];
  T.dtl = 0.f;
  T.w0 = sd[4];
  T.dw = 0.f;
  T.dy = 0.f;
  T.dz = 0.f;
  T.ya = 0.f;
  T.za = 0.f;
  seed_cov_of(A, T);
  int st = st0;
  double chi2sum = 0.0;
  int nacc = 0;
  float xref = 0.f;
  float out_p[5], out_c[15];
  int64_t smoothed_from = e;  // clusters [smoothed_from, e) hold smoothed values
  if (st0 != ST_BAD_INPUT) {  // BAD_INPUT here = offsets out of range: touch nothing of the frame
    const int n = (int)(e - a);
    if (n > 0) {
      T.ya = A.y[a];
      T.za = A.z[a];
      xref = A.x[a];
    }
    state_of(T, out_p);  // the outputs of a track that is not fitted
    cov_of(T, out_c);
    float xcur = xref;
    int fw_done = 0;  // clusters the forward filter updated with
#pragma unroll
    for (int w = 0; w < kSmoothBitWords; ++w) bits[w * kSmoothBlock] = 0u;
    if (st0 == ST_OK) {
      const Gate gate = make_gate(A.chi2_max, A.chi2_max_d);
      const int lead = chunk_lead(A, a);
      const uint32_t rsh = (uint32_t)((reinterpret_cast<uintptr_t>(A.row) + (uintptr_t)(a - lead)) & 3u);
      const int nch = (lead + n + kChunk - 1) / kChunk;
      // ---------------- forward filter (outward pass) ----------------
      int kc = 0;
      int staged = nch < kStageBufs ? nch : kStageBufs;  // chunks 0 .. staged-1 issued
      for (int c = 0; c < staged; ++c) stage_chunk<kSmoothBlock>(A, a, e, lead, rsh, c, c, f4, wrow);
      cp_async_wait_all();
      int cbuf = 0;  // buffer of the current chunk
      uint32_t rows_cur = staged_rows<kSmoothBlock>(wrow, 0, rsh);
      Clu cand = read_staged<kSmoothBlock>(f4, lead, 0, rows_cur);
      int nacc_out = 0, rprev = -1;
      const int r0 = cand.r;  // predictions are kept by row step r - r0
      uint32_t ow = 0u, obit = 1u;  // forward accept bits of the current 32-cluster word
      for (int r = cand.r, step = 0;; ++r, ++step) {
        if (step > 0 && (step & (kChunk - 1)) == 0) {  // staging step (warp-uniform)
          cp_async_wait_all();
          if (staged < nch && staged <= ((kc + lead) >> 2) + 2) {  // the buffer of chunk staged-3 is consumed
            stage_chunk<kSmoothBlock>(A, a, e, lead, rsh, staged, staged % kStageBufs, f4, wrow);
            ++staged;
          }
        }
        {  // the next cluster, validated as in the fit before any propagation towards it
          const int vs = check_cluster(cand.r, rprev, A.n_rows, cand.x, cand.y, cand.z, cand.vy, cand.vz);
          if (vs != ST_OK) { st = vs; break; }
        }
        const bool has = (cand.r == r);
        const float xt = has ? cand.x : s_rowx[r];
        if (!propagate(T, xt - xcur, A.b, A.snp_max)) { st = ST_SNP_LIMIT; break; }
        xcur = xt;
        {  // the prediction at every row step, also on rows without a cluster (never read back there):
           // the warp's stores then cover whole sectors, which L2 takes without reading them from DRAM
          float pm[5], cm[15];
          state_of(T, pm);
          cov_of(T, cm);
          store_pred(pred, r - r0, pm, cm);
        }
        if (has) {
          bool acc;
          double chi2;
          const int ust = update(T, cand.y, cand.z, cand.vy, cand.vz, gate, false, acc, chi2);
          if (ust != ST_OK) { st = ust; break; }
          if (acc) ow |= obit;
          nacc_out += acc ? 1 : 0;
          ++fw_done;
          rprev = cand.r;
          obit = __funnelshift_l(obit, obit, 1);  // rotate: the bit of cluster kc + 1 in its word
          if (obit == 1u) {                      // clusters kc - 31 .. kc complete a word
            bits[(kc >> 5) * kSmoothBlock] = ow;
            ow = 0u;
          }
          if (++kc < n) {
            const int p = kc + lead;
            if ((p & 3) == 0) {  // entering chunk p/4 (arrived)
              cbuf = cbuf == kStageBufs - 1 ? 0 : cbuf + 1;
              rows_cur = staged_rows<kSmoothBlock>(wrow, cbuf, rsh);
            }
            cand = read_staged<kSmoothBlock>(f4, p & 3, cbuf, rows_cur);
          }
        }
        if (A.xx0 > 0.f) ms_noise(T, A.xx0, A.mass2);
        if (kc == n) break;
      }
      if (kc & 31) bits[(kc >> 5) * kSmoothBlock] = ow;  // the last, partial word
      if (st == ST_OK) {
        // ---------------- restart, as the fit's inward pass ----------------
        // cand holds the outermost cluster n-1
        const bool fw_valid = 100 * nacc_out >= A.reseed_pct * n;
        if (!fw_valid) {
          float p[5];
          const int64_t m = a + n / 2;
          seed3(cand.x, cand.y, cand.z, A.x[m], A.y[m], A.x[a], A.y[a], A.z[a], A.b, p);
          T.sp = -p[2];
          T.spl = 0.f;
          T.tl0 = -p[3];
          T.dtl = 0.f;
          T.w0 = -p[4];
          T.dw = 0.f;
          T.ya = cand.y;
          T.za = cand.z;
          T.dy = 0.f;
          T.dz = 0.f;
          seed_cov_of(A, T);
        } else {
          const float d0 = fminf(A.restart_scale * T.c[0], A.seed_cov[0]);
          const float d1 = fminf(A.restart_scale * T.c[2], A.seed_cov[1]);
          const float d2 = fminf(A.restart_scale * (T.c[5] + T.c5l), A.seed_cov[2]);
          const float d3 = fminf(A.restart_scale * (T.c[9] + T.c9l), A.seed_cov[3]);
          const float d4 = fminf(A.restart_scale * (T.c[14] + T.c14l), A.seed_cov[4]);
#pragma unroll
          for (int i = 0; i < 15; ++i) T.c[i] = 0.f;
          T.c[0] = d0;
          T.c[2] = d1;
          T.c[5] = d2;
          T.c[9] = d3;
          T.c[14] = d4;
          T.clear_comp();
        }
        // ---------------- backward filter and combination ----------------
        // the ring holds the last kStageBufs chunks, arrived; the last is current
        kc = n - 1;
        int lowest = nch > kStageBufs ? nch - kStageBufs : 0;  // the lowest chunk issued
        float pm[5], cm[15];  // the forward prediction at the current cluster, loaded a step ahead of its use
        if (fw_valid) load_pred(pred, cand.r - r0, pm, cm);
        for (int r = cand.r, step = 0;; --r, ++step) {
          if (step > 0 && (step & (kChunk - 1)) == 0) {  // staging step (warp-uniform)
            cp_async_wait_all();
            if (lowest > 0 && lowest + 1 >= ((kc + lead) >> 2)) {  // the buffer of chunk lowest+2 is consumed
              --lowest;
              stage_chunk<kSmoothBlock>(A, a, e, lead, rsh, lowest, lowest % kStageBufs, f4, wrow);
            }
          }
          const bool has = (cand.r == r);
          const float xt = has ? cand.x : s_rowx[r];
          if (!propagate(T, xt - xcur, A.b, A.snp_max)) { st = ST_SNP_LIMIT; break; }
          xcur = xt;
          if (step > 0 && A.xx0 > 0.f) ms_noise(T, A.xx0, A.mass2);  // the row's kink lies beyond its measurement
          if (has) {
            bool acc;
            double chi2;
            const int ust = update(T, cand.y, cand.z, cand.vy, cand.vz, gate, true, acc, chi2);
            if (ust != ST_OK) { st = ust; break; }
            chi2sum += __longlong_as_double(acc ? __double_as_longlong(chi2) : 0ll);
            nacc += acc ? 1 : 0;
            const int64_t k = a + kc;
            A.accept[k] = (uint8_t)(((bits[(kc >> 5) * kSmoothBlock] >> (kc & 31)) & 1u) | (acc ? 2u : 0u));
            float ps[5], cs[15];
            {
              float pp[5], cp[15];
              state_of(T, pp);
              cov_of(T, cp);
              if (fw_valid) {
                if (!combine(pm, cm, pp, cp, ps, cs)) { st = ST_NOT_PD; break; }
              } else {
                store5(ps, pp);
                store15(cs, cp);
              }
            }
            if (--kc >= 0) {
              const int p = kc + lead;
              if ((p & 3) == 3) {  // entering chunk p/4 from above (arrived)
                cbuf = cbuf == 0 ? kStageBufs - 1 : cbuf - 1;
                rows_cur = staged_rows<kSmoothBlock>(wrow, cbuf, rsh);
              }
              cand = read_staged<kSmoothBlock>(f4, p & 3, cbuf, rows_cur);
              if (fw_valid) load_pred(pred, cand.r - r0, pm, cm);  // the next cluster's, a step ahead
            }
            store_vec<5>(A.sm_state + 5 * k, ps);
            store_vec<15>(A.sm_cov + 15 * k, cs);
            smoothed_from = k;
            if (kc < 0) {
              store5(out_p, ps);
              store15(out_c, cs);
              break;
            }
          }
        }
        if (st == ST_OK) {
          bool fin = true;
#pragma unroll
          for (int i = 0; i < 5; ++i) fin = fin && isfinite(out_p[i]);
#pragma unroll
          for (int i = 0; i < 15; ++i) fin = fin && isfinite(out_c[i]);
          if (!fin) st = ST_NONFINITE;
        }
        if (st == ST_OK && 100 * nacc < kSmoothDerailPct * n) st = ST_DERAILED;
      }
      cp_async_wait_all();  // no copy may land in the column after this track
      if (st != ST_OK && st != ST_DERAILED) {  // a failed fit: the state where it stopped
        state_of(T, out_p);
        cov_of(T, out_c);
      }
    }
    // clusters without a smoothed state (the backward filter wrote the accept
    // bytes of the others): their forward bit, 0 where the forward filter did
    // not reach (the backward filter runs only after a complete forward pass,
    // so a + fw_done <= smoothed_from whenever fw_done < n)
    for (int64_t q = a; q < smoothed_from; ++q) {
#pragma unroll
      for (int i = 0; i < 5; ++i) A.sm_state[5 * q + i] = qnan;
#pragma unroll
      for (int i = 0; i < 15; ++i) A.sm_cov[15 * q + i] = qnan;
      const int j = (int)(q - a);
      A.accept[q] = j < fw_done ? (uint8_t)((bits[(j >> 5) * kSmoothBlock] >> (j & 31)) & 1u) : (uint8_t)0u;
    }
  }
  if (st0 == ST_BAD_INPUT) {
    state_of(T, out_p);
    cov_of(T, out_c);
  }
  A.x_ref[t] = xref;
  store5(A.state + 5 * t, out_p);
  store15(A.cov + 15 * t, out_c);
  A.chi2[t] = chi2sum;
  A.ndf[t] = 2 * nacc - 5;
  A.status[t] = st;
}

// Shared memory of k_smooth: the fit's staging (pad-row table, chunk ring,
// row words) and the forward accept bits, over kSmoothBlock track columns.
constexpr size_t kSmoothSmem = stage_smem<kSmoothBlock>() + (size_t)kSmoothBitWords * kSmoothBlock * sizeof(uint32_t);

__global__ void __launch_bounds__(kSmoothBlock) k_smooth(FitArgs A) {
  __shared__ __align__(16) unsigned char smem[kSmoothSmem];
  float *s_rowx = reinterpret_cast<float *>(smem);
  float *s_f4 = reinterpret_cast<float *>(smem + kSmemRowx);
  uint32_t *s_w = reinterpret_cast<uint32_t *>(smem + kSmemRowx + smem_f4<kSmoothBlock>());
  uint32_t *s_bits = s_w + kStageBufs * 2 * kSmoothBlock;
  for (int i = threadIdx.x; i < kMaxRows; i += blockDim.x) s_rowx[i] = A.row_x[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const size_t warp = ((size_t)blockIdx.x * kSmoothBlock + threadIdx.x) >> 5;
  float *pred = A.sm_pred + warp * (size_t)A.n_rows * (32 * 4 * kPredVec) + 4 * lane;  // this warp's scratch, this lane's column
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(A.work, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= (unsigned long long)A.n_tracks) break;
    const int64_t i = (int64_t)base + lane;
    if (i < A.n_tracks)
      smooth_track(A, A.perm ? (int64_t)A.perm[i] : i, s_rowx, s_f4 + 4 * threadIdx.x, s_w + threadIdx.x,
                   s_bits + threadIdx.x, pred);
    __syncwarp();
  }
}

}  // namespace

int smooth_grid() {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_smooth, kSmoothBlock, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int per_sm = occ < 4 ? (occ > 0 ? occ : 1) : 4;  // up to 512 tracks per SM (its prediction scratch grows with the grid)
  return sms * per_sm;
}

// Scratch of the forward predictions: per warp of the grid, 80 bytes for
// each of up to n_rows clusters of each of its 32 lanes' tracks (a track has
// at most one cluster per pad row).
size_t smooth_pred_bytes(int grid, int n_rows) {
  return (size_t)grid * (kSmoothBlock / 32) * (size_t)n_rows * 32 * 4 * kPredVec * sizeof(float);
}

cudaError_t launch_smooth(const FitArgs &a, int grid, cudaStream_t stream) {
  if (a.n_tracks <= 0) return cudaSuccess;
  if (!a.sm_state || !a.sm_cov || !a.sm_pred || grid <= 0) return cudaErrorInvalidValue;
  k_smooth<<<grid, kSmoothBlock, 0, stream>>>(fit_args_for_launch(a));  // with stage_vec set
  return cudaGetLastError();
}

}  // namespace tpcfit
