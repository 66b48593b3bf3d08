// CUDA kernels of the batched TPC Kalman track fit (sm_103a); the track state,
// propagation, scattering and update they share with track following are in
// fit_device.cuh.
//
// The paper (Sec. 5, Tables 1-2; Sec. 6) puts full TPC tracking on the GPU as
// the dominant reconstruction step; the fit computed here is the textbook
// Kalman track fit (Fruhwirth 1987) with an exact helix in a uniform field and
// PDG Highland scattering, in an outward then an inward pass.
//
// Launch sequence of one frame:
//   k_prepare   thread per track: offset checks, 3-point seed, status preset,
//               sort key (pad rows crossed) histogram
//   k_sort_*    counting sort of tracks by pad rows crossed, longest first
//   k_fit       persistent grid; each warp claims 32 consecutive tracks of the
//               sorted order, one thread per track, and steps pad row by pad
//               row through the outward and the inward pass (every lane
//               propagates each step; lanes with a cluster on the row update).
// Serving fits the prepared parts of several frames with k_fit_parts instead:
// the same fit of each track, the warps claiming (part, 32-track group)
// descriptors from a device table.
//
// Precision: propagation, covariance transport and the gain/update are FP32.
// The innovation-matrix determinant, the reciprocal correction of chi2 =
// r^T S^-1 r and the chi2 sum are FP64.  GB300 executes FP64 at ~1/64 of the
// FP32 rate and a warp-wide FP64 instruction costs the same with one active
// lane as with 32, so the FP64 island is kept to 2 instructions per outward
// update (det; the gate is decided in FP64 only within 2^-19 of its boundary,
// else in binary32 with the same outcome) and 6 per inward update (det,
// reciprocal correction and chi2, sum); the quadratic form of the residual is
// formed in twice the binary32 precision on the FP32 pipe, every FP32->FP64
// widening is done with integer operations, and warps are filled with tracks
// of equal length so that the FP64 instructions of a step serve (almost)
// every lane.
//
// Track positions are carried as FP32 offsets (dy, dz) from the last
// cluster's coordinates: residuals are then formed from small numbers and the
// chi2 near the gate keeps FP64-level agreement with an FP64 fit.

#include <cuda_runtime.h>

#include <atomic>
#include <math.h>
#include <stdint.h>

#include "fit_device.cuh"
#include "stage_device.cuh"
#include "tpcfit_internal.h"

namespace tpcfit {



constexpr int kBitWords = kMaxRows / 32;  // outward accept bits of one track (<= 256 clusters)
// A completed fit whose (last) inward pass accepted fewer than this percentage
// of the track's clusters lost the track for a stretch: status DERAILED.
constexpr int kDerailPct = 80;
// Dynamic shared memory of k_fit over NCOL track columns (threads x tracks
// per lane): the staging (row table, chunks, row words) and the outward
// accept bits ([word][column]).
template <int NCOL> __host__ __device__ constexpr size_t fit_smem() {
  return stage_smem<NCOL>() + (size_t)kBitWords * NCOL * sizeof(uint32_t);
}

// ---------------------------------------------------------------------------
// k_prepare: per-track offset checks, status preset, seed, key histogram.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_prepare(FitArgs A) {
  __shared__ uint32_t s_hist[kKeyBins];
  for (int i = threadIdx.x; i < kKeyBins; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < A.n_tracks) {
    if (t == 0 && (A.off[0] - A.off_base != 0 || A.off[A.n_tracks] - A.off_base != A.n_clusters))
      atomicOr(A.frame_error, 1);
    const int64_t a = A.off[t] - A.off_base, e = A.off[t + 1] - A.off_base;
    int st = ST_OK;
    int64_t n = 0;
    if (a < 0 || e < a || e > A.n_clusters) {
      st = ST_BAD_INPUT;
      atomicOr(A.frame_error, 1);
    } else {
      n = e - a;
      if (n < A.min_clusters || n < 3) st = ST_TOO_FEW;
    }
    float p[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (st == ST_OK) {
      const int64_t m = a + n / 2, l = e - 1;
      seed3(A.x[a], A.y[a], A.z[a], A.x[m], A.y[m], A.x[l], A.y[l], A.z[l], A.b, p);
      if (fabsf(p[2]) >= A.snp_max) st = ST_SNP_LIMIT;  // NaN passes
    }
    float *sd = A.seed + 5 * t;
#pragma unroll
    for (int i = 0; i < 5; ++i) sd[i] = p[i];
    A.status[t] = st;
    int key = 0;  // rows crossed, so that warps get tracks with the same number of row steps
    if (st == ST_OK) {
      const int rr = (int)A.row[e - 1] - (int)A.row[a] + 1;
      key = rr < 1 ? 1 : (rr > kMaxRows ? kMaxRows : rr);
    }
    atomicAdd(&s_hist[key], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kKeyBins; i += blockDim.x)
    if (s_hist[i]) atomicAdd(&A.hist[i], s_hist[i]);
}

// ---------------------------------------------------------------------------
// Counting sort by key, descending: exclusive scan of the histogram (one block)
// then a block-aggregated scatter.
// ---------------------------------------------------------------------------
__global__ void k_sort_scan(uint32_t *hist) {
  // hist[0..kKeyBins) counts -> hist[kKeyBins..2*kKeyBins) start positions, key descending
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int k = kKeyBins - 1; k >= 0; --k) {
      hist[kKeyBins + k] = acc;
      acc += hist[k];
    }
  }
}

__device__ __forceinline__ int track_key(const FitArgs &A, int64_t t) {
  if (A.status[t] != ST_OK) return 0;
  const int64_t a = A.off[t] - A.off_base, e = A.off[t + 1] - A.off_base;
  const int rr = (int)A.row[e - 1] - (int)A.row[a] + 1;
  return rr < 1 ? 1 : (rr > kMaxRows ? kMaxRows : rr);
}

__global__ void __launch_bounds__(256) k_sort_scatter(FitArgs A) {
  __shared__ uint32_t s_cnt[kKeyBins];
  __shared__ uint32_t s_base[kKeyBins];
  for (int i = threadIdx.x; i < kKeyBins; i += blockDim.x) s_cnt[i] = 0;
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int key = 0;
  uint32_t rank = 0;
  if (t < A.n_tracks) {
    key = track_key(A, t);
    rank = atomicAdd(&s_cnt[key], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kKeyBins; i += blockDim.x)
    s_base[i] = s_cnt[i] ? atomicAdd(&A.hist[kKeyBins + i], s_cnt[i]) : 0u;
  __syncthreads();
  if (t < A.n_tracks) A.perm[s_base[key] + rank] = (int32_t)t;
}

// ---------------------------------------------------------------------------
// k_fit: persistent warps over the (sorted) track list, one track per lane;
// each lane stages its track's clusters as stage_device.cuh describes.
// ---------------------------------------------------------------------------

// Fitted state and covariance all finite.
__device__ __forceinline__ bool state_finite(const Trk &T) {
  bool fin = isfinite(T.dy) && isfinite(T.dz) && isfinite(T.snp()) && isfinite(T.tl()) && isfinite(T.w());
#pragma unroll
  for (int i = 0; i < 15; ++i) fin = fin && isfinite(T.c[i]);
  return fin;
}

// Fit of track t by one lane: outward pass, restart, inward pass (and, in the
// variant, energy loss, seed iterations and the per-cluster diagnostics:
// chi2 of every update and the inward restart state).  NCOL = threads of the block: the
// lane's staging and accept-bit columns are strided by it.
template <int NCOL, bool VAR>
__device__ void fit_track(const FitArgs &A, int64_t t, uint32_t *bits, const float *s_rowx, float *f4,
                          uint32_t *wrow) {
  const int64_t a = A.off[t] - A.off_base, e = A.off[t + 1] - A.off_base;
  const int st0 = A.status[t];
  const float *sd = A.seed + 5 * t;
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
#pragma unroll
  for (int i = 0; i < 15; ++i) T.c[i] = 0.f;
  T.c[0] = A.seed_cov[0];
  T.c[2] = A.seed_cov[1];
  T.c[5] = A.seed_cov[2];
  T.c[9] = A.seed_cov[3];
  T.c[14] = A.seed_cov[4];
  T.clear_comp();
  int st = st0;
  double chi2sum = 0.0;
  int nacc = 0;
  float xref = 0.f;
  if (st0 != ST_BAD_INPUT) {  // BAD_INPUT here = offsets out of range: touch nothing of the frame
    const int n = (int)(e - a);
    if (n > 0) {
      T.ya = A.y[a];
      T.za = A.z[a];
      xref = A.x[a];
    }
    float xcur = xref;
#pragma unroll
    for (int w = 0; w < kBitWords; ++w) bits[NCOL * w] = 0u;
    uint8_t *const acc_t = A.accept + a;  // this track's accept bytes
    int done = 0;      // clusters (from the outer end) whose accept byte is final
    int out_done = 0;  // clusters the outward pass updated with
    if (st0 == ST_OK) {
      const Gate gate = make_gate(A.chi2_max, A.chi2_max_d);
      const int lead = chunk_lead(A, a);
      const uint32_t rsh = (uint32_t)((reinterpret_cast<uintptr_t>(A.row) + (uintptr_t)(a - lead)) & 3u);
      const int nch = (lead + n + kChunk - 1) / kChunk;
      // passes: one outward + inward pair, or (the variant) 1 + n_iter of them
      for (int it = 0;; ++it) {
        int nacc_out = 0;
        // outward accept bits of the current 32-cluster word, written to the
        // track's shared-memory words when complete and after the pass
        uint32_t ow = 0u, obit = 1u;
        // candidate: the next cluster to use, read from the track's staged chunks.
        // The chunks sit in a ring of kStageBufs buffers; copies are issued and
        // waited for at warp-uniform steps, every kChunk rows of a pass (the
        // same rows for all lanes of a warp, whose tracks cross as many rows),
        // so the lanes stage in step.  After each step the lane's current chunk
        // and the next one have arrived, and a lane reaches at most one new
        // chunk before the next step.  After an inward pass the ring already
        // holds chunks 0..2, arrived.
        int kc = 0;
        int staged = nch < kStageBufs ? nch : kStageBufs;  // outward: chunks 0 .. staged-1 issued
        if (it == 0)
          for (int c = 0; c < staged; ++c) stage_chunk<NCOL>(A, a, e, lead, rsh, c, c, f4, wrow);
        cp_async_wait_all();
        int cbuf = 0;  // buffer of the current chunk
        uint32_t rows_cur = staged_rows<NCOL>(wrow, 0, rsh);
        Clu cand = read_staged<NCOL>(f4, lead, 0, rows_cur);
        int rprev = -1;
        // ---------------- outward pass: rows row[0] .. row[n-1] ----------------
        for (int r = cand.r, step = 0;; ++r, ++step) {
          if (step > 0 && (step & (kChunk - 1)) == 0) {  // staging step (warp-uniform)
            cp_async_wait_all();
            if (staged < nch && staged <= ((kc + lead) >> 2) + 2) {  // the buffer of chunk staged-3 is consumed
              stage_chunk<NCOL>(A, a, e, lead, rsh, staged, staged % kStageBufs, f4, wrow);
              ++staged;
            }
          }
          {  // the next cluster is validated when the pass reaches it, before any
             // propagation towards it (checked at every row until it is used: the
             // values were read at the end of the previous step, so the test does
             // not wait for them)
            const int vs = check_cluster(cand.r, rprev, A.n_rows, cand.x, cand.y, cand.z, cand.vy, cand.vz);
            if (vs != ST_OK) { st = vs; break; }
          }
          const bool has = (cand.r == r);
          const float xt = has ? cand.x : s_rowx[r];
          if (!propagate(T, xt - xcur, A.b, A.snp_max)) { st = ST_SNP_LIMIT; break; }
          xcur = xt;
          if (has) {
            bool acc;
            double chi2;
            const int ust = update(T, cand.y, cand.z, cand.vy, cand.vz, gate,
                                   VAR && A.chi2_out_c != nullptr, acc, chi2);
            if (ust != ST_OK) { st = ust; break; }
            if (acc) ow |= obit;
            if (VAR && A.chi2_out_c) A.chi2_out_c[a + kc] = chi2;
            ++out_done;
            nacc_out += acc ? 1 : 0;
            rprev = cand.r;
            obit = __funnelshift_l(obit, obit, 1);  // rotate: the bit of cluster kc + 1 in its word
            if (obit == 1u) {                      // clusters kc - 31 .. kc complete a word
              bits[NCOL * (kc >> 5)] = ow;
              ow = 0u;
            }
            if (++kc < n) {
              const int p = kc + lead;
              if ((p & 3) == 0) {  // entering chunk p/4 (arrived)
                cbuf = cbuf == kStageBufs - 1 ? 0 : cbuf + 1;
                rows_cur = staged_rows<NCOL>(wrow, cbuf, rsh);
              }
              cand = read_staged<NCOL>(f4, p & 3, cbuf, rows_cur);
            }
          }
          if (A.xx0 > 0.f) ms_noise(T, A.xx0, A.mass2);
          if (VAR && A.xrho > 0.f && !eloss(T, A.xrho, A.el_kza, A.el_a, A.el_ratio, A.mass2, 1.0f)) {
            st = ST_STOPPED;
            break;
          }
          if (kc == n) break;
        }
        if (kc & 31) bits[NCOL * (kc >> 5)] = ow;  // the last, partial word
        // ---------------- restart ----------------
        if (st == ST_OK) {
          // cand holds the outermost cluster n-1
          if (100 * nacc_out < A.reseed_pct * n) {
            // the outward pass accepted fewer than reseed_pct % of the clusters: re-seed
            // at the outermost cluster (circle through clusters n-1, n/2, 0 for
            // motion towards cluster 0, reversed) with the seed covariance
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
#pragma unroll
            for (int i = 0; i < 15; ++i) T.c[i] = 0.f;
            T.c[0] = A.seed_cov[0];
            T.c[2] = A.seed_cov[1];
            T.c[5] = A.seed_cov[2];
            T.c[9] = A.seed_cov[3];
            T.c[14] = A.seed_cov[4];
          } else {
            // inward restart: diagonal, outward variances inflated, capped at the seed's
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
          }
          T.clear_comp();
          if (VAR && A.restart_state) {
            float *rs = A.restart_state + 5 * t;
            rs[0] = T.ya + T.dy;
            rs[1] = T.za + T.dz;
            rs[2] = T.snp();
            rs[3] = T.tl();
            rs[4] = T.w();
          }
          // ---------------- inward pass: rows row[n-1] .. row[0] ----------------
          kc = n - 1;
          uint32_t iw = bits[NCOL * (kc >> 5)] << (31 - (kc & 31));  // the outward bit of cluster kc in bit 31
          // the ring holds the last kStageBufs chunks (the outward pass reached
          // the last one, so all of them have arrived); the last is current
          int lowest = nch > kStageBufs ? nch - kStageBufs : 0;  // inward: the lowest chunk issued
          for (int r = cand.r, step = 0;; --r, ++step) {
            if (step > 0 && (step & (kChunk - 1)) == 0) {  // staging step (warp-uniform)
              cp_async_wait_all();
              if (lowest > 0 && lowest + 1 >= ((kc + lead) >> 2)) {  // the buffer of chunk lowest+2 is consumed
                --lowest;
                stage_chunk<NCOL>(A, a, e, lead, rsh, lowest, lowest % kStageBufs, f4, wrow);
              }
            }
            const bool has = (cand.r == r);
            const float xt = has ? cand.x : s_rowx[r];
            if (!propagate(T, xt - xcur, A.b, A.snp_max)) { st = ST_SNP_LIMIT; break; }
            xcur = xt;
            // the layer of row r lies beyond the plane in outward motion: its loss is added back first
            if (VAR && A.xrho > 0.f && !eloss(T, A.xrho, A.el_kza, A.el_a, A.el_ratio, A.mass2, -1.0f)) {
              st = ST_STOPPED;
              break;
            }
            if (has) {
              bool acc;
              double chi2;
              const int ust = update(T, cand.y, cand.z, cand.vy, cand.vz, gate, true, acc,
                                     chi2);
              if (ust != ST_OK) { st = ust; break; }
              if (VAR && A.chi2_in_c) A.chi2_in_c[a + kc] = chi2;
              chi2sum += __longlong_as_double(acc ? __double_as_longlong(chi2) : 0ll);
              nacc += acc ? 1 : 0;
              acc_t[kc] = (uint8_t)((iw >> 31) | (acc ? 2u : 0u));
              ++done;
              if (--kc >= 0) {
                if ((kc & 31) == 31)
                  iw = bits[NCOL * (kc >> 5)];
                else
                  iw <<= 1;
                const int p = kc + lead;
                if ((p & 3) == 3) {  // entering chunk p/4 from above (arrived)
                  cbuf = cbuf == 0 ? kStageBufs - 1 : cbuf - 1;
                  rows_cur = staged_rows<NCOL>(wrow, cbuf, rsh);
                }
                cand = read_staged<NCOL>(f4, p & 3, cbuf, rows_cur);
              }
            }
            if (A.xx0 > 0.f) ms_noise(T, A.xx0, A.mass2);
            if (kc < 0) break;
          }
        }
        if (!VAR || st != ST_OK || it >= A.n_iter) break;
        // seed iteration: the fitted state at the innermost cluster (xcur) seeds
        // another outward pass with the seed covariance; a non-finite state ends
        // the fit instead.  The ring holds chunks 0..2: the inward pass ended on chunk 0.
        if (!state_finite(T)) {
          st = ST_NONFINITE;
          break;
        }
#pragma unroll
        for (int i = 0; i < 15; ++i) T.c[i] = 0.f;
        T.c[0] = A.seed_cov[0];
        T.c[2] = A.seed_cov[1];
        T.c[5] = A.seed_cov[2];
        T.c[9] = A.seed_cov[3];
        T.c[14] = A.seed_cov[4];
        T.clear_comp();
#pragma unroll
        for (int w = 0; w < kBitWords; ++w) bits[NCOL * w] = 0u;
        done = 0;
        out_done = 0;
        chi2sum = 0.0;
        nacc = 0;
      }  // passes
      cp_async_wait_all();  // no copy may land in the column after this track
      if (st == ST_OK && !state_finite(T)) st = ST_NONFINITE;
      if (st == ST_OK && 100 * nacc < kDerailPct * n) st = ST_DERAILED;  // the last inward pass lost the track
    }
    // accept bytes not written by the inward pass (failed or unfitted tracks): outward bits only
    for (int64_t k = a; k < e - done; ++k) {
      const int lk = (int)(k - a);
      A.accept[k] = (lk < kMaxRows) ? (uint8_t)((bits[NCOL * (lk >> 5)] >> (lk & 31)) & 1u) : (uint8_t)0;
    }
    if (VAR && A.chi2_in_c)
      for (int64_t k = a; k < e - done; ++k) A.chi2_in_c[k] = __longlong_as_double(0x7ff8000000000000ll);
    if (VAR && A.chi2_out_c)
      for (int64_t k = a + out_done; k < e; ++k) A.chi2_out_c[k] = __longlong_as_double(0x7ff8000000000000ll);
  }
  A.x_ref[t] = xref;
  float *ps = A.state + 5 * t;
  ps[0] = T.ya + T.dy;
  ps[1] = T.za + T.dz;
  ps[2] = T.snp();
  ps[3] = T.tl();
  ps[4] = T.w();
  float *pc = A.cov + 15 * t;
  T.fold_comp();
#pragma unroll
  for (int i = 0; i < 15; ++i) pc[i] = T.c[i];
  A.chi2[t] = chi2sum;
  A.ndf[t] = 2 * nacc - 5;
  A.status[t] = st;
}

// VAR: the variant -- energy loss, seed iteration and the diagnostic
// outputs, each checked at run time (a separate instantiation, so that the
// plain fit keeps its own register allocation and schedule).
template <int BLOCK, int MINB, bool VAR>
__global__ void __launch_bounds__(BLOCK, MINB) k_fit(FitArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  float *s_rowx = reinterpret_cast<float *>(smem);
  float *s_f4 = reinterpret_cast<float *>(smem + kSmemRowx);
  uint32_t *s_w = reinterpret_cast<uint32_t *>(smem + kSmemRowx + smem_f4<BLOCK>());
  uint32_t *s_bits = s_w + kStageBufs * 2 * BLOCK;
  for (int i = threadIdx.x; i < kMaxRows; i += blockDim.x) s_rowx[i] = A.row_x[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(A.work, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= (unsigned long long)A.n_tracks) break;
    const int64_t i = (int64_t)base + lane;
    if (i < A.n_tracks) {
      const int64_t t = A.perm ? (int64_t)A.perm[i] : i;
      fit_track<BLOCK, VAR>(A, t, s_bits + threadIdx.x, s_rowx, s_f4 + 4 * threadIdx.x, s_w + threadIdx.x);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// k_fit_parts: one persistent launch over the resident parts of several time
// frames (the serving engine).  The track groups of all parts -- 32
// consecutive tracks of a part's sorted order -- form one range, part p's
// being [prefix[p], prefix[p+1]); each warp claims the next group with an
// atomic cursor, fits it with the part's arguments (copied into the warp's
// shared-memory slot when the part changes), and counts the part's remaining
// groups down.  The warp that fits a part's last group makes the part's
// results visible system-wide and sets the part's flag in host-mapped memory,
// so the host copies that part's results back while the launch still fits
// the others.
// ---------------------------------------------------------------------------
template <int BLOCK, int MINB, bool VAR>
__global__ void __launch_bounds__(BLOCK, MINB) k_fit_parts(PartsArgs P) {
  extern __shared__ __align__(16) unsigned char smem[];
  float *s_rowx = reinterpret_cast<float *>(smem);
  float *s_f4 = reinterpret_cast<float *>(smem + kSmemRowx);
  uint32_t *s_w = reinterpret_cast<uint32_t *>(smem + kSmemRowx + smem_f4<BLOCK>());
  uint32_t *s_bits = s_w + kStageBufs * 2 * BLOCK;
  FitArgs *s_args = reinterpret_cast<FitArgs *>(smem + fit_smem<BLOCK>());  // one per warp
  // the parts come from one handle and share its pad-row table
  for (int i = threadIdx.x; i < kMaxRows; i += blockDim.x) s_rowx[i] = P.parts[0].row_x[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  FitArgs *wa = s_args + (threadIdx.x >> 5);
  const unsigned long long total = P.prefix[P.n_parts];
  int cur = -1;  // part whose arguments are in the warp's slot
  for (;;) {
    unsigned long long g = 0;
    if (lane == 0) g = atomicAdd(P.cursor, 1ull);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= total) break;
    int lo = 0, hi = P.n_parts;  // the part p with prefix[p] <= g < prefix[p+1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (P.prefix[mid] <= g) lo = mid;
      else hi = mid;
    }
    if (lo != cur) {  // warp-uniform
      __syncwarp();
      const uint32_t *src = reinterpret_cast<const uint32_t *>(P.parts + lo);
      uint32_t *dst = reinterpret_cast<uint32_t *>(wa);
      for (int k = lane; k < (int)(sizeof(FitArgs) / 4); k += 32) dst[k] = src[k];
      __syncwarp();
      cur = lo;
    }
    const FitArgs &A = *wa;
    const int64_t i = (int64_t)(g - P.prefix[lo]) * 32 + lane;
    if (i < A.n_tracks) {
      const int64_t t = A.perm ? (int64_t)A.perm[i] : i;
      fit_track<BLOCK, VAR>(A, t, s_bits + threadIdx.x, s_rowx, s_f4 + 4 * threadIdx.x, s_w + threadIdx.x);
    }
    __threadfence();  // this lane's results, before the group counts as fitted
    __syncwarp();
    if (lane == 0 && atomicSub(P.remaining + lo, 1u) == 1u) {
      __threadfence_system();
      P.done_flag[lo] = 1;
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_prepare(const FitArgs &a, cudaStream_t stream) {
  if (a.n_tracks <= 0) return cudaSuccess;
  const int64_t blocks = (a.n_tracks + 255) / 256;
  k_prepare<<<(unsigned)blocks, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sort(const FitArgs &a, cudaStream_t stream, int *launches) {
  if (a.n_tracks <= 0 || !a.perm) return cudaSuccess;
  k_sort_scan<<<1, 32, 0, stream>>>(a.hist);
  const int64_t blocks = (a.n_tracks + 255) / 256;
  k_sort_scatter<<<(unsigned)blocks, 256, 0, stream>>>(a);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

// Raise the dynamic shared memory limit of one k_fit instantiation, once per
// device (the attribute belongs to the function in the current device's context).
template <int BLOCK, int MINB, bool VAR> static cudaError_t set_fit_smem() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(k_fit<BLOCK, MINB, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fit_smem<BLOCK>());
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

template <int BLOCK, int MINB, bool VAR> static cudaError_t launch_fit_as(const FitArgs &a, int grid,
                                                                             cudaStream_t stream) {
  cudaError_t e = set_fit_smem<BLOCK, MINB, VAR>();
  if (e != cudaSuccess) return e;
  k_fit<BLOCK, MINB, VAR><<<grid, BLOCK, fit_smem<BLOCK>(), stream>>>(a);
  return cudaGetLastError();
}

// The five cluster arrays share their position within 16-byte lines: whole
// aligned chunks are then staged as one 16-byte copy per array.
static bool same_16b_phase(const FitArgs &a) {
  const uintptr_t p = reinterpret_cast<uintptr_t>(a.x) & 15u;
  return (reinterpret_cast<uintptr_t>(a.y) & 15u) == p && (reinterpret_cast<uintptr_t>(a.z) & 15u) == p &&
         (reinterpret_cast<uintptr_t>(a.sy2) & 15u) == p && (reinterpret_cast<uintptr_t>(a.sz2) & 15u) == p;
}

// The variant instantiation: energy loss, seed iteration or diagnostic outputs.
static bool fit_variant(const FitArgs &a) {
  return a.xrho > 0.0f || a.n_iter > 0 || a.chi2_out_c || a.chi2_in_c || a.restart_state;
}

// SMs of the current device.
static int current_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms;
}

// The plain fit in blocks of 128 has two instantiations: for 4 resident
// blocks per SM (up to 128 registers per thread) and for 5 (up to 102): a
// grid of more than 4 blocks per SM runs the second, whose 640 tracks per SM
// fit the Pb-Pb frame 2 % faster although more of their clusters leave L2
// between the two passes (76 against 61 B of DRAM traffic per cluster).  A
// frame with no more tracks than 4 blocks per SM hold gains nothing from the
// fifth block and runs the first (its tracks' steps are shorter).  The
// variant and the serving engine keep 4 blocks of 128 per SM (a larger grid is
// cut to that: the warps claim their work, so the results do not change).
constexpr int kMaxBlocks128 = 5;

cudaError_t fit_set_attributes(const FitArgs &a, int block) {
  if (fit_variant(a)) return block == 128 ? set_fit_smem<128, 4, true>() : set_fit_smem<256, 2, true>();
  if (block != 128) return set_fit_smem<256, 2, false>();
  const cudaError_t e = set_fit_smem<128, 4, false>();
  return e != cudaSuccess ? e : set_fit_smem<128, kMaxBlocks128, false>();
}

cudaError_t launch_fit(const FitArgs &a_in, int grid, int block, cudaStream_t stream) {
  if (a_in.n_tracks <= 0) return cudaSuccess;
  FitArgs a = a_in;
  a.stage_vec = same_16b_phase(a) ? 1 : 0;
  if (block != 128)
    return fit_variant(a) ? launch_fit_as<256, 2, true>(a, grid, stream) : launch_fit_as<256, 2, false>(a, grid, stream);
  const int sms = current_sms();
  const bool over4 = sms > 0 && grid > 4 * sms;
  if (fit_variant(a) || (over4 && a.n_tracks <= (int64_t)4 * sms * 128))
    return fit_variant(a) ? launch_fit_as<128, 4, true>(a, over4 ? 4 * sms : grid, stream)
                          : launch_fit_as<128, 4, false>(a, 4 * sms, stream);
  return over4 ? launch_fit_as<128, kMaxBlocks128, false>(a, grid, stream) : launch_fit_as<128, 4, false>(a, grid, stream);
}

// Occupancy of the plain fit (the variant, compiled for 4 blocks of 128 or 2
// of 256, reaches 512 threads per SM).
int fit_blocks_per_sm(int block) {
  int n = 0;
  cudaError_t e;
  if (block == 128) {
    set_fit_smem<128, kMaxBlocks128, false>();
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fit<128, kMaxBlocks128, false>, 128, fit_smem<128>());
  } else {
    set_fit_smem<256, 2, false>();
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fit<256, 2, false>, 256, fit_smem<256>());
  }
  if (e != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

// Resident blocks per SM when the caller leaves the choice to the library:
// 640 tracks per SM for the plain fit in blocks of 128, else 512.  With 768
// tracks per SM in flight their clusters do not stay in L2 between the
// outward and the inward pass (DRAM reads of 170 B per cluster against 60 B
// with 512 and 72 B with 640, measured on GB300).
int fit_default_blocks_per_sm(int block, bool variant) {
  const int occ = fit_blocks_per_sm(block);
  const int want = block == 128 ? (variant ? 4 : kMaxBlocks128) : 2;
  return occ < want ? occ : want;
}

template <int BLOCK, int MINB, bool VAR> static cudaError_t launch_parts_as(const PartsArgs &p, int grid,
                                                                               cudaStream_t stream) {
  static std::atomic<unsigned long long> done{0};
  constexpr size_t smem = fit_smem<BLOCK>() + (BLOCK / 32) * sizeof(FitArgs);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(k_fit_parts<BLOCK, MINB, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    done.fetch_or(bit, std::memory_order_acq_rel);
  }
  k_fit_parts<BLOCK, MINB, VAR><<<grid, BLOCK, smem, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_fit_parts(const PartsArgs &p, bool variant, int grid, int block, cudaStream_t stream) {
  if (p.n_parts <= 0) return cudaSuccess;
  if (block == 128) {  // compiled for 4 resident blocks of 128
    const int sms = current_sms();
    if (sms > 0 && grid > 4 * sms) grid = 4 * sms;
  }
  if (variant)
    return block == 128 ? launch_parts_as<128, 4, true>(p, grid, stream) : launch_parts_as<256, 2, true>(p, grid, stream);
  return block == 128 ? launch_parts_as<128, 4, false>(p, grid, stream) : launch_parts_as<256, 2, false>(p, grid, stream);
}

FitArgs fit_args_for_launch(const FitArgs &a) {
  FitArgs b = a;
  b.stage_vec = same_16b_phase(a) ? 1 : 0;
  return b;
}

int fit_regs_per_thread(int block, bool variant, int blocks_per_sm) {
  cudaFuncAttributes at;
  cudaError_t e;
  if (block == 128 && !variant && blocks_per_sm > 4)
    e = cudaFuncGetAttributes(&at, k_fit<128, kMaxBlocks128, false>);
  else if (block == 128)
    e = variant ? cudaFuncGetAttributes(&at, k_fit<128, 4, true>) : cudaFuncGetAttributes(&at, k_fit<128, 4, false>);
  else
    e = variant ? cudaFuncGetAttributes(&at, k_fit<256, 2, true>) : cudaFuncGetAttributes(&at, k_fit<256, 2, false>);
  if (e != cudaSuccess) return -1;
  return at.numRegs;
}

}  // namespace tpcfit
