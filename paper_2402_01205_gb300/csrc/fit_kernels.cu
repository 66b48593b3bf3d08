// CUDA kernels of the batched TPC Kalman track fit (sm_103a).
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
//
// Precision: propagation, covariance transport and the gain/update are FP32.
// The innovation-matrix determinant and reciprocal, the quadratic form
// chi2 = r^T S^-1 r, the gate decision and the chi2 sum are FP64.  GB300
// executes FP64 at ~1/64 of the FP32 rate and a warp-wide FP64 instruction
// costs the same with one active lane as with 32, so the FP64 island is kept
// to 4 instructions per outward update (det, gate) and 7 per inward update
// (det, reciprocal, chi2, sum); the quadratic form of the residual is formed
// in twice the binary32 precision on the FP32 pipe, every FP32->FP64 widening
// is done with integer operations, and warps are filled with tracks of equal
// length so that the FP64 instructions of a step serve (almost) every lane.
//
// Track positions are carried as FP32 offsets (dy, dz) from the last
// cluster's coordinates: residuals are then formed from small numbers and the
// chi2 near the gate keeps FP64-level agreement with an FP64 fit.

#include <cuda_runtime.h>

#include <atomic>
#include <math.h>
#include <stdint.h>

#include "tpcfit_internal.h"

namespace tpcfit {

enum { ST_OK = 0, ST_TOO_FEW = 1, ST_SNP_LIMIT = 2, ST_NOT_PD = 3, ST_NONFINITE = 4, ST_BAD_INPUT = 5 };


constexpr int kBitWords = kMaxRows / 32;  // outward accept bits of one track (<= 256 clusters)
constexpr int kChunk = 4;                 // clusters per staged chunk (per lane)
constexpr int kStageArrays = 5;           // x, y, z, sy2, sz2
// dynamic shared memory of k_fit: row table, outward accept bits, staged clusters
constexpr size_t kSmemRowx = kMaxRows * sizeof(float);
template <int BLOCK> __host__ __device__ constexpr size_t smem_bits() { return (size_t)(BLOCK / 32) * kBitWords * 32 * sizeof(uint32_t); }
// staged floats [buf][array][slot][lane], then staged row words [buf][word][lane]
constexpr int kStageFloats = 2 * kStageArrays * kChunk;  // per lane
constexpr int kStageRowWords = 2 * 2;                     // per lane: two aligned words per buffer
template <int BLOCK> __host__ __device__ constexpr size_t smem_stage() { return (size_t)(kStageFloats + kStageRowWords) * BLOCK * sizeof(float); }
template <int BLOCK> __host__ __device__ constexpr size_t fit_smem() { return kSmemRowx + smem_bits<BLOCK>() + smem_stage<BLOCK>(); }

// 4-byte asynchronous global->shared copy (zero-fill when !valid; the source
// address is then still a valid element and is not read).
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// ---------------------------------------------------------------------------
// binary32 -> binary64 widening with integer operations (IEEE 754: the
// exponent is re-biased by 1023-127 = 896 and the 23-bit fraction moves to the
// top of the 52-bit fraction).  The FP64 pipe's own conversion costs as much
// as an FP64 multiply, so the island widens its inputs on the integer pipe.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double join64(uint32_t hi, uint32_t lo) {
  double d;
  asm("mov.b64 %0, {%1, %2};" : "=d"(d) : "r"(lo), "r"(hi));
  return d;
}
// The two halves of a binary64 value, taken with an opaque move so that the
// compiler keeps integer operations and does not turn the tests below back
// into FP64-pipe instructions (which cost as much as the arithmetic they guard).
__device__ __forceinline__ void split64(double x, uint32_t &hi, uint32_t &lo) {
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
}
// Halves of the widened value of a finite binary32 f: exact for normal f; a
// zero or subnormal f gives a value of the same sign and magnitude in
// [2^-127, 2^-126), i.e. zero to within 2^-126 absolute.
__device__ __forceinline__ void widen_halves(float f, uint32_t &hi, uint32_t &lo) {
  const uint32_t u = __float_as_uint(f);
  hi = (((u >> 3) & 0x0fffffffu) + (896u << 20)) | (u & 0x80000000u);
  lo = u << 29;
}
__device__ __forceinline__ double widen(float f) {
  uint32_t hi, lo;
  widen_halves(f, hi, lo);
  return join64(hi, lo);
}
// Exact widening of a positive normal binary32 value.
__device__ __forceinline__ double widen_pos(float f) {
  const uint32_t u = __float_as_uint(f);
  return join64((u >> 3) + (896u << 20), u << 29);
}
// x <= 0 for a finite x (-0 included).
__device__ __forceinline__ bool le0_finite64(double x) {
  uint32_t hi, lo;
  split64(x, hi, lo);
  return (int32_t)hi < 0 || (hi | lo) == 0u;
}
// x <= g for a finite x and a positive finite g given as (ghi, glo).
__device__ __forceinline__ bool le_finite64(double x, uint32_t ghi, uint32_t glo) {
  uint32_t hi, lo;
  split64(x, hi, lo);
  return (int32_t)hi < (int32_t)ghi || (hi == ghi && lo <= glo);
}

// Error-free sum of two binary32 numbers (Knuth's TwoSum): a + b = s + e
// exactly.  The error-free transformations use the _rn intrinsics, which the
// compiler never contracts into a fused multiply-add: the proofs need each
// sum and product rounded on its own.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Dekker's Fast2Sum: the same when |a| >= |b| (a variance plus a smaller
// increment, or minus a smaller decrement).
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// ---------------------------------------------------------------------------
// Seed: circle through three clusters (a, b, c) in the (x, y) plane; state at a.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float asin_over_u_f(float u) {
  const float u2 = u * u;
  if (fabsf(u) < 0.1f) return 1.0f + u2 * (1.0f / 6.0f + u2 * (3.0f / 40.0f + u2 * (5.0f / 112.0f)));
  return asinf(u) / u;
}

__device__ __noinline__ void seed3(float xa, float ya, float za, float xb, float yb, float xc, float yc, float zc, float b,
                      float p[5]) {
  const float abx = xb - xa, aby = yb - ya, acx = xc - xa, acy = yc - ya, bcx = xc - xb, bcy = yc - yb;
  const float cross = abx * acy - aby * acx;
  const float lab = sqrtf(abx * abx + aby * aby), lac = sqrtf(acx * acx + acy * acy),
              lbc = sqrtf(bcx * bcx + bcy * bcy);
  const float kappa = 2.0f * cross / (lab * lac * lbc);
  float u = 0.5f * kappa * lac;
  u = fminf(1.0f, fmaxf(-1.0f, u));
  const float phi = atan2f(acy, acx) - asinf(u);
  const float s_ac = lac * asin_over_u_f(u);
  p[0] = ya;
  p[1] = za;
  p[2] = sinf(phi);
  p[3] = (zc - za) / s_ac;
  p[4] = kappa / b;  // q/pT = -kappa/(kB Bz) = kappa / b
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
// Fit of one track: device helpers.
// ---------------------------------------------------------------------------
// Track state in FP32 with extended precision where the Kalman recursion
// accumulates many small increments onto a large value:
//  - y, z:       offsets (dy, dz) from the last cluster's coordinates (ya, za)
//  - sinphi:     compensated sum sp + spl (TwoSum on every increment)
//  - tanlambda:  anchor tl0 + offset dtl;  q/pT: anchor w0 + offset dw
//  - variances of tanlambda and q/pT: compensated sums c[9] + c9l, c[14] + c14l
//    (transport leaves them unchanged; after a restart they shrink by orders of
//    magnitude through many small decrements)
struct Trk {
  float dy, dz, sp, spl, tl0, dtl, w0, dw;
  float ya, za;
  float c[15];  // covariance, packed lower triangle
  float c9l, c14l;
  __device__ __forceinline__ float tl() const { return tl0 + dtl; }
  __device__ __forceinline__ float w() const { return w0 + dw; }
  __device__ __forceinline__ float snp() const { return sp + spl; }
};

// Exact helix transport x1 -> x1+dx with Jacobian applied to the covariance.
// Returns false on the |sinphi| limit (NaN passes).
__device__ __forceinline__ bool propagate(Trk &T, float dx, float b, float snp_max) {
  const float tl = T.tl();
  const float C = b * T.w();
  const float s1 = T.snp(), s2 = fmaf(C, dx, s1);
  if (fabsf(s1) >= snp_max || fabsf(s2) >= snp_max) return false;
  const float q1 = fmaf(-s1, s1, 1.0f), q2 = fmaf(-s2, s2, 1.0f);
  const float ic1 = rsqrtf(q1), ic2 = rsqrtf(q2);
  const float c1 = q1 * ic1, c2 = q2 * ic2;  // cos phi at both planes
  const float iB = __fdividef(1.0f, c1 + c2);
  const float Tn = (s1 + s2) * iB;           // tangent of the chord direction
  const float kk2 = fmaf(Tn, Tn, 1.0f);
  const float ik = rsqrtf(kk2);
  const float L = dx * (kk2 * ik);           // signed chord
  const float u = 0.5f * C * L;
  const float u2 = u * u;
  float g, h;
  if (fabsf(u) < 0.1f) {
    g = 1.0f + u2 * (1.0f / 6.0f + u2 * (3.0f / 40.0f + u2 * (5.0f / 112.0f)));
    h = 1.0f / 6.0f + u2 * (3.0f / 20.0f + u2 * (15.0f / 112.0f + u2 * (35.0f / 288.0f)));
  } else {
    g = asinf(u) / u;
    h = (rsqrtf(1.0f - u2) - g) / (2.0f * u2);
  }
  const float sT = L * g;                    // signed transverse arc length
  T.dy = fmaf(dx, Tn, T.dy);
  T.dz = fmaf(tl, sT, T.dz);
  {  // sinphi += C dx, compensated
    float hi, e;
    two_sum(T.sp, C * dx, hi, e);
    T.sp = hi;
    T.spl += e;
  }
  // Jacobian
  const float Q = fmaf(c1, c2, fmaf(s1, s2, 1.0f)) * iB * iB;
  const float dTds = Q * (ic1 + ic2);
  const float bdx = b * dx;
  const float dTdw = Q * ic2 * bdx;
  const float Jys = dx * dTds, Jyw = dx * dTdw;
  const float dsdL = rsqrtf(fmaf(-u, u, 1.0f));
  const float dLdT = dx * Tn * ik;
  const float dsdC = L * L * u * h;
  const float a1 = dsdL * dLdT;
  const float Jzs = tl * a1 * dTds;
  const float Jzt = sT;
  const float Jzw = tl * fmaf(a1, dTdw, dsdC * b);
  const float Jsw = bdx;
  float *c = T.c;
  // F C (rows 0..2 differ from C), entries needed by F C F^T
  const float FC00 = fmaf(Jys, c[3], fmaf(Jyw, c[10], c[0]));
  const float FC02 = fmaf(Jys, c[5], fmaf(Jyw, c[12], c[3]));
  const float FC04 = fmaf(Jys, c[12], fmaf(Jyw, c[14], c[10]));
  const float FC10 = fmaf(Jzs, c[3], fmaf(Jzt, c[6], fmaf(Jzw, c[10], c[1])));
  const float FC11 = fmaf(Jzs, c[4], fmaf(Jzt, c[7], fmaf(Jzw, c[11], c[2])));
  const float FC12 = fmaf(Jzs, c[5], fmaf(Jzt, c[8], fmaf(Jzw, c[12], c[4])));
  const float FC13 = fmaf(Jzs, c[8], fmaf(Jzt, c[9], fmaf(Jzw, c[13], c[7])));
  const float FC14 = fmaf(Jzs, c[12], fmaf(Jzt, c[13], fmaf(Jzw, c[14], c[11])));
  const float FC20 = fmaf(Jsw, c[10], c[3]);
  const float FC21 = fmaf(Jsw, c[11], c[4]);
  const float FC22 = fmaf(Jsw, c[12], c[5]);
  const float FC23 = fmaf(Jsw, c[13], c[8]);
  const float FC24 = fmaf(Jsw, c[14], c[12]);
  // (F C) F^T, lower triangle; rows 3 and 4 of F C equal those of C
  const float n30 = fmaf(Jys, c[8], fmaf(Jyw, c[13], c[6]));
  const float n31 = fmaf(Jzs, c[8], fmaf(Jzt, c[9], fmaf(Jzw, c[13], c[7])));
  const float n32 = fmaf(Jsw, c[13], c[8]);
  const float n40 = fmaf(Jys, c[12], fmaf(Jyw, c[14], c[10]));
  const float n41 = fmaf(Jzs, c[12], fmaf(Jzt, c[13], fmaf(Jzw, c[14], c[11])));
  const float n42 = fmaf(Jsw, c[14], c[12]);
  c[0] = fmaf(Jys, FC02, fmaf(Jyw, FC04, FC00));
  c[1] = fmaf(Jys, FC12, fmaf(Jyw, FC14, FC10));
  c[2] = fmaf(Jzs, FC12, fmaf(Jzt, FC13, fmaf(Jzw, FC14, FC11)));
  c[3] = fmaf(Jys, FC22, fmaf(Jyw, FC24, FC20));
  c[4] = fmaf(Jzs, FC22, fmaf(Jzt, FC23, fmaf(Jzw, FC24, FC21)));
  c[5] = fmaf(Jsw, FC24, FC22);
  c[6] = n30;
  c[7] = n31;
  c[8] = n32;
  c[10] = n40;
  c[11] = n41;
  c[12] = n42;
  // c[9], c[13], c[14] unchanged
  return true;
}

// Highland multiple-scattering noise of one pad row.
__device__ __forceinline__ void ms_noise(Trk &T, float xx0, float mass2) {
  const float s = T.snp(), t = T.tl(), w = T.w();
  const float tt = fmaf(t, t, 1.0f);
  const float cs2 = fmaf(-s, s, 1.0f);
  const float itt = __fdividef(1.0f, tt);
  const float pinv2 = w * w * itt;                  // 1/p^2
  const float ib2 = fmaf(mass2, pinv2, 1.0f);       // 1/beta^2
  const float eps = xx0 * (tt * rsqrtf(tt * cs2));  // xx0 sqrt(tt / cs2)
  const float lg = fmaf(0.038f, __logf(eps * ib2), 1.0f);
  const float th2 = (0.0136f * 0.0136f) * pinv2 * ib2 * eps * lg * lg;
  T.c[5] = fmaf(th2, cs2 * tt, T.c[5]);
  fast_two_sum(T.c[9], fmaf(th2, tt * tt, T.c9l), T.c[9], T.c9l);
  fast_two_sum(T.c[14], fmaf(th2, w * w * t * t, T.c14l), T.c[14], T.c14l);
  T.c[13] = fmaf(th2, tt * w * t, T.c[13]);
}

// Error-free product of two binary32 numbers: a * b = p + e exactly.
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
  p = __fmul_rn(a, b);
  e = fmaf(a, b, -p);
}

// The quadratic form r^T adj(S) r = S11 r0^2 - 2 S10 r0 r1 + S00 r1^2 as an
// unevaluated sum qh + ql of two binary32 numbers, from error-free products
// and sums (the compensated dot product of Ogita, Rump and Oishi, 2005, in
// nested form r0 (S11 r0 - 2 S10 r1) + S00 r1 r1): relative error of order
// 2^-46 of the sum of the magnitudes of the three terms, which for a positive
// definite S bounds it by a small multiple of the form itself.  On GB300 these
// 31 binary32 operations cost less than the 5 binary64 ones they replace.
__device__ __forceinline__ void quad_form2(float S00, float S10, float S11, float r0, float r1, float &qh,
                                           float &ql) {
  float p1, e1, p2, e2, uh, ul, vh, t, tl, wh;
  two_prod(S11, r0, p1, e1);
  two_prod(-2.0f * S10, r1, p2, e2);  // -2 S10 exact
  two_sum(p1, p2, uh, ul);
  ul += e1 + e2;                       // u = S11 r0 - 2 S10 r1 = uh + ul
  vh = __fmul_rn(r0, uh);
  const float vl = fmaf(r0, ul, fmaf(r0, uh, -vh));  // r0 u = vh + vl
  two_prod(r1, r1, t, tl);
  wh = __fmul_rn(S00, t);
  const float wl = fmaf(S00, tl, fmaf(S00, t, -wh));  // S00 r1^2 = wh + wl
  two_sum(vh, wh, qh, ql);
  ql += vl + wl;
}

// Gated Kalman update with the cluster (yc, zc, vy, vz).  FP64 island: the
// determinant of S, and where the chi2 value is needed (inward pass,
// diagnostics) the reciprocal of det (Newton step from an FP32 seed), chi2 =
// q / det and (by the caller) the chi2 sum; otherwise the gate is decided in
// FP64 as q - chi2_max det <= 0.  The quadratic form q = r^T adj(S) r enters
// as the exact binary64 sum of its two binary32 parts.  Non-finite innovation
// matrices or residuals give chi2 = NaN and a rejected cluster, as in FP64.
// Returns the status (OK / NOT_PD).
__device__ __forceinline__ int update(Trk &T, float yc, float zc, float vy, float vz, double gate, uint32_t gate_hi,
                                      uint32_t gate_lo, bool want_chi2, bool &acc, double &chi2) {
  float *c = T.c;
  const float r0 = (yc - T.ya) - T.dy;
  const float r1 = (zc - T.za) - T.dz;
  const float S00 = c[0] + vy, S10 = c[1], S11 = c[2] + vz;
  float qh, ql;
  quad_form2(S00, S10, S11, r0, r1, qh, ql);
  const bool fin = fabsf((S00 + S11) + (S10 + qh)) < INFINITY;
  const float det32 = fmaf(S00, S11, -(S10 * S10));
  const float i32 = __fdividef(1.0f, det32);  // FP32 seed of 1/det, and the gain's 1/det
  // ---- FP64 island ----
  const double s00 = widen_pos(S00), s11 = widen_pos(S11), s10 = widen(S10);
  const double det = fma(s00, s11, -(s10 * s10));
  const double qhd = widen(qh), qld = widen(ql);
  if (want_chi2) {
    const double y0 = widen_pos(i32);
    const double ey = fma(-det, y0, 1.0);
    const double inv = fma(y0, ey, y0);  // 1/det, one Newton step
    chi2 = fma(qhd, inv, qld * inv);
    acc = le_finite64(chi2, gate_hi, gate_lo);
  } else {
    acc = le0_finite64(fma(-gate, det, qhd) + qld);
  }
  const bool notpd = fin && (le0_finite64(det) || !(S00 > 0.0f) || !(S11 > 0.0f));
  // ---- back to FP32 ----
  if (!fin) {
    acc = false;
    chi2 = __longlong_as_double(0x7ff8000000000000ll);
  }
  if (notpd) {
    acc = false;
    return ST_NOT_PD;
  }
  const float Si00 = S11 * i32, Si10 = -S10 * i32, Si11 = S00 * i32;
  if (acc) {
    float K0[5], K1[5];
    const int col0[5] = {0, 1, 3, 6, 10}, col1[5] = {1, 2, 4, 7, 11};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const float ci0 = c[col0[i]], ci1 = c[col1[i]];
      K0[i] = fmaf(ci0, Si00, ci1 * Si10);
      K1[i] = fmaf(ci0, Si10, ci1 * Si11);
    }
    // new position offsets relative to this cluster (the new anchor)
    T.dy = fmaf(K0[0] - 1.0f, r0, K1[0] * r1);
    T.dz = fmaf(K0[1], r0, (K1[1] - 1.0f) * r1);
    {
      float hi, e;
      two_sum(T.sp, fmaf(K0[2], r0, fmaf(K1[2], r1, T.spl)), hi, e);
      T.sp = hi;
      T.spl = e;
    }
    T.dtl = fmaf(K0[3], r0, fmaf(K1[3], r1, T.dtl));
    T.dw = fmaf(K0[4], r0, fmaf(K1[4], r1, T.dw));
    // C -= K (H C).  For the measured columns (j = y, z) this equals K V
    // exactly (C_iH - C_iH S^-1 C_HH = C_iH S^-1 V), computed without
    // cancellation; the angle block uses the subtraction form.
    float h0[5], h1[5];
#pragma unroll
    for (int j = 2; j < 5; ++j) {
      h0[j] = c[col0[j]];
      h1[j] = c[col1[j]];
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      c[col0[i]] = K0[i] * vy;  // C'(i,0)
      if (i >= 1) c[col1[i]] = K1[i] * vz;  // C'(i,1)
    }
    c[5] = fmaf(-K0[2], h0[2], fmaf(-K1[2], h1[2], c[5]));
    c[8] = fmaf(-K0[3], h0[2], fmaf(-K1[3], h1[2], c[8]));
    fast_two_sum(c[9], T.c9l - fmaf(K0[3], h0[3], K1[3] * h1[3]), c[9], T.c9l);
    c[12] = fmaf(-K0[4], h0[2], fmaf(-K1[4], h1[2], c[12]));
    c[13] = fmaf(-K0[4], h0[3], fmaf(-K1[4], h1[3], c[13]));
    fast_two_sum(c[14], T.c14l - fmaf(K0[4], h0[4], K1[4] * h1[4]), c[14], T.c14l);
  } else {
    T.dy = -r0;
    T.dz = -r1;
  }
  T.ya = yc;
  T.za = zc;
  return ST_OK;
}

__device__ __forceinline__ bool finite5(float a, float b, float c, float d, float e) {
  return isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d) && isfinite(e);
}

// ---------------------------------------------------------------------------
// k_fit: persistent warps over the (sorted) track list.
// ---------------------------------------------------------------------------
// Validation of a cluster when the outward pass reaches it (before any
// propagation towards it): row inside the geometry and above the previous
// one, finite values, positive variances.
__device__ __forceinline__ int check_cluster(int r, int rprev, int n_rows, float x, float y, float z, float vy,
                                             float vz) {
  if (r >= n_rows || r <= rprev) return ST_BAD_INPUT;
  if (!finite5(x, y, z, vy, vz)) return ST_NONFINITE;
  if (!(vy > 0.f) || !(vz > 0.f)) return ST_BAD_INPUT;
  return ST_OK;
}

struct Clu {
  float x, y, z, vy, vz;
  int r;
};

// Issue the copies of chunk c (clusters a+4c .. a+4c+3, clipped to the track)
// into buffer c&1 of this lane's staging column.  The chunk's four row bytes
// are copied as the two aligned 32-bit words that hold them (the second only
// when it holds a byte of the track; an aligned word that holds a byte of an
// allocation lies inside it, allocations being at least 4-byte granular).
template <int BLOCK>
__device__ __forceinline__ void stage_chunk(const FitArgs &A, int64_t a, int64_t e, int c, float *stg) {
  const int buf = c & 1;
  const int64_t k0 = a + (int64_t)kChunk * c;
  float *dst0 = stg + (buf * kStageArrays) * kChunk * BLOCK;
  if (k0 + kChunk <= e) {  // full chunk: four consecutive clusters of each array
    const float *src[kStageArrays] = {A.x + k0, A.y + k0, A.z + k0, A.sy2 + k0, A.sz2 + k0};
#pragma unroll
    for (int j = 0; j < kStageArrays; ++j)
#pragma unroll
      for (int s = 0; s < kChunk; ++s) cp_async4(dst0 + (j * kChunk + s) * BLOCK, src[j] + s, true);
  } else {  // the track's last chunk: slots past the end are zero-filled from an in-range address
#pragma unroll
    for (int s = 0; s < kChunk; ++s) {
      const int64_t k = k0 + s;
      const bool v = k < e;
      const int64_t kk = v ? k : e - 1;
      float *dst = dst0 + s * BLOCK;
      cp_async4(dst + 0 * kChunk * BLOCK, A.x + kk, v);
      cp_async4(dst + 1 * kChunk * BLOCK, A.y + kk, v);
      cp_async4(dst + 2 * kChunk * BLOCK, A.z + kk, v);
      cp_async4(dst + 3 * kChunk * BLOCK, A.sy2 + kk, v);
      cp_async4(dst + 4 * kChunk * BLOCK, A.sz2 + kk, v);
    }
  }
  const uint8_t *p0 = A.row + k0;
  const uint32_t *w0 = reinterpret_cast<const uint32_t *>(reinterpret_cast<uintptr_t>(p0) & ~(uintptr_t)3);
  const bool v1 = reinterpret_cast<const uint8_t *>(w0 + 1) < A.row + e;
  float *rdst = stg + (kStageFloats + 2 * buf) * BLOCK;
  cp_async4(rdst, w0, true);
  cp_async4(rdst + BLOCK, v1 ? w0 + 1 : w0, v1);
  cp_async_commit();
}

// Rows of the staged chunk c (current), one byte per cluster; `rsh` is the
// byte offset of the track's first row byte within its aligned word.
template <int BLOCK>
__device__ __forceinline__ uint32_t staged_rows(const float *stg, int c, uint32_t rsh) {
  const float *src = stg + (kStageFloats + 2 * (c & 1)) * BLOCK;
  return __funnelshift_r(__float_as_uint(src[0]), __float_as_uint(src[BLOCK]), 8u * rsh);
}

// Cluster lk of the track from the staged chunk lk/4 (which must be current).
template <int BLOCK>
__device__ __forceinline__ Clu read_staged(const float *stg, int lk, uint32_t rows_cur) {
  const int ch = lk / kChunk, slot = lk % kChunk;
  const float *src = stg + (((ch & 1) * kStageArrays) * kChunk + slot) * BLOCK;
  Clu c;
  c.x = src[0];
  c.y = src[kChunk * BLOCK];
  c.z = src[2 * kChunk * BLOCK];
  c.vy = src[3 * kChunk * BLOCK];
  c.vz = src[4 * kChunk * BLOCK];
  c.r = (rows_cur >> (8 * slot)) & 0xffu;
  return c;
}

// ---------------------------------------------------------------------------
// Track-model compression residuals (Sec. 5: TPC clusters are stored as
// residuals to their track instead of absolute coordinates).  The fitted
// helix (state at x0, no scattering) is evaluated at each cluster's x in one
// exact step of the chord form; the residual is quantised to an int16 code.
// ---------------------------------------------------------------------------
// (y, z) of the helix through (y0, z0) at x0 with sinphi s0, tanlambda tl and
// curvature C, at x0 + dx; false if the helix does not reach that plane.
// Correctly rounded division and square roots: this pass is off the hot loop.
__device__ __forceinline__ bool helix_at(float y0, float z0, float s0, float tl, float C, float dx, float &y,
                                         float &z) {
  const float s2 = fmaf(C, dx, s0);
  if (!(fabsf(s0) < 1.0f) || !(fabsf(s2) < 1.0f)) return false;
  const float c1 = sqrtf(fmaf(-s0, s0, 1.0f)), c2 = sqrtf(fmaf(-s2, s2, 1.0f));
  const float Tn = (s0 + s2) / (c1 + c2);  // tangent of the chord direction
  const float L = dx * sqrtf(fmaf(Tn, Tn, 1.0f));
  const float u = 0.5f * C * L;            // sine of half the turning angle
  float g;                                 // arc / chord = asin(u) / u
  if (fabsf(u) < 0.1f) {
    const float u2 = u * u;
    g = 1.0f + u2 * (1.0f / 6.0f + u2 * (3.0f / 40.0f + u2 * (5.0f / 112.0f)));
  } else {
    g = asinf(u) / u;
  }
  y = fmaf(dx, Tn, y0);
  z = fmaf(tl, L * g, z0);
  return isfinite(y) && isfinite(z);
}

// Residual in code units -> int16 code: round half to even, clipped to
// +-32767; -32768 (not encoded) for a non-finite residual.
__device__ __forceinline__ int16_t res_code(float r, float inv_step) {
  const float q = r * inv_step;
  if (isnan(q)) return (int16_t)-32768;
  if (!(fabsf(q) < 32767.5f)) return q > 0.0f ? (int16_t)32767 : (int16_t)-32767;
  return (int16_t)__float2int_rn(q);
}

template <int BLOCK>
__device__ void fit_track(const FitArgs &A, int64_t t, uint32_t *bits, const float *s_rowx, float *stg) {
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
  T.c9l = 0.f;
  T.c14l = 0.f;
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
    for (int w = 0; w < kBitWords; ++w) bits[32 * w] = 0u;
    uint8_t *const acc_t = A.accept + a;  // this track's accept bytes
    int done = 0;      // clusters (from the outer end) whose accept byte is final
    int out_done = 0;  // clusters the outward pass updated with
    if (st0 == ST_OK) {
      uint32_t gate_hi, gate_lo;
      split64(A.chi2_max_d, gate_hi, gate_lo);
      int nacc_out = 0;
      // candidate: the next cluster to use, read from the lane's staged chunk;
      // the following chunk is in flight (cp.async) while this one is used
      const int nch = (n + kChunk - 1) / kChunk;
      int kc = 0;
      const uint32_t rsh = (uint32_t)(reinterpret_cast<uintptr_t>(A.row + a) & 3u);
      stage_chunk<BLOCK>(A, a, e, 0, stg);
      cp_async_wait_all();
      uint32_t rows_cur = staged_rows<BLOCK>(stg, 0, rsh);
      if (nch > 1) stage_chunk<BLOCK>(A, a, e, 1, stg);
      Clu cand = read_staged<BLOCK>(stg, 0, rows_cur);
      int rprev = -1;
      st = check_cluster(cand.r, rprev, A.n_rows, cand.x, cand.y, cand.z, cand.vy, cand.vz);
      // ---------------- outward pass: rows row[0] .. row[n-1] ----------------
      for (int r = cand.r; st == ST_OK; ++r) {
        const bool has = (cand.r == r);
        const float xt = has ? cand.x : s_rowx[r];
        if (!propagate(T, xt - xcur, A.b, A.snp_max)) { st = ST_SNP_LIMIT; break; }
        xcur = xt;
        if (has) {
          bool acc;
          double chi2;
          const int ust = update(T, cand.y, cand.z, cand.vy, cand.vz, A.chi2_max_d, gate_hi, gate_lo,
                                 A.chi2_out_c != nullptr, acc, chi2);
          if (ust != ST_OK) { st = ust; break; }
          if (acc) bits[32 * (kc >> 5)] |= 1u << (kc & 31);
          if (A.chi2_out_c) A.chi2_out_c[a + kc] = chi2;
          ++out_done;
          nacc_out += acc ? 1 : 0;
          rprev = cand.r;
          if (++kc < n) {
            if (kc % kChunk == 0) {  // entering chunk kc/4
              cp_async_wait_all();
              rows_cur = staged_rows<BLOCK>(stg, kc / kChunk, rsh);
              if (kc / kChunk + 1 < nch) stage_chunk<BLOCK>(A, a, e, kc / kChunk + 1, stg);
            }
            cand = read_staged<BLOCK>(stg, kc, rows_cur);
            const int vs = check_cluster(cand.r, rprev, A.n_rows, cand.x, cand.y, cand.z, cand.vy, cand.vz);
            if (vs != ST_OK) { st = vs; break; }
          }
        }
        if (A.xx0 > 0.f) ms_noise(T, A.xx0, A.mass2);
        if (kc == n) break;
      }
      // ---------------- restart ----------------
      if (st == ST_OK) {
        // cand holds the outermost cluster n-1
        if (10 * nacc_out < 9 * n) {
          // the outward pass accepted fewer than 90 % of the clusters: re-seed
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
          const float d2 = fminf(A.restart_scale * T.c[5], A.seed_cov[2]);
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
        T.c9l = 0.f;
        T.c14l = 0.f;
        if (A.restart_state) {
          float *rs = A.restart_state + 5 * t;
          rs[0] = T.ya + T.dy;
          rs[1] = T.za + T.dz;
          rs[2] = T.snp();
          rs[3] = T.tl();
          rs[4] = T.w();
        }
        // ---------------- inward pass: rows row[n-1] .. row[0] ----------------
        kc = n - 1;
        // the last chunk is current; restage the one below it into the other buffer
        if (nch > 1) stage_chunk<BLOCK>(A, a, e, nch - 2, stg);
        for (int r = cand.r;; --r) {
          const bool has = (cand.r == r);
          const float xt = has ? cand.x : s_rowx[r];
          if (!propagate(T, xt - xcur, A.b, A.snp_max)) { st = ST_SNP_LIMIT; break; }
          xcur = xt;
          if (has) {
            bool acc;
            double chi2;
            const int ust = update(T, cand.y, cand.z, cand.vy, cand.vz, A.chi2_max_d, gate_hi, gate_lo, true, acc,
                                   chi2);
            if (ust != ST_OK) { st = ust; break; }
            if (A.chi2_in_c) A.chi2_in_c[a + kc] = chi2;
            chi2sum += __longlong_as_double(acc ? __double_as_longlong(chi2) : 0ll);
            nacc += acc ? 1 : 0;
            const uint32_t ob = (bits[32 * (kc >> 5)] >> (kc & 31)) & 1u;
            acc_t[kc] = (uint8_t)(ob | (acc ? 2u : 0u));
            ++done;
            if (--kc >= 0) {
              if (kc % kChunk == kChunk - 1) {  // entering chunk kc/4 from above
                cp_async_wait_all();
                rows_cur = staged_rows<BLOCK>(stg, kc / kChunk, rsh);
                if (kc / kChunk > 0) stage_chunk<BLOCK>(A, a, e, kc / kChunk - 1, stg);
              }
              cand = read_staged<BLOCK>(stg, kc, rows_cur);
            }
          }
          if (A.xx0 > 0.f) ms_noise(T, A.xx0, A.mass2);
          if (kc < 0) break;
        }
      }
      cp_async_wait_all();  // no copy may land in the column after this track
      if (st == ST_OK) {
        bool fin = isfinite(T.dy) && isfinite(T.dz) && isfinite(T.snp()) && isfinite(T.tl()) && isfinite(T.w());
#pragma unroll
        for (int i = 0; i < 15; ++i) fin = fin && isfinite(T.c[i]);
        if (!fin) st = ST_NONFINITE;
      }
    }
    // accept bytes not written by the inward pass (failed or unfitted tracks): outward bits only
    for (int64_t k = a; k < e - done; ++k) {
      const int lk = (int)(k - a);
      A.accept[k] = (lk < kMaxRows) ? (uint8_t)((bits[32 * (lk >> 5)] >> (lk & 31)) & 1u) : (uint8_t)0;
    }
    if (A.chi2_in_c)
      for (int64_t k = a; k < e - done; ++k) A.chi2_in_c[k] = __longlong_as_double(0x7ff8000000000000ll);
    if (A.chi2_out_c)
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
  T.c[9] += T.c9l;
  T.c[14] += T.c14l;
#pragma unroll
  for (int i = 0; i < 15; ++i) pc[i] = T.c[i];
  A.chi2[t] = chi2sum;
  A.ndf[t] = 2 * nacc - 5;
  A.status[t] = st;
}

template <int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_fit(FitArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  float *s_rowx = reinterpret_cast<float *>(smem);
  uint32_t *s_bits = reinterpret_cast<uint32_t *>(smem + kSmemRowx);
  float *s_stage = reinterpret_cast<float *>(smem + kSmemRowx + smem_bits<BLOCK>());
  for (int i = threadIdx.x; i < kMaxRows; i += blockDim.x) s_rowx[i] = A.row_x[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t *bits = s_bits + wib * kBitWords * 32 + lane;  // word w of this lane at bits[32*w]
  float *stg = s_stage + threadIdx.x;                      // this lane's staging column
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(A.work, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= (unsigned long long)A.n_tracks) break;
    const int64_t i = (int64_t)base + lane;
    if (i < A.n_tracks) {
      const int64_t t = A.perm ? (int64_t)A.perm[i] : i;
      fit_track<BLOCK>(A, t, bits, s_rowx, stg);
    }
    __syncwarp();
  }
}

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
  T.c9l = T.c14l = 0.f;
  uint32_t gate_hi, gate_lo;
  split64(A.chi2_max_d, gate_hi, gate_lo);
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
    int32_t best = -1;
    int64_t bpos = -1;
    float bchi = INFINITY;
    const float S01 = T.c[1];
    for (int iz = iz0; iz <= iz1; ++iz) {
      const int64_t row0 = (base + iz) * A.ny;
      const uint32_t q0 = A.cell_start[row0 + iy0], q1 = A.cell_start[row0 + iy1 + 1];
      for (uint32_t q = q0; q < q1; ++q) {
        const float r0v = (A.cy[q] - T.ya) - T.dy, r1v = (A.cz[q] - T.za) - T.dz;
        if (fabsf(r0v) > wy || fabsf(r1v) > wz) continue;
        const float S00 = T.c[0] + A.cvy[q], S11 = T.c[2] + A.cvz[q];
        const float det = fmaf(S00, S11, -S01 * S01);
        const float chi = (r0v * fmaf(S11, r0v, -S01 * r1v) + r1v * fmaf(S00, r1v, -S01 * r0v)) / det;
        const int32_t k = A.cidx[q];
        if (chi < bchi || (chi == bchi && k < best)) {
          bchi = chi;
          best = k;
          bpos = q;
        }
      }
    }
    bool acc = false;
    if (best >= 0) {
      double chi2;
      const int ust = update(T, A.cy[bpos], A.cz[bpos], A.cvy[bpos], A.cvz[bpos], A.chi2_max_d, gate_hi, gate_lo,
                             false, acc, chi2);
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
template <int BLOCK, int MINB> static cudaError_t set_fit_smem() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(k_fit<BLOCK, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fit_smem<BLOCK>());
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
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

cudaError_t launch_fit(const FitArgs &a, int grid, int block, cudaStream_t stream) {
  if (a.n_tracks <= 0) return cudaSuccess;
  cudaError_t e;
  if (block == 128) {
    if ((e = set_fit_smem<128, 4>()) != cudaSuccess) return e;
    k_fit<128, 4><<<grid, 128, fit_smem<128>(), stream>>>(a);
  } else {
    if ((e = set_fit_smem<256, 2>()) != cudaSuccess) return e;
    k_fit<256, 2><<<grid, 256, fit_smem<256>(), stream>>>(a);
  }
  return cudaGetLastError();
}

int fit_blocks_per_sm(int block) {
  int n = 0;
  cudaError_t e;
  if (block == 128) {
    set_fit_smem<128, 4>();
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fit<128, 4>, 128, fit_smem<128>());
  } else {
    set_fit_smem<256, 2>();
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fit<256, 2>, 256, fit_smem<256>());
  }
  if (e != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

// Resident blocks per SM when the caller leaves the choice to the library:
// 512 tracks per SM.  With 768 tracks per SM in flight their clusters do not
// stay in L2 between the outward and the inward pass (DRAM reads of 170 B per
// cluster against 60 B with 512, measured on GB300), so the instantiations are
// compiled for 512 threads per SM (up to 128 registers per thread).
int fit_default_blocks_per_sm(int block) {
  const int occ = fit_blocks_per_sm(block);
  const int want = 512 / (block == 128 ? 128 : 256);
  return occ < want ? occ : want;
}

int fit_regs_per_thread() {
  cudaFuncAttributes at;
  if (cudaFuncGetAttributes(&at, k_fit<256, 2>) != cudaSuccess) return -1;
  return at.numRegs;
}

}  // namespace tpcfit
