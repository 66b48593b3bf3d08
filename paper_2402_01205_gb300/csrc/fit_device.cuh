// Device code shared by the fit kernel (fit_kernels.cu) and the track
// following and residual kernels (track_kernels.cu): track state, exact
// helix propagation with covariance transport, Highland scattering, the
// gated Kalman update with its FP64 island, and the fitted-helix residuals.
#pragma once

#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>

namespace tpcfit {

enum { ST_OK = 0, ST_TOO_FEW = 1, ST_SNP_LIMIT = 2, ST_NOT_PD = 3, ST_NONFINITE = 4, ST_BAD_INPUT = 5,
       ST_STOPPED = 6, ST_DERAILED = 7 };

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

// ---------------------------------------------------------------------------
// FP32 arithmetic of the fit, every operation rounded as written: vmul and
// vadd are never contracted into a fused multiply-add (vfma is one), so the
// error-free transformations below hold and the results do not depend on the
// compiler's contraction choices.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Error-free sum of two binary32 numbers (Knuth's TwoSum): a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = vadd(a, b);
  const float bb = vsub(s, a);
  e = vadd(vsub(a, vsub(s, bb)), vsub(b, bb));
}
// Dekker's Fast2Sum: the same when |a| >= |b| (a variance plus a smaller
// increment, or minus a smaller decrement).
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = vadd(a, b);
  e = vsub(b, vsub(s, a));
}
// Two Fast2Sums at once, (a0 + b0, a1 + b1) = (s0 + e0, s1 + e1), with the
// paired binary32 instructions of sm_100 and later (each half rounds as the
// scalar instruction does; s - a and b - z as fused multiply-adds by -1,
// which round the difference once).
__device__ __forceinline__ void fast_two_sum_x2(float a0, float a1, float b0, float b1, float &s0, float &s1,
                                                float &e0, float &e1) {
  const float2 m1 = make_float2(-1.0f, -1.0f);
  const float2 a = make_float2(a0, a1), b = make_float2(b0, b1);
  const float2 s = __fadd2_rn(a, b);
  const float2 e = __ffma2_rn(__ffma2_rn(a, m1, s), m1, b);  // b - (s - a)
  s0 = s.x;
  s1 = s.y;
  e0 = e.x;
  e1 = e.y;
}
// Error-free product of two binary32 numbers: a * b = p + e exactly.
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
  p = vmul(a, b);
  e = vfma(a, b, -p);
}

// ---------------------------------------------------------------------------
// Fit of one track: device helpers.
// ---------------------------------------------------------------------------
// Track state in FP32 with extended precision where the Kalman recursion
// accumulates many small increments onto a large value:
//  - y, z:       offsets (dy, dz) from the last cluster's coordinates (ya, za)
//  - sinphi:     compensated sum sp + spl
//  - tanlambda:  anchor tl0 + offset dtl;  q/pT: anchor w0 + offset dw
//  - variances of tanlambda and q/pT: compensated sums c[9] + c9l, c[14] + c14l
//    (transport leaves them unchanged; after a restart they shrink by orders of
//    magnitude through many small decrements)
//  - variance of sinphi and its covariance with q/pT: compensated sums
//    c[5] + c5l, c[12] + c12l.  On a curved track sinphi and q/pT become
//    almost fully correlated, and binary32 storage of these two entries
//    alone (every other step in FP64) moves the fitted covariance of a track
//    that was lost and found again in the outward pass by up to 1.2e-4 of
//    its diagonal; with them compensated, by less than 2e-5.
// Each compensated sum adds (increment + low part) to the high part with
// Fast2Sum, which is exact when the high part is the larger; where an
// increment exceeds it (a covariance or sinphi passing through zero) that
// step's error is at most half a binary32 ulp of the increment, i.e. the
// step is as accurate as an uncompensated binary32 sum of small values.
// The sums are done in pairs with the paired binary32 instructions.
struct Trk {
  float dy, dz, sp, spl, tl0, dtl, w0, dw;
  float ya, za;
  float c[15];  // covariance, packed lower triangle
  float c9l, c14l, c5l, c12l, c3l;
  __device__ __forceinline__ void clear_comp() { c9l = c14l = c5l = c12l = c3l = 0.f; }
  // the covariance with the compensation terms added in (binary32)
  __device__ __forceinline__ void fold_comp() {
    c[3] = vadd(c[3], c3l);
    c[5] = vadd(c[5], c5l);
    c[9] = vadd(c[9], c9l);
    c[12] = vadd(c[12], c12l);
    c[14] = vadd(c[14], c14l);
    clear_comp();
  }
  __device__ __forceinline__ float tl() const { return vadd(tl0, dtl); }
  __device__ __forceinline__ float w() const { return vadd(w0, dw); }
  __device__ __forceinline__ float snp() const { return vadd(sp, spl); }
};

// Exact helix transport x1 -> x1+dx with Jacobian applied to the covariance.
// Returns false on the |sinphi| limit (NaN passes), with T unchanged.
__device__ __forceinline__ bool propagate(Trk &T, float dx, float b, float snp_max) {
  const float tl = T.tl();
  const float C = vmul(b, T.w());
  const float s1 = T.snp(), s2 = vfma(C, dx, s1);
  if (fabsf(s1) >= snp_max || fabsf(s2) >= snp_max) return false;
  const float q1 = vfma(-s1, s1, 1.0f), q2 = vfma(-s2, s2, 1.0f);
  const float ic1 = rsqrtf(q1), ic2 = rsqrtf(q2);
  const float2 cc = __fmul2_rn(make_float2(q1, q2), make_float2(ic1, ic2));
  const float c1 = cc.x, c2 = cc.y;  // cos phi at both planes
  const float iB = __fdividef(1.0f, vadd(c1, c2));
  const float Tn = vmul(vadd(s1, s2), iB);             // tangent of the chord direction
  const float kk2 = vfma(Tn, Tn, 1.0f);
  const float ik = rsqrtf(kk2);
  const float L = vmul(dx, vmul(kk2, ik));             // signed chord
  const float u = vmul(vmul(0.5f, C), L);
  const float u2 = vmul(u, u);
  // arc / chord g = asin(u)/u and h = (g' / u) / 2 = (1/sqrt(1-u^2) - g) / (2 u^2):
  // series for |u| < 0.1, else the functions themselves
  float g, h;
  if (fabsf(u) < 0.1f) {
    g = vfma(u2, vfma(u2, vfma(u2, 5.0f / 112.0f, 3.0f / 40.0f), 1.0f / 6.0f), 1.0f);
    h = vfma(u2, vfma(u2, vfma(u2, 35.0f / 288.0f, 15.0f / 112.0f), 3.0f / 20.0f), 1.0f / 6.0f);
  } else {
    g = asinf(u) / u;
    h = (rsqrtf(1.0f - u2) - g) / (2.0f * u2);
  }
  const float sT = vmul(L, g);                         // signed transverse arc length
  {
    const float2 d = __ffma2_rn(make_float2(dx, tl), make_float2(Tn, sT), make_float2(T.dy, T.dz));
    T.dy = d.x;
    T.dz = d.y;
  }
  // Jacobian
  const float Q = vmul(vmul(vfma(c1, c2, vfma(s1, s2, 1.0f)), iB), iB);
  const float dTds = vmul(Q, vadd(ic1, ic2));
  const float bdx = vmul(b, dx);
  const float dTdw = vmul(vmul(Q, ic2), bdx);
  const float Jys = vmul(dx, dTds), Jyw = vmul(dx, dTdw);
  const float dsdL = rsqrtf(vfma(-u, u, 1.0f));
  const float dLdT = vmul(vmul(dx, Tn), ik);
  const float dsdC = vmul(vmul(vmul(L, L), u), h);
  const float a1 = vmul(dsdL, dLdT);
  const float Jzs = vmul(vmul(tl, a1), dTds);
  const float Jzt = sT;
  const float Jzw = vmul(tl, vfma(a1, dTdw, vmul(dsdC, b)));
  const float Jsw = bdx;
  float *c = T.c;
  // F C (rows 0..2 differ from C), entries needed by F C F^T
  const float FC00 = vfma(Jys, c[3], vfma(Jyw, c[10], c[0]));
  const float FC02 = vfma(Jys, c[5], vfma(Jyw, c[12], c[3]));
  const float FC04 = vfma(Jys, c[12], vfma(Jyw, c[14], c[10]));
  const float FC10 = vfma(Jzs, c[3], vfma(Jzt, c[6], vfma(Jzw, c[10], c[1])));
  const float FC11 = vfma(Jzs, c[4], vfma(Jzt, c[7], vfma(Jzw, c[11], c[2])));
  const float FC12 = vfma(Jzs, c[5], vfma(Jzt, c[8], vfma(Jzw, c[12], c[4])));
  const float FC13 = vfma(Jzs, c[8], vfma(Jzt, c[9], vfma(Jzw, c[13], c[7])));
  const float FC14 = vfma(Jzs, c[12], vfma(Jzt, c[13], vfma(Jzw, c[14], c[11])));
  const float FC21 = vfma(Jsw, c[11], c[4]);
  const float FC22 = vfma(Jsw, c[12], c[5]);
  const float FC23 = vfma(Jsw, c[13], c[8]);
  const float FC24 = vfma(Jsw, c[14], c[12]);
  // (F C) F^T, lower triangle; rows 3 and 4 of F C equal those of C, so
  // entries (3,1), (4,0) and (4,1) are FC13, FC04 and FC14
  const float n30 = vfma(Jys, c[8], vfma(Jyw, c[13], c[6]));
  const float n32 = vfma(Jsw, c[13], c[8]);
  // compensated C_sw' = C_sw + Jsw C_ww and C_ss' = C_ss + Jsw (2 C_sw + Jsw C_ww)
  const float dsw = vmul(Jsw, vadd(c[14], T.c14l));
  const float dss = vmul(Jsw, vfma(2.0f, c[12], dsw));
  c[0] = vfma(Jys, FC02, vfma(Jyw, FC04, FC00));
  c[1] = vfma(Jys, FC12, vfma(Jyw, FC14, FC10));
  c[2] = vfma(Jzs, FC12, vfma(Jzt, FC13, vfma(Jzw, FC14, FC11)));
  c[4] = vfma(Jzs, FC22, vfma(Jzt, FC23, vfma(Jzw, FC24, FC21)));
  // compensated sums, two at a time: (C_ys, C_ss) and (sinphi, C_sw)
  fast_two_sum_x2(c[3], c[5], vfma(Jys, FC22, vfma(Jyw, FC24, vfma(Jsw, c[10], T.c3l))), vadd(dss, T.c5l), c[3],
                  c[5], T.c3l, T.c5l);
  fast_two_sum_x2(T.sp, c[12], vfma(C, dx, T.spl), vadd(dsw, T.c12l), T.sp, c[12], T.spl, T.c12l);
  c[6] = n30;
  c[7] = FC13;
  c[8] = n32;
  c[10] = FC04;
  c[11] = FC14;
  // c[9], c[13], c[14] unchanged
  return true;
}

// Highland multiple-scattering noise of one pad row.
__device__ __forceinline__ void ms_noise(Trk &T, float xx0, float mass2) {
  const float s = T.snp(), t = T.tl(), w = T.w();
  const float tt = vfma(t, t, 1.0f);
  const float cs2 = vfma(-s, s, 1.0f);
  const float itt = __fdividef(1.0f, tt);
  const float pinv2 = vmul(vmul(w, w), itt);                    // 1/p^2
  const float ib2 = vfma(mass2, pinv2, 1.0f);                   // 1/beta^2
  const float eps = vmul(xx0, vmul(tt, rsqrtf(vmul(tt, cs2))));  // xx0 sqrt(tt / cs2)
  const float lg = vfma(0.038f, __logf(vmul(eps, ib2)), 1.0f);
  const float th2 = vmul(vmul(vmul(vmul(vmul(0.0136f * 0.0136f, pinv2), ib2), eps), lg), lg);
  fast_two_sum(T.c[5], vfma(th2, vmul(cs2, tt), T.c5l), T.c[5], T.c5l);
  fast_two_sum_x2(T.c[9], T.c[14], vfma(th2, vmul(tt, tt), T.c9l), vfma(th2, vmul(vmul(vmul(w, w), t), t), T.c14l),
                  T.c[9], T.c[14], T.c9l, T.c14l);
  T.c[13] = vfma(th2, vmul(vmul(tt, w), t), T.c[13]);
}

// Mean stopping power (Bethe formula, PDG Review of Particle Physics, passage
// of particles through matter; |charge| 1, no density effect) from 1/p^2.
// With m2p = m^2/p^2:  1/beta^2 = 1 + m2p,  (beta gamma)^2 = bg2 = min(1/m2p, 1e10),
//   W_max = 2 m_e bg2 / D,  D = 1 + 2 gamma m_e/M + (m_e/M)^2,
//   -dE/dx = K Z/A (1/beta^2) [ln(2 m_e bg2 W_max / I^2)/2 - beta^2]
//          = kza ((1/beta^2) ln(a^2/D)/2 - 1),  a = (2 m_e / I) bg2,
// clamped at 0 where the formula turns negative (GeV cm^2/g).
__device__ __forceinline__ float stopping_power(float pinv2, float kza, float a_coef, float ratio, float mass2) {
  const float m2p = mass2 * pinv2;
  const float ib2 = 1.0f + m2p;
  const float bg2 = fminf(1.0f / m2p, 1e10f);
  const float gam = sqrtf(1.0f + bg2);
  const float aa = a_coef * bg2;
  const float D = fmaf(2.0f * gam, ratio, fmaf(ratio, ratio, 1.0f));
  return fmaxf(kza * fmaf(0.5f * ib2, logf(aa * (aa / D)), -1.0f), 0.0f);
}

// The energy-loss layer of one pad row: x rho along the row normal, so
// xrho / (cos lambda cos phi) along the path.  dir = +1 (outward: the particle
// loses dE, evaluated at its momentum before the layer) or -1 (inward: the
// loss is added back; the energy before the layer solves E_b - dE(E_b) = E,
// taken with one fixed-point step from dE(E), error O(dE^3)).
// p'^2 = p^2 (1 - r) with r = s (2E - s) / p^2, s = dir dE, written without
// E - m cancellation; q/pT grows by k = (1 - r)^-1/2, applied as w (k - 1) with
// k - 1 = r / (sqrt(1-r) (1 + sqrt(1-r))), exact to rounding even when r is
// of order 1e-7; row/column 4 of the covariance scale by k.  Returns false
// when |r| > 1/2 (the fit stops there); momenta above 1e15 GeV lose nothing.
__device__ __forceinline__ bool eloss(Trk &T, float xrho, float kza, float a_coef, float ratio, float mass2,
                                      float dir) {
  const float s = T.snp(), t = T.tl(), w = T.w();
  const float tt = fmaf(t, t, 1.0f);
  const float cs2 = fmaf(-s, s, 1.0f);
  const float pinv2 = (w * w) / tt;  // 1/p^2
  if (!(pinv2 > 1e-30f)) return true;
  const float path = xrho * sqrtf(tt / cs2);
  const float e2p = 2.0f * sqrtf(fmaf(mass2, pinv2, 1.0f) * pinv2);  // 2 E / p^2
  float sd = dir * (stopping_power(pinv2, kza, a_coef, ratio, mass2) * path);
  float r = sd * fmaf(-sd, pinv2, e2p);
  if (dir < 0.0f) {
    if (fabsf(r) > 0.5f) return false;
    sd = -(stopping_power(pinv2 / (1.0f - r), kza, a_coef, ratio, mass2) * path);
    r = sd * fmaf(-sd, pinv2, e2p);
  }
  if (fabsf(r) > 0.5f) return false;
  const float q = sqrtf(1.0f - r);
  const float km1 = r / (q * (1.0f + q));
  T.dw = fmaf(w, km1, T.dw);
  const float k = 1.0f + km1, k2 = k * k;
  T.c[10] *= k;
  T.c[11] *= k;
  T.c[12] *= k;
  T.c12l *= k;
  T.c[13] *= k;
  T.c[14] *= k2;
  T.c14l *= k2;
  return true;
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
  float p1, e1, p2, e2, uh, ul, t, tl;
  two_prod(S11, r0, p1, e1);
  two_prod(vmul(-2.0f, S10), r1, p2, e2);  // -2 S10 exact
  two_sum(p1, p2, uh, ul);
  ul = vadd(ul, vadd(e1, e2));             // u = S11 r0 - 2 S10 r1 = uh + ul
  const float vh = vmul(r0, uh);
  const float vl = vfma(r0, ul, vfma(r0, uh, -vh));  // r0 u = vh + vl
  two_prod(r1, r1, t, tl);
  const float wh = vmul(S00, t);
  const float wl = vfma(S00, tl, vfma(S00, t, -wh));  // S00 r1^2 = wh + wl
  two_sum(vh, wh, qh, ql);
  ql = vadd(ql, vadd(vl, wl));
}

// The chi2 gate of the Kalman update: chi2_max (configured in binary32) as
// binary64, its two 32-bit halves (integer comparisons of FP64 values) and
// as binary32.
struct Gate {
  double d;
  uint32_t hi, lo;
  float f;
};
__device__ __forceinline__ Gate make_gate(float chi2_max, double chi2_max_d) {
  Gate g;
  g.d = chi2_max_d;
  split64(chi2_max_d, g.hi, g.lo);
  g.f = chi2_max;
  return g;
}

// Gated Kalman update with the cluster (yc, zc, vy, vz).  FP64 island: the
// inversion of S -- its determinant det = S00 S11 - S10^2 (the products of
// the binary32 entries are exact in binary64, rounded once) and, where the
// chi2 value is needed (inward pass, diagnostics), chi2 = q / det with one
// FP64 Newton correction of the binary32 reciprocal, and (by the caller) the
// chi2 sum.  The quadratic form q = r^T adj(S) r is an unevaluated sum of two
// binary32 numbers (quad_form2).  Without the chi2 value the gate
// q - chi2_max det <= 0 is decided in binary32 from det narrowed toward zero
// when its margin exceeds 2^-19 of the magnitudes of its terms (every rounding
// of that evaluation stays below 2^-21 of them, so its sign is that of the
// exact value, which the FP64 evaluation also gives), else in FP64: the same
// decision as the FP64 evaluation, at 2 FP64 operations per outward update
// instead of 4.  The gain's S^-1 = adj(S) / det takes its 1/det from the FP64
// determinant (narrowed to binary32 by integer operations), so that the
// cancellation in det of a strongly correlated S does not reach the gain.
// Non-finite innovation matrices or residuals give chi2 = NaN and a rejected
// cluster, as in FP64.  Returns the status (OK, or NOT_PD with T unchanged).
__device__ __forceinline__ int update(Trk &T, float yc, float zc, float vy, float vz, const Gate &G, bool want_chi2,
                                      bool &acc, double &chi2) {
  float *c = T.c;
  // residual (yc - ya) - dy, (zc - za) - dz as a pair (a fused multiply-add by -1 rounds a difference once)
  const float2 m1 = make_float2(-1.0f, -1.0f);
  const float2 rr =
      __ffma2_rn(make_float2(T.dy, T.dz), m1, __ffma2_rn(make_float2(T.ya, T.za), m1, make_float2(yc, zc)));
  const float r0 = rr.x, r1 = rr.y;
  const float S00 = vadd(c[0], vy), S10 = c[1], S11 = vadd(c[2], vz);
  float qh, ql;
  quad_form2(S00, S10, S11, r0, r1, qh, ql);
  const bool fin = fabsf(vadd(vadd(S00, S11), vadd(S10, qh))) < INFINITY;
  // ---- FP64 island ----
  const double s00 = widen_pos(S00), s11 = widen_pos(S11), s10 = widen(S10);
  const double det = __fma_rn(s00, s11, -__dmul_rn(s10, s10));  // exact products of the binary32 S: rounded once
  // det narrowed to binary32 toward zero (relative error below 2^-23) where it
  // lies in the normal binary32 range (d_in); the gain's 1/det and the seed of
  // the FP64 reciprocal come from it
  uint32_t dhi, dlo;
  split64(det, dhi, dlo);
  const bool d_in = dhi - (897u << 20) < (254u << 20);
  const float d32 = __uint_as_float(((dhi - (896u << 20)) << 3) | (dlo >> 29));
  const float i32 = __fdividef(1.0f, d_in ? d32 : vfma(S00, S11, -vmul(S10, S10)));
  chi2 = 0.0;
  if (want_chi2) {
    // q / det = q y0 / (1 - e) with y0 = i32 and e = 1 - det y0 (|e| < 2^-21):
    // q y0 = p + pl to twice the binary32 precision (q renormalised so that
    // its low part is below half an ulp of its high part, the error-free
    // product of the high part and y0, plus the low part times y0), times
    // (1 + e) in FP64: relative error O(e^2), about 2^-42
    float qn, qnl, p, pe;
    fast_two_sum(qh, ql, qn, qnl);
    two_prod(qn, i32, p, pe);
    const float pl = vfma(qnl, i32, pe);
    const double e = __fma_rn(-det, widen_pos(i32), 1.0);
    const double P = widen(p);
    chi2 = __dadd_rn(P, __fma_rn(P, e, widen(pl)));
    acc = le_finite64(chi2, G.hi, G.lo);
  } else {
    const float m = vadd(vfma(-G.f, d32, qh), ql);
    const float mag = vadd(vfma(G.f, d32, fabsf(qh)), fabsf(ql));
    acc = m < 0.0f;
    if (!(d_in && fabsf(m) > vmul(0x1p-19f, mag)))  // near the boundary, or det outside binary32
      acc = le0_finite64(__dadd_rn(__fma_rn(-G.d, det, widen(qh)), widen(ql)));
  }
  // ---- back to FP32 ----
  if (!fin) {
    acc = false;
    chi2 = __longlong_as_double(0x7ff8000000000000ll);
  }
  if (fin && (le0_finite64(det) || !(S00 > 0.0f) || !(S11 > 0.0f))) {
    acc = false;
    return ST_NOT_PD;
  }
  if (acc) {
    const float Si00 = vmul(S11, i32), Si10 = vmul(-S10, i32), Si11 = vmul(S00, i32);
    float K0[5], K1[5];
    const int col0[5] = {0, 1, 3, 6, 10}, col1[5] = {1, 2, 4, 7, 11};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const float ci0 = c[col0[i]], ci1 = c[col1[i]];
      K0[i] = vfma(ci0, Si00, vmul(ci1, Si10));
      K1[i] = vfma(ci0, Si10, vmul(ci1, Si11));
    }
    // new position offsets relative to this cluster (the new anchor)
    T.dy = vfma(vsub(K0[0], 1.0f), r0, vmul(K1[0], r1));
    T.dz = vfma(K0[1], r0, vmul(vsub(K1[1], 1.0f), r1));
    T.dtl = vfma(K0[3], r0, vfma(K1[3], r1, T.dtl));
    T.dw = vfma(K0[4], r0, vfma(K1[4], r1, T.dw));
    // C -= K (H C).  For the measured columns (j = y, z) this equals K V
    // exactly (C_iH - C_iH S^-1 C_HH = C_iH S^-1 V), computed without
    // cancellation; the angle block uses the subtraction form.
    float h0[5], h1[5];
#pragma unroll
    for (int j = 2; j < 5; ++j) {
      h0[j] = c[col0[j]];
      h1[j] = c[col1[j]];
    }
    T.c3l = 0.f;  // C'(2,0) below is a fresh product
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      if (i == 1 || i >= 3) {  // C'(i,0), C'(i,1) as a pair
        const float2 v = __fmul2_rn(make_float2(K0[i], K1[i]), make_float2(vy, vz));
        c[col0[i]] = v.x;
        c[col1[i]] = v.y;
      } else {
        c[col0[i]] = vmul(K0[i], vy);              // C'(i,0)
        if (i >= 1) c[col1[i]] = vmul(K1[i], vz);  // C'(i,1)
      }
    }
    fast_two_sum(c[5], vsub(T.c5l, vfma(K0[2], h0[2], vmul(K1[2], h1[2]))), c[5], T.c5l);
    c[8] = vfma(-K0[3], h0[2], vfma(-K1[3], h1[2], c[8]));
    fast_two_sum_x2(T.sp, c[12], vfma(K0[2], r0, vfma(K1[2], r1, T.spl)),
                    vsub(T.c12l, vfma(K0[4], h0[2], vmul(K1[4], h1[2]))), T.sp, c[12], T.spl, T.c12l);
    c[13] = vfma(-K0[4], h0[3], vfma(-K1[4], h1[3], c[13]));
    fast_two_sum_x2(c[9], c[14], vsub(T.c9l, vfma(K0[3], h0[3], vmul(K1[3], h1[3]))),
                    vsub(T.c14l, vfma(K0[4], h0[4], vmul(K1[4], h1[4]))), c[9], c[14], T.c9l, T.c14l);
  } else {  // a rejected cluster still becomes the anchor: offsets to the predicted position
    T.dy = -r0;
    T.dz = -r1;
  }
  T.ya = yc;
  T.za = zc;
  return ST_OK;
}

// ---------------------------------------------------------------------------
// Seed: circle through three clusters (a, b, c) in the (x, y) plane; state at a.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float asin_over_u_f(float u) {
  const float u2 = u * u;
  if (fabsf(u) < 0.1f) return 1.0f + u2 * (1.0f / 6.0f + u2 * (3.0f / 40.0f + u2 * (5.0f / 112.0f)));
  return asinf(u) / u;
}

static __device__ __noinline__ void seed3(float xa, float ya, float za, float xb, float yb, float xc, float yc, float zc, float b,
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

__device__ __forceinline__ bool finite5(float a, float b, float c, float d, float e) {
  return isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d) && isfinite(e);
}

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

}  // namespace tpcfit
