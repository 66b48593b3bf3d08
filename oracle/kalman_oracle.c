/*
 * FP64 CPU ORACLE for the batched TPC Kalman track fit.  TEST INFRASTRUCTURE:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code with the CUDA library.
 *
 * What it computes.  The paper (Eulisse & Rohr, Sec. 5 and Sec. 6) places full
 * TPC tracking on the GPU as the dominant synchronous step (Table 1) and the
 * dominant asynchronous step (Table 2), but it does not write out the fit.  The
 * fit below is the textbook Kalman filter (Kalman 1960) applied to track
 * fitting (Fruhwirth 1987, NIM A262 444), with an exact helix in a uniform
 * solenoid field and PDG Highland multiple scattering, in the local frame of a
 * TPC sector:
 *   state p = (y, z, sinphi, tanlambda, q/pT) on the plane of constant x,
 *   covariance C (5x5), measurement H = [I2 0], V = diag(sy2, sz2).
 * Plain and slow on purpose: full 5x5 matrices, explicit products, explicit
 * inverse, one track at a time (a track range per thread).
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   curvature C = -kB*Bz*(q/pT); seed = circle through clusters 0, n/2, n-1;
 *   seed covariance diag(1,1,0.01,0.01,1); chi2 gate 16 (equality accepts);
 *   |sinphi| limit 0.999; MS after the (possible) update at every crossed row;
 *   inward pass restarts from the outward state with a diagonal covariance:
 *   the outward variances times restart_scale (100), capped at the seed's;
 *   if the outward pass accepted fewer than reseed_pct % (50 %) of the
 *   clusters (a pass that lost the track, typically after an outlier at the
 *   first cluster) it restarts instead from a fresh three-point seed at the
 *   outermost cluster;
 *   outputs at the innermost cluster;
 *   optional mean energy loss in a thin layer at every crossed row, crossed
 *   right after the row's cluster in outward motion (outward pass: after the
 *   update and the scattering; inward pass: added back before the update);
 *   optional seed iteration: the fitted state seeds another outward pass
 *   (seed covariance), restart and inward pass, n_iterations times.
 * Status rule: clusters are validated when the outward pass reaches them, so the
 * first offending cluster decides; NaN never trips a numerical limit (it flows
 * to that cluster), a completed fit with a non-finite state or covariance
 * is marked NONFINITE, and a completed fit whose last inward pass accepted
 * fewer than derail_pct % (80 %) of the track's clusters is marked DERAILED
 * (the pass lost the track for a stretch: its estimate does not describe it).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_KB 0.299792458e-2 /* GeV / (cm T) */
#define ORC_ME 0.51099895e-3  /* electron mass, GeV */
#define ORC_K 0.307075e-3     /* 4 pi N_A r_e^2 m_e c^2, GeV cm^2 / mol */

enum { ST_OK = 0, ST_TOO_FEW = 1, ST_SNP_LIMIT = 2, ST_NOT_PD = 3, ST_NONFINITE = 4, ST_BAD_INPUT = 5,
       ST_STOPPED = 6, ST_DERAILED = 7 };

typedef struct {
  double bz;            /* Tesla */
  double chi2_max;      /* gate on the 2-dof chi2 of one cluster */
  double xx0;           /* x/X0 per crossed pad row (0: no scattering) */
  double mass;          /* GeV, for beta in the Highland formula */
  double snp_max;       /* |sinphi| limit */
  double seed_cov[5];   /* diagonal of the seed covariance (also caps the restart covariance) */
  int32_t min_clusters;
  int32_t n_rows;
  const float *row_x;   /* n_rows pad-row plane positions (cm) */
  double restart_scale; /* inward restart covariance: diag(min(restart_scale * C_out_ii, seed_cov_i)) */
  double xrho;          /* energy-loss layer per crossed row, g/cm^2 (0: no energy loss) */
  double eloss_za;      /* Z/A of its material */
  double eloss_i;       /* mean excitation energy of its material, GeV */
  int32_t n_iterations; /* refits seeded from the previous fit's state (0: none) */
  int32_t reseed_pct;   /* the inward pass re-seeds when the outward pass accepted < reseed_pct % of the clusters */
  int32_t derail_pct;   /* a completed fit whose inward pass accepted < derail_pct % of the clusters is DERAILED */
} orc_config;

typedef struct {
  double *state;  /* nt*5 */
  double *cov;    /* nt*15 packed lower triangle (00,10,11,20,...,44) */
  double *x_ref;  /* nt */
  double *chi2;   /* nt */
  int32_t *ndf;   /* nt */
  int32_t *status;/* nt */
  uint8_t *accept;/* nc: bit0 outward, bit1 inward */
  /* optional per-cluster diagnostics (may be NULL) */
  double *chi2_out_c;  /* nc: chi2 of the cluster in the outward pass (NaN if not reached) */
  double *chi2_in_c;   /* nc: chi2 of the cluster in the inward pass */
  double *state_in_c;  /* nc*5: inward state after the cluster's update, before its scattering */
  double *state_out_t; /* nt*5: state the inward pass restarts from */
  double *restart_t;   /* nt*5: diagonal of the covariance the inward pass restarts with */
} orc_result;

/* ---------------------------------------------------------------------------
 * Propagation of the state from plane x1 to plane x2 along the exact helix.
 * d(sinphi)/dx = C, so sinphi2 = sinphi1 + C dx; y2 - y1 = (r1 - r2)/C written
 * in the cancellation-free form dx (s1+s2)/(r1+r2); z advances by tanlambda
 * times the transverse arc length s = L asin(CL/2)/(CL/2), L the chord.
 * F receives the Jacobian d p2 / d p1 (row-major 5x5), derived analytically.
 * Returns 0, or ST_SNP_LIMIT if |sinphi1| or |sinphi2| >= snp_max.
 * ------------------------------------------------------------------------- */
static double asin_over_u(double u) {
  /* asin(u)/u, power series near 0 */
  if (fabs(u) < 1e-3) { double u2 = u * u; return 1.0 + u2 * (1.0 / 6.0 + u2 * (3.0 / 40.0 + u2 * (5.0 / 112.0))); }
  return asin(u) / u;
}
static double dsdc_over_l2u(double u) {
  /* (1/sqrt(1-u^2) - asin(u)/u) / (2 u^2)  ==  d s / d C divided by L^2 u,
     series near 0: 1/6 + 3/20 u^2 + 15/112 u^4 + ... */
  if (fabs(u) < 1e-2) { double u2 = u * u; return 1.0 / 6.0 + u2 * (3.0 / 20.0 + u2 * (15.0 / 112.0 + u2 * (35.0 / 288.0))); }
  return (1.0 / sqrt(1.0 - u * u) - asin(u) / u) / (2.0 * u * u);
}

int orc_propagate(const double p1[5], double x1, double x2, double bz, double snp_max, double p2[5], double F[25]) {
  const double b = -ORC_KB * bz; /* dC/dw */
  double dx = x2 - x1;
  double C = b * p1[4];
  double s1 = p1[2], s2 = s1 + C * dx;
  /* NaN passes (it is reported where the pass meets the offending input) */
  if (fabs(s1) >= snp_max || fabs(s2) >= snp_max) return ST_SNP_LIMIT;
  double r1 = sqrt(1.0 - s1 * s1), r2 = sqrt(1.0 - s2 * s2);
  double T = (s1 + s2) / (r1 + r2);     /* tan of the mean chord direction */
  double k = sqrt(1.0 + T * T);
  double L = dx * k;                    /* signed chord length */
  double u = 0.5 * C * L;
  double g = asin_over_u(u);
  double sT = L * g;                    /* signed transverse arc length */
  p2[0] = p1[0] + dx * T;
  p2[1] = p1[1] + p1[3] * sT;
  p2[2] = s2;
  p2[3] = p1[3];
  p2[4] = p1[4];
  /* Jacobian */
  double Q = (1.0 + r1 * r2 + s1 * s2) / ((r1 + r2) * (r1 + r2));
  double dT_ds1 = Q * (1.0 / r1 + 1.0 / r2);       /* includes d s2 / d s1 = 1 */
  double dT_dw = Q / r2 * (b * dx);                 /* via s2 only */
  double dL_dT = dx * T / k;
  double ds_dL = 1.0 / sqrt(1.0 - u * u);
  double ds_dC = L * L * u * dsdc_over_l2u(u);
  for (int i = 0; i < 25; ++i) F[i] = 0.0;
  for (int i = 0; i < 5; ++i) F[i * 5 + i] = 1.0;
  F[0 * 5 + 2] = dx * dT_ds1;
  F[0 * 5 + 4] = dx * dT_dw;
  F[1 * 5 + 2] = p1[3] * ds_dL * dL_dT * dT_ds1;
  F[1 * 5 + 3] = sT;
  F[1 * 5 + 4] = p1[3] * (ds_dL * dL_dT * dT_dw + ds_dC * b);
  F[2 * 5 + 4] = b * dx;
  return ST_OK;
}

/* C <- F C F^T, plain 5x5 products. */
static void cov_transport(double C[25], const double F[25]) {
  double FC[25], R[25];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      double s = 0.0;
      for (int k = 0; k < 5; ++k) s += F[i * 5 + k] * C[k * 5 + j];
      FC[i * 5 + j] = s;
    }
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      double s = 0.0;
      for (int k = 0; k < 5; ++k) s += FC[i * 5 + k] * F[j * 5 + k];
      R[i * 5 + j] = s;
    }
  memcpy(C, R, sizeof(R));
}

/* ---------------------------------------------------------------------------
 * Kalman update with one (y, z) cluster: S = H C H^T + V, chi2 = r^T S^-1 r,
 * accept iff chi2 <= chi2_max; then K = C H^T S^-1, p += K r, C -= K (H C),
 * symmetrised.  Returns 0 or ST_NOT_PD (S not positive definite).
 * ------------------------------------------------------------------------- */
int orc_update(double p[5], double C[25], double yc, double zc, double sy2, double sz2, double chi2_max,
               double *chi2_out, int *accepted) {
  double S00 = C[0] + sy2, S01 = C[1], S11 = C[6] + sz2;
  double det = S00 * S11 - S01 * S01;
  *accepted = 0;
  if (det <= 0.0 || S00 <= 0.0) { *chi2_out = NAN; return ST_NOT_PD; } /* NaN passes, chi2 NaN is rejected */
  double Si00 = S11 / det, Si01 = -S01 / det, Si11 = S00 / det;
  double r0 = yc - p[0], r1 = zc - p[1];
  double chi2 = r0 * (Si00 * r0 + Si01 * r1) + r1 * (Si01 * r0 + Si11 * r1);
  *chi2_out = chi2;
  if (!(chi2 <= chi2_max)) return ST_OK;
  double K[10];
  for (int i = 0; i < 5; ++i) {
    K[i * 2 + 0] = C[i * 5 + 0] * Si00 + C[i * 5 + 1] * Si01;
    K[i * 2 + 1] = C[i * 5 + 0] * Si01 + C[i * 5 + 1] * Si11;
  }
  double HC[10];
  for (int j = 0; j < 5; ++j) { HC[0 * 5 + j] = C[0 * 5 + j]; HC[1 * 5 + j] = C[1 * 5 + j]; }
  for (int i = 0; i < 5; ++i) p[i] += K[i * 2 + 0] * r0 + K[i * 2 + 1] * r1;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) C[i * 5 + j] -= K[i * 2 + 0] * HC[0 * 5 + j] + K[i * 2 + 1] * HC[1 * 5 + j];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < i; ++j) { double m = 0.5 * (C[i * 5 + j] + C[j * 5 + i]); C[i * 5 + j] = C[j * 5 + i] = m; }
  *accepted = 1;
  return ST_OK;
}

/* ---------------------------------------------------------------------------
 * Multiple scattering in one pad row (PDG Highland formula): momentum
 * p = |1/w| sqrt(1+t^2), beta = p / sqrt(p^2+m^2), path through the plane of
 * constant x: eps = xx0 sqrt(1+t^2)/sqrt(1-sinphi^2),
 * theta0 = 0.0136/(beta p) sqrt(eps) (1 + 0.038 ln(eps/beta^2)).
 * Two independent small kicks (in phi and in lambda) at fixed |p| give the
 * added noise on (sinphi, tanlambda, q/pT).
 * ------------------------------------------------------------------------- */
void orc_ms_noise(const double p[5], double C[25], double xx0, double mass) {
  if (!(xx0 > 0.0)) return;
  double s = p[2], t = p[3], w = p[4];
  double tt = 1.0 + t * t;
  if (w == 0.0) return; /* infinite momentum: no deflection */
  double mom = sqrt(tt) / fabs(w);
  double beta = mom / sqrt(mom * mom + mass * mass);
  double eps = xx0 * sqrt(tt) / sqrt(1.0 - s * s);
  double th0 = 0.0136 / (beta * mom) * sqrt(eps) * (1.0 + 0.038 * log(eps / (beta * beta)));
  double th2 = th0 * th0;
  C[2 * 5 + 2] += th2 * (1.0 - s * s) * tt;
  C[3 * 5 + 3] += th2 * tt * tt;
  C[4 * 5 + 4] += th2 * w * w * t * t;
  C[3 * 5 + 4] += th2 * tt * w * t;
  C[4 * 5 + 3] += th2 * tt * w * t;
}

/* ---------------------------------------------------------------------------
 * Mean ionisation energy loss (Bethe formula as in the PDG Review of Particle
 * Physics, passage of particles through matter, for |charge| 1 and without the
 * density-effect term):
 *   -dE/dx = K (Z/A) (1/beta^2) [ 1/2 ln(2 m_e c^2 beta^2 gamma^2 W_max / I^2) - beta^2 ],
 *   W_max = 2 m_e c^2 beta^2 gamma^2 / (1 + 2 gamma m_e/M + (m_e/M)^2),
 * in GeV cm^2/g for momentum p and mass M (GeV).  Readings: beta gamma is
 * capped at 1e5 and the value clamped at 0 where the formula turns negative.
 * ------------------------------------------------------------------------- */
double orc_dedx(double p, double mass, double za, double i_gev) {
  double E = sqrt(p * p + mass * mass);
  double beta2 = (p * p) / (E * E);
  double bg2 = (p * p) / (mass * mass);
  if (bg2 > 1e10) bg2 = 1e10;
  double gamma = sqrt(1.0 + bg2);
  double ratio = ORC_ME / mass;
  double wmax = 2.0 * ORC_ME * bg2 / (1.0 + 2.0 * gamma * ratio + ratio * ratio);
  double v = ORC_K * za / beta2 * (0.5 * log(2.0 * ORC_ME * bg2 * wmax / (i_gev * i_gev)) - beta2);
  return v > 0.0 ? v : 0.0;
}

/* ---------------------------------------------------------------------------
 * The energy-loss layer of one pad row: x rho along the row normal, so
 * xrho sqrt(1+t^2)/sqrt(1-sinphi^2) along the path.  dir = +1 when the pass
 * moves with the particle (outward): E' = E - dE(E), the loss taken at the
 * energy before the layer.  dir = -1 against it (inward): the energy before
 * the layer solves E' - dE(E') = E; one fixed-point step from dE(E) gives it
 * to O(dE^3).  The momentum scales by p'/p at fixed angles, so
 * q/pT -> q/pT * k with k = p/p', and the covariance transforms with the
 * Jacobian diag(1,1,1,1,k) (the loss taken as fixed).  Returns ST_STOPPED
 * when p'^2 differs from p^2 by more than 50 % (also for the first estimate
 * of the inward step).
 * ------------------------------------------------------------------------- */
int orc_eloss(double p[5], double C[25], const orc_config *c, double dir) {
  if (!(c->xrho > 0.0)) return ST_OK;
  double s = p[2], t = p[3], w = p[4];
  double tt = 1.0 + t * t;
  if (!(w * w / tt > 1e-30)) return ST_OK; /* p above 1e15 GeV (or infinite): no loss */
  double mom = sqrt(tt) / fabs(w);
  double m = sqrt(c->mass * c->mass);
  double E = sqrt(mom * mom + m * m);
  double path = c->xrho * sqrt(tt) / sqrt(1.0 - s * s);
  double dE = orc_dedx(mom, m, c->eloss_za, c->eloss_i) * path;
  double E2 = E - dir * dE;
  double p2sq = E2 * E2 - m * m;
  if (dir < 0.0) {
    if (fabs(p2sq / (mom * mom) - 1.0) > 0.5) return ST_STOPPED;
    dE = orc_dedx(sqrt(p2sq), m, c->eloss_za, c->eloss_i) * path;
    E2 = E + dE;
    p2sq = E2 * E2 - m * m;
  }
  if (fabs(p2sq / (mom * mom) - 1.0) > 0.5) return ST_STOPPED;
  double k = mom / sqrt(p2sq);
  p[4] = w * k;
  for (int j = 0; j < 5; ++j) {
    C[4 * 5 + j] *= k;
    C[j * 5 + 4] *= k;
  }
  return ST_OK;
}

/* ---------------------------------------------------------------------------
 * Three-point seed: circle through clusters a=0, b=n/2, c=n-1 in the (x, y)
 * plane.  Signed curvature from the triangle (kappa = 2 cross / (|ab||ac||bc|)),
 * direction at a from the chord a->c minus half the turned angle,
 * tanlambda from (z_c - z_a) over the transverse arc a->c, q/pT = -C/(kB Bz).
 * ------------------------------------------------------------------------- */
void orc_seed(const double xa[3], const double xb[3], const double xc[3], double bz, double p[5]) {
  double abx = xb[0] - xa[0], aby = xb[1] - xa[1];
  double acx = xc[0] - xa[0], acy = xc[1] - xa[1];
  double bcx = xc[0] - xb[0], bcy = xc[1] - xb[1];
  double cross = abx * acy - aby * acx;
  double lab = sqrt(abx * abx + aby * aby), lac = sqrt(acx * acx + acy * acy), lbc = sqrt(bcx * bcx + bcy * bcy);
  double kappa = 2.0 * cross / (lab * lac * lbc);
  double u = 0.5 * kappa * lac;
  if (u > 1.0) u = 1.0;
  if (u < -1.0) u = -1.0;
  double phi = atan2(acy, acx) - asin(u);
  double s_ac = lac * asin_over_u(u);
  p[0] = xa[1];
  p[1] = xa[2];
  p[2] = sin(phi);
  p[3] = (xc[2] - xa[2]) / s_ac;
  p[4] = -kappa / (ORC_KB * bz);
}

static void pack_cov(const double C[25], double *out15) {
  int k = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j) out15[k++] = C[i * 5 + j];
}
static void seed_cov(const orc_config *c, double C[25]) {
  for (int i = 0; i < 25; ++i) C[i] = 0.0;
  for (int i = 0; i < 5; ++i) C[i * 5 + i] = c->seed_cov[i];
}
static int finite_cluster(const float *x, const float *y, const float *z, const float *sy2, const float *sz2, int64_t k) {
  return isfinite(x[k]) && isfinite(y[k]) && isfinite(z[k]) && isfinite(sy2[k]) && isfinite(sz2[k]);
}

/* One track: seed, outward pass over every crossed row, restart, inward pass. */
static void fit_track(const orc_config *c, int64_t t, const int64_t *off, const float *x, const float *y, const float *z,
                      const float *sy2, const float *sz2, const uint8_t *row, const orc_result *o) {
  int64_t a = off[t], e = off[t + 1];
  int64_t n = e - a;
  double p[5] = {0, 0, 0, 0, 0}, C[25], F[25], pn[5];
  int status = ST_OK;
  double chi2_in = 0.0;
  int nacc_in = 0;
  for (int64_t k = a; k < e; ++k) {
    o->accept[k] = 0;
    if (o->chi2_out_c) o->chi2_out_c[k] = NAN;
    if (o->chi2_in_c) o->chi2_in_c[k] = NAN;
    if (o->state_in_c) for (int i = 0; i < 5; ++i) o->state_in_c[5 * k + i] = NAN;
  }
  seed_cov(c, C);
  double xref = (n > 0) ? (double)x[a] : 0.0;
  if (n < c->min_clusters || n < 3) {
    status = ST_TOO_FEW;
    goto emit;
  }
  {
    double A[3] = {x[a], y[a], z[a]}, B[3] = {x[a + n / 2], y[a + n / 2], z[a + n / 2]},
           D[3] = {x[e - 1], y[e - 1], z[e - 1]};
    orc_seed(A, B, D, c->bz, p);
  }
  if (fabs(p[2]) >= c->snp_max) { status = ST_SNP_LIMIT; goto emit; }
  int iteration = 0;

refit:;
  /* ---- outward pass: rows row[a] .. row[e-1] ---- */
  double xcur = x[a];
  for (int64_t k = a; k < e; ++k) {
    /* validation of cluster k when the pass reaches it */
    if (row[k] >= c->n_rows || (k > a && row[k] <= row[k - 1])) { status = ST_BAD_INPUT; goto emit; }
    if (!finite_cluster(x, y, z, sy2, sz2, k)) { status = ST_NONFINITE; goto emit; }
    if (!(sy2[k] > 0.0f) || !(sz2[k] > 0.0f)) { status = ST_BAD_INPUT; goto emit; }
    /* rows crossed without a cluster */
    if (k > a) {
      for (int r = row[k - 1] + 1; r < row[k]; ++r) {
        double xr = c->row_x[r];
        if ((status = orc_propagate(p, xcur, xr, c->bz, c->snp_max, pn, F)) != ST_OK) goto emit;
        memcpy(p, pn, sizeof(pn));
        cov_transport(C, F);
        xcur = xr;
        orc_ms_noise(p, C, c->xx0, c->mass);
        if ((status = orc_eloss(p, C, c, 1.0)) != ST_OK) goto emit;
      }
    }
    if ((status = orc_propagate(p, xcur, x[k], c->bz, c->snp_max, pn, F)) != ST_OK) goto emit;
    memcpy(p, pn, sizeof(pn));
    cov_transport(C, F);
    xcur = x[k];
    double chi2;
    int acc;
    if ((status = orc_update(p, C, y[k], z[k], sy2[k], sz2[k], c->chi2_max, &chi2, &acc)) != ST_OK) goto emit;
    if (o->chi2_out_c) o->chi2_out_c[k] = chi2;
    if (acc) o->accept[k] |= 1;
    orc_ms_noise(p, C, c->xx0, c->mass);
    /* the energy-loss layer of row[k], crossed after its cluster */
    if ((status = orc_eloss(p, C, c, 1.0)) != ST_OK) goto emit;
  }

  /* ---- inward pass restart.  If the outward pass accepted at least
     reseed_pct % of the clusters: from the outward state with a diagonal covariance, the
     outward variances inflated by restart_scale and capped at the seed's.
     Otherwise the outward pass is not trusted: a fresh three-point seed at the
     outermost cluster (circle through clusters n-1, n/2, 0, taken for motion
     from the outer end, then reversed) with the seed covariance. ---- */
  {
    int nacc_out = 0;
    for (int64_t k = a; k < e; ++k) nacc_out += o->accept[k] & 1;
    if (100 * (int64_t)nacc_out < (int64_t)c->reseed_pct * n) {
      double A[3] = {x[e - 1], y[e - 1], z[e - 1]}, B[3] = {x[a + n / 2], y[a + n / 2], z[a + n / 2]},
             D[3] = {x[a], y[a], z[a]};
      orc_seed(A, B, D, c->bz, p);
      /* the seed describes motion towards cluster 0: reversing the motion
         flips the direction (sinphi), the dip (tanlambda) and the curvature */
      p[2] = -p[2];
      p[3] = -p[3];
      p[4] = -p[4];
      seed_cov(c, C);
    } else {
      double d[5];
      for (int i = 0; i < 5; ++i) {
        d[i] = c->restart_scale * C[i * 5 + i];
        if (!(d[i] <= c->seed_cov[i])) d[i] = c->seed_cov[i];
      }
      for (int i = 0; i < 25; ++i) C[i] = 0.0;
      for (int i = 0; i < 5; ++i) C[i * 5 + i] = d[i];
    }
    if (o->state_out_t) for (int i = 0; i < 5; ++i) o->state_out_t[5 * t + i] = p[i];
    if (o->restart_t) for (int i = 0; i < 5; ++i) o->restart_t[5 * t + i] = C[i * 5 + i];
  }
  for (int64_t k = e - 1; k >= a; --k) {
    if (k < e - 1) {
      for (int r = row[k + 1] - 1; r > row[k]; --r) {
        double xr = c->row_x[r];
        if ((status = orc_propagate(p, xcur, xr, c->bz, c->snp_max, pn, F)) != ST_OK) goto emit;
        memcpy(p, pn, sizeof(pn));
        cov_transport(C, F);
        xcur = xr;
        if ((status = orc_eloss(p, C, c, -1.0)) != ST_OK) goto emit;
        orc_ms_noise(p, C, c->xx0, c->mass);
      }
    }
    if ((status = orc_propagate(p, xcur, x[k], c->bz, c->snp_max, pn, F)) != ST_OK) goto emit;
    memcpy(p, pn, sizeof(pn));
    cov_transport(C, F);
    xcur = x[k];
    /* moving inward, the layer of row[k] comes before its cluster: its loss is added back first */
    if ((status = orc_eloss(p, C, c, -1.0)) != ST_OK) goto emit;
    double chi2;
    int acc;
    if ((status = orc_update(p, C, y[k], z[k], sy2[k], sz2[k], c->chi2_max, &chi2, &acc)) != ST_OK) goto emit;
    if (o->chi2_in_c) o->chi2_in_c[k] = chi2;
    if (acc) { o->accept[k] |= 2; chi2_in += chi2; ++nacc_in; }
    if (o->state_in_c) for (int i = 0; i < 5; ++i) o->state_in_c[5 * k + i] = p[i];
    orc_ms_noise(p, C, c->xx0, c->mass);
  }

  /* a fit that completed with a non-finite state or covariance */
  for (int i = 0; i < 25; ++i)
    if (!isfinite(C[i]) || (i < 5 && !isfinite(p[i]))) { status = ST_NONFINITE; break; }

  /* seed iteration: the fitted state at the innermost cluster seeds a new
     outward pass with the seed covariance, then restart and inward pass */
  if (status == ST_OK && iteration < c->n_iterations) {
    ++iteration;
    seed_cov(c, C);
    chi2_in = 0.0;
    nacc_in = 0;
    for (int64_t k = a; k < e; ++k) {
      o->accept[k] = 0;
      if (o->chi2_out_c) o->chi2_out_c[k] = NAN;
      if (o->chi2_in_c) o->chi2_in_c[k] = NAN;
      if (o->state_in_c) for (int i = 0; i < 5; ++i) o->state_in_c[5 * k + i] = NAN;
    }
    goto refit;
  }
  /* a completed fit that kept fewer than derail_pct % of its clusters lost the track */
  if (status == ST_OK && 100 * (int64_t)nacc_in < (int64_t)c->derail_pct * n) status = ST_DERAILED;

emit:
  for (int i = 0; i < 5; ++i) o->state[5 * t + i] = p[i];
  pack_cov(C, o->cov + 15 * t);
  o->x_ref[t] = xref;
  o->chi2[t] = chi2_in;
  o->ndf[t] = 2 * nacc_in - 5;
  o->status[t] = status;
}

typedef struct {
  const orc_config *c;
  int64_t nt;
  const int64_t *off;
  const float *x, *y, *z, *sy2, *sz2;
  const uint8_t *row;
  const orc_result *o;
  int tid, nth;
} job_t;

static void *worker(void *arg) {
  job_t *j = (job_t *)arg;
  int64_t per = (j->nt + j->nth - 1) / j->nth;
  int64_t s = (int64_t)j->tid * per, e = s + per < j->nt ? s + per : j->nt;
  for (int64_t t = s; t < e; ++t) fit_track(j->c, t, j->off, j->x, j->y, j->z, j->sy2, j->sz2, j->row, j->o);
  return NULL;
}

/* Frame-level entry.  Returns 0, or -1 if the offsets are malformed
 * (off[0] != 0, decreasing, or off[nt] != nc): nothing is fitted then. */
int oracle_fit(const orc_config *c, int64_t nt, int64_t nc, const int64_t *off, const float *x, const float *y,
               const float *z, const float *sy2, const float *sz2, const uint8_t *row, const orc_result *o,
               int n_threads) {
  if (nt < 0 || nc < 0 || !off) return -1;
  if (off[0] != 0 || off[nt] != nc) return -1;
  for (int64_t t = 0; t < nt; ++t)
    if (off[t + 1] < off[t]) return -1;
  int nth = n_threads > 0 ? n_threads : 1;
  if (nth > 512) nth = 512;
  if ((int64_t)nth > nt) nth = nt > 0 ? (int)nt : 1;
  pthread_t th[512];
  job_t jobs[512];
  for (int i = 0; i < nth; ++i) {
    job_t jj = {c, nt, off, x, y, z, sy2, sz2, row, o, i, nth};
    jobs[i] = jj;
    if (nth == 1) worker(&jobs[i]);
    else pthread_create(&th[i], NULL, worker, &jobs[i]);
  }
  if (nth > 1) for (int i = 0; i < nth; ++i) pthread_join(th[i], NULL);
  return 0;
}

/* ---------------------------------------------------------------------------
 * Two-filter smoother (fit variant): the state at every cluster from all of
 * the track's clusters.  Model (the fit's outward reading): the particle
 * moves outward; at each crossed row it is first measured (if the row has a
 * cluster) and then scattered, x_{r+1} = f(x_r + w_r).
 *  - forward filter: the outward pass of fit_track; at cluster k it records
 *    the prediction (p-, C-) before the update (clusters 0..k-1 and the seed
 *    prior at cluster 0);
 *  - backward filter: starts at the outermost cluster as the inward pass of
 *    fit_track does (the forward state with the diagonal restart covariance,
 *    or the fresh reversed seed when the forward filter accepted fewer than
 *    reseed_pct % of the clusters), so its prior carries about 1 % of the
 *    forward information (the restart inflates the variances 100-fold);
 *    moving
 *    inward it propagates to each crossed row, adds that row's scattering
 *    (the kink lies outward of the row's measurement in the model above),
 *    and then updates with the row's cluster: after the update at cluster k
 *    it holds (p+, C+) from clusters k..n-1 and its own seed prior;
 *  - the two estimates of the state arriving at cluster k are independent
 *    and combine as p = p- + K (p+ - p-), C = C- - K C-, K = C- (C- + C+)^-1;
 *    when the forward filter lost the track (it accepted fewer than
 *    reseed_pct % of the clusters, so that the backward filter re-seeds) its
 *    predictions carry no valid information and the smoothed state is the
 *    backward filter's.
 * Track outputs: the smoothed state and covariance at cluster 0; chi2, ndf
 * and accept bit 1 from the backward filter; bit 0 from the forward filter;
 * status as for fit_track (DERAILED when the backward filter kept fewer than
 * derail_pct % of the clusters).  No energy loss, no seed iteration.
 * ------------------------------------------------------------------------- */
static int solve5(const double A[25], const double B[25], double X[25]) {
  /* X = A^-1 B for a symmetric positive definite A, by Gauss-Jordan
     elimination with partial pivoting; returns 0, or -1 if A is singular */
  double M[5][10];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) { M[i][j] = A[i * 5 + j]; M[i][5 + j] = B[i * 5 + j]; }
  for (int c = 0; c < 5; ++c) {
    int pr = c;
    for (int i = c + 1; i < 5; ++i) if (fabs(M[i][c]) > fabs(M[pr][c])) pr = i;
    if (!(fabs(M[pr][c]) > 0.0)) return -1;
    if (pr != c) for (int j = 0; j < 10; ++j) { double t = M[c][j]; M[c][j] = M[pr][j]; M[pr][j] = t; }
    double d = M[c][c];
    for (int j = 0; j < 10; ++j) M[c][j] /= d;
    for (int i = 0; i < 5; ++i) {
      if (i == c) continue;
      double f = M[i][c];
      for (int j = 0; j < 10; ++j) M[i][j] -= f * M[c][j];
    }
  }
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) X[i * 5 + j] = M[i][5 + j];
  return 0;
}

static void smooth_track(const orc_config *c, int64_t t, const int64_t *off, const float *x, const float *y,
                         const float *z, const float *sy2, const float *sz2, const uint8_t *row, const orc_result *o,
                         double *sm_state, double *sm_cov) {
  int64_t a = off[t], e = off[t + 1];
  int64_t n = e - a;
  double p[5] = {0, 0, 0, 0, 0}, C[25], F[25], pn[5];
  int status = ST_OK;
  double chi2_in = 0.0;
  int nacc_in = 0;
  double *fp = NULL, *fC = NULL; /* forward predictions at each cluster */
  for (int64_t k = a; k < e; ++k) {
    o->accept[k] = 0;
    for (int i = 0; i < 5; ++i) sm_state[5 * k + i] = NAN;
    for (int i = 0; i < 15; ++i) sm_cov[15 * k + i] = NAN;
  }
  seed_cov(c, C);
  double xref = (n > 0) ? (double)x[a] : 0.0;
  if (n < c->min_clusters || n < 3) { status = ST_TOO_FEW; goto emit; }
  {
    double A[3] = {x[a], y[a], z[a]}, B[3] = {x[a + n / 2], y[a + n / 2], z[a + n / 2]},
           D[3] = {x[e - 1], y[e - 1], z[e - 1]};
    orc_seed(A, B, D, c->bz, p);
  }
  if (fabs(p[2]) >= c->snp_max) { status = ST_SNP_LIMIT; goto emit; }
  fp = malloc((size_t)n * 5 * sizeof(double));
  fC = malloc((size_t)n * 25 * sizeof(double));
  if (!fp || !fC) { status = ST_NONFINITE; goto emit; }
  /* ---- forward filter (the outward pass), predictions recorded ---- */
  double xcur = x[a];
  for (int64_t k = a; k < e; ++k) {
    if (row[k] >= c->n_rows || (k > a && row[k] <= row[k - 1])) { status = ST_BAD_INPUT; goto emit; }
    if (!finite_cluster(x, y, z, sy2, sz2, k)) { status = ST_NONFINITE; goto emit; }
    if (!(sy2[k] > 0.0f) || !(sz2[k] > 0.0f)) { status = ST_BAD_INPUT; goto emit; }
    if (k > a) {
      for (int r = row[k - 1] + 1; r < row[k]; ++r) {
        double xr = c->row_x[r];
        if ((status = orc_propagate(p, xcur, xr, c->bz, c->snp_max, pn, F)) != ST_OK) goto emit;
        memcpy(p, pn, sizeof(pn));
        cov_transport(C, F);
        xcur = xr;
        orc_ms_noise(p, C, c->xx0, c->mass);
      }
    }
    if ((status = orc_propagate(p, xcur, x[k], c->bz, c->snp_max, pn, F)) != ST_OK) goto emit;
    memcpy(p, pn, sizeof(pn));
    cov_transport(C, F);
    xcur = x[k];
    memcpy(fp + 5 * (k - a), p, 5 * sizeof(double));
    memcpy(fC + 25 * (k - a), C, 25 * sizeof(double));
    double chi2;
    int acc;
    if ((status = orc_update(p, C, y[k], z[k], sy2[k], sz2[k], c->chi2_max, &chi2, &acc)) != ST_OK) goto emit;
    if (acc) o->accept[k] |= 1;
    orc_ms_noise(p, C, c->xx0, c->mass);
  }
  /* ---- backward filter: from the forward state (or a fresh reversed seed) with the seed covariance ---- */
  int fw_valid = 1;
  {
    int nacc_out = 0;
    for (int64_t k = a; k < e; ++k) nacc_out += o->accept[k] & 1;
    if (100 * (int64_t)nacc_out < (int64_t)c->reseed_pct * n) {
      fw_valid = 0;
      double A[3] = {x[e - 1], y[e - 1], z[e - 1]}, B[3] = {x[a + n / 2], y[a + n / 2], z[a + n / 2]},
             D[3] = {x[a], y[a], z[a]};
      orc_seed(A, B, D, c->bz, p);
      p[2] = -p[2];
      p[3] = -p[3];
      p[4] = -p[4];
      seed_cov(c, C);
    } else {
      double d[5];
      for (int i = 0; i < 5; ++i) {
        d[i] = c->restart_scale * C[i * 5 + i];
        if (!(d[i] <= c->seed_cov[i])) d[i] = c->seed_cov[i];
      }
      for (int i = 0; i < 25; ++i) C[i] = 0.0;
      for (int i = 0; i < 5; ++i) C[i * 5 + i] = d[i];
    }
    if (o->state_out_t) for (int i = 0; i < 5; ++i) o->state_out_t[5 * t + i] = p[i];
    if (o->restart_t) for (int i = 0; i < 5; ++i) o->restart_t[5 * t + i] = C[i * 5 + i];
  }
  for (int64_t k = e - 1; k >= a; --k) {
    if (k < e - 1) {
      /* rows crossed without a cluster between cluster k+1 and cluster k */
      for (int r = row[k + 1] - 1; r > row[k]; --r) {
        double xr = c->row_x[r];
        if ((status = orc_propagate(p, xcur, xr, c->bz, c->snp_max, pn, F)) != ST_OK) goto emit;
        memcpy(p, pn, sizeof(pn));
        cov_transport(C, F);
        xcur = xr;
        orc_ms_noise(p, C, c->xx0, c->mass);
      }
      if ((status = orc_propagate(p, xcur, x[k], c->bz, c->snp_max, pn, F)) != ST_OK) goto emit;
      memcpy(p, pn, sizeof(pn));
      cov_transport(C, F);
      xcur = x[k];
      orc_ms_noise(p, C, c->xx0, c->mass); /* the kink of row k lies outward of its measurement */
    }
    double chi2;
    int acc;
    if ((status = orc_update(p, C, y[k], z[k], sy2[k], sz2[k], c->chi2_max, &chi2, &acc)) != ST_OK) goto emit;
    if (acc) { o->accept[k] |= 2; chi2_in += chi2; ++nacc_in; }
    /* combine with the forward prediction at cluster k */
    if (!fw_valid) {
      for (int i = 0; i < 5; ++i) sm_state[5 * k + i] = p[i];
      pack_cov(C, sm_cov + 15 * k);
    } else {
      const double *pm = fp + 5 * (k - a), *Cm = fC + 25 * (k - a);
      double S[25], K[25], Kt[25], ps[5], Cs[25];
      for (int i = 0; i < 25; ++i) S[i] = Cm[i] + C[i];
      /* K^T = S^-1 Cm (S and Cm symmetric), so K = Cm S^-1 */
      if (solve5(S, Cm, Kt) != 0) { status = ST_NOT_PD; goto emit; }
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) K[i * 5 + j] = Kt[j * 5 + i];
      for (int i = 0; i < 5; ++i) {
        double v = pm[i];
        for (int j = 0; j < 5; ++j) v += K[i * 5 + j] * (p[j] - pm[j]);
        ps[i] = v;
      }
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
          double v = Cm[i * 5 + j];
          for (int m = 0; m < 5; ++m) v -= K[i * 5 + m] * Cm[m * 5 + j];
          Cs[i * 5 + j] = v;
        }
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j < i; ++j) { double m = 0.5 * (Cs[i * 5 + j] + Cs[j * 5 + i]); Cs[i * 5 + j] = Cs[j * 5 + i] = m; }
      for (int i = 0; i < 5; ++i) sm_state[5 * k + i] = ps[i];
      pack_cov(Cs, sm_cov + 15 * k);
      if (k == a) { memcpy(p, ps, sizeof(ps)); memcpy(C, Cs, sizeof(Cs)); } /* the track output */
    }
  }
  for (int i = 0; i < 25; ++i)
    if (!isfinite(C[i]) || (i < 5 && !isfinite(p[i]))) { status = ST_NONFINITE; break; }
  if (status == ST_OK && 100 * (int64_t)nacc_in < (int64_t)c->derail_pct * n) status = ST_DERAILED;
emit:
  free(fp);
  free(fC);
  for (int i = 0; i < 5; ++i) o->state[5 * t + i] = p[i];
  pack_cov(C, o->cov + 15 * t);
  o->x_ref[t] = xref;
  o->chi2[t] = chi2_in;
  o->ndf[t] = 2 * nacc_in - 5;
  o->status[t] = status;
}

typedef struct {
  const orc_config *c;
  int64_t nt;
  const int64_t *off;
  const float *x, *y, *z, *sy2, *sz2;
  const uint8_t *row;
  const orc_result *o;
  double *sm_state, *sm_cov;
  int tid, nth;
} smooth_job;

static void *smooth_worker(void *arg) {
  smooth_job *j = (smooth_job *)arg;
  for (int64_t t = j->tid; t < j->nt; t += j->nth)
    smooth_track(j->c, t, j->off, j->x, j->y, j->z, j->sy2, j->sz2, j->row, j->o, j->sm_state, j->sm_cov);
  return NULL;
}

/* Frame-level entry of the smoother: track outputs in *o (accept flags
 * included), smoothed state (nc*5) and covariance (nc*15, packed) at every
 * cluster (NaN where the fit did not complete).  Returns 0, or -1 on
 * malformed offsets. */
int oracle_smooth(const orc_config *c, int64_t nt, int64_t nc, const int64_t *off, const float *x, const float *y,
                  const float *z, const float *sy2, const float *sz2, const uint8_t *row, const orc_result *o,
                  double *sm_state, double *sm_cov, int n_threads) {
  if (nt < 0 || nc < 0 || !off) return -1;
  if (off[0] != 0 || off[nt] != nc) return -1;
  for (int64_t t = 0; t < nt; ++t)
    if (off[t + 1] < off[t]) return -1;
  int nth = n_threads > 0 ? n_threads : 1;
  if (nth > 512) nth = 512;
  if ((int64_t)nth > nt) nth = nt > 0 ? (int)nt : 1;
  pthread_t th[512];
  smooth_job jobs[512];
  for (int i = 0; i < nth; ++i) {
    smooth_job jj = {c, nt, off, x, y, z, sy2, sz2, row, o, sm_state, sm_cov, i, nth};
    jobs[i] = jj;
    if (nth == 1) smooth_worker(&jobs[i]);
    else pthread_create(&th[i], NULL, smooth_worker, &jobs[i]);
  }
  if (nth > 1) for (int i = 0; i < nth; ++i) pthread_join(th[i], NULL);
  return 0;
}

/* ---------------------------------------------------------------------------
 * Track-model compression residuals.  The paper's TPC compression stores
 * cluster-to-track residuals instead of absolute coordinates (Sec. 5) and
 * gives no formula.  Reading: for a track with status OK, the residual of
 * cluster k is its (y, z) minus the fitted helix -- the fit's output state at
 * x_ref, transported without scattering in one exact-helix step to the
 * cluster's x; its code is round-half-even(residual / step), clipped to
 * +-32767.  Clusters of other tracks, and clusters the helix does not reach,
 * get -32768.  raw_y / raw_z (may be NULL) receive residual / step in FP64.
 * Returns 0, or -1 on malformed offsets.
 * ------------------------------------------------------------------------- */
static int16_t orc_code(double q) {
  if (isnan(q)) return (int16_t)-32768;
  if (!(fabs(q) < 32767.5)) return q > 0 ? (int16_t)32767 : (int16_t)-32767;
  return (int16_t)nearbyint(q); /* default rounding mode: half to even */
}

int oracle_residuals(double bz, double step_y, double step_z, int64_t nt, int64_t nc, const int64_t *off,
                     const float *x, const float *y, const float *z, const double *state, const double *x_ref,
                     const int32_t *status, int16_t *res_y, int16_t *res_z, double *raw_y, double *raw_z) {
  if (nt < 0 || nc < 0 || !off || off[0] != 0 || off[nt] != nc) return -1;
  for (int64_t t = 0; t < nt; ++t)
    if (off[t + 1] < off[t]) return -1;
  for (int64_t t = 0; t < nt; ++t) {
    for (int64_t k = off[t]; k < off[t + 1]; ++k) {
      double qy = NAN, qz = NAN;
      if (status[t] == ST_OK) {
        double pn[5], F[25];
        /* no |sinphi| limit short of 1: a reachable plane is always encoded */
        if (orc_propagate(state + 5 * t, x_ref[t], (double)x[k], bz, 1.0, pn, F) == ST_OK) {
          qy = ((double)y[k] - pn[0]) / step_y;
          qz = ((double)z[k] - pn[1]) / step_z;
        }
      }
      res_y[k] = orc_code(qy);
      res_z[k] = orc_code(qz);
      if (raw_y) raw_y[k] = qy;
      if (raw_z) raw_z[k] = qz;
    }
  }
  return 0;
}


/* ---------------------------------------------------------------------------
 * Track following: the tracking step in front of the fit (the paper runs the
 * full TPC tracking on the GPU, Sec. 5 and Sec. 6, and describes no
 * algorithm).  Reading: a seed (state at the plane of pad row r0, sector s,
 * diagonal covariance) is carried row by row with the fit's own propagation,
 * update and scattering; at each row the candidate clusters are those of its
 * sector and row with |y_c - y| <= k sqrt(C_yy + v) and |z_c - z| <= k
 * sqrt(C_zz + v) (k = window_sigma, v = nominal_v); the candidate with the
 * smallest chi2 (its own variances; ties: lowest cluster index) is attached
 * if its chi2 passes the gate.  MS noise after the (possible) update at every
 * row.  Following ends at the last row, at the sector edge (|y| > x tan_edge),
 * at |z| > z_max (status END), after max_miss consecutive rows without a
 * cluster (MISSES), or on a numerical failure (SNP_LIMIT, NOT_PD).
 * Diagnostics per (seed, row), for the comparison with other arithmetic:
 * the best and second-best candidate chi2 and the smallest relative distance
 * of any cluster of the row to the window edge.
 * ------------------------------------------------------------------------- */
typedef struct {
  double window_sigma;
  double nominal_v;
  int32_t max_miss;
  double tan_edge;
  double z_max;
} orc_follow_cfg;

enum { FL_END = 0, FL_MISSES = 1 };

static const float *g_sort_y; /* qsort comparator context (set per call under a lock) */
static int cmp_y_idx(const void *a, const void *b) {
  const int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
  if (g_sort_y[i] < g_sort_y[j]) return -1;
  if (g_sort_y[i] > g_sort_y[j]) return 1;
  return (i > j) - (i < j);
}
static pthread_mutex_t g_sort_mu = PTHREAD_MUTEX_INITIALIZER;

typedef struct {
  const orc_config *c;
  const orc_follow_cfg *fc;
  const float *y, *z, *sy2, *sz2;
  const int64_t *bstart; /* n_buckets + 1 */
  const int64_t *bidx;   /* cluster indices, bucket by bucket, by y */
  int64_t ns;
  const double *seed_state, *seed_cov;
  const uint8_t *seed_row, *seed_sector;
  int32_t *att, *n_att, *status;
  double *state_out, *best2, *edge;
  int tid, nth;
} follow_job;

static void follow_seed(const follow_job *J, int64_t s) {
  const orc_config *c = J->c;
  const orc_follow_cfg *fc = J->fc;
  const int nr = c->n_rows;
  double p[5], C[25], pn[5], F[25];
  for (int i = 0; i < 5; ++i) p[i] = J->seed_state[5 * s + i];
  memset(C, 0, sizeof(C));
  for (int i = 0; i < 5; ++i) C[i * 5 + i] = J->seed_cov[i];
  for (int r = 0; r < nr; ++r) {
    J->att[s * nr + r] = -1;
    if (J->best2) J->best2[(s * nr + r) * 2] = J->best2[(s * nr + r) * 2 + 1] = NAN;
    if (J->edge) J->edge[s * nr + r] = NAN;
  }
  int status = FL_END, misses = 0, n = 0;
  const int r0 = J->seed_row[s], sec = J->seed_sector[s];
  double xcur = c->row_x[r0 < nr ? r0 : 0];
  for (int r = r0; r < nr; ++r) {
    const double xr = c->row_x[r];
    if (r > r0) {
      if ((status = orc_propagate(p, xcur, xr, c->bz, c->snp_max, pn, F)) != ST_OK) break;
      memcpy(p, pn, sizeof(pn));
      cov_transport(C, F);
      xcur = xr;
    }
    if (fabs(p[0]) > xr * fc->tan_edge || fabs(p[1]) > fc->z_max) { status = FL_END; break; }
    const double wy = fc->window_sigma * sqrt(C[0] + fc->nominal_v);
    const double wz = fc->window_sigma * sqrt(C[6] + fc->nominal_v);
    const int64_t b = (int64_t)sec * nr + r;
    const int64_t lo0 = J->bstart[b], hi0 = J->bstart[b + 1];
    /* first cluster with y >= p0 - 1.01 wy (binary search over the bucket sorted by y) */
    int64_t lo = lo0, hi = hi0;
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if ((double)J->y[J->bidx[mid]] < p[0] - 1.01 * wy) lo = mid + 1;
      else hi = mid;
    }
    int64_t best = -1;
    double c1 = INFINITY, c2 = INFINITY, edge = INFINITY;
    for (int64_t q = lo; q < hi0; ++q) {
      const int64_t k = J->bidx[q];
      const double dy = (double)J->y[k] - p[0], dz = (double)J->z[k] - p[1];
      if (dy > 1.01 * wy) break;
      if (fabs(dz) > 1.01 * wz) continue;
      const double ey = fabs(fabs(dy) - wy) / wy, ez = fabs(fabs(dz) - wz) / wz;
      edge = fmin(edge, fmin(ey, ez));
      if (fabs(dy) > wy || fabs(dz) > wz) continue;
      const double S00 = C[0] + J->sy2[k], S01 = C[1], S11 = C[6] + J->sz2[k];
      const double det = S00 * S11 - S01 * S01;
      const double chi2 = (dy * (S11 * dy - S01 * dz) + dz * (S00 * dz - S01 * dy)) / det;
      if (chi2 < c1 || (chi2 == c1 && k < best)) { c2 = c1; c1 = chi2; best = k; }
      else if (chi2 < c2) c2 = chi2;
    }
    if (J->best2) { J->best2[(s * nr + r) * 2] = c1; J->best2[(s * nr + r) * 2 + 1] = c2; }
    if (J->edge) J->edge[s * nr + r] = edge;
    int acc = 0;
    if (best >= 0) {
      double chi2;
      if ((status = orc_update(p, C, J->y[best], J->z[best], J->sy2[best], J->sz2[best], c->chi2_max, &chi2, &acc)) !=
          ST_OK)
        break;
    }
    if (acc) { J->att[s * nr + r] = (int32_t)best; ++n; misses = 0; }
    else if (++misses > fc->max_miss) { status = FL_MISSES; break; }
    orc_ms_noise(p, C, c->xx0, c->mass);
  }
  J->n_att[s] = n;
  J->status[s] = status;
  if (J->state_out) for (int i = 0; i < 5; ++i) J->state_out[5 * s + i] = p[i];
}

static void *follow_worker(void *arg) {
  follow_job *j = (follow_job *)arg;
  for (int64_t s = j->tid; s < j->ns; s += j->nth) follow_seed(j, s);
  return NULL;
}

/* Follow ns seeds through the clusters (x is the row plane; rows and sectors
 * per cluster).  att: ns*n_rows cluster indices by row (-1: none).  Returns 0,
 * or -1 on bad arguments. */
int oracle_follow(const orc_config *c, const orc_follow_cfg *fc, int64_t nc, const float *y, const float *z,
                  const float *sy2, const float *sz2, const uint8_t *row, const uint8_t *sector, int64_t ns,
                  const double *seed_state, const uint8_t *seed_row, const uint8_t *seed_sector, const double *seed_cov,
                  int32_t *att, int32_t *n_att, int32_t *status, double *state_out, double *best2, double *edge,
                  int n_threads) {
  if (nc < 0 || ns < 0 || c->n_rows < 1 || c->n_rows > 256) return -1;
  const int64_t nb = 256 * (int64_t)c->n_rows;
  int64_t *bstart = calloc((size_t)nb + 1, sizeof(int64_t));
  int64_t *bidx = malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int64_t));
  int64_t *cur = calloc((size_t)nb + 1, sizeof(int64_t));
  if (!bstart || !bidx || !cur) { free(bstart); free(bidx); free(cur); return -1; }
  for (int64_t k = 0; k < nc; ++k) {
    if (row[k] >= c->n_rows) continue;
    ++bstart[(int64_t)sector[k] * c->n_rows + row[k] + 1];
  }
  for (int64_t b = 0; b < nb; ++b) bstart[b + 1] += bstart[b];
  memcpy(cur, bstart, (size_t)nb * sizeof(int64_t));
  for (int64_t k = 0; k < nc; ++k) {
    if (row[k] >= c->n_rows) continue;
    bidx[cur[(int64_t)sector[k] * c->n_rows + row[k]]++] = k;
  }
  pthread_mutex_lock(&g_sort_mu);
  g_sort_y = y;
  for (int64_t b = 0; b < nb; ++b)
    if (bstart[b + 1] - bstart[b] > 1) qsort(bidx + bstart[b], (size_t)(bstart[b + 1] - bstart[b]), sizeof(int64_t), cmp_y_idx);
  pthread_mutex_unlock(&g_sort_mu);
  int nth = n_threads > 0 ? n_threads : 1;
  if (nth > 512) nth = 512;
  if ((int64_t)nth > ns) nth = ns > 0 ? (int)ns : 1;
  pthread_t th[512];
  follow_job jobs[512];
  for (int i = 0; i < nth; ++i) {
    follow_job jj = {c, fc, y, z, sy2, sz2, bstart, bidx, ns, seed_state, seed_cov, seed_row, seed_sector,
                     att, n_att, status, state_out, best2, edge, i, nth};
    jobs[i] = jj;
    if (nth == 1) follow_worker(&jobs[i]);
    else pthread_create(&th[i], NULL, follow_worker, &jobs[i]);
  }
  if (nth > 1) for (int i = 0; i < nth; ++i) pthread_join(th[i], NULL);
  free(bstart); free(bidx); free(cur);
  return 0;
}
