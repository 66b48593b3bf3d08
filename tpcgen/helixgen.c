/*
 * Seeded synthetic TPC time-frame generator (test and benchmark input only).
 *
 * Produces helix tracks in a uniform solenoid field crossing the TPC pad-row
 * planes of one sector frame, with Gaussian cluster noise, optional Highland
 * multiple-scattering kicks, optional mean ionisation energy loss in every
 * crossed row, random cluster dropout and uniformly displaced outlier clusters.  This stands in for the ALICE Monte-Carlo and Pb-Pb data of
 * the paper's Sec. 7, which are not available.
 *
 * The trajectory is represented as a GLOBAL CIRCLE (centre, radius) in the
 * sector frame and intersected with each pad-row plane x = x_row; it shares no
 * code and no parametrisation with any track fitter.  It holds none of the
 * fitting arithmetic: it only draws inputs and records the true state.
 *
 * Random numbers: a counter-based SplitMix64 stream keyed by (seed, track id,
 * attempt), so each track is reproducible on its own and the output does not
 * depend on the number of threads.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GEN_KB 0.299792458e-2 /* GeV / (cm T): p_T [GeV] = KB * B [T] * R [cm] */

typedef struct {
  uint64_t seed;
  int64_t n_tracks;
  int32_t n_rows;
  int32_t min_clusters;
  double row_x0, row_pitch; /* pad row i at x = float(row_x0 + i*row_pitch) */
  double bz;                /* Tesla */
  double xx0;               /* radiation-length fraction per crossed row; 0 = none */
  double mass;              /* GeV */
  double sigma_y, sigma_z;  /* cluster noise, cm */
  double p_drop;            /* probability a crossing leaves no cluster */
  double p_outlier;         /* probability a kept cluster is an outlier */
  double outlier_half;      /* outlier shift ~ U(-h, h) in y and in z, cm */
  int32_t pt_mode;          /* 0: log-uniform [pt_min, pt_max]; 1: exponential(pt_mean) floored at pt_min */
  int32_t n_phi_sectors;    /* 1: every track labelled sector 0; 18: sectors 0..35 with z side */
  double pt_min, pt_max, pt_mean;
  double sector_half_angle; /* radians */
  double vtx_sigma;         /* cm, per coordinate */
  double tgl_max;
  double z_max;             /* cm */
  double snp_max;           /* stop when |sin phi| >= snp_max at a crossing */
  int32_t max_attempts;
  int32_t n_threads;
  int64_t track_id_offset;  /* added to the track index to key the RNG */
  double xrho;              /* g/cm^2 of material per crossed row (mean energy loss); 0 = none */
  double eloss_za;          /* its Z/A */
  double eloss_i_ev;        /* its mean excitation energy, eV */
  int32_t var_mode;         /* 0: every cluster has sigma_y^2, sigma_z^2; 1: per-cluster variances */
  double var_lo, var_hi;    /* var_mode 1: sy2 and sz2 drawn independently, log-uniform in [var_lo, var_hi] cm^2 */
} tpcgen_config;

typedef struct {
  int64_t *offsets; /* n_tracks+1 (fill pass) */
  int32_t *counts;  /* n_tracks (count pass) */
  float *x, *y, *z, *sy2, *sz2;
  uint8_t *row, *sector;
  double *truth;    /* 5 per cluster: y, z, sin phi, tan lambda, q/pT at arrival (before the kick) */
  uint8_t *flags;   /* per cluster: bit0 outlier */
  double *truth_vertex; /* 6 per track: vx, vy, vz, phi0, tanl0, q/pT0 */
} tpcgen_out;

/* Mean stopping power in MeV cm^2/g of a singly charged particle of momentum
 * p and mass m (GeV) in a material (Z/A, I in eV): the Bethe formula of the
 * PDG review (no density effect), with the maximum energy transfer to one
 * electron in MeV. */
static double stopping_power(double p, double m, double za, double i_ev) {
  const double me_mev = 0.51099895;
  double e = sqrt(p * p + m * m);
  double beta = p / e, gam = e / m, bg = p / m;
  double mr = 0.51099895e-3 / m;
  double tmax = 2.0 * me_mev * bg * bg / (1.0 + 2.0 * gam * mr + mr * mr);
  double i_mev = i_ev * 1e-6;
  double L = 0.5 * log(2.0 * me_mev * bg * bg * tmax / (i_mev * i_mev)) - beta * beta;
  double v = 0.307075 * za * L / (beta * beta);
  return v > 0 ? v : 0;
}

/* ---- counter-based RNG ---------------------------------------------------- */
typedef struct { uint64_t s; } rng_t;
static inline uint64_t splitmix64(uint64_t *s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static inline double u01(rng_t *r) { /* (0,1) */
  return ((double)(splitmix64(&r->s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}
static inline double gauss(rng_t *r) { /* Box-Muller, one value per call */
  double u1 = u01(r), u2 = u01(r);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}
static rng_t key_rng(uint64_t seed, uint64_t track, uint64_t attempt) {
  uint64_t s = seed * 0xD1342543DE82EF95ULL + 0x2545F4914F6CDD1DULL;
  rng_t r; r.s = s;
  r.s ^= splitmix64(&s) + track * 0x9E3779B97F4A7C15ULL;
  r.s ^= (attempt + 1) * 0xC2B2AE3D27D4EB4FULL;
  (void)splitmix64(&r.s);
  return r;
}

static double row_x(const tpcgen_config *c, int i) {
  return (double)(float)(c->row_x0 + (double)i * c->row_pitch);
}

/* One attempt at one track. Returns the number of clusters written (or counted
 * when the output pointers are NULL). */
static int gen_one(const tpcgen_config *c, rng_t *r, int64_t base, const tpcgen_out *o,
                   int write, uint8_t *sector_out, double *vtx_out) {
  const double twopi = 6.283185307179586;
  double vx = c->vtx_sigma * gauss(r), vy = c->vtx_sigma * gauss(r), vz = c->vtx_sigma * gauss(r);
  double phi = (2.0 * u01(r) - 1.0) * c->sector_half_angle;
  double tgl = (2.0 * u01(r) - 1.0) * c->tgl_max;
  double pt;
  if (c->pt_mode == 0) {
    pt = c->pt_min * exp(u01(r) * log(c->pt_max / c->pt_min));
  } else {
    pt = -c->pt_mean * log(u01(r));
    if (pt < c->pt_min) pt = c->pt_min;
  }
  double q = (u01(r) < 0.5) ? -1.0 : 1.0;
  int sec = 0;
  if (c->n_phi_sectors > 1) {
    sec = (int)(u01(r) * c->n_phi_sectors);
    if (sec >= c->n_phi_sectors) sec = c->n_phi_sectors - 1;
    if (tgl < 0) sec += c->n_phi_sectors;
  }
  if (sector_out) *sector_out = (uint8_t)sec;
  if (vtx_out) { vtx_out[0] = vx; vtx_out[1] = vy; vtx_out[2] = vz; vtx_out[3] = phi; vtx_out[4] = tgl; vtx_out[5] = q / pt; }

  /* current point, direction and momentum */
  double px = vx, py = vy, pz = vz;
  double p = pt * sqrt(1.0 + tgl * tgl);
  double tan_edge = tan(c->sector_half_angle);
  int n = 0;
  for (int i = 0; i < c->n_rows; ++i) {
    double X = row_x(c, i);
    /* signed curvature: a positive charge in +Bz turns clockwise (F = q v x B) */
    double kap = -GEN_KB * c->bz * q / pt;
    double R = 1.0 / fabs(kap);
    /* centre on the left of the direction for anticlockwise motion (kap > 0) */
    double xc = px - sin(phi) / kap, yc = py + cos(phi) / kap;
    double dx = X - xc;
    if (fabs(dx) > R) break; /* no crossing: the track curls before this row */
    double h = sqrt(R * R - dx * dx);
    double th_p = atan2(py - yc, px - xc);
    double best_s = -1.0, best_y = 0.0, best_th = 0.0;
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      double qy = yc + sgn * h;
      double th_q = atan2(qy - yc, X - xc);
      double dth = (th_q - th_p) * (kap > 0 ? 1.0 : -1.0);
      dth = fmod(dth, twopi);
      if (dth < 0) dth += twopi;
      double s = R * dth;
      if (s > 1e-9 && (best_s < 0 || s < best_s)) { best_s = s; best_y = qy; best_th = th_q; }
    }
    if (best_s < 0) break;
    /* tangent at the crossing, oriented along the motion */
    double dirx = (kap > 0) ? -sin(best_th) : sin(best_th);
    double diry = (kap > 0) ? cos(best_th) : -cos(best_th);
    double phi_q = atan2(diry, dirx);
    double zq = pz + tgl * best_s;
    double snp = sin(phi_q);
    if (fabs(snp) >= c->snp_max) break;
    if (fabs(best_y) > X * tan_edge) break;
    if (fabs(zq) > c->z_max) break;

    int dropped = (c->p_drop > 0) && (u01(r) < c->p_drop);
    if (!dropped) {
      /* measurement variances of this cluster, and noise drawn with them */
      double vy = c->sigma_y * c->sigma_y, vz = c->sigma_z * c->sigma_z;
      if (c->var_mode == 1) {
        const double lr = log(c->var_hi / c->var_lo);
        vy = (double)(float)(c->var_lo * exp(u01(r) * lr));
        vz = (double)(float)(c->var_lo * exp(u01(r) * lr));
      }
      double ny = vy > 0 ? sqrt(vy) * gauss(r) : 0.0;
      double nz = vz > 0 ? sqrt(vz) * gauss(r) : 0.0;
      int outl = (c->p_outlier > 0) && (u01(r) < c->p_outlier);
      if (outl) {
        ny += (2.0 * u01(r) - 1.0) * c->outlier_half;
        nz += (2.0 * u01(r) - 1.0) * c->outlier_half;
      }
      if (write) {
        int64_t k = base + n;
        o->x[k] = (float)X;
        o->y[k] = (float)(best_y + ny);
        o->z[k] = (float)(zq + nz);
        o->sy2[k] = (float)(vy > 0 ? vy : 1e-6);
        o->sz2[k] = (float)(vz > 0 ? vz : 1e-6);
        o->row[k] = (uint8_t)i;
        if (o->truth) {
          double *tr = o->truth + 5 * k;
          tr[0] = best_y; tr[1] = zq; tr[2] = snp; tr[3] = tgl; tr[4] = q / pt;
        }
        if (o->flags) o->flags[k] = (uint8_t)(outl ? 1 : 0);
      }
      ++n;
    }
    /* move to the crossing */
    px = X; py = best_y; pz = zq; phi = phi_q;
    /* multiple-scattering kick: two Gaussian angles perpendicular to the
       direction, momentum magnitude kept (PDG Highland width) */
    if (c->xx0 > 0) {
      double cl = 1.0 / sqrt(1.0 + tgl * tgl), sl = tgl * cl;
      double beta = p / sqrt(p * p + c->mass * c->mass);
      double eps = c->xx0 / (cl * fabs(cos(phi)));
      double th0 = 0.0136 / (beta * p) * sqrt(eps) * (1.0 + 0.038 * log(eps / (beta * beta)));
      double a1 = th0 * gauss(r), a2 = th0 * gauss(r);
      double cp = cos(phi), sp = sin(phi);
      double dx3 = cl * cp + a1 * (-sp) + a2 * (-sl * cp);
      double dy3 = cl * sp + a1 * (cp) + a2 * (-sl * sp);
      double dz3 = sl + a2 * cl;
      double dt = sqrt(dx3 * dx3 + dy3 * dy3);
      phi = atan2(dy3, dx3);
      tgl = dz3 / dt;
      pt = p * dt / sqrt(dt * dt + dz3 * dz3);
    }
    /* mean energy loss in the row's layer (thickness xrho along x), after the kick */
    if (c->xrho > 0) {
      double path = c->xrho * sqrt(1.0 + tgl * tgl) / fabs(cos(phi));
      double de = 1e-3 * stopping_power(p, c->mass, c->eloss_za, c->eloss_i_ev) * path; /* GeV */
      double e2 = sqrt(p * p + c->mass * c->mass) - de;
      if (!(e2 > c->mass * (1.0 + 1e-6))) break; /* stopped in this row */
      double p2 = sqrt(e2 * e2 - c->mass * c->mass);
      pt *= p2 / p;
      p = p2;
    }
  }
  return n;
}

static int gen_track(const tpcgen_config *c, int64_t t, int64_t base, const tpcgen_out *o, int write) {
  uint64_t tid = (uint64_t)(t + c->track_id_offset);
  for (int a = 0; a < c->max_attempts; ++a) {
    rng_t r = key_rng(c->seed, tid, (uint64_t)a);
    uint8_t sec = 0;
    double vtx[6];
    int n = gen_one(c, &r, base, o, 0, &sec, vtx);
    if (n >= c->min_clusters || a == c->max_attempts - 1) {
      if (write) {
        rng_t r2 = key_rng(c->seed, tid, (uint64_t)a);
        (void)gen_one(c, &r2, base, o, 1, &sec, vtx);
        if (o->sector) o->sector[t] = sec;
        if (o->truth_vertex) memcpy(o->truth_vertex + 6 * t, vtx, sizeof(vtx));
      }
      return n;
    }
  }
  return 0;
}

typedef struct {
  const tpcgen_config *c;
  const tpcgen_out *o;
  int tid, nthreads, write;
} job_t;

static void *worker(void *arg) {
  job_t *j = (job_t *)arg;
  const int64_t chunk = 256;
  for (int64_t s = (int64_t)j->tid * chunk; s < j->c->n_tracks; s += (int64_t)j->nthreads * chunk) {
    int64_t e = s + chunk < j->c->n_tracks ? s + chunk : j->c->n_tracks;
    for (int64_t t = s; t < e; ++t) {
      if (j->write) gen_track(j->c, t, j->o->offsets[t], j->o, 1);
      else j->o->counts[t] = gen_track(j->c, t, 0, j->o, 0);
    }
  }
  return NULL;
}

static void run(const tpcgen_config *c, const tpcgen_out *o, int write) {
  int nt = c->n_threads > 0 ? c->n_threads : 1;
  if (nt > 256) nt = 256;
  pthread_t th[256];
  job_t jobs[256];
  for (int i = 0; i < nt; ++i) {
    jobs[i].c = c; jobs[i].o = o; jobs[i].tid = i; jobs[i].nthreads = nt; jobs[i].write = write;
    if (nt == 1) worker(&jobs[i]);
    else pthread_create(&th[i], NULL, worker, &jobs[i]);
  }
  if (nt > 1) for (int i = 0; i < nt; ++i) pthread_join(th[i], NULL);
}

/* Pass 1: per-track cluster counts. */
int tpcgen_count(const tpcgen_config *c, int32_t *counts) {
  if (!c || !counts || c->n_tracks < 0 || c->n_rows <= 0 || c->n_rows > 256) return -1;
  tpcgen_out o; memset(&o, 0, sizeof(o)); o.counts = counts;
  run(c, &o, 0);
  return 0;
}

/* Pass 2: fill the SoA arrays at the CSR offsets computed from pass 1. */
int tpcgen_fill(const tpcgen_config *c, const tpcgen_out *o) {
  if (!c || !o || !o->offsets || !o->x || !o->y || !o->z || !o->sy2 || !o->sz2 || !o->row) return -1;
  run(c, o, 1);
  return 0;
}

/* Event sizes for batched or served workloads: log-normal with median m and
 * log-width s, redrawn outside [lo, hi]. */
int tpcgen_lognormal_sizes(uint64_t seed, int64_t n, double median, double sigma_ln, double lo, double hi,
                           int64_t *out) {
  rng_t r = key_rng(seed ^ 0x5eedfacecafef00dULL, 0xFFFFFFFFULL, 0);
  for (int64_t i = 0; i < n; ++i) {
    double v;
    int guard = 0;
    do { v = median * exp(sigma_ln * gauss(&r)); } while ((v < lo || v > hi) && ++guard < 1000);
    if (v < lo) v = lo;
    if (v > hi) v = hi;
    out[i] = (int64_t)llround(v);
  }
  return 0;
}

/* Exponential inter-arrival times (Poisson process with the given rate). */
int tpcgen_poisson_arrivals(uint64_t seed, int64_t n, double rate_hz, double *t_out) {
  rng_t r = key_rng(seed ^ 0xa11a11a11a11a11aULL, 0xFFFFFFFEULL, 0);
  double t = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    t += -log(u01(&r)) / rate_hz;
    t_out[i] = t;
  }
  return 0;
}
