/*
 * FP64 CPU oracle — TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Signal model (arXiv 2305.14176, Sec. II-A, Eqs. 1-3) with the separable reading:
 *   tau_i(j) = (d_i + 2 v_i j T_d) / c              Eq. 1, chirps spaced by T_d
 *   t_n      = n T_c / N_s                          fast time, n = 0 .. N_s-1
 *   phase    = mu t_n tau_i(0) + f_c tau_i(j)       Eq. 2 (mu t dtau_i(j) dropped)
 *            + k s sin(az) cos(el) / lambda          Eq. 7 in the far field
 *            + phi0_i / 2pi                          per-ray start phase
 * which, per ray, is a sum of four cycle counts:
 *   f_c d / c + phi0/2pi,  n * B d / (c N_s),  m * 2 v f_c T_d / c,  k * s f_c sin cos / c.
 *
 * Compiled with -O2 -ffp-contract=off; no -ffast-math.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_C 299792458.0 /* speed of light, m/s (exact SI value) */
#define ORC_TWO_PI 6.283185307179586476925286766559

int orc_default_threads(void) {
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

static int nv_of(const orc_radar *p) { return p->n_tx * p->n_rx; }

/* antenna spacing in carrier wavelengths: s f_c / c, or exactly 1/2 when unset */
static double spacing_wl(const orc_radar *p) {
  if (p->element_spacing_m == 0.0) return 0.5;
  return (p->element_spacing_m * p->carrier_hz) / ORC_C;
}

static double frac(double x) { return x - floor(x); }

double orc_sin_rep(double x);
double orc_cos_rep(double x);

/* amplitude after the antenna pattern of Eq. 2, A(az, el) = (cos az cos el)^q: the labels'
   fixed-point energies follow it too, so it uses the same polynomial cosine and q products
   in order */
static double pattern_amp(const orc_radar *p, double a, double az, double el) {
  if (p->pattern_exp <= 0) return a;
  const double c = orc_cos_rep(az) * orc_cos_rep(el);
  for (int e = 0; e < p->pattern_exp; ++e) a = a * c;
  return a;
}

/* transmitter of virtual channel k = tx N_rx + rx */
static int64_t tx_of(const orc_radar *p, int64_t k) {
  return k / p->n_rx;
}

/* --------------------------------------------------------------- per-ray cycle counts */
typedef struct {
  double carrier; /* frac(f_c d / c) + phi0 / 2pi, cycles */
  double nu_r;    /* cycles per fast-time sample: B d / (c N_s)  (mu t tau, t = n T_c/N_s) */
  double nu_d;    /* cycles per chirp: 2 v f_c T_d / c             (f_c dtau per T_d) */
  double nu_a;    /* cycles per virtual channel: s sin(az) cos(el) / lambda */
  double eps;     /* exact model: cycles per (sample x chirp), mu dt (2 v T_d / c); else 0 */
  double nu_t;    /* cycles per transmitter slot: 2 v f_c T_slot / c (TDM-MIMO) */
  double eps_t;   /* exact model: cycles per (sample x slot), mu dt (2 v T_slot / c); else 0 */
  double amp;
} ray_cycles;

static void ray_cycles_of(const orc_radar *p, const orc_rays *r, int64_t i, ray_cycles *o) {
  const double d = r->range_rt_m[i];
  const double v = (double)r->radial_velocity_mps[i];
  const double az = (double)r->azimuth_rad[i];
  const double el = (double)r->elevation_rad[i];
  const double tau = d / ORC_C;                                   /* Eq. 1 */
  const double mu = p->bandwidth_hz / p->sweep_time_s;            /* Eq. 3 */
  const double dt = p->sweep_time_s / p->n_samples;               /* sample spacing */
  o->carrier = frac(p->carrier_hz * tau) + frac((double)r->phase0_rad[i] / ORC_TWO_PI);
  o->nu_r = mu * dt * tau;                                        /* mu t_n tau per n */
  o->nu_d = p->carrier_hz * (2.0 * v * p->chirp_period_s) / ORC_C; /* f_c dtau per chirp */
  o->nu_a = spacing_wl(p) * sin(az) * cos(el);                   /* far-field Eq. 7 */
  /* exact Eq. 2 keeps mu t_n (tau_i(j) - tau_i(0)) = n j mu dt 2 v T_d / c */
  o->eps = p->model == 1 ? mu * dt * (2.0 * v * p->chirp_period_s) / ORC_C : 0.0;
  /* transmitter t of a TDM-MIMO frame sends chirp j at j T_d + t T_slot: its delays
     tau_i(j, t) = (d + 2 v (j T_d + t T_slot)) / c add t nu_t to the carrier term of Eq. 2 and,
     in the exact model, n t eps_t to the range-migration product */
  o->nu_t = p->carrier_hz * (2.0 * v * p->tdm_slot_s) / ORC_C;
  o->eps_t = p->model == 1 ? mu * dt * (2.0 * v * p->tdm_slot_s) / ORC_C : 0.0;
  o->amp = pattern_amp(p, (double)r->amplitude[i], az, el);
}

/* e^{2 pi i x} for a cycle count x */
static void cis_cycles(double x, double *re, double *im) {
  double t = x - nearbyint(x);
  *re = cos(ORC_TWO_PI * t);
  *im = sin(ORC_TWO_PI * t);
}

/* --------------------------------------------------------------- thread helper */
typedef struct {
  void (*fn)(void *ctx, int64_t lo, int64_t hi);
  void *ctx;
  int64_t lo, hi;
} orc_job;

static void *orc_job_main(void *a) {
  orc_job *j = (orc_job *)a;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

/* split [0, n) into contiguous blocks over nthreads threads */
static void parallel_for(int64_t n, int nthreads, void (*fn)(void *, int64_t, int64_t), void *ctx) {
  if (nthreads <= 0) nthreads = orc_default_threads();
  if (nthreads > n) nthreads = (int)(n > 0 ? n : 1);
  if (nthreads <= 1) {
    fn(ctx, 0, n);
    return;
  }
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
  orc_job *jobs = (orc_job *)malloc(sizeof(orc_job) * (size_t)nthreads);
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = fn;
    jobs[t].ctx = ctx;
    jobs[t].lo = n * t / nthreads;
    jobs[t].hi = n * (t + 1) / nthreads;
    pthread_create(&th[t], NULL, orc_job_main, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

/* --------------------------------------------------------------- signal (Eq. 2) */
typedef struct {
  const orc_radar *p;
  const orc_rays *r;
  const ray_cycles *rc;
  double *out;
  int64_t npts;
  const int64_t *idx;
} sig_ctx;

/* one (k, m) row: s[k][m][n] = sum_i a_i e^{2 pi i (carrier + k nu_a + m nu_d + n nu_r)} */
static void signal_rows(void *vctx, int64_t lo, int64_t hi) {
  sig_ctx *c = (sig_ctx *)vctx;
  const int ns = c->p->n_samples, nc = c->p->n_chirps;
  for (int64_t row = lo; row < hi; ++row) {
    const int k = (int)(row / nc), m = (int)(row % nc), tx = (int)tx_of(c->p, k);
    double *o = c->out + row * (int64_t)ns * 2;
    memset(o, 0, sizeof(double) * 2 * (size_t)ns);
    for (int64_t i = 0; i < c->r->n; ++i) {
      const ray_cycles *q = &c->rc[i];
      const double base = q->carrier + frac(k * q->nu_a) + frac(m * q->nu_d) + frac(tx * q->nu_t);
      for (int n = 0; n < ns; ++n) {
        double re, im;
        cis_cycles(base + frac(n * q->nu_r) + frac((double)n * m * q->eps) + frac((double)n * tx * q->eps_t),
                   &re, &im);
        o[2 * n] += q->amp * re;
        o[2 * n + 1] += q->amp * im;
      }
    }
  }
}

static ray_cycles *all_cycles(const orc_radar *p, const orc_rays *r) {
  ray_cycles *rc = (ray_cycles *)malloc(sizeof(ray_cycles) * (size_t)(r->n > 0 ? r->n : 1));
  for (int64_t i = 0; i < r->n; ++i) ray_cycles_of(p, r, i, &rc[i]);
  return rc;
}

void orc_signal(const orc_radar *p, const orc_rays *r, double *out, int nthreads) {
  ray_cycles *rc = all_cycles(p, r);
  sig_ctx c = {p, r, rc, out, 0, NULL};
  parallel_for((int64_t)nv_of(p) * p->n_chirps, nthreads, signal_rows, &c);
  free(rc);
}

static void signal_points(void *vctx, int64_t lo, int64_t hi) {
  sig_ctx *c = (sig_ctx *)vctx;
  const int64_t ns = c->p->n_samples, nc = c->p->n_chirps;
  for (int64_t t = lo; t < hi; ++t) {
    const int64_t f = c->idx[t];
    const int64_t n = f % ns, m = (f / ns) % nc, k = f / (ns * nc), tx = tx_of(c->p, k);
    double sr = 0.0, si = 0.0;
    for (int64_t i = 0; i < c->r->n; ++i) {
      const ray_cycles *q = &c->rc[i];
      double re, im;
      cis_cycles(q->carrier + frac(k * q->nu_a) + frac(m * q->nu_d) + frac(tx * q->nu_t) + frac(n * q->nu_r) +
                     frac((double)n * m * q->eps) + frac((double)n * tx * q->eps_t), &re, &im);
      sr += q->amp * re;
      si += q->amp * im;
    }
    c->out[2 * t] = sr;
    c->out[2 * t + 1] = si;
  }
}

void orc_signal_at(const orc_radar *p, const orc_rays *r, int64_t npts, const int64_t *idx,
                   double *out, int nthreads) {
  ray_cycles *rc = all_cycles(p, r);
  sig_ctx c = {p, r, rc, out, npts, idx};
  parallel_for(npts, nthreads, signal_points, &c);
  free(rc);
}

/* --------------------------------------------------------------- windows */
static double window_value(int type, int t, int len) {
  switch (type) {
    case 1: /* periodic Hann */
      return 0.5 * (1.0 - cos(ORC_TWO_PI * t / len));
    case 2: /* symmetric Hann */
      return len > 1 ? 0.5 * (1.0 - cos(ORC_TWO_PI * t / (len - 1))) : 1.0;
    case 3: /* Hann over len+2 points with both zero end points removed */
      return 0.5 * (1.0 - cos(ORC_TWO_PI * (t + 1) / (len + 1)));
    default:
      return 1.0;
  }
}

static int axis_len(const orc_radar *p, int axis) {
  return axis == 0 ? p->n_samples : axis == 1 ? p->n_chirps : nv_of(p);
}

void orc_window(const orc_radar *p, int axis, double *out) {
  const int len = axis_len(p, axis);
  for (int t = 0; t < len; ++t) out[t] = window_value(p->window[axis], t, len);
}

/* --------------------------------------------------------------- spectrum (Eq. 4) */
/* X[q] = sum_t w[t] x[t] e^{-2 pi i t q / N}, naive, with exact integer reduction of t q mod N */
typedef struct {
  const orc_radar *p;
  const double *in;
  double *out;
  const double *w;
  const double *tw; /* twiddle table cos/sin(2 pi j / N), j < N */
  int axis;
} dft_ctx;

static void dft_lines(void *vctx, int64_t lo, int64_t hi) {
  dft_ctx *c = (dft_ctx *)vctx;
  const int64_t ns = c->p->n_samples, nc = c->p->n_chirps, nv = nv_of(c->p), na = c->p->n_angle;
  int64_t len, nout, stride_in, stride_out;
  if (c->axis == 0) { len = ns; nout = ns; stride_in = 1; stride_out = 1; }
  else if (c->axis == 1) { len = nc; nout = nc; stride_in = ns; stride_out = ns; }
  else { len = nv; nout = na; stride_in = nc * ns; stride_out = nc * ns; }
  for (int64_t line = lo; line < hi; ++line) {
    int64_t base_in, base_out;
    if (c->axis == 0) { base_in = line * ns; base_out = base_in; }
    else if (c->axis == 1) {
      const int64_t k = line / ns, q = line % ns;
      base_in = k * nc * ns + q; base_out = base_in;
    } else { base_in = line; base_out = line; }
    for (int64_t f = 0; f < nout; ++f) {
      double sr = 0.0, si = 0.0;
      for (int64_t t = 0; t < len; ++t) {
        const double xr = c->in[2 * (base_in + t * stride_in)] * c->w[t];
        const double xi = c->in[2 * (base_in + t * stride_in) + 1] * c->w[t];
        const int64_t j = (t * f) % nout;
        const double cr = c->tw[2 * j], ci = -c->tw[2 * j + 1]; /* e^{-2 pi i j/N} */
        sr += xr * cr - xi * ci;
        si += xr * ci + xi * cr;
      }
      c->out[2 * (base_out + f * stride_out)] = sr;
      c->out[2 * (base_out + f * stride_out) + 1] = si;
    }
  }
}

static double *twiddles(int64_t n) {
  double *t = (double *)malloc(sizeof(double) * 2 * (size_t)n);
  for (int64_t j = 0; j < n; ++j) {
    t[2 * j] = cos(ORC_TWO_PI * (double)j / (double)n);
    t[2 * j + 1] = sin(ORC_TWO_PI * (double)j / (double)n);
  }
  return t;
}

void orc_spectrum(const orc_radar *p, const double *signal, double *out, int nthreads) {
  const int64_t ns = p->n_samples, nc = p->n_chirps, nv = nv_of(p), na = p->n_angle;
  const size_t cube_v = (size_t)(nv * nc * ns * 2);
  double *t1 = (double *)malloc(sizeof(double) * cube_v);
  double *t2 = (double *)malloc(sizeof(double) * cube_v);
  double *wr = (double *)malloc(sizeof(double) * (size_t)ns);
  double *wd = (double *)malloc(sizeof(double) * (size_t)nc);
  double *wa = (double *)malloc(sizeof(double) * (size_t)nv);
  orc_window(p, 0, wr);
  orc_window(p, 1, wd);
  orc_window(p, 2, wa);
  double *tr = twiddles(ns), *td = twiddles(nc), *ta = twiddles(na);
  dft_ctx c0 = {p, signal, t1, wr, tr, 0};
  parallel_for(nv * nc, nthreads, dft_lines, &c0); /* range: along n */
  dft_ctx c1 = {p, t1, t2, wd, td, 1};
  parallel_for(nv * ns, nthreads, dft_lines, &c1); /* Doppler: along m */
  dft_ctx c2 = {p, t2, out, wa, ta, 2};
  parallel_for(nc * ns, nthreads, dft_lines, &c2); /* angle: along k, zero padded to N_a */
  free(t1); free(t2); free(wr); free(wd); free(wa); free(tr); free(td); free(ta);
}

/* --------------------------------------------------------------- per-cell windowed DTFT */
/* X[qa,qd,qr] = sum_i a_i e^{2 pi i carrier_i} W_a(nu_a - qa/N_a) W_d(nu_d - qd/N_c) W_r(nu_r - qr/N_s),
   W(delta) = sum_{t < L} w[t] e^{2 pi i delta t}: the separable sum of the signal model
   pushed through the three windowed DFTs term by term (linearity, Eq. 5). */
typedef struct {
  const orc_radar *p;
  const orc_rays *r;
  const ray_cycles *rc;
  const int64_t *cells;
  double *out;
  const double *w[3];
} dtft_ctx;

static void wdtft(const double *w, int len, double nu, int64_t q, int64_t nfft, double *re, double *im) {
  double sr = 0.0, si = 0.0;
  for (int t = 0; t < len; ++t) {
    double cr, ci;
    cis_cycles(frac(t * nu) - (double)((t * q) % nfft) / (double)nfft, &cr, &ci);
    sr += w[t] * cr;
    si += w[t] * ci;
  }
  *re = sr;
  *im = si;
}

/* the angle factor with transmitter slot offsets: sum_k w[k] e^{2 pi i (k nu_a + t(k) nu_t - k q / N)},
   t(k) = k / N_rx; it is wdtft when nu_t = 0 */
static void wdtft_tdm(const orc_radar *p, const double *w, int len, double nu, double nu_t, int64_t q,
                      int64_t nfft, double *re, double *im) {
  double sr = 0.0, si = 0.0;
  for (int t = 0; t < len; ++t) {
    double cr, ci;
    cis_cycles(frac(t * nu) + frac(tx_of(p, t) * nu_t) - (double)((t * q) % nfft) / (double)nfft, &cr, &ci);
    sr += w[t] * cr;
    si += w[t] * ci;
  }
  *re = sr;
  *im = si;
}

static void dtft_cells(void *vctx, int64_t lo, int64_t hi) {
  dtft_ctx *c = (dtft_ctx *)vctx;
  const int64_t ns = c->p->n_samples, nc = c->p->n_chirps, na = c->p->n_angle;
  const int nv = nv_of(c->p);
  for (int64_t t = lo; t < hi; ++t) {
    const int64_t f = c->cells[t];
    const int64_t qr = f % ns, qd = (f / ns) % nc, qa = f / (ns * nc);
    double sr = 0.0, si = 0.0;
    for (int64_t i = 0; i < c->r->n; ++i) {
      const ray_cycles *q = &c->rc[i];
      double ar, ai, dr, di, rr, ri, cr, ci;
      if (q->nu_t != 0.0)
        wdtft_tdm(c->p, c->w[2], nv, q->nu_a, q->nu_t, qa, na, &ar, &ai);
      else
        wdtft(c->w[2], nv, q->nu_a, qa, na, &ar, &ai);
      wdtft(c->w[1], (int)nc, q->nu_d, qd, nc, &dr, &di);
      wdtft(c->w[0], (int)ns, q->nu_r, qr, ns, &rr, &ri);
      cis_cycles(q->carrier, &cr, &ci);
      /* product of four complex factors, left to right */
      double xr = cr * ar - ci * ai, xi = cr * ai + ci * ar;
      double yr = xr * dr - xi * di, yi = xr * di + xi * dr;
      double zr = yr * rr - yi * ri, zi = yr * ri + yi * rr;
      sr += q->amp * zr;
      si += q->amp * zi;
    }
    c->out[2 * t] = sr;
    c->out[2 * t + 1] = si;
  }
}

void orc_cell_dtft(const orc_radar *p, const orc_rays *r, int64_t ncells, const int64_t *cells,
                   double *out, int nthreads) {
  ray_cycles *rc = all_cycles(p, r);
  double *wr = (double *)malloc(sizeof(double) * (size_t)p->n_samples);
  double *wd = (double *)malloc(sizeof(double) * (size_t)p->n_chirps);
  double *wa = (double *)malloc(sizeof(double) * (size_t)nv_of(p));
  orc_window(p, 0, wr);
  orc_window(p, 1, wd);
  orc_window(p, 2, wa);
  dtft_ctx c = {p, r, rc, cells, out, {wr, wd, wa}};
  parallel_for(ncells, nthreads, dtft_cells, &c);
  free(rc); free(wr); free(wd); free(wa);
}

/* --------------------------------------------------------------- virtual snapshots (Eq. 6, Eq. 7) */
/* hit h at chirp snapshot j: the stored barycentric coordinates applied to the triangle's
   vertices at that snapshot, p = (1 - u - v) v1 + u v2 + v v3 (Eq. 6) */
static void hit_position(const orc_geometry *g, int64_t j, int64_t h, double out[3]) {
  const int32_t *tri = g->triangles + 3 * (int64_t)g->hit_triangle[h];
  const double *V = g->vertices + j * g->n_vertices * 3;
  const double u = (double)g->hit_u[h], v = (double)g->hit_v[h];
  const double w = 1.0 - u - v;
  for (int c = 0; c < 3; ++c) {
    out[c] = w * V[3 * tri[0] + c] + u * V[3 * tri[1] + c] + v * V[3 * tri[2] + c];
  }
}

static double distance3(const double a[3], const double b[3]) {
  const double x = a[0] - b[0], y = a[1] - b[1], z = a[2] - b[2];
  return sqrt(x * x + y * y + z * z);
}

/* length between the first and the last hit at snapshot j */
static double inner_length(const orc_geometry *g, int64_t i, int64_t j) {
  double s = 0.0, prev[3], cur[3];
  hit_position(g, j, g->hit_offset[i], prev);
  for (int64_t h = g->hit_offset[i] + 1; h < g->hit_offset[i + 1]; ++h) {
    hit_position(g, j, h, cur);
    s += distance3(prev, cur);
    prev[0] = cur[0]; prev[1] = cur[1]; prev[2] = cur[2];
  }
  return s;
}

/* Eq. 7: the traced length minus the legs to the traced antennas at snapshot 0, plus the legs
   to transmitter t and receiver r at snapshot j; the path between the first and last hit is
   re-measured at snapshot j (the hits move with their triangles, Eq. 6) */
static double path_length(const orc_geometry *g, const orc_rays *r, int64_t i, int64_t j, int t, int rx) {
  const int64_t f = g->hit_offset[i], l = g->hit_offset[i + 1] - 1;
  double pf0[3], pl0[3], pfj[3], plj[3];
  hit_position(g, 0, f, pf0);
  hit_position(g, 0, l, pl0);
  hit_position(g, j, f, pfj);
  hit_position(g, j, l, plj);
  return r->range_rt_m[i] - distance3(pf0, g->ref_tx) + distance3(pfj, g->tx_pos + 3 * t) -
         inner_length(g, i, 0) + inner_length(g, i, j) - distance3(pl0, g->ref_rx) +
         distance3(plj, g->rx_pos + 3 * rx);
}

typedef struct {
  const orc_radar *p;
  const orc_rays *r;
  const orc_geometry *g;
  double *out;
  const int64_t *idx;
} geom_ctx;

static void paths_rays(void *vctx, int64_t lo, int64_t hi) {
  geom_ctx *c = (geom_ctx *)vctx;
  const int nc = c->p->n_chirps, nv = nv_of(c->p);
  for (int64_t i = lo; i < hi; ++i)
    for (int j = 0; j < nc; ++j)
      for (int k = 0; k < nv; ++k)
        c->out[(i * nc + j) * nv + k] = path_length(c->g, c->r, i, j, k / c->p->n_rx, k % c->p->n_rx);
}

void orc_paths(const orc_radar *p, const orc_rays *r, const orc_geometry *g, double *out, int nthreads) {
  geom_ctx c = {p, r, g, out, NULL};
  parallel_for(r->n, nthreads, paths_rays, &c);
}

/* one output sample of Eq. 2 with tau = l / c: sum_i a_i e^{2 pi i (f_c tau + mu t_n tau) + i phi0} */
static void geom_point(const geom_ctx *c, int64_t k, int64_t m, int64_t n, double *sr, double *si) {
  const orc_radar *p = c->p;
  const double mu = p->bandwidth_hz / p->sweep_time_s, dt = p->sweep_time_s / p->n_samples;
  double accr = 0.0, acci = 0.0;
  for (int64_t i = 0; i < c->r->n; ++i) {
    const double tau = path_length(c->g, c->r, i, m, (int)(k / p->n_rx), (int)(k % p->n_rx)) / ORC_C;
    const double amp = pattern_amp(p, (double)c->r->amplitude[i], (double)c->r->azimuth_rad[i],
                                   (double)c->r->elevation_rad[i]);
    double re, im;
    cis_cycles(frac(p->carrier_hz * tau) + frac((double)c->r->phase0_rad[i] / ORC_TWO_PI) +
                   frac(mu * (double)n * dt * tau), &re, &im);
    accr += amp * re;
    acci += amp * im;
  }
  *sr = accr;
  *si = acci;
}

static void geom_rows(void *vctx, int64_t lo, int64_t hi) {
  geom_ctx *c = (geom_ctx *)vctx;
  const int64_t ns = c->p->n_samples, nc = c->p->n_chirps;
  for (int64_t row = lo; row < hi; ++row)
    for (int64_t n = 0; n < ns; ++n)
      geom_point(c, row / nc, row % nc, n, &c->out[2 * (row * ns + n)], &c->out[2 * (row * ns + n) + 1]);
}

static void geom_points(void *vctx, int64_t lo, int64_t hi) {
  geom_ctx *c = (geom_ctx *)vctx;
  const int64_t ns = c->p->n_samples, nc = c->p->n_chirps;
  for (int64_t t = lo; t < hi; ++t) {
    const int64_t f = c->idx[t];
    geom_point(c, f / (ns * nc), (f / ns) % nc, f % ns, &c->out[2 * t], &c->out[2 * t + 1]);
  }
}

void orc_signal_geom(const orc_radar *p, const orc_rays *r, const orc_geometry *g, double *out, int nthreads) {
  geom_ctx c = {p, r, g, out, NULL};
  parallel_for((int64_t)nv_of(p) * p->n_chirps, nthreads, geom_rows, &c);
}

void orc_signal_geom_at(const orc_radar *p, const orc_rays *r, const orc_geometry *g, int64_t npts,
                        const int64_t *idx, double *out, int nthreads) {
  geom_ctx c = {p, r, g, out, idx};
  parallel_for(npts, nthreads, geom_points, &c);
}

/* --------------------------------------------------------------- polynomial sin / cos */
/* Cody-Waite reduction by pi/2 split into two doubles (P1 + P2), then Taylor series
   of sin and cos on [-pi/4, pi/4] in Horner form with fused multiply-adds in a fixed
   order.  |x| <= pi keeps the quotient k in -2..2 so k*P1 and k*P2 are exact and
   x - k*P1 is exact (Sterbenz). */
static const double CW_P1 = 0x1.921fb54442d18p+0;   /* pi/2 rounded to double */
static const double CW_P2 = 0x1.1a62633145c07p-54;  /* pi/2 - P1 rounded to double */
static const double CW_2_OVER_PI = 0x1.45f306dc9c883p-1;

static double taylor_sin(double r) {
  const double z = r * r;
  double p = 1.0 / 355687428096000.0;        /* +1/17! */
  p = fma(p, z, -1.0 / 1307674368000.0);     /* -1/15! */
  p = fma(p, z, 1.0 / 6227020800.0);         /* +1/13! */
  p = fma(p, z, -1.0 / 39916800.0);          /* -1/11! */
  p = fma(p, z, 1.0 / 362880.0);             /* +1/9!  */
  p = fma(p, z, -1.0 / 5040.0);              /* -1/7!  */
  p = fma(p, z, 1.0 / 120.0);                /* +1/5!  */
  p = fma(p, z, -1.0 / 6.0);                 /* -1/3!  */
  return fma(r * z, p, r);
}

static double taylor_cos(double r) {
  const double z = r * r;
  double q = -1.0 / 6402373705728000.0;      /* -1/18! */
  q = fma(q, z, 1.0 / 20922789888000.0);     /* +1/16! */
  q = fma(q, z, -1.0 / 87178291200.0);       /* -1/14! */
  q = fma(q, z, 1.0 / 479001600.0);          /* +1/12! */
  q = fma(q, z, -1.0 / 3628800.0);           /* -1/10! */
  q = fma(q, z, 1.0 / 40320.0);              /* +1/8!  */
  q = fma(q, z, -1.0 / 720.0);               /* -1/6!  */
  q = fma(q, z, 1.0 / 24.0);                 /* +1/4!  */
  q = fma(q, z, -1.0 / 2.0);                 /* -1/2!  */
  return fma(z, q, 1.0);
}

static void reduce_half_pi(double x, double *r, int *quadrant) {
  const double k = nearbyint(x * CW_2_OVER_PI);
  *r = (x - k * CW_P1) - k * CW_P2;
  *quadrant = ((int)k) & 3;
}

double orc_sin_rep(double x) {
  double r;
  int q;
  reduce_half_pi(x, &r, &q);
  switch (q) {
    case 0: return taylor_sin(r);
    case 1: return taylor_cos(r);
    case 2: return -taylor_sin(r);
    default: return -taylor_cos(r);
  }
}

double orc_cos_rep(double x) {
  double r;
  int q;
  reduce_half_pi(x, &r, &q);
  switch (q) {
    case 0: return taylor_cos(r);
    case 1: return -taylor_sin(r);
    case 2: return -taylor_cos(r);
    default: return taylor_sin(r);
  }
}

/* --------------------------------------------------------------- bins and labels */
/* Analytic bin coordinates of a ray, in the fixed operation order the labels use:
     x_r = (B d) / c                      range bin: the beat frequency mu tau over f_s/N_s
     x_d = ((((2 v) f_c) T_d) N_c) / c    Doppler bin: cycles per chirp times N_c
     x_a = (N_a s_wl) (sin(az) cos(el))   angle bin: cycles per channel times N_a
   q_x = floor(x + 0.5) reduced into [0, N_x); cell = (q_a N_c + q_d) N_s + q_r;
   energy = min(rint(a^2 2^32), 2^41). */
static int64_t bin_of(double x, int64_t n) {
  int64_t q = (int64_t)floor(x + 0.5);
  q %= n;
  if (q < 0) q += n;
  return q;
}

void orc_bins(const orc_radar *p, const orc_rays *r, double *xr, double *xd, double *xa,
              int64_t *cell, int64_t *energy) {
  const int64_t ns = p->n_samples, nc = p->n_chirps, na = p->n_angle;
  const double ka = (double)p->n_angle * spacing_wl(p);
  for (int64_t i = 0; i < r->n; ++i) {
    const double d = r->range_rt_m[i];
    const double v = (double)r->radial_velocity_mps[i];
    const double x_r = (p->bandwidth_hz * d) / ORC_C;
    const double x_d = ((((2.0 * v) * p->carrier_hz) * p->chirp_period_s) * (double)p->n_chirps) / ORC_C;
    const double x_a = ka * (orc_sin_rep((double)r->azimuth_rad[i]) * orc_cos_rep((double)r->elevation_rad[i]));
    if (xr) xr[i] = x_r;
    if (xd) xd[i] = x_d;
    if (xa) xa[i] = x_a;
    if (cell) cell[i] = (bin_of(x_a, na) * nc + bin_of(x_d, nc)) * ns + bin_of(x_r, ns);
    if (energy) {
      const double a = pattern_amp(p, (double)r->amplitude[i], (double)r->azimuth_rad[i],
                                   (double)r->elevation_rad[i]);
      double e = nearbyint(ldexp(a * a, 32));
      if (e > 2199023255552.0) e = 2199023255552.0; /* 2^41 */
      energy[i] = (int64_t)e;
    }
  }
}

typedef struct {
  int64_t cell;
  int32_t obj;
  int64_t e;
} cell_obj;

static int cmp_cell_obj(const void *a, const void *b) {
  const cell_obj *x = (const cell_obj *)a, *y = (const cell_obj *)b;
  if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
  if (x->obj != y->obj) return x->obj < y->obj ? -1 : 1;
  return 0;
}

int64_t orc_cell_object_energy(const orc_radar *p, const orc_rays *r, const int32_t *object_id,
                               int64_t *cell, int32_t *obj, int64_t *energy) {
  const int64_t n = r->n;
  if (n == 0) return 0;
  int64_t *c = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *e = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  orc_bins(p, r, NULL, NULL, NULL, c, e);
  cell_obj *v = (cell_obj *)malloc(sizeof(cell_obj) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    v[i].cell = c[i];
    v[i].obj = object_id[i];
    v[i].e = e[i];
  }
  qsort(v, (size_t)n, sizeof(cell_obj), cmp_cell_obj);
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (m > 0 && cell[m - 1] == v[i].cell && obj[m - 1] == v[i].obj) {
      energy[m - 1] += v[i].e;
    } else {
      cell[m] = v[i].cell;
      obj[m] = v[i].obj;
      energy[m] = v[i].e;
      ++m;
    }
  }
  free(c); free(e); free(v);
  return m;
}

void orc_labels(const orc_radar *p, const orc_rays *r, const int32_t *object_id, int32_t *labels) {
  const int64_t ncell = (int64_t)p->n_angle * p->n_chirps * p->n_samples;
  for (int64_t t = 0; t < ncell; ++t) labels[t] = -1;
  const int64_t n = r->n;
  if (n == 0) return;
  int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int32_t *obj = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int64_t *e = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  const int64_t m = orc_cell_object_energy(p, r, object_id, cell, obj, e);
  /* pairs are sorted by (cell, obj): the first strict maximum in each cell is the
     largest energy with the smallest id */
  int64_t best_e = -1;
  for (int64_t t = 0; t < m; ++t) {
    if (t == 0 || cell[t] != cell[t - 1]) best_e = -1;
    if (e[t] > best_e) {
      best_e = e[t];
      labels[cell[t]] = obj[t];
    }
  }
  free(cell); free(obj); free(e);
}
