/*
 * FP64 CPU oracle for the FMCW ray-sum -> range-Doppler-angle spectrum -> label path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: it exists so that the tests, the smoke check and the CPU
 * baseline of the benchmark can compare the CUDA library against a plain,
 * slow, obviously correct restatement of the paper's signal model.  It shares
 * no code, header, table or constant with the CUDA library.
 *
 * Paper: Schuessler et al., "Achieving Efficient and Realistic Full-Radar
 * Simulations and Automatic Data Annotation by exploiting Ray Meta Data of a
 * Radar Ray Tracing Simulator" (arXiv 2305.14176).
 *   Eq. 1  tau_i = d_i(j) / c                          (Sec. II-A)
 *   Eq. 2  s_IF(t,j) = sum_i A exp(2 pi j (mu t tau_i(j) + f_c tau_i(j)))
 *   Eq. 3  mu = B / T_c
 *   Eq. 4  S_IF(f_r, f_d) = DFT_2d(s_IF(t, j))  (zero padding, windows omitted)
 *   Eq. 5  s_IF = sum_h s_IF^h                      (Sec. II-C, decomposition)
 *   Eq. 7  far-field antenna displacement            (Sec. II-E)
 *
 * Every floating-point quantity is FP64; the library is compiled with
 * -ffp-contract=off so the written operation order is the evaluated one.
 */
#ifndef RADAR_ORACLE_H
#define RADAR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double carrier_hz;        /* f_c */
  double bandwidth_hz;      /* B */
  double sweep_time_s;      /* T_c: sweep = sampling window (Eq. 3) */
  double chirp_period_s;    /* T_d: time between chirps (Sec. II-A) */
  int32_t n_samples;        /* N_s fast-time samples per chirp */
  int32_t n_chirps;         /* N_c chirps */
  int32_t n_tx, n_rx;       /* virtual channel k = tx * n_rx + rx */
  double element_spacing_m; /* virtual ULA spacing; 0 => half a wavelength */
  int32_t n_angle;          /* angle DFT length N_a >= N_v (zero padded) */
  int32_t window[3];        /* range, Doppler, angle: 0 none, 1 periodic Hann,
                               2 symmetric Hann, 3 Hann without zero end points */
  int32_t model;            /* 0: separable Eq. 2; 1: Eq. 2 with mu t (tau_i(j) - tau_i(0)) */
  int32_t pattern_exp;      /* antenna pattern A(az, el) = (cos az cos el)^q; 0: isotropic */
  double tdm_slot_s;        /* TDM-MIMO: transmitter t sends chirp j at j T_d + t tdm_slot_s */
} orc_radar;

typedef struct {
  int64_t n;
  const double *range_rt_m;        /* round-trip path length d_i */
  const float *amplitude;          /* a_i */
  const float *radial_velocity_mps;/* v_i, > 0 receding */
  const float *azimuth_rad;
  const float *elevation_rad;
  const float *phase0_rad;         /* start phase phi0_i */
} orc_rays;

/* Beat-signal cube s[k][m][n] (complex, interleaved re/im), k < N_v, m < N_c, n < N_s. */
void orc_signal(const orc_radar *p, const orc_rays *r, double *out, int nthreads);
/* The same sum evaluated only at flat indices (k*N_c + m)*N_s + n. */
void orc_signal_at(const orc_radar *p, const orc_rays *r, int64_t npts, const int64_t *idx,
                   double *out, int nthreads);
/* Windowed, zero-padded DFT of a signal cube: X[a][p][q], a < N_a (naive O(N^2) per axis). */
void orc_spectrum(const orc_radar *p, const double *signal, double *out, int nthreads);
/* Spectrum cells evaluated directly from the rays by the windowed-DTFT form:
   flat cell index (a*N_c + p)*N_s + q. */
void orc_cell_dtft(const orc_radar *p, const orc_rays *r, int64_t ncells, const int64_t *cells,
                   double *out, int nthreads);
/* Window w[t] for axis 0 (range), 1 (Doppler), 2 (angle, length N_v). */
void orc_window(const orc_radar *p, int axis, double *out);
/* Per-ray analytic bin coordinates x_r, x_d, x_a, cell index and fixed-point energy. */
void orc_bins(const orc_radar *p, const orc_rays *r, double *xr, double *xd, double *xa,
              int64_t *cell, int64_t *energy);
/* Per-cell labels int32[N_a][N_c][N_s]: object with the largest summed energy, ties to
   the smallest id, -1 for cells no ray falls in. */
void orc_labels(const orc_radar *p, const orc_rays *r, const int32_t *object_id, int32_t *labels);
/* Per-(cell, object) summed energies for the cells rays fall in, sorted by (cell, object).
   Returns the number of pairs; arrays must hold r->n entries. */
int64_t orc_cell_object_energy(const orc_radar *p, const orc_rays *r, const int32_t *object_id,
                               int64_t *cell, int32_t *obj, int64_t *energy);
/* Moving scene for virtual snapshots (Sec. II-D, Eq. 6) and antenna displacement (Sec. II-E,
   Eq. 7).  Ray i hit the triangles hit_triangle[h], h = hit_offset[i] .. hit_offset[i+1]-1, in
   path order (first hit first), at barycentric coordinates (hit_u, hit_v); its traced path
   length d_i runs from ref_tx over those hits to ref_rx at snapshot 0. */
typedef struct {
  int64_t n_vertices, n_triangles;
  const double *vertices;    /* [N_c][n_vertices][3]: vertex positions at t = j T_d (m) */
  const int32_t *triangles;  /* [n_triangles][3] vertex indices */
  const double *tx_pos;      /* [n_tx][3] transmitter positions */
  const double *rx_pos;      /* [n_rx][3] receiver positions */
  double ref_tx[3], ref_rx[3];
  const int64_t *hit_offset; /* [n + 1] */
  const int32_t *hit_triangle;
  const float *hit_u, *hit_v;
} orc_geometry;

/* Path length of every ray at every chirp snapshot and virtual channel k = tx N_rx + rx:
   out[i][j][k] (Eq. 6 hit positions, Eq. 7 antenna displacement, inner path updated). */
void orc_paths(const orc_radar *p, const orc_rays *r, const orc_geometry *g, double *out, int nthreads);
/* Eq. 2 with those path lengths, tau_i(j, k) = l_i(j, k) / c in both the beat and the carrier
   term: the signal cube, or its values at flat indices (k*N_c + m)*N_s + n. */
void orc_signal_geom(const orc_radar *p, const orc_rays *r, const orc_geometry *g, double *out, int nthreads);
void orc_signal_geom_at(const orc_radar *p, const orc_rays *r, const orc_geometry *g, int64_t npts,
                        const int64_t *idx, double *out, int nthreads);

/* The polynomial sine/cosine used for the angle bin (Cody-Waite + Taylor). |x| <= pi. */
double orc_sin_rep(double x);
double orc_cos_rep(double x);
/* Number of host threads used when nthreads <= 0. */
int orc_default_threads(void);

#ifdef __cplusplus
}
#endif
#endif
