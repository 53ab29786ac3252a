/*
 * radarsim — GB300 (sm_103a) FMCW radar data from ray-tracer output and meta data.
 *
 * C ABI of libradarsim.so.  It turns the per-ray output of a radar ray tracer
 * (round-trip path length, amplitude, radial velocity, azimuth/elevation,
 * start phase) and its meta data (object id, material id) into
 *   1. the complex beat-signal cube s[k][m][n] of every virtual channel k,
 *      chirp m and fast-time sample n (arXiv 2305.14176, Sec. II-A, Eqs. 1-3,
 *      with the far-field antenna adjustment of Sec. II-E, Eq. 7),
 *   2. its windowed range-Doppler-angle spectrum (Sec. II-A, Eq. 4, extended
 *      along the virtual channels), and
 *   3. a per-cell object label: the id whose rays deposit the most energy in
 *      the cell (Sec. II-C, Eq. 5 decomposition by meta data, and the automatic
 *      annotation that follows it).
 *
 * Signal model (separable reading of Eq. 2):
 *   s[k][m][n] = sum_i a_i exp(2 pi j (phi_i + k nu_a,i + m nu_d,i + n nu_r,i))
 *   phi_i  = f_c d_i / c + phase0_i / 2pi           carrier phase (Eq. 2, f_c tau)
 *   nu_r,i = B d_i / (c N_s)                        Eq. 2 mu t tau, t = n T_c / N_s, Eq. 3
 *   nu_d,i = 2 v_i f_c T_d / c                      Eq. 2 f_c tau_i(j), d grows 2 v T_d per chirp
 *   nu_a,i = s f_c sin(az_i) cos(el_i) / c          Eq. 7 in the far field, ULA spacing s
 * with c = 299792458 m/s.  Virtual channel k = tx * n_rx + rx sits at k * s.  With a TDM
 * slot time the phase gains tx nu_t,i (see tdm_slot_s); the labels keep the physical cell.
 *
 * Spectrum X[a][p][q] = sum_{k<N_v, m<N_c, n<N_s} w_a[k] w_d[m] w_r[n] s[k][m][n]
 *                        e^{-2 pi j (k a / N_a + m p / N_c + n q / N_s)}
 * forward, unnormalised, natural order (bin 0 = DC); the angle axis is zero
 * padded from N_v to N_a.
 *
 * Labels: each ray's cell is (q_a, q_d, q_r) with q_x = floor(x + 0.5) mod N_x,
 *   x_r = (B d) / c, x_d = ((((2 v) f_c) T_d) N_c) / c,
 *   x_a = (N_a s f_c / c) (sin(az) cos(el)),
 * in FP64 in exactly this order (sin, cos by Cody-Waite reduction and Taylor
 * series in a fixed fused-multiply-add order); its energy is
 * min(rint(a'^2 2^32), 2^41) as int64, a' = a (cos(az) cos(el))^q the amplitude after the
 * antenna pattern (q = pattern_exp; the same cos polynomial, q multiplications in order).  A cell's label is the object id with the
 * largest summed energy, ties to the smallest id, -1 for a cell no ray falls in.
 *
 * Layouts (row-major, last index fastest, complex = interleaved float re, im):
 *   signal    complex64[N_v][N_c][N_s]
 *   spectrum  complex64[N_a][N_c][N_s]
 *   labels    int32[N_a][N_c][N_s]
 *
 * Errors: every call returns an int status (SIM_OK or a negative SIM_E_*);
 * nothing aborts or throws across the ABI.  All calls are thread-safe.
 */
#ifndef RADARSIM_H
#define RADARSIM_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RADARSIM_ABI_VERSION 1

#if defined(__GNUC__)
#define SIM_API __attribute__((visibility("default")))
#else
#define SIM_API
#endif

/* status codes */
#define SIM_OK 0
#define SIM_E_INVALID (-1)        /* bad parameters or ray values */
#define SIM_E_NOMEM (-2)          /* device or host allocation failed */
#define SIM_E_BUSY (-3)           /* admission refused: memory budget or queue full */
#define SIM_E_TIMEOUT (-4)        /* sim_fetch timed out; the ticket stays valid */
#define SIM_E_NOT_READY (-5)      /* ticket not finished (timeout_ms == 0) */
#define SIM_E_UNKNOWN_TICKET (-6) /* ticket never issued, already fetched or for another context */
#define SIM_E_CUDA (-7)           /* a CUDA runtime call failed */
#define SIM_E_DEVICE (-8)         /* a kernel reported an internal limit (status word) */

/* window codes */
#define SIM_WIN_NONE 0
#define SIM_WIN_HANN_PERIODIC 1   /* w[t] = (1 - cos(2 pi t / L)) / 2 */
#define SIM_WIN_HANN_SYMMETRIC 2  /* w[t] = (1 - cos(2 pi t / (L - 1))) / 2 */
#define SIM_WIN_HANN_NOZERO 3     /* w[t] = (1 - cos(2 pi (t + 1) / (L + 1))) / 2 */

/* ray-sum arithmetic */
#define SIM_PREC_FP32_DIRECT 0    /* one FP32 sin/cos per ray and output sample */
#define SIM_PREC_BF16 1           /* tensor-core GEMM, BF16 operands, FP32 accumulation */
#define SIM_PREC_BF16_SPLIT 2     /* BF16 hi + lo operands, three MMAs */
#define SIM_PREC_FP16 3
#define SIM_PREC_FP16_SPLIT 4

/* signal model */
#define SIM_MODEL_SEPARABLE 0     /* Eq. 2 without the range-migration product (a GEMM) */
#define SIM_MODEL_EXACT 1         /* Eq. 2 with mu t (tau_i(j) - tau_i(0)): phase + n m eps_i,
                                     eps_i = B 2 v_i T_d / (c N_s); any precision.  The tensor-core
                                     precisions expand the coupling about each output tile's centre
                                     (4 Taylor or 4, 6, 8 Chebyshev terms, truncation <= 1e-6 of a contribution at
                                     hi + lo, 1e-5 single pass); a scene beyond that bound runs per
                                     chirp instead.  With tdm_slot_s > 0 they need n_samples >= 32,
                                     and a scene beyond the bound is reported as SIM_E_INVALID. */

/* outputs bitmask */
#define SIM_OUT_SIGNAL 1
#define SIM_OUT_SPECTRUM 2
#define SIM_OUT_LABELS 4

typedef struct sim_ctx sim_ctx; /* opaque: one radar configuration */

typedef struct {
  uint32_t struct_size;      /* sizeof(sim_radar_params) of the caller's header */
  double carrier_hz;         /* f_c > 0 */
  double bandwidth_hz;       /* B > 0 */
  double sweep_time_s;       /* T_c > 0: sweep and sampling window */
  double chirp_period_s;     /* T_d > 0: chirp repetition period */
  int32_t n_samples;         /* N_s: power of two, 16 .. 4096 */
  int32_t n_chirps;          /* N_c: power of two, 2 .. 4096 */
  int32_t n_tx, n_rx;        /* >= 1 each; N_v = n_tx * n_rx <= 1024 */
  double element_spacing_m;  /* virtual ULA spacing s >= 0; 0 means lambda / 2 */
  int32_t n_angle;           /* N_a: power of two >= N_v, <= 1024; 0 means max(16, nextpow2(N_v)) */
  int32_t window[3];         /* range, Doppler, angle: SIM_WIN_* */
  int32_t precision;         /* SIM_PREC_* */
  int32_t outputs;           /* SIM_OUT_* bitmask, nonzero */
  int64_t max_rays;          /* 1 .. 2^21 (keeps the int64 energy sums exact) */
  int32_t model;             /* SIM_MODEL_SEPARABLE or SIM_MODEL_EXACT */
  int32_t pattern_exp;       /* antenna pattern A = (cos(az) cos(el))^q, q = 0 .. 16 (0: isotropic) */
  double tdm_slot_s;         /* TDM-MIMO slot time T_slot >= 0: transmitter tx sends chirp m at
                                m T_d + tx T_slot, adding tx nu_t,i = tx 2 v_i f_c T_slot / c cycles
                                (and, in the exact model, n tx B 2 v_i T_slot / (c N_s)); 0 = none */
} sim_radar_params;

/* Structure-of-arrays rays.  Each pointer holds n elements; pointers may be
   host (pageable or pinned) or device memory of the current device. */
typedef struct {
  int64_t n;                        /* 0 .. max_rays */
  const double *range_rt_m;         /* d_i >= 0: Tx -> scatterers -> Rx path length */
  const float *amplitude;           /* a_i >= 0 */
  const float *radial_velocity_mps; /* v_i, > 0 receding; finite */
  const float *azimuth_rad;         /* |az| <= pi */
  const float *elevation_rad;       /* |el| <= pi/2 */
  const float *phase0_rad;          /* finite */
} sim_rays;

typedef struct {
  const int32_t *object_id;   /* >= 0; required when SIM_OUT_LABELS is requested */
  const int32_t *material_id; /* may be NULL; used by sim_decompose's span rules */
  const int32_t *n_hits;      /* may be NULL; number of scatterer hits on the ray's path */
} sim_meta;

/* Validate params, derive the radar constants and upload the window and twiddle
   tables.  *out receives a context owned by the caller until sim_destroy.
   Errors: SIM_E_INVALID (bad params, *out untouched), SIM_E_NOMEM, SIM_E_CUDA. */
SIM_API int sim_create(const sim_radar_params *params, sim_ctx **out);

/* Queue one scene.  The ray arrays (and meta arrays) are copied before the call
   returns; the caller may reuse them at once.  Work starts on the device as soon
   as the engine admits the scene (free memory budget and a free slot); otherwise it
   waits in a bounded queue.  A slot (a stream) frees when its scene finishes on the
   device; memory frees when a result is fetched.  Admitted scenes run concurrently.
   *ticket_out identifies the result for sim_fetch.
   Errors: SIM_E_INVALID (n out of range, NULL array, a host ray with a bad value),
   SIM_E_BUSY (queue full, or the scene alone exceeds the memory budget),
   SIM_E_NOMEM, SIM_E_CUDA.  Invalid values in device-resident rays are reported
   by sim_fetch as SIM_E_INVALID. */
SIM_API int sim_submit(sim_ctx *ctx, const sim_rays *rays, const sim_meta *meta, uint64_t *ticket_out);

/* Wait for a ticket and copy its results out.  spectrum (complex64), signal
   (complex64) and labels (int32) are caller-owned host or device buffers in the
   layouts above; each may be NULL if not wanted and must be NULL if the context
   was created without that output.  timeout_ms < 0 waits forever, 0 polls.
   On SIM_OK the ticket is consumed and its device memory released.
   A queued ticket is admitted only when earlier results are fetched (their memory and
   slots free up): fetching it while no other fetch is under way and the queue head cannot
   be admitted returns SIM_E_BUSY at once (ticket kept) instead of waiting forever.
   Errors: SIM_E_UNKNOWN_TICKET, SIM_E_TIMEOUT / SIM_E_NOT_READY / SIM_E_BUSY (ticket kept),
   SIM_E_INVALID (the scene held an invalid ray, or - exact model with TDM slots on tensor
   cores - a range migration beyond the expansion's bound; ticket consumed, outputs undefined),
   SIM_E_DEVICE, SIM_E_CUDA. */
SIM_API int sim_fetch(sim_ctx *ctx, uint64_t ticket, void *spectrum_c64, void *signal_c64,
              int32_t *labels, int32_t timeout_ms);

/* Release a context.  Unfetched tickets of the context are waited for and dropped. */
SIM_API int sim_destroy(sim_ctx *ctx);

/* Static string for a status code. */
SIM_API const char *sim_status_string(int status);

/* ---- virtual snapshots and antenna displacement (Sec. II-D Eq. 6, Sec. II-E Eq. 7) ----
   A ray traced once (first chirp, one transmitter / receiver pair) keeps its hits as
   (triangle, u, v).  At chirp j a hit sits at (1 - u - v) v1 + u v2 + v v3 of its triangle's
   vertices at that snapshot (Eq. 6); the ray's path to transmitter t and receiver r is its
   traced length d with both antenna legs replaced (Eq. 7) and the stretch between its first
   and last hit measured again at snapshot j:
     l(j, t, r) = d + [inner(j) - inner(0)] + |p_f(j) - x_t| - |p_f(0) - ref_tx|
                    + |p_l(j) - x_r| - |p_l(0) - ref_rx|.
   Coordinates in metres, FP64. */
typedef struct {
  int64_t n_vertices;         /* V, 1 .. 2^31 */
  int64_t n_triangles;        /* 1 .. 2^31 */
  const double *vertices;     /* [N_c][V][3]: vertex positions at t = j T_d, one snapshot per chirp */
  const int32_t *triangles;   /* [n_triangles][3] vertex indices in [0, V) */
  const double *tx_pos;       /* [n_tx][3] transmitter positions */
  const double *rx_pos;       /* [n_rx][3] receiver positions */
  double ref_tx[3];           /* the transmitter and receiver the rays were traced between */
  double ref_rx[3];
} sim_geometry;

/* Hit lists in CSR form: ray i hit triangle[h] at (u[h], v[h]) for h = offset[i] ..
   offset[i+1] - 1, first hit first; offset[0] = 0 and every ray has at least one hit. */
typedef struct {
  const int64_t *offset;      /* [n + 1] */
  const int32_t *triangle;    /* [offset[n]] indices in [0, n_triangles) */
  const float *u;             /* [offset[n]] barycentric coordinates */
  const float *v;
} sim_hits;

/* Path lengths l(j, t, r) of every ray into paths, double[n][N_c][N_v] (k = t N_rx + r), host or
   device.  The context gives N_c, n_tx, n_rx (any precision: the paths do not depend on it)
   and must have no TDM slot time.  The reference legs are carried in float-float arithmetic
   (~48 bits, ~1e-12 m on a 100 m leg), the antenna offsets from them in FP32 (~3e-7 of the
   offset).  All arrays host or device (as for sim_submit).  Synchronous.  Its working memory
   stays in the context between calls (grown when a call needs more, freed by sim_destroy);
   a call made while another one holds it allocates its own for its duration.
   SIM_E_INVALID for bad arguments, a hit list or index out of range (checked before any
   access) or a ray failing sim_submit's checks. */
SIM_API int sim_snapshot_paths(sim_ctx *ctx, const sim_rays *rays, const sim_hits *hits, const sim_geometry *geom,
                               double *paths);

/* The scene through Eq. 2 with tau = l(j, t, r) / c in both the beat and the carrier term
   (channel k = t N_rx + r, chirp m = j):
     s[k][m][n] = sum_i a_i' exp(2 pi j (f_c l / c + n B l / (c N_s)) + j phase0_i),
   a_i' the amplitude after the antenna pattern; then the spectrum and the labels as for
   sim_fetch (labels from the rays' analytic cells of d, v, az, el).  Any of spectrum,
   signal, labels may be NULL (not all); spectrum and labels need the context's outputs
   bit.  Same context limits, memory and errors as sim_snapshot_paths.  Rays go in chunks
   whose phase words (8 bytes per ray, chirp and antenna) fit 3 GiB.  SIM_PREC_FP32_DIRECT sums each chunk directly; the
   tensor-core precisions expand each tile's coupling of samples and rows about its centre,
   the exact-model expansion with every row's own phase words (4 Taylor or 4, 6, 8
   Chebyshev terms, truncation
   <= 1e-6 of a contribution at hi + lo, 1e-5 single pass, chosen on the device per chunk).
   A chunk beyond that bound, or N_s < 32, is summed directly in FP32. */
SIM_API int sim_snapshot_run(sim_ctx *ctx, const sim_rays *rays, const sim_meta *meta, const sim_hits *hits,
                             const sim_geometry *geom, void *spectrum, void *signal, int32_t *labels);

/* ---- decomposition by ray meta data (Sec. II-C, Eq. 5) ----
   A span rule selects rays by meta data; a ray belongs to the span when every set field
   matches (then `exclude` complements the result):
     object_id >= 0    : object (mesh) id equals it (needs meta.object_id)
     material_id >= 0  : material id equals it (needs meta.material_id)
     min_hits > 0 or max_hits >= 0 : min_hits <= n_hits <= max_hits, max_hits -1 = no upper
                         bound (needs meta.n_hits)
   e.g. "any hit on the pedestrian", "more than one hit" (ghosts: min_hits 2), "line of
   sight of object 7" (object_id 7, min_hits 1, max_hits 1). */
typedef struct {
  int32_t object_id;
  int32_t material_id;
  int32_t min_hits;
  int32_t max_hits;
  int32_t exclude;
} sim_span_rule;

/* Split one scene into n_spans parts s^h by the rules (1 <= n_spans <= 64), each summed over
   its rays only with the context's ray-sum arithmetic and model, and transformed like the
   spectrum.  span_spectra[h] (nullable array / entries): complex64[N_a][N_c][N_s] per span.
   span_labels (nullable): int32[N_a][N_c][N_s], per cell the span h with the largest
   |X_h|^2 among spans with |X_h|^2 >= threshold^2 * max_{h, cells} |X_h|^2 (a binary
   segmentation of each span image; ties to the lower h), -1 if none passes.  0 <= threshold
   <= 1. Rays and meta: host or device, as for sim_submit. Synchronous; its working memory,
   outside the engine's budget, stays in the context between calls as for sim_snapshot_paths.
   Each span's rays are packed in ray order and summed alone (up to four spans at once, on their
   own streams), so a span costs its own ray count and its part is the scene of its rays alone:
   bit for bit with SIM_PREC_FP32_DIRECT or the exact model, and with the other precisions up to
   the regrouping of FP32 sums (a span's tensor-core sum is split into fewer parts than a scene
   alone, since the spans share the GPU: ~1e-6 of the norm at hi + lo, ~1e-5 single pass).
   Repeated calls give the same bits. The parts of spans that partition the rays add up to the
   whole scene (Eq. 5). Errors: SIM_E_INVALID (bad rule, missing meta a rule needs, bad ray),
   SIM_E_NOMEM, SIM_E_CUDA, SIM_E_DEVICE. */
SIM_API int sim_decompose(sim_ctx *ctx, const sim_rays *rays, const sim_meta *meta, int32_t n_spans,
                          const sim_span_rule *rules, void *const *span_spectra, int32_t *span_labels,
                          float threshold);

/* ---- engine controls and measurement (not part of the paper's method) ---- */

/* Device-memory budget of the engine in bytes (0 = default: 90 % of the free
   memory when the engine starts), the number of concurrent slots (streams; 2 unless
   configured) and the queue length (64 unless configured).
   Must be called before the first sim_create; SIM_E_INVALID afterwards. */
SIM_API int sim_engine_configure(int64_t memory_budget_bytes, int32_t slots, int32_t max_queue);

/* Device bytes the engine holds for one submitted scene of n_rays rays on this context (its
   inputs, per-ray data, signal, spectrum, labels, label tables and ray-sum workspace): the
   amount the memory budget of sim_engine_configure is charged while the scene is admitted,
   for callers that plan a budget.  Not a compute call; the result follows the current tuning
   table.  Errors: SIM_E_INVALID (null pointers, n_rays < 0 or above the context's max_rays). */
SIM_API int sim_scene_bytes(const sim_ctx *ctx, int64_t n_rays, int64_t *bytes);

/* Per-stage device time in milliseconds of the most recently fetched ticket of
   this context, from CUDA events on the stream the scene ran on: [0] ingest
   copies, [1] per-ray prep, [2] ray-sum main kernel, [3] ray-sum split reduction,
   [4] FFTs, [5] labels (they run on a second stream beside the ray sum once the prep is done;
   this is the time they add after the FFTs), [6] whole device pipeline; n is the array
   length (<= 8).
   Entries for stages that did not run are 0.  sim_snapshot_run also records its
   stages here: [1] holds the prep and the path / phase-word kernels, [2] the direct
   sums, [6] prep to labels (its input copies happen before, synchronously).  So does a
   successful sim_decompose: [1] prep and the span sizes, [2] the spans' packing, ray sums
   and FFTs (they overlap on up to four streams), [5] the span labels, [6] prep to labels
   (including the wait for the span sizes and the allocation of the spans' scratch). */
SIM_API int sim_last_stage_ms(sim_ctx *ctx, float *ms, int32_t n);

/* Number of kernels the most recently fetched ticket of this context launched (or the last
   sim_snapshot_run or sim_decompose on it). */
SIM_API int sim_last_kernel_count(sim_ctx *ctx, int32_t *count);

/* Which form the tensor-core ray sum of the exact model (Sec. II-A, Eq. 2 with the
   range-migration term) or of virtual snapshots (Sec. II-D and II-E, Eq. 6 and 7) took in the
   most recently fetched ticket of this context (or the last sim_snapshot_run or sim_decompose
   on it), as a bit mask over its ray chunks and spans: bit P (P = 4, 6 or 8) when one ran the
   per-tile expansion of the coupling phase with P Taylor terms, bit 16 + P with P Chebyshev
   (Jacobi-Anger) terms; bit 0 when one lay beyond the expansion's bound and ran the per-chirp
   product (snapshots: the direct pair sum).  0 when no
   ray sum chose a term count (the separable model, SIM_PREC_FP32_DIRECT, fewer than 32
   samples, no ray) and after a failed sim_fetch; a failed sim_snapshot_run or sim_decompose
   leaves it, like the stage times, as it was.  Errors: SIM_E_INVALID (null pointer). */
SIM_API int sim_last_expansion_terms(sim_ctx *ctx, uint32_t *mask);

/* Run a batch of scenes as one device pipeline: per-scene prep, ONE persistent
   tensor-core launch over the (scene, tile, split) work units of all scenes, longest
   first, then per-scene split reduction, FFTs and labels.  The pipeline is captured into
   a CUDA graph the first time a batch shape (every scene's radar constants and ray count,
   in order) is seen, and replayed on later calls of the same shape (a few shapes are
   cached).  Each scene gives bit-identical results to sim_submit/sim_fetch of it alone.
   ctxs[i] may repeat or differ; all must use one tensor-core precision (not FP32_DIRECT).
   rays[i], meta[i]: as for sim_submit (host or device).  spectra / signals / labels:
   arrays of n output pointers (host or device, layouts as for sim_fetch), each array or
   entry may be NULL.  Synchronous.  device_ms (nullable) receives the device time of the
   pipeline without the input and output copies; kernel_count (nullable) the number of
   kernels it launched.
   Errors: SIM_E_INVALID, SIM_E_NOMEM, SIM_E_CUDA, SIM_E_DEVICE. */
SIM_API int sim_run_batch(int32_t n, sim_ctx *const *ctxs, const sim_rays *rays, const sim_meta *meta,
                          void *const *spectra, void *const *signals, int32_t *const *labels, float *device_ms,
                          int32_t *kernel_count);

/* ---- autotuner ----
   sim_autotune times, on the device and with synthetic rays of the context's shape,
   the tensor-core ray sum in its built-in plan and at several split-K counts and the FFT
   passes at several tile widths, and stores the fastest choice in a process-wide table keyed by (N_v, N_c,
   N_s, N_a, precision, ceil(log2 n_rays)).  Every later launch of that shape uses it
   (single scenes, batches, sim_raysum_noalloc), so tune before serving: results of one
   shape stay bit-identical for as long as the table does.  out (nullable) receives the
   choice and its timings.  Errors: SIM_E_INVALID, SIM_E_NOMEM, SIM_E_CUDA. */
typedef struct {
  int32_t splits;            /* split-K count of the ray sum (0: the built-in plan, which at hi + lo
                                precisions divides the work stream-K; FP32 direct is not tuned) */
  int32_t fft_range_points;  /* points per block of the range FFT (0: built-in choice) */
  int32_t fft_doppler_strip; /* samples per block of the Doppler FFT (0: built-in) */
  int32_t fft_angle_strip;   /* (m, n) positions per block of the angle FFT (0: built-in) */
  float ray_sum_ms;          /* device time of the chosen ray sum */
  float fft_ms;              /* device time of the chosen FFTs */
} sim_tuning;
SIM_API int sim_autotune(sim_ctx *ctx, int64_t n_rays, sim_tuning *out);
/* Write / read the table as a JSON array, one object per line.  Loading adds to the
   table (entries with out-of-range values are skipped).  The engine loads the file named
   by the environment variable RADARSIM_TUNE_CACHE when it starts. */
SIM_API int sim_tuning_save(const char *path);
SIM_API int sim_tuning_load(const char *path);
SIM_API int sim_tuning_clear(void);
/* number of tuned shapes in the table (not a status) */
SIM_API int sim_tuning_count(void);

/* Self-test of the tensor-core tile path on caller data (not a simulation call):
   D[M][N] = A[M][K] * B[N][K]^T with A, B row-major 16-bit (f16 bit 0 set: FP16, else
   BF16; bit 1 set: the instruction descriptor's negate-B bit, D = -A B^T) device matrices and D row-major FP32 device memory, through the same shared
   memory layout, descriptors and tcgen05 pipeline the ray sum uses.  N a multiple of
   16 in 32 .. 512 (a multiple of 256 above 256), K even, M >= 1.  stream is a
   cudaStream_t (NULL = default stream); the call synchronizes it.
   Errors: SIM_E_INVALID, SIM_E_NOMEM, SIM_E_CUDA, SIM_E_DEVICE (a pipeline wait ran out). */
SIM_API int sim_selftest_umma(int32_t f16, int32_t m, int32_t n, int64_t k, const void *a, const void *b,
                              float *d, void *stream);

/* Self-test of the bounded waits (not a simulation call): one GPU thread waits on an
   mbarrier that nothing arrives on, with the wait every pipeline kernel uses and a limit of
   limit_ms (1 .. 1000) instead of their 4 s.  Expected result: SIM_E_DEVICE (the wait ran out
   and the kernel reported it in its status word) with *waited_ms about limit_ms; the context
   stays usable.  stream is a cudaStream_t (NULL = default); the call synchronizes it. */
SIM_API int sim_selftest_wait(int32_t limit_ms, int32_t *waited_ms, void *stream);

/* Self-test of the two-SM tensor-core tile (not a simulation call): one CTA pair computes
   D[256][N] = A[256][K] * B[N][K]^T with tcgen05.mma.cta_group::2, each CTA holding 128 rows
   of A and N/2 rows of B in its shared memory.  A, B row-major 16-bit device matrices (f16 1:
   FP16, 0: BF16), D row-major FP32 device memory; N a multiple of 16 in 32 .. 256, K even.
   stream is a cudaStream_t (NULL = default); the call synchronizes it.
   Errors: SIM_E_INVALID, SIM_E_NOMEM, SIM_E_CUDA, SIM_E_DEVICE (a wait ran out). */
SIM_API int sim_selftest_umma_pair(int32_t f16, int32_t n, int64_t k, const void *a, const void *b, float *d,
                                   void *stream);

/* Ray sum without any device allocation.
   Some callers cannot call cudaMalloc: a host application whose framework allocator has
   already reserved the GPU's memory, a real-time loop that must not take the implicit
   device synchronisation and unbounded latency of cudaMalloc/cudaFree, or a deployment
   that forbids allocation after start-up.  For them this call computes the beat-signal
   cube s[k][m][n] (complex64[N_v][N_c][N_s], same model, precision and result within
   the same tolerance as the signal of sim_submit/sim_fetch) with all of its working
   memory in one static device array of 128 MiB that every device which loads the
   library holds until the process exits.  The caller passes device-resident ray arrays
   (meta data is not needed) and a device output buffer, and a cudaStream_t (NULL = the
   default stream); the call runs on that stream and synchronizes it before returning.
   Limits: n <= min(max_rays, 262144); on the tensor-core precisions one FP32 copy of
   the whole cube, 8 N_v N_c N_s bytes, must also fit beside the 72 bytes per ray of
   per-ray data, 88 in the exact model (the automotive 12 x 256 x 512 cube does; a 192 x 512 x 1024 imaging
   cube does not).  The exact model runs here per chirp on the tensor-core precisions, a
   form without the TDM slot term that keeps one FP32 cube per split of its rays: the
   exact model with tdm_slot_s > 0 on a tensor-core precision is refused, and so is an
   exact-model scene whose splits do not fit beside its per-ray data.  Beyond a limit,
   with pointers that are not device memory of the current device, or in those cases it
   returns SIM_E_INVALID before launching anything.
   The first call on each device also looks up the array's device address (set-up).
   Every call on a device shares the one
   array and finds the previous call's contents in it (the call clears what must start
   at zero), so calls whose work overlaps on the GPU, from several streams or host
   threads, race: serialise them.
   Errors: SIM_E_INVALID, SIM_E_CUDA, SIM_E_DEVICE (a pipeline wait ran out); an invalid
   ray value is reported as SIM_E_INVALID after the run. */
SIM_API int sim_raysum_noalloc(const sim_radar_params *params, const sim_rays *rays, void *signal_c64,
                               void *stream);

#ifdef __cplusplus
}
#endif
#endif
