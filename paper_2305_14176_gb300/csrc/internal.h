// Internal declarations shared by the CUDA translation units of libradarsim.
// Nothing here is part of the C ABI (include/radarsim.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "radarsim.h"

namespace rs {

constexpr double kC = 299792458.0;  // speed of light, m/s

// device status word bits (written by kernels with atomicOr, read at fetch).  A scene's status
// block is 256 bytes: word 0 holds these bits, word 1 the route mask of the expansion's term
// chooser (bit P for a P-term chunk, bit 0 for one handed to the per-chirp or pair-sum form).
enum : uint32_t {
  kStatusBadRay = 1u,        // a ray failed validation in the prep kernel
  kStatusHashFull = 2u,      // a label hash probe ran past its limit
  kStatusWaitLimit = 4u,     // a tensor-core pipeline wait ran past its limit
  kStatusBadLaunch = 8u,     // a kernel saw a launch shape it was not built for
  kStatusBadGeometry = 16u,  // a hit list, triangle or vertex index was out of range
  kStatusModelRange = 32u,   // exact model with TDM slots on tensor cores: the range migration is
                             // beyond the per-tile expansion's bound (reported as invalid rays)
};

// Term counts P the per-tile expansion (umma_taylor.cu) is built for.  Its term chooser writes
// one of them, or 0 when none meets the bound; the per-chirp and pair-sum kernels then own the
// scene, and each kernel of either route returns at once when the other one owns it.
__host__ __device__ inline bool expansion_terms(uint32_t p) { return p == 4u || p == 6u || p == 8u; }

// Radar constants derived on the host in FP64 from sim_radar_params.
struct Derived {
  double fc, bw, tc, td;
  int ns, nc, ntx, nrx, nv, na;
  int log2_ns, log2_nc, log2_na;
  double spacing_wl;  // antenna spacing in carrier wavelengths: s f_c / c, or exactly 1/2
  double ka;          // N_a * spacing_wl: angle-bin coordinate per unit sin(az) cos(el)
  int win[3];
  int precision, outputs, model, pattern_exp;
  double tslot;  // TDM-MIMO slot time (s), 0 = none
  int64_t max_rays;
  int64_t n_sig;   // N_v N_c N_s
  int64_t n_cell;  // N_a N_c N_s
};

// Rays as handed to the device (structure of arrays)
struct RaysIn {
  const double *d;
  const float *a, *v, *az, *el, *p0;
  const int32_t *obj;
};

// Per-ray quantities produced by the prep kernel (Q0.64 phases are fractions of a cycle
// times 2^64; integer addition wraps exactly modulo one cycle).
struct RaysPrep {
  uint64_t *carrier;  // frac(f_c d / c) + phase0 / 2 pi
  uint64_t *nu_r;     // cycles per fast-time sample
  uint64_t *nu_d;     // cycles per chirp
  uint64_t *nu_a;     // cycles per virtual channel
  float *amp;         // amplitude (0 for an invalid ray)
  int32_t *cell;      // flat label cell, -1 for an invalid ray
  uint64_t *energy;   // min(rint(a^2 2^32), 2^41)
  float2 *step_d;     // e^{2 pi j 32 nu_d}: phasor step over 32 chirps (exact Q0.64 product, ~1.5 ulp)
  float2 *step_r;     // e^{2 pi j 32 nu_r}: phasor step over 32 samples
  uint64_t *eps;      // exact Eq. 2 only (else null): range-migration cycles per sample x chirp
  uint64_t *nu_tx;    // cycles per transmitter: N_rx nu_a + nu_t (nu_t = TDM slot Doppler, 0 = none)
  uint64_t *eps_t;    // exact Eq. 2 only (else null): range-migration cycles per sample x TDM slot
};

// Scratch for the label kernels: two open-addressing hash tables
struct LabelScratch {
  uint64_t *pair_key;    // (cell << 32) | object id, ~0 = empty
  uint64_t *pair_energy;
  uint32_t *cell_key;    // cell, ~0 = empty
  uint64_t *cell_max;
  uint32_t *cell_obj;    // smallest object id at the cell maximum
  int64_t capacity;      // power of two, >= 2 * rays
};

int64_t label_capacity(int64_t n_rays);

// window / twiddle tables for one radar configuration (device memory)
struct Tables {
  float *win_r, *win_d, *win_a;   // lengths N_s, N_c, N_v
  float2 *tw_r, *tw_d, *tw_a;     // e^{-2 pi i j / N}, j < N/2
};

// ---- launchers (each returns the number of kernels it launched) ----
int launch_prep(const Derived &g, RaysIn in, int64_t n, RaysPrep out, uint32_t *status, cudaStream_t s);
// copy device-resident input arrays (obj may be null) into a scene's block in one launch
struct IngestArgs {
  const double *d;
  const float *a, *v, *az, *el, *p0;
  const int32_t *obj;
  double *dst_d;
  float *dst_a, *dst_v, *dst_az, *dst_el, *dst_p0;
  int32_t *dst_obj;
};
int launch_ingest(const IngestArgs &x, int64_t n, cudaStream_t s);
// separable direct sum; `workspace` (may be null: one ray part) of direct_workspace_bytes(g, n)
// lets the rays go in parts that fill the SMs
int64_t direct_workspace_bytes(const Derived &g, int64_t n);
int launch_direct_sum(const Derived &g, RaysPrep p, int64_t n, float2 *sig, void *workspace, cudaStream_t s);
// Launch calls that hand back their error instead of leaving it for cudaGetLastError
// (cudaLaunchKernelEx, cudaFuncSetAttribute) report it through note_launch.  A call clears the
// record with launches_begin() before its first launch, and its final check takes
// launches_ok(), which also reads and clears cudaGetLastError: a launch the runtime refused
// fails the call instead of leaving its outputs unwritten.  The record is per host thread.
void note_launch(cudaError_t e);
void launches_begin();
bool launches_ok();
// Runs a runtime call whose failure is expected and handled (a pointer or occupancy query) in
// the middle of a pipeline: its own error is cleared, and an earlier launch's error that the
// thread's last-error slot held is kept in the launch record instead of being lost with it.
template <class F>
cudaError_t handled_call(F f) {
  const cudaError_t prior = cudaGetLastError();
  const cudaError_t rc = f();
  if (rc != cudaSuccess) cudaGetLastError();
  note_launch(prior);
  return rc;
}
// Runs f() once per device for the flag `done` (bit d: done on device d).  Function attributes
// such as the dynamic shared-memory size belong to a device's context, so each device the
// process launches on needs its own call; several host threads may arrive at once, and f() may
// then run more than once, which setting an attribute allows.
template <class F>
void once_per_device(std::atomic<uint64_t> &done, F f) {
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0ull;
  if (bit != 0 && (done.load(std::memory_order_acquire) & bit) != 0) return;
  f();
  if (bit != 0) done.fetch_or(bit, std::memory_order_acq_rel);
}
// store a synchronous call's stage times (7 entries, the sim_last_stage_ms order), kernel count
// and route mask (status word 1)
void record_stage_ms(sim_ctx *c, const float *ms, int kernels, uint32_t route);
// direct sum over per-(ray, chirp, transmitter) and per-(ray, chirp, receiver) Q0.32 phase
// words (base, per-sample step): w_tx[(m N_tx + t) stride + i], w_rx[(m N_rx + r) stride + i]
// `workspace` (may be null: one ray part) of pair_workspace_bytes(g, n) lets the rays go in
// parts that fill the SMs
int64_t pair_workspace_bytes(const Derived &g, int64_t n);
// `gate` (device word, may be null) holding a term count (expansion_terms) makes both of its
// kernels return at once
int launch_pair_sum(const Derived &g, const uint2 *w_tx, const uint2 *w_rx, const float *amp, int64_t n,
                    int64_t stride, bool accumulate, float2 *sig, void *workspace, const uint32_t *gate,
                    cudaStream_t s);
// virtual snapshots on tensor cores, one chunk of phase words (umma_taylor.cu): the per-tile
// expansion, or the pair sum when the expansion's bound fails; workspace of
// snap_tensor_workspace_bytes(g, chunk), pair_ws of pair_workspace_bytes(g, chunk).  The
// expansion's reference antennas are the central ones; `rec` holds, per (ray, chirp m) at
// [m stride + ray], the step S(m, t_c, r_c) and the largest and smallest signed difference
// S(m, t, r) - S(m, t_c, r_c) over the antennas, as the Q0.32 words hold them, which bound
// the expansion's argument.
inline int snap_ref_tx(const Derived &g) { return g.ntx / 2; }
inline int snap_ref_rx(const Derived &g) { return g.nrx / 2; }
struct SnapRec {
  const uint32_t *s;
  const int32_t *d_hi, *d_lo;
};
int64_t snap_tensor_workspace_bytes(const Derived &g, int64_t chunk);
int launch_snap_tensor(const Derived &g, const uint2 *w_tx, const uint2 *w_rx, SnapRec rec, int64_t stride,
                       const float *amp, int64_t cnt, bool accumulate, float2 *sig, void *workspace, void *pair_ws,
                       uint32_t *status, cudaStream_t s);
int launch_fft(const Derived &g, const Tables &t, const float2 *sig, float2 *tmp, float2 *spec, cudaStream_t s);
// The same passes for many cubes of one shape held in spectrum slots of n_cell elements: the
// range pass of one signal into the first n_sig elements of its slot, then the Doppler and angle
// passes in place over `count` consecutive slots at once (the same arithmetic per cube, so the
// same bits as launch_fft).
int launch_fft_range_into(const Derived &g, const Tables &t, const float2 *sig, float2 *slot, cudaStream_t s);
int launch_fft_planes(const Derived &g, const Tables &t, float2 *slots, int count, cudaStream_t s);
int launch_labels(const Derived &g, RaysPrep p, const int32_t *obj, int64_t n, LabelScratch sc,
                  int32_t *labels, uint32_t *status, cudaStream_t s);

// exact Eq. 2 on tensor cores (samples x channels tiles per chirp), used by launch_umma_sum
// for SIM_MODEL_EXACT contexts
int64_t exact_workspace_bytes(const Derived &g, int64_t n);
int launch_exact_sum(const Derived &g, RaysPrep p, int64_t n, float2 *sig, void *workspace, uint32_t *status,
                     cudaStream_t s, cudaEvent_t after_main);
// its two halves; `gate` (device word, may be null) holding a term count makes both return at once
int launch_exact_main(const Derived &g, RaysPrep p, int64_t n, void *workspace, uint32_t *status, cudaStream_t s,
                      const uint32_t *gate);
int launch_exact_reduce(const Derived &g, int64_t n, float2 *sig, void *workspace, cudaStream_t s,
                        const uint32_t *gate);
// exact Eq. 2 on tensor cores through the per-tile expansion of the range-migration phase
// (umma_taylor.cu), falling back on the device to the per-chirp kernel when the expansion's
// bound is not met; the workspace covers both
int64_t exact_tensor_workspace_bytes(const Derived &g, int64_t n);
int launch_exact_tensor(const Derived &g, RaysPrep p, int64_t n, float2 *sig, void *workspace, uint32_t *status,
                        cudaStream_t s, cudaEvent_t after_main);
// tensor-core ray sum: workspace bytes it needs and its launcher
// A scene in a batch keeps the plan it has alone, so its results are the same bits.  Every step
// of a batch (work list, workspace, split-K reduction) takes that plan from one function
// (batch_workspace_bytes, umma_units_of, launch_umma_post).
int64_t batch_workspace_bytes(const Derived &g, int64_t n);
// `waves`: the plan's minimum waves of CTAs; `min_chunk` (> 0): at least that many rays per
// split; launch_umma_sum takes the same values
int64_t umma_workspace_bytes(const Derived &g, int64_t n, float waves = 4.f, int64_t min_chunk = 0);
// `after_main` (may be null) is recorded on `s` right after the GEMM kernel, before the
// split reduction, so the GEMM can be timed on its own stream.
int launch_umma_sum(const Derived &g, RaysPrep p, int64_t n, float2 *sig, void *workspace,
                    uint32_t *status, cudaStream_t s, cudaEvent_t after_main, float waves = 4.f,
                    int64_t min_chunk = 0);

// ---- batched tensor-core ray sum (one persistent launch over several scenes)
struct UmmaBatch {
  unsigned *counter;  // work-list cursors (device): [0] two-SM list, [1] one-SM list
  void *args;         // per-scene kernel arguments (device)
  void *units;        // two-SM work list (256-row tiles), longest first (device)
  int n_units;
  void *units1;       // one-SM work list (128-row tiles), longest first (device)
  int n_units1;
  int n_scenes, bn_max, bn_max1;  // widest tile (real columns) of each list
  bool f16, split, fast;
};
// device bytes of the batch's descriptors and counter
int64_t umma_batch_scratch_bytes(int n_scenes, int64_t n_units);
// work units (tiles x splits) of one scene: the same decomposition as a single-scene launch
int64_t umma_units_of(const Derived &g, int64_t n);
// upload the descriptors (synchronous, not for stream capture); all scenes share one
// tensor-core precision, else SIM_E_INVALID
int prepare_umma_batch(int n_scenes, const Derived *const *gs, const RaysPrep *ps, const int64_t *ns,
                       void *const *workspaces, uint32_t *const *statuses, void *scratch, cudaStream_t s,
                       UmmaBatch *out);
int launch_umma_batch(const UmmaBatch &b, cudaStream_t s);
int launch_umma_pre(const Derived &g, RaysPrep p, int64_t n, void *workspace, cudaStream_t s);
int launch_umma_post(const Derived &g, int64_t n, float2 *sig, void *workspace, cudaStream_t s);

// ---- autotuned launch shapes (table in tune.cu), keyed by the radar shape, precision and
// the ray count's power-of-two bucket.  0 in a field means "use the built-in heuristic".
struct Tuning {
  int splits;             // tensor-core split-K count
  int fft_range_points;   // points per block of the range FFT (1024 .. 4096)
  int fft_doppler_strip;  // samples per block of the Doppler FFT
  int fft_angle_strip;    // (m, n) positions per block of the angle FFT
};
bool tuning_lookup(const Derived &g, int64_t n, Tuning *t);
// FFTs with explicit tile choices (zeros: heuristic)
int launch_fft_with(const Derived &g, const Tables &t, const float2 *sig, float2 *tmp, float2 *spec,
                    cudaStream_t s, const Tuning &tu);
// tensor-core ray sum with a forced split count (autotuner), or with splits = 0 the plan a
// scene takes without a table entry (stream-K at split precision); workspace sized for it
int launch_umma_sum_splits(const Derived &g, RaysPrep p, int64_t n, float2 *sig, void *workspace, uint32_t *status,
                           cudaStream_t s, int splits);
int64_t umma_workspace_bytes_splits(const Derived &g, int splits);
// partial slots of that built-in plan (its workspace is umma_workspace_bytes_splits of them)
int umma_builtin_splits(const Derived &g, int64_t n);
// the split counts the tuner tries for a shape (heuristic first)
int umma_split_candidates(const Derived &g, int64_t n, int *out, int max_out);

// Validate sim_radar_params and derive the radar constants (SIM_OK or SIM_E_INVALID).
int derive_radar(const sim_radar_params *p, Derived *g);

// Tensor-core ray sum inside a caller-provided workspace of `ws_bytes`: the split-K count
// is lowered until the partials fit.  Returns the number of kernels launched, or -1 when
// even a single split does not fit.
int launch_umma_sum_in(const Derived &g, RaysPrep p, int64_t n, float2 *sig, void *workspace, int64_t ws_bytes,
                       uint32_t *status, cudaStream_t s);

}  // namespace rs

// One radar configuration (the C ABI's opaque handle).
namespace rs {
// A context's device scratch for its synchronous calls (sim_decompose, sim_snapshot_*): grown on
// demand and kept until sim_destroy, so that repeated calls neither allocate nor free device
// memory (cudaFree waits for the whole device).  One call holds a slot at a time.
struct ScratchSlot {
  std::mutex m;
  void *p = nullptr;
  size_t bytes = 0;
};
enum { kSlotDecompose = 0, kSlotDecomposeLanes = 1, kSlotSnapshot = 2, kSlots = 3 };
// One call's use of a slot: the slot's buffer, grown to the size asked for, or, when another
// call holds the slot, a buffer of this call's own.  Released (or freed) on destruction, which
// must follow the last device work on it.  get() may be called again with a smaller size after
// it returned null (out of memory).
class ScratchLease {
 public:
  ScratchLease() = default;
  ScratchLease(const ScratchLease &) = delete;
  ScratchLease &operator=(const ScratchLease &) = delete;
  ~ScratchLease();
  void *get(ScratchSlot &slot, size_t bytes);

 private:
  ScratchSlot *held_ = nullptr;
  void *own_ = nullptr;
};
}  // namespace rs

struct sim_ctx {
  rs::Derived g;
  rs::Tables t;
  void *table_mem = nullptr;  // window and twiddle tables (device)
  size_t table_bytes = 0;
  float last_ms[8] = {};
  int last_kernels = 0;
  uint32_t last_route = 0;    // route mask of the last fetched scene (sim_last_expansion_terms)
  std::atomic<int> live{0};   // tickets not yet fetched
  rs::ScratchSlot scratch[rs::kSlots];
};

