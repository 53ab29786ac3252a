// Engine and C ABI of libradarsim (include/radarsim.h).
//
// The engine is a process-wide singleton bound to the device that is current at the
// first sim_create.  It owns
//   * a dedicated stream-ordered device memory pool and a byte budget,
//   * `slots` CUDA streams: each admitted scene runs on one, so scenes submitted while
//     others are on the GPU overlap on the device (continuous batching),
//   * a bounded queue of scenes waiting for memory or a slot, drained by a host worker
//     thread whenever a fetch releases resources.
// A scene's device buffers live in one block from the pool: inputs, per-ray prep,
// signal, FFT scratch, spectrum, labels, label hash tables and the ray-sum workspace.
// Results stay on the device until sim_fetch copies them out and releases the block.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

using namespace rs;

namespace {

constexpr int kNumEvents = 7;  // start, ingest, prep, ray-sum main kernel, ray sum done, fft, labels/end

struct Job;

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev[kNumEvents] = {};
  // the labels need only the prep: they run on a second stream beside the ray sum and FFTs,
  // between lab[0] and lab[1], and the slot's stream waits for lab[1] before its last event
  cudaStream_t side = nullptr;
  cudaEvent_t lab[2] = {};
  bool busy = false;
  Job *job = nullptr;  // the scene running on this slot
};

struct Plan {  // byte offsets of one scene's buffers inside its device block
  size_t d, a, v, az, el, p0, obj;
  size_t carrier, nu_r, nu_d, nu_a, amp, cell, energy, step_d, step_r, eps, nu_tx, eps_t;
  size_t status;
  size_t sig, tmp, spec, labels;
  size_t pk, pe, ck, cm, co;
  size_t ws;
  int64_t cap;
  size_t total;
};

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

}  // namespace

namespace {

// A scene's life: queued (pending, host copy of its inputs) -> running (a slot: stream and
// events) -> done on the device (slot released, device block and stage times kept) ->
// fetched (block freed, ticket gone).
struct Job {
  uint64_t ticket = 0;
  sim_ctx *ctx = nullptr;
  int64_t n = 0;
  bool has_obj = false;
  Plan plan{};
  bool pending = true;
  bool done = false;
  bool claimed = false;            // a fetch has taken it
  std::vector<uint8_t> host_copy;  // inputs held while the scene waits in the queue
  uint8_t *block = nullptr;
  int slot = -1;
  int kernels = 0;
  int launch_error = 0;
  cudaError_t device_error = cudaSuccess;
  float ms[8] = {};
};

struct Engine {
  std::mutex mu;
  std::condition_variable cv;
  int device = -1;
  int64_t budget = 0, used = 0;
  int max_queue = 64;
  std::vector<Slot> slots;
  std::vector<cudaStream_t> egress;  // streams for the result copies of sim_fetch
  std::deque<Job *> queue;
  std::unordered_map<uint64_t, Job *> jobs;
  uint64_t next_ticket = 1;
  int fetching = 0;  // threads inside sim_fetch
  cudaMemPool_t pool = nullptr;
  bool ready = false;
  // configuration requested before start
  int64_t cfg_budget = 0;
  // two scenes on the device at a time: the same throughput as four (e2e 7.15e13 against
  // 7.20e13 contributions/s with six frames in flight), and a lower median latency under
  // Poisson load, since co-running scenes share the SMs (200 automotive frames/s: p50 12.9
  // against 15.9 ms, p99 78.8 against 78.4 ms; 150/s: p50 9.0 against 9.5, p99 27.5 against
  // 31.6 ms)
  int cfg_slots = 2;
  int cfg_queue = 64;
};

Engine &engine() {
  static Engine *e = new Engine();  // never destroyed: the worker thread may outlive statics
  return *e;
}

Plan make_plan(const Derived &g, int64_t n, bool has_obj) {
  Plan p{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes > 0 ? bytes : 1);
    return o;
  };
  const size_t un = static_cast<size_t>(n);
  const size_t up = (un + 31) / 32 * 32;  // per-ray prep arrays padded to whole 32-ray stages
  p.d = take(8 * un);
  p.a = take(4 * un);
  p.v = take(4 * un);
  p.az = take(4 * un);
  p.el = take(4 * un);
  p.p0 = take(4 * un);
  p.obj = take(has_obj ? 4 * un : 0);
  p.carrier = take(8 * up);
  p.nu_r = take(8 * up);
  p.nu_d = take(8 * up);
  p.nu_a = take(8 * up);
  p.amp = take(4 * up);
  p.cell = take(4 * up);
  p.energy = take(8 * up);
  p.step_d = take(8 * up);
  p.step_r = take(8 * up);
  p.eps = take(g.model == SIM_MODEL_EXACT ? 8 * up : 0);
  p.nu_tx = take(8 * up);
  p.eps_t = take(g.model == SIM_MODEL_EXACT ? 8 * up : 0);
  p.status = take(256);
  p.sig = take(8 * static_cast<size_t>(g.n_sig));
  const bool spec = g.outputs & SIM_OUT_SPECTRUM;
  const bool lab = g.outputs & SIM_OUT_LABELS;
  p.tmp = take(spec ? 8 * static_cast<size_t>(g.n_sig) : 0);
  p.spec = take(spec ? 8 * static_cast<size_t>(g.n_cell) : 0);
  p.labels = take(lab ? 4 * static_cast<size_t>(g.n_cell) : 0);
  p.cap = lab ? label_capacity(n) : 0;
  const size_t cap = static_cast<size_t>(p.cap);
  p.pk = take(8 * cap);
  p.pe = take(8 * cap);
  p.ck = take(4 * cap);
  p.cm = take(8 * cap);
  p.co = take(4 * cap);
  p.ws = take(static_cast<size_t>(g.precision == SIM_PREC_FP32_DIRECT ? direct_workspace_bytes(g, n)
                                                                      : umma_workspace_bytes(g, n)));
  p.total = off;
  return p;
}

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// same acceptance rule as the prep kernel
bool host_ray_ok(double d, float a, float v, float az, float el, float p0) {
  return (d >= 0.0 && d <= 1.0e7) && (a >= 0.0f && a <= 3.0e38f) && (fabsf(v) <= 1.0e5f) &&
         (fabsf(az) <= 3.14159274f) && (fabsf(el) <= 1.57079637f) && (fabsf(p0) <= 1.0e6f);
}

int start_engine_locked(Engine &e);

// Launch a scene on its slot: ingest copies, prep, ray sum, FFTs, labels.
// `src` holds the caller's pointers (or the host copy's).  Returns a SIM status.
int launch_job(Engine &e, Job *j, const sim_rays &src, const int32_t *src_obj) {
  launches_begin();
  Slot &sl = e.slots[j->slot];
  cudaStream_t s = sl.stream;
  const Derived &g = j->ctx->g;
  const Plan &p = j->plan;
  void *blk = nullptr;
  if (cudaMallocFromPoolAsync(&blk, p.total, e.pool, s) != cudaSuccess) {
    cudaGetLastError();
    return SIM_E_NOMEM;
  }
  j->block = static_cast<uint8_t *>(blk);
  uint8_t *b = j->block;
  const size_t un = static_cast<size_t>(j->n);
  cudaEventRecord(sl.ev[0], s);
  const bool dev_src = j->n > 0 && is_device_ptr(src.range_rt_m) && is_device_ptr(src.amplitude) &&
                       is_device_ptr(src.radial_velocity_mps) && is_device_ptr(src.azimuth_rad) &&
                       is_device_ptr(src.elevation_rad) && is_device_ptr(src.phase0_rad) &&
                       (!j->has_obj || is_device_ptr(src_obj));
  int ingest_kernels = 0;
  if (dev_src) {
    IngestArgs x{src.range_rt_m, src.amplitude, src.radial_velocity_mps, src.azimuth_rad, src.elevation_rad,
                 src.phase0_rad, j->has_obj ? src_obj : nullptr, reinterpret_cast<double *>(b + p.d),
                 reinterpret_cast<float *>(b + p.a), reinterpret_cast<float *>(b + p.v),
                 reinterpret_cast<float *>(b + p.az), reinterpret_cast<float *>(b + p.el),
                 reinterpret_cast<float *>(b + p.p0), reinterpret_cast<int32_t *>(b + p.obj)};
    ingest_kernels = launch_ingest(x, j->n, s);
  } else if (j->n > 0) {
    cudaMemcpyAsync(b + p.d, src.range_rt_m, 8 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + p.a, src.amplitude, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + p.v, src.radial_velocity_mps, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + p.az, src.azimuth_rad, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + p.el, src.elevation_rad, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + p.p0, src.phase0_rad, 4 * un, cudaMemcpyDefault, s);
    if (j->has_obj) cudaMemcpyAsync(b + p.obj, src_obj, 4 * un, cudaMemcpyDefault, s);
  }
  cudaMemsetAsync(b + p.status, 0, 256, s);
  cudaEventRecord(sl.ev[1], s);

  RaysIn in{reinterpret_cast<const double *>(b + p.d), reinterpret_cast<const float *>(b + p.a),
            reinterpret_cast<const float *>(b + p.v), reinterpret_cast<const float *>(b + p.az),
            reinterpret_cast<const float *>(b + p.el), reinterpret_cast<const float *>(b + p.p0),
            j->has_obj ? reinterpret_cast<const int32_t *>(b + p.obj) : nullptr};
  RaysPrep rp{reinterpret_cast<uint64_t *>(b + p.carrier), reinterpret_cast<uint64_t *>(b + p.nu_r),
              reinterpret_cast<uint64_t *>(b + p.nu_d), reinterpret_cast<uint64_t *>(b + p.nu_a),
              reinterpret_cast<float *>(b + p.amp), reinterpret_cast<int32_t *>(b + p.cell),
              reinterpret_cast<uint64_t *>(b + p.energy), reinterpret_cast<float2 *>(b + p.step_d),
              reinterpret_cast<float2 *>(b + p.step_r),
              g.model == SIM_MODEL_EXACT ? reinterpret_cast<uint64_t *>(b + p.eps) : nullptr,
              reinterpret_cast<uint64_t *>(b + p.nu_tx),
              g.model == SIM_MODEL_EXACT ? reinterpret_cast<uint64_t *>(b + p.eps_t) : nullptr};
  uint32_t *status = reinterpret_cast<uint32_t *>(b + p.status);
  float2 *sig = reinterpret_cast<float2 *>(b + p.sig);
  int kernels = ingest_kernels;
  kernels += launch_prep(g, in, j->n, rp, status, s);
  cudaEventRecord(sl.ev[2], s);
  const bool labels = (g.outputs & SIM_OUT_LABELS) != 0;
  if (labels) {
    cudaStreamWaitEvent(sl.side, sl.ev[2], 0);
    cudaEventRecord(sl.lab[0], sl.side);
    LabelScratch sc{reinterpret_cast<uint64_t *>(b + p.pk), reinterpret_cast<uint64_t *>(b + p.pe),
                    reinterpret_cast<uint32_t *>(b + p.ck), reinterpret_cast<uint64_t *>(b + p.cm),
                    reinterpret_cast<uint32_t *>(b + p.co), p.cap};
    kernels += launch_labels(g, rp, in.obj, j->n, sc, reinterpret_cast<int32_t *>(b + p.labels), status, sl.side);
    cudaEventRecord(sl.lab[1], sl.side);
  }
  if (g.precision == SIM_PREC_FP32_DIRECT) {
    kernels += launch_direct_sum(g, rp, j->n, sig, b + p.ws, s);
    cudaEventRecord(sl.ev[3], s);
  } else {
    kernels += launch_umma_sum(g, rp, j->n, sig, b + p.ws, status, s, sl.ev[3]);
  }
  cudaEventRecord(sl.ev[4], s);
  if (g.outputs & SIM_OUT_SPECTRUM)
    kernels += launch_fft(g, j->ctx->t, sig, reinterpret_cast<float2 *>(b + p.tmp),
                          reinterpret_cast<float2 *>(b + p.spec), s);
  cudaEventRecord(sl.ev[5], s);
  if (labels) cudaStreamWaitEvent(s, sl.lab[1], 0);  // join: the scene ends when its labels do
  cudaEventRecord(sl.ev[6], s);
  j->kernels = kernels;
  if (!launches_ok()) return SIM_E_CUDA;
  return SIM_OK;
}

// does the queue head fit the memory budget now? (lock held; slots free up on their own)
bool head_fits_locked(Engine &e) {
  if (e.queue.empty()) return true;
  return e.used + static_cast<int64_t>(e.queue.front()->plan.total) <= e.budget;
}

// try to reserve memory and a slot for `j` (lock held)
bool try_reserve_locked(Engine &e, Job *j) {
  if (e.used + static_cast<int64_t>(j->plan.total) > e.budget) return false;
  for (size_t i = 0; i < e.slots.size(); ++i) {
    if (!e.slots[i].busy) {
      e.slots[i].busy = true;
      e.slots[i].job = j;
      j->slot = static_cast<int>(i);
      e.used += static_cast<int64_t>(j->plan.total);
      return true;
    }
  }
  return false;
}

// the scene finished on the device: keep its stage times, give its slot to the next scene
void finish_on_device_locked(Engine &e, Job *j, cudaError_t err) {
  Slot &sl = e.slots[j->slot];
  for (int i = 0; i + 1 < kNumEvents; ++i) {
    j->ms[i] = 0.f;
    cudaEventElapsedTime(&j->ms[i], sl.ev[i], sl.ev[i + 1]);
  }
  cudaEventElapsedTime(&j->ms[kNumEvents - 1], sl.ev[0], sl.ev[kNumEvents - 1]);
  cudaGetLastError();
  j->device_error = err;
  j->done = true;
  sl.busy = false;
  sl.job = nullptr;
  j->slot = -1;
}

// poll the running scenes (lock held); true if any finished
bool reap_locked(Engine &e) {
  bool any = false;
  for (auto &sl : e.slots) {
    if (!sl.busy || !sl.job || sl.job->pending) continue;
    const cudaError_t q = cudaEventQuery(sl.ev[kNumEvents - 1]);
    if (q == cudaErrorNotReady) continue;
    finish_on_device_locked(e, sl.job, q);
    any = true;
  }
  if (any) cudaGetLastError();
  return any;
}

bool any_running_locked(const Engine &e) {
  return std::any_of(e.slots.begin(), e.slots.end(), [](const Slot &s) { return s.busy; });
}

sim_rays host_copy_view(Job *j, const int32_t **obj) {
  uint8_t *h = j->host_copy.data();
  const size_t un = static_cast<size_t>(j->n);
  sim_rays r;
  r.n = j->n;
  r.range_rt_m = reinterpret_cast<const double *>(h);
  r.amplitude = reinterpret_cast<const float *>(h + 8 * un);
  r.radial_velocity_mps = reinterpret_cast<const float *>(h + 12 * un);
  r.azimuth_rad = reinterpret_cast<const float *>(h + 16 * un);
  r.elevation_rad = reinterpret_cast<const float *>(h + 20 * un);
  r.phase0_rad = reinterpret_cast<const float *>(h + 24 * un);
  *obj = j->has_obj ? reinterpret_cast<const int32_t *>(h + 28 * un) : nullptr;
  return r;
}

// worker: notice scenes that finished on the device (their slots free up) and admit queued
// scenes in arrival order as memory and slots allow
void worker_main() {
  Engine &e = engine();
  cudaSetDevice(e.device);
  std::unique_lock<std::mutex> lk(e.mu);
  for (;;) {
    if (reap_locked(e)) e.cv.notify_all();
    while (!e.queue.empty()) {
      Job *j = e.queue.front();
      if (!try_reserve_locked(e, j)) break;
      e.queue.pop_front();
      lk.unlock();
      const int32_t *obj = nullptr;
      sim_rays src = host_copy_view(j, &obj);
      const int rc = launch_job(e, j, src, obj);
      lk.lock();
      j->launch_error = rc;
      j->pending = false;
      j->host_copy.clear();
      j->host_copy.shrink_to_fit();
      if (rc != SIM_OK) finish_on_device_locked(e, j, cudaSuccess);
      e.cv.notify_all();
    }
    if (any_running_locked(e)) e.cv.wait_for(lk, std::chrono::microseconds(100));
    else e.cv.wait(lk);
  }
}

int start_engine_locked(Engine &e) {
  if (e.ready) return SIM_OK;
  if (cudaGetDevice(&e.device) != cudaSuccess) return SIM_E_CUDA;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return SIM_E_CUDA;
  e.budget = e.cfg_budget > 0 ? e.cfg_budget : static_cast<int64_t>(0.9 * static_cast<double>(free_b));
  e.max_queue = e.cfg_queue;
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = e.device;
  if (cudaMemPoolCreate(&e.pool, &props) != cudaSuccess) return SIM_E_CUDA;
  uint64_t keep = ~0ull;  // keep freed blocks cached in the pool
  cudaMemPoolSetAttribute(e.pool, cudaMemPoolAttrReleaseThreshold, &keep);
  e.slots.resize(static_cast<size_t>(e.cfg_slots));
  for (auto &s : e.slots) {
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) return SIM_E_CUDA;
    for (auto &ev : s.ev)
      if (cudaEventCreate(&ev) != cudaSuccess) return SIM_E_CUDA;
    if (cudaStreamCreateWithFlags(&s.side, cudaStreamNonBlocking) != cudaSuccess) return SIM_E_CUDA;
    for (auto &ev : s.lab)
      if (cudaEventCreate(&ev) != cudaSuccess) return SIM_E_CUDA;
  }
  e.egress.resize(4);
  for (auto &st : e.egress)
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SIM_E_CUDA;
  std::thread(worker_main).detach();
  e.ready = true;
  if (const char *tc = getenv("RADARSIM_TUNE_CACHE")) sim_tuning_load(tc);
  return SIM_OK;
}

bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }
int ilog2(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}
bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

int derive(const sim_radar_params *p, Derived *g) {
  if (!p || p->struct_size < sizeof(sim_radar_params)) return SIM_E_INVALID;
  if (!finite_pos(p->carrier_hz) || !finite_pos(p->bandwidth_hz) || !finite_pos(p->sweep_time_s) ||
      !finite_pos(p->chirp_period_s))
    return SIM_E_INVALID;
  if (!pow2(p->n_samples) || p->n_samples < 16 || p->n_samples > 4096) return SIM_E_INVALID;
  if (!pow2(p->n_chirps) || p->n_chirps < 2 || p->n_chirps > 4096) return SIM_E_INVALID;
  if (p->n_tx < 1 || p->n_rx < 1 || p->n_tx > 1024 || p->n_rx > 1024 || p->n_tx * p->n_rx > 1024)
    return SIM_E_INVALID;
  if (!(isfinite(p->element_spacing_m) && p->element_spacing_m >= 0.0)) return SIM_E_INVALID;
  const int nv = p->n_tx * p->n_rx;
  int na = p->n_angle;
  if (na == 0) {
    na = 16;
    while (na < nv) na <<= 1;
  }
  if (!pow2(na) || na < nv || na > 1024) return SIM_E_INVALID;
  for (int i = 0; i < 3; ++i)
    if (p->window[i] < SIM_WIN_NONE || p->window[i] > SIM_WIN_HANN_NOZERO) return SIM_E_INVALID;
  if (p->precision < SIM_PREC_FP32_DIRECT || p->precision > SIM_PREC_FP16_SPLIT) return SIM_E_INVALID;
  if (p->outputs <= 0 || p->outputs > 7) return SIM_E_INVALID;
  if (p->max_rays < 1 || p->max_rays > (int64_t{1} << 21)) return SIM_E_INVALID;
  if (p->model != SIM_MODEL_SEPARABLE && p->model != SIM_MODEL_EXACT) return SIM_E_INVALID;
  // the exact model with TDM slots on tensor cores needs the per-tile expansion, which needs
  // two-SM tiles of at least 32 samples (the per-chirp product has no slot term)
  if (p->model == SIM_MODEL_EXACT && p->precision != SIM_PREC_FP32_DIRECT && p->tdm_slot_s != 0.0 &&
      p->n_samples < 32)
    return SIM_E_INVALID;
  if (p->pattern_exp < 0 || p->pattern_exp > 16) return SIM_E_INVALID;
  if (!(isfinite(p->tdm_slot_s) && p->tdm_slot_s >= 0.0 && p->tdm_slot_s <= 1.0)) return SIM_E_INVALID;
  const int64_t n_cell = static_cast<int64_t>(na) * p->n_chirps * p->n_samples;
  if (n_cell >= (int64_t{1} << 31)) return SIM_E_INVALID;
  g->fc = p->carrier_hz;
  g->bw = p->bandwidth_hz;
  g->tc = p->sweep_time_s;
  g->td = p->chirp_period_s;
  g->ns = p->n_samples;
  g->nc = p->n_chirps;
  g->ntx = p->n_tx;
  g->nrx = p->n_rx;
  g->nv = nv;
  g->na = na;
  g->log2_ns = ilog2(g->ns);
  g->log2_nc = ilog2(g->nc);
  g->log2_na = ilog2(g->na);
  g->spacing_wl = p->element_spacing_m == 0.0 ? 0.5 : (p->element_spacing_m * p->carrier_hz) / kC;
  g->ka = static_cast<double>(na) * g->spacing_wl;
  for (int i = 0; i < 3; ++i) g->win[i] = p->window[i];
  g->precision = p->precision;
  g->outputs = p->outputs;
  g->model = p->model;
  g->pattern_exp = p->pattern_exp;
  g->tslot = p->tdm_slot_s;
  g->max_rays = p->max_rays;
  g->n_sig = static_cast<int64_t>(nv) * g->nc * g->ns;
  g->n_cell = n_cell;
  return SIM_OK;
}

double window_value(int type, int t, int len) {
  const double two_pi = 6.283185307179586476925286766559;
  switch (type) {
    case SIM_WIN_HANN_PERIODIC: return 0.5 * (1.0 - cos(two_pi * t / len));
    case SIM_WIN_HANN_SYMMETRIC: return len > 1 ? 0.5 * (1.0 - cos(two_pi * t / (len - 1))) : 1.0;
    case SIM_WIN_HANN_NOZERO: return 0.5 * (1.0 - cos(two_pi * (t + 1) / (len + 1)));
    default: return 1.0;
  }
}

int upload_tables(sim_ctx *c) {
  const Derived &g = c->g;
  const int lens[3] = {g.ns, g.nc, g.nv};
  const int ffts[3] = {g.ns, g.nc, g.na};
  size_t bytes = 0;
  for (int a = 0; a < 3; ++a) bytes += align256(4 * static_cast<size_t>(lens[a])) + align256(8 * static_cast<size_t>(ffts[a] / 2));
  std::vector<uint8_t> h(bytes, 0);
  size_t off = 0;
  size_t win_off[3], tw_off[3];
  const double two_pi = 6.283185307179586476925286766559;
  for (int a = 0; a < 3; ++a) {
    win_off[a] = off;
    float *w = reinterpret_cast<float *>(h.data() + off);
    for (int t = 0; t < lens[a]; ++t) w[t] = static_cast<float>(window_value(g.win[a], t, lens[a]));
    off += align256(4 * static_cast<size_t>(lens[a]));
    tw_off[a] = off;
    float *tw = reinterpret_cast<float *>(h.data() + off);
    for (int j = 0; j < ffts[a] / 2; ++j) {
      tw[2 * j] = static_cast<float>(cos(two_pi * j / ffts[a]));
      tw[2 * j + 1] = static_cast<float>(-sin(two_pi * j / ffts[a]));
    }
    off += align256(8 * static_cast<size_t>(ffts[a] / 2));
  }
  c->table_bytes = bytes;
  if (cudaMalloc(&c->table_mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return SIM_E_NOMEM;
  }
  if (cudaMemcpy(c->table_mem, h.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) return SIM_E_CUDA;
  uint8_t *d = static_cast<uint8_t *>(c->table_mem);
  c->t.win_r = reinterpret_cast<float *>(d + win_off[0]);
  c->t.win_d = reinterpret_cast<float *>(d + win_off[1]);
  c->t.win_a = reinterpret_cast<float *>(d + win_off[2]);
  c->t.tw_r = reinterpret_cast<float2 *>(d + tw_off[0]);
  c->t.tw_d = reinterpret_cast<float2 *>(d + tw_off[1]);
  c->t.tw_a = reinterpret_cast<float2 *>(d + tw_off[2]);
  return SIM_OK;
}

}  // namespace

int rs::derive_radar(const sim_radar_params *p, Derived *g) { return derive(p, g); }

namespace rs {
namespace {
thread_local cudaError_t t_launch_error = cudaSuccess;
}
void note_launch(cudaError_t e) {
  if (e != cudaSuccess && t_launch_error == cudaSuccess) t_launch_error = e;
}
void launches_begin() { t_launch_error = cudaSuccess; }
bool launches_ok() {
  const bool ok = cudaGetLastError() == cudaSuccess && t_launch_error == cudaSuccess;
  t_launch_error = cudaSuccess;
  return ok;
}

void record_stage_ms(sim_ctx *c, const float *ms, int kernels, uint32_t route) {
  Engine &e = engine();
  std::lock_guard<std::mutex> lk(e.mu);
  for (int i = 0; i < kNumEvents; ++i) c->last_ms[i] = ms[i];
  c->last_kernels = kernels;
  c->last_route = route;
}
}  // namespace rs

namespace rs {

void *ScratchLease::get(ScratchSlot &slot, size_t bytes) {
  if (!held_ && !own_ && slot.m.try_lock()) held_ = &slot;
  if (held_) {
    if (held_->bytes < bytes) {
      if (held_->p) cudaFree(held_->p);
      held_->p = nullptr;
      held_->bytes = 0;
      if (cudaMalloc(&held_->p, bytes) != cudaSuccess) {
        cudaGetLastError();
        held_->p = nullptr;
        return nullptr;
      }
      held_->bytes = bytes;
    }
    return held_->p;
  }
  if (own_) cudaFree(own_);
  own_ = nullptr;
  if (cudaMalloc(&own_, bytes) != cudaSuccess) {
    cudaGetLastError();
    own_ = nullptr;
  }
  return own_;
}

ScratchLease::~ScratchLease() {
  if (own_) cudaFree(own_);
  if (held_) held_->m.unlock();
}

}  // namespace rs

extern "C" {

const char *sim_status_string(int s) {
  switch (s) {
    case SIM_OK: return "ok";
    case SIM_E_INVALID: return "invalid argument or ray value";
    case SIM_E_NOMEM: return "out of memory";
    case SIM_E_BUSY: return "busy: memory budget or queue full";
    case SIM_E_TIMEOUT: return "timed out";
    case SIM_E_NOT_READY: return "not ready";
    case SIM_E_UNKNOWN_TICKET: return "unknown ticket";
    case SIM_E_CUDA: return "CUDA runtime error";
    case SIM_E_DEVICE: return "device-side limit reached";
    default: return "unknown status";
  }
}

int sim_engine_configure(int64_t memory_budget_bytes, int32_t slots, int32_t max_queue) {
  Engine &e = engine();
  std::lock_guard<std::mutex> lk(e.mu);
  if (e.ready) return SIM_E_INVALID;
  if (memory_budget_bytes < 0 || slots < 1 || slots > 64 || max_queue < 0) return SIM_E_INVALID;
  e.cfg_budget = memory_budget_bytes;
  e.cfg_slots = slots;
  e.cfg_queue = max_queue;
  return SIM_OK;
}

int sim_create(const sim_radar_params *params, sim_ctx **out) {
  if (!out) return SIM_E_INVALID;
  Derived g;
  int rc = derive(params, &g);
  if (rc != SIM_OK) return rc;
  Engine &e = engine();
  {
    std::lock_guard<std::mutex> lk(e.mu);
    rc = start_engine_locked(e);
    if (rc != SIM_OK) return rc;
  }
  cudaSetDevice(e.device);
  sim_ctx *c = new sim_ctx();
  c->g = g;
  rc = upload_tables(c);
  if (rc != SIM_OK) {
    if (c->table_mem) cudaFree(c->table_mem);
    delete c;
    return rc;
  }
  *out = c;
  return SIM_OK;
}

int sim_scene_bytes(const sim_ctx *c, int64_t n_rays, int64_t *bytes) {
  if (!c || !bytes || n_rays < 0 || n_rays > c->g.max_rays) return SIM_E_INVALID;
  const bool want_labels = (c->g.outputs & SIM_OUT_LABELS) != 0;
  *bytes = static_cast<int64_t>(make_plan(c->g, n_rays, want_labels && n_rays > 0).total);
  return SIM_OK;
}

int sim_submit(sim_ctx *c, const sim_rays *rays, const sim_meta *meta, uint64_t *ticket_out) {
  if (!c || !rays || !ticket_out) return SIM_E_INVALID;
  const int64_t n = rays->n;
  if (n < 0 || n > c->g.max_rays) return SIM_E_INVALID;
  const bool want_labels = (c->g.outputs & SIM_OUT_LABELS) != 0;
  const int32_t *obj = meta ? meta->object_id : nullptr;
  if (n > 0) {
    if (!rays->range_rt_m || !rays->amplitude || !rays->radial_velocity_mps || !rays->azimuth_rad ||
        !rays->elevation_rad || !rays->phase0_rad)
      return SIM_E_INVALID;
    if (want_labels && !obj) return SIM_E_INVALID;
  }
  Engine &e = engine();
  cudaSetDevice(e.device);
  // host-resident arrays are validated here; device-resident ones by the prep kernel
  if (n > 0 && !is_device_ptr(rays->range_rt_m) && !is_device_ptr(rays->amplitude) &&
      !is_device_ptr(rays->radial_velocity_mps) && !is_device_ptr(rays->azimuth_rad) &&
      !is_device_ptr(rays->elevation_rad) && !is_device_ptr(rays->phase0_rad)) {
    for (int64_t i = 0; i < n; ++i)
      if (!host_ray_ok(rays->range_rt_m[i], rays->amplitude[i], rays->radial_velocity_mps[i],
                       rays->azimuth_rad[i], rays->elevation_rad[i], rays->phase0_rad[i]))
        return SIM_E_INVALID;
  }
  if (n > 0 && want_labels && !is_device_ptr(obj)) {
    for (int64_t i = 0; i < n; ++i)
      if (obj[i] < 0) return SIM_E_INVALID;
  }
  Job *j = new Job();
  j->ctx = c;
  j->n = n;
  j->has_obj = want_labels && n > 0;
  j->plan = make_plan(c->g, n, j->has_obj);
  bool run_now = false;
  {
    std::lock_guard<std::mutex> lk(e.mu);
    if (static_cast<int64_t>(j->plan.total) > e.budget) {
      delete j;
      return SIM_E_BUSY;
    }
    if (e.queue.empty() && try_reserve_locked(e, j)) {
      run_now = true;
    } else if (static_cast<int>(e.queue.size()) < e.max_queue) {
      // hold a private copy of the inputs until the scene is admitted
      const size_t un = static_cast<size_t>(n);
      j->host_copy.resize(32 * un + 1);
      uint8_t *h = j->host_copy.data();
      if (n > 0) {
        cudaMemcpy(h, rays->range_rt_m, 8 * un, cudaMemcpyDefault);
        cudaMemcpy(h + 8 * un, rays->amplitude, 4 * un, cudaMemcpyDefault);
        cudaMemcpy(h + 12 * un, rays->radial_velocity_mps, 4 * un, cudaMemcpyDefault);
        cudaMemcpy(h + 16 * un, rays->azimuth_rad, 4 * un, cudaMemcpyDefault);
        cudaMemcpy(h + 20 * un, rays->elevation_rad, 4 * un, cudaMemcpyDefault);
        cudaMemcpy(h + 24 * un, rays->phase0_rad, 4 * un, cudaMemcpyDefault);
        if (j->has_obj) cudaMemcpy(h + 28 * un, obj, 4 * un, cudaMemcpyDefault);
      }
      if (cudaGetLastError() != cudaSuccess) {
        delete j;
        return SIM_E_CUDA;
      }
      e.queue.push_back(j);
    } else {
      delete j;
      return SIM_E_BUSY;
    }
    j->ticket = e.next_ticket++;
    e.jobs[j->ticket] = j;
    c->live++;
    e.cv.notify_all();
  }
  if (run_now) {
    const int rc = launch_job(e, j, *rays, obj);
    if (rc == SIM_OK) cudaEventSynchronize(e.slots[j->slot].ev[1]);  // inputs consumed
    std::lock_guard<std::mutex> lk(e.mu);
    j->pending = false;
    if (rc != SIM_OK) {
      // undo: the scene never ran
      cudaStream_t st = e.slots[j->slot].stream;
      if (j->block) cudaFreeAsync(j->block, st);
      cudaStreamSynchronize(st);
      finish_on_device_locked(e, j, cudaSuccess);
      e.used -= static_cast<int64_t>(j->plan.total);
      e.jobs.erase(j->ticket);
      c->live--;
      delete j;
      e.cv.notify_all();
      return rc;
    }
    e.cv.notify_all();  // the worker watches for its completion
  }
  *ticket_out = j->ticket;
  return SIM_OK;
}

int sim_fetch(sim_ctx *c, uint64_t ticket, void *spectrum, void *signal, int32_t *labels, int32_t timeout_ms) {
  if (!c) return SIM_E_INVALID;
  Engine &e = engine();
  if ((spectrum && !(c->g.outputs & SIM_OUT_SPECTRUM)) || (signal && !(c->g.outputs & SIM_OUT_SIGNAL)) ||
      (labels && !(c->g.outputs & SIM_OUT_LABELS)))
    return SIM_E_INVALID;
  cudaSetDevice(e.device);
  const auto t0 = std::chrono::steady_clock::now();
  auto expired = [&] {
    if (timeout_ms < 0) return false;
    return std::chrono::steady_clock::now() - t0 >= std::chrono::milliseconds(timeout_ms);
  };
  std::unique_lock<std::mutex> lk(e.mu);
  auto it = e.jobs.find(ticket);
  if (it == e.jobs.end() || it->second->ctx != c || it->second->claimed) return SIM_E_UNKNOWN_TICKET;
  Job *j = it->second;
  ++e.fetching;
  int rc = SIM_OK;
  for (;;) {
    if (j->done) break;
    if (!j->pending) {
      // running: poll its final event here too, without waiting for the worker
      const cudaError_t q = cudaEventQuery(e.slots[j->slot].ev[kNumEvents - 1]);
      if (q != cudaErrorNotReady) {
        finish_on_device_locked(e, j, q);
        e.cv.notify_all();
        break;
      }
      cudaGetLastError();
    } else if (j->slot < 0 && e.fetching == 1 && !head_fits_locked(e)) {
      // still queued, behind memory that only fetches free, and no other fetch is under way
      rc = SIM_E_BUSY;
      break;
    }
    if (timeout_ms == 0) {
      rc = SIM_E_NOT_READY;
      break;
    }
    if (expired()) {
      rc = SIM_E_TIMEOUT;
      break;
    }
    e.cv.wait_for(lk, std::chrono::microseconds(50));
    if (e.jobs.find(ticket) == e.jobs.end()) {
      rc = SIM_E_UNKNOWN_TICKET;
      break;
    }
  }
  --e.fetching;
  if (rc != SIM_OK) return rc;
  j->claimed = true;
  e.jobs.erase(ticket);
  cudaStream_t s = e.egress[ticket % e.egress.size()];
  lk.unlock();

  uint32_t st[2] = {0, 0};  // status bits, route mask
  cudaError_t sync_rc = j->device_error;
  if (j->launch_error == SIM_OK && j->block) {
    const Derived &g = c->g;
    const Plan &p = j->plan;
    if (spectrum) cudaMemcpyAsync(spectrum, j->block + p.spec, 8 * static_cast<size_t>(g.n_cell), cudaMemcpyDefault, s);
    if (signal) cudaMemcpyAsync(signal, j->block + p.sig, 8 * static_cast<size_t>(g.n_sig), cudaMemcpyDefault, s);
    if (labels) cudaMemcpyAsync(labels, j->block + p.labels, 4 * static_cast<size_t>(g.n_cell), cudaMemcpyDefault, s);
    cudaMemcpyAsync(st, j->block + p.status, 8, cudaMemcpyDeviceToHost, s);
    const cudaError_t cr = cudaStreamSynchronize(s);
    if (sync_rc == cudaSuccess) sync_rc = cr;
  }
  if (j->block) cudaFreeAsync(j->block, s);
  {
    std::lock_guard<std::mutex> g2(e.mu);
    for (int i = 0; i < kNumEvents; ++i) c->last_ms[i] = j->ms[i];
    c->last_kernels = j->kernels;
    c->last_route = st[0] == 0 && sync_rc == cudaSuccess ? st[1] : 0u;
    e.used -= static_cast<int64_t>(j->plan.total);
    c->live--;
    e.cv.notify_all();
  }
  const int launch_error = j->launch_error;
  delete j;
  if (launch_error != SIM_OK) return launch_error;
  if (sync_rc != cudaSuccess) return SIM_E_CUDA;
  if (st[0] & (kStatusBadRay | kStatusModelRange)) return SIM_E_INVALID;
  if (st[0]) return SIM_E_DEVICE;
  return SIM_OK;
}

int sim_destroy(sim_ctx *c) {
  if (!c) return SIM_E_INVALID;
  Engine &e = engine();
  cudaSetDevice(e.device);
  std::vector<uint64_t> mine;
  {
    std::lock_guard<std::mutex> lk(e.mu);
    // queued scenes of this context never start
    for (auto it = e.queue.begin(); it != e.queue.end();) {
      if ((*it)->ctx == c) {
        Job *j = *it;
        e.jobs.erase(j->ticket);
        c->live--;
        delete j;
        it = e.queue.erase(it);
      } else {
        ++it;
      }
    }
    for (auto &kv : e.jobs)
      if (kv.second->ctx == c && !kv.second->claimed) mine.push_back(kv.first);
    e.cv.notify_all();
  }
  for (uint64_t t : mine) sim_fetch(c, t, nullptr, nullptr, nullptr, -1);
  while (c->live.load() > 0) std::this_thread::sleep_for(std::chrono::milliseconds(1));
  if (c->table_mem) cudaFree(c->table_mem);
  for (auto &slot : c->scratch) {
    std::lock_guard<std::mutex> lk(slot.m);  // a synchronous call still running ends first
    if (slot.p) cudaFree(slot.p);
    slot.p = nullptr;
  }
  delete c;
  return SIM_OK;
}

int sim_last_stage_ms(sim_ctx *c, float *ms, int32_t n) {
  if (!c || !ms || n < 0 || n > 8) return SIM_E_INVALID;
  Engine &e = engine();
  std::lock_guard<std::mutex> lk(e.mu);
  for (int i = 0; i < n; ++i) ms[i] = c->last_ms[i];
  return SIM_OK;
}

int sim_last_kernel_count(sim_ctx *c, int32_t *count) {
  if (!c || !count) return SIM_E_INVALID;
  Engine &e = engine();
  std::lock_guard<std::mutex> lk(e.mu);
  *count = c->last_kernels;
  return SIM_OK;
}

int sim_last_expansion_terms(sim_ctx *c, uint32_t *mask) {
  if (!c || !mask) return SIM_E_INVALID;
  Engine &e = engine();
  std::lock_guard<std::mutex> lk(e.mu);
  *mask = c->last_route;
  return SIM_OK;
}

}  // extern "C"
