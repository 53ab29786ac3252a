// sim_run_batch: many scenes, possibly of different radar configurations, as one device
// pipeline (see include/radarsim.h).
//
//   per scene: per-ray prep (+ amplitude maximum for FP16), then its labels
//   all scenes: ONE persistent tensor-core launch; CTAs take (scene, tile, split) units
//               longest first from an atomic work list
//   per scene: split reduction, windowed FFTs
//
// The per-scene stages go to eight side streams (graph branches), so the scenes' small kernels
// overlap one another and the labels overlap the persistent launch.
//
// Each scene's units are exactly those of its single-scene launch, and a unit's result does
// not depend on which CTA runs it, so every scene gives the same bits in the batch as alone.
// The pipeline of a batch shape (the scenes' radar constants and ray counts) is run once
// eagerly, then captured into a CUDA graph that later calls of the same shape replay.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

using namespace rs;

namespace {

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct SceneBufs {
  size_t d, a, v, az, el, p0, obj;
  size_t carrier, nu_r, nu_d, nu_a, amp, cell, energy, step_d, step_r, nu_tx;
  size_t sig, tmp, spec, labels, pk, pe, ck, cm, co, ws, tables;
  int64_t cap;
};

struct BatchPlan {
  std::vector<Derived> gs;
  std::vector<int64_t> ns;
  std::vector<Tables> tables;
  std::vector<SceneBufs> bufs;
  size_t status_off = 0, scratch_off = 0, total = 0;
  uint8_t *block = nullptr;
  UmmaBatch ub{};
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
  ~BatchPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (block) cudaFree(block);
  }
};

// shape key: the radar constants that select kernels and layouts, and the ray count
using Key = std::vector<std::tuple<double, double, double, double, int, int, int, int, double, int, int, int,
                                   int, int, int, int, int, double, int64_t>>;

std::mutex g_mu;
std::map<Key, std::unique_ptr<BatchPlan>> g_plans;
cudaStream_t g_stream = nullptr;
cudaEvent_t g_ev0 = nullptr, g_ev1 = nullptr;
constexpr size_t kMaxPlans = 4;
// Per-scene stages run on kBranches side streams (branches of the captured graph), scene i on
// branch i % kBranches, so the small kernels of different scenes overlap each other and the
// labels overlap the persistent launch; the main stream forks before the preps and joins
// before and after the persistent launch.
constexpr int kBranches = 8;
cudaStream_t g_branch[kBranches] = {};
cudaEvent_t g_fork = nullptr, g_gemm = nullptr, g_pre[kBranches] = {}, g_post[kBranches] = {};

Key key_of(int n, sim_ctx *const *ctxs, const sim_rays *rays) {
  Key k;
  for (int i = 0; i < n; ++i) {
    const Derived &g = ctxs[i]->g;
    k.emplace_back(g.fc, g.bw, g.tc, g.td, g.ns, g.nc, g.ntx, g.nrx, g.spacing_wl, g.na, g.win[0], g.win[1],
                   g.win[2], g.precision, g.outputs, g.model, g.pattern_exp, g.tslot, rays[i].n);
  }
  return k;
}

// the stages of one batch, forked from and joined back into stream s; returns the number of
// kernels launched
int enqueue(BatchPlan &p, cudaStream_t s) {
  uint8_t *b = p.block;
  const int n = static_cast<int>(p.gs.size());
  uint32_t *status = reinterpret_cast<uint32_t *>(b + p.status_off);
  int kernels = 0;
  cudaMemsetAsync(status, 0, 4 * static_cast<size_t>(n), s);
  cudaEventRecord(g_fork, s);
  for (int k = 0; k < kBranches; ++k) cudaStreamWaitEvent(g_branch[k], g_fork, 0);
  std::vector<RaysPrep> preps(static_cast<size_t>(n));
  for (int i = 0; i < n; ++i) {
    cudaStream_t bs = g_branch[i % kBranches];
    const SceneBufs &q = p.bufs[static_cast<size_t>(i)];
    const Derived &g = p.gs[static_cast<size_t>(i)];
    const bool lab = g.outputs & SIM_OUT_LABELS;
    RaysIn in{reinterpret_cast<const double *>(b + q.d), reinterpret_cast<const float *>(b + q.a),
              reinterpret_cast<const float *>(b + q.v), reinterpret_cast<const float *>(b + q.az),
              reinterpret_cast<const float *>(b + q.el), reinterpret_cast<const float *>(b + q.p0),
              lab ? reinterpret_cast<const int32_t *>(b + q.obj) : nullptr};
    RaysPrep rp{reinterpret_cast<uint64_t *>(b + q.carrier), reinterpret_cast<uint64_t *>(b + q.nu_r),
                reinterpret_cast<uint64_t *>(b + q.nu_d), reinterpret_cast<uint64_t *>(b + q.nu_a),
                reinterpret_cast<float *>(b + q.amp), reinterpret_cast<int32_t *>(b + q.cell),
                reinterpret_cast<uint64_t *>(b + q.energy), reinterpret_cast<float2 *>(b + q.step_d),
                reinterpret_cast<float2 *>(b + q.step_r), nullptr, reinterpret_cast<uint64_t *>(b + q.nu_tx),
                nullptr};
    preps[static_cast<size_t>(i)] = rp;
    kernels += launch_prep(g, in, p.ns[static_cast<size_t>(i)], rp, status + i, bs);
    kernels += launch_umma_pre(g, rp, p.ns[static_cast<size_t>(i)], b + q.ws, bs);
  }
  for (int k = 0; k < kBranches; ++k) {
    cudaEventRecord(g_pre[k], g_branch[k]);
    cudaStreamWaitEvent(s, g_pre[k], 0);
  }
  // the labels need only the prep: they run beside the persistent launch
  for (int i = 0; i < n; ++i) {
    const SceneBufs &q = p.bufs[static_cast<size_t>(i)];
    const Derived &g = p.gs[static_cast<size_t>(i)];
    if (g.outputs & SIM_OUT_LABELS) {
      LabelScratch sc{reinterpret_cast<uint64_t *>(b + q.pk), reinterpret_cast<uint64_t *>(b + q.pe),
                      reinterpret_cast<uint32_t *>(b + q.ck), reinterpret_cast<uint64_t *>(b + q.cm),
                      reinterpret_cast<uint32_t *>(b + q.co), q.cap};
      kernels += launch_labels(g, preps[static_cast<size_t>(i)], reinterpret_cast<const int32_t *>(b + q.obj),
                               p.ns[static_cast<size_t>(i)], sc, reinterpret_cast<int32_t *>(b + q.labels),
                               status + i, g_branch[i % kBranches]);
    }
  }
  kernels += launch_umma_batch(p.ub, s);
  cudaEventRecord(g_gemm, s);
  for (int k = 0; k < kBranches; ++k) cudaStreamWaitEvent(g_branch[k], g_gemm, 0);
  for (int i = 0; i < n; ++i) {
    cudaStream_t bs = g_branch[i % kBranches];
    const SceneBufs &q = p.bufs[static_cast<size_t>(i)];
    const Derived &g = p.gs[static_cast<size_t>(i)];
    float2 *sig = reinterpret_cast<float2 *>(b + q.sig);
    kernels += launch_umma_post(g, p.ns[static_cast<size_t>(i)], sig, b + q.ws, bs);
    if (g.outputs & SIM_OUT_SPECTRUM)
      kernels += launch_fft(g, p.tables[static_cast<size_t>(i)], sig, reinterpret_cast<float2 *>(b + q.tmp),
                            reinterpret_cast<float2 *>(b + q.spec), bs);
  }
  for (int k = 0; k < kBranches; ++k) {
    cudaEventRecord(g_post[k], g_branch[k]);
    cudaStreamWaitEvent(s, g_post[k], 0);
  }
  return kernels;
}

int build_plan(int n, sim_ctx *const *ctxs, const sim_rays *rays, BatchPlan &p) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes > 0 ? bytes : 1);
    return o;
  };
  int64_t total_units = 0;
  for (int i = 0; i < n; ++i) {
    const Derived &g = ctxs[i]->g;
    const int64_t r = rays[i].n;
    const size_t un = static_cast<size_t>(r), up = (un + 31) / 32 * 32;
    const bool spec = g.outputs & SIM_OUT_SPECTRUM, lab = g.outputs & SIM_OUT_LABELS;
    SceneBufs q{};
    q.d = take(8 * un);
    q.a = take(4 * un);
    q.v = take(4 * un);
    q.az = take(4 * un);
    q.el = take(4 * un);
    q.p0 = take(4 * un);
    q.obj = take(lab ? 4 * un : 0);
    q.carrier = take(8 * up);
    q.nu_r = take(8 * up);
    q.nu_d = take(8 * up);
    q.nu_a = take(8 * up);
    q.amp = take(4 * up);
    q.cell = take(4 * up);
    q.energy = take(8 * up);
    q.step_d = take(8 * up);
    q.step_r = take(8 * up);
    q.nu_tx = take(8 * up);
    q.sig = take(8 * static_cast<size_t>(g.n_sig));
    q.tmp = take(spec ? 8 * static_cast<size_t>(g.n_sig) : 0);
    q.spec = take(spec ? 8 * static_cast<size_t>(g.n_cell) : 0);
    q.labels = take(lab ? 4 * static_cast<size_t>(g.n_cell) : 0);
    q.cap = lab ? label_capacity(r) : 0;
    const size_t cap = static_cast<size_t>(q.cap);
    q.pk = take(8 * cap);
    q.pe = take(8 * cap);
    q.ck = take(4 * cap);
    q.cm = take(8 * cap);
    q.co = take(4 * cap);
    q.ws = take(static_cast<size_t>(batch_workspace_bytes(g, r)));
    q.tables = take(ctxs[i]->table_bytes);
    p.bufs.push_back(q);
    p.gs.push_back(g);
    p.ns.push_back(r);
    total_units += umma_units_of(g, r);
  }
  p.status_off = take(4 * static_cast<size_t>(n));
  p.scratch_off = take(static_cast<size_t>(umma_batch_scratch_bytes(n, total_units)));
  p.total = off;
  if (cudaMalloc(&p.block, p.total) != cudaSuccess) {
    cudaGetLastError();
    p.block = nullptr;
    return SIM_E_NOMEM;
  }
  // private copies of each scene's window and twiddle tables
  for (int i = 0; i < n; ++i) {
    const sim_ctx *c = ctxs[i];
    uint8_t *dst = p.block + p.bufs[static_cast<size_t>(i)].tables;
    if (cudaMemcpyAsync(dst, c->table_mem, c->table_bytes, cudaMemcpyDeviceToDevice, g_stream) != cudaSuccess)
      return SIM_E_CUDA;
    const uint8_t *src = static_cast<const uint8_t *>(c->table_mem);
    auto rebase = [&](const void *ptr) { return dst + (static_cast<const uint8_t *>(ptr) - src); };
    Tables t;
    t.win_r = reinterpret_cast<float *>(rebase(c->t.win_r));
    t.win_d = reinterpret_cast<float *>(rebase(c->t.win_d));
    t.win_a = reinterpret_cast<float *>(rebase(c->t.win_a));
    t.tw_r = reinterpret_cast<float2 *>(rebase(c->t.tw_r));
    t.tw_d = reinterpret_cast<float2 *>(rebase(c->t.tw_d));
    t.tw_a = reinterpret_cast<float2 *>(rebase(c->t.tw_a));
    p.tables.push_back(t);
  }
  std::vector<const Derived *> gp;
  std::vector<RaysPrep> rp;
  std::vector<void *> ws;
  std::vector<uint32_t *> st;
  for (int i = 0; i < n; ++i) {
    const SceneBufs &q = p.bufs[static_cast<size_t>(i)];
    gp.push_back(&p.gs[static_cast<size_t>(i)]);
    RaysPrep r{reinterpret_cast<uint64_t *>(p.block + q.carrier), reinterpret_cast<uint64_t *>(p.block + q.nu_r),
               reinterpret_cast<uint64_t *>(p.block + q.nu_d), reinterpret_cast<uint64_t *>(p.block + q.nu_a),
               reinterpret_cast<float *>(p.block + q.amp), reinterpret_cast<int32_t *>(p.block + q.cell),
               reinterpret_cast<uint64_t *>(p.block + q.energy), reinterpret_cast<float2 *>(p.block + q.step_d),
               reinterpret_cast<float2 *>(p.block + q.step_r), nullptr,
               reinterpret_cast<uint64_t *>(p.block + q.nu_tx), nullptr};
    rp.push_back(r);
    ws.push_back(p.block + q.ws);
    st.push_back(reinterpret_cast<uint32_t *>(p.block + p.status_off) + i);
  }
  return prepare_umma_batch(n, gp.data(), rp.data(), p.ns.data(), ws.data(), st.data(), p.block + p.scratch_off,
                            g_stream, &p.ub);
}

}  // namespace

extern "C" SIM_API int sim_run_batch(int32_t n, sim_ctx *const *ctxs, const sim_rays *rays, const sim_meta *meta,
                                     void *const *spectra, void *const *signals, int32_t *const *labels,
                                     float *device_ms, int32_t *kernel_count) {
  if (n < 1 || n > 4096 || !ctxs || !rays) return SIM_E_INVALID;
  launches_begin();
  for (int i = 0; i < n; ++i) {
    const sim_ctx *c = ctxs[i];
    if (!c) return SIM_E_INVALID;
    const Derived &g = c->g;
    if (g.precision == SIM_PREC_FP32_DIRECT || g.precision != ctxs[0]->g.precision) return SIM_E_INVALID;
    if (rays[i].n < 0 || rays[i].n > g.max_rays) return SIM_E_INVALID;
    if (rays[i].n > 0 && (!rays[i].range_rt_m || !rays[i].amplitude || !rays[i].radial_velocity_mps ||
                          !rays[i].azimuth_rad || !rays[i].elevation_rad || !rays[i].phase0_rad))
      return SIM_E_INVALID;
    if ((g.outputs & SIM_OUT_LABELS) && rays[i].n > 0 && (!meta || !meta[i].object_id)) return SIM_E_INVALID;
    if ((spectra && spectra[i] && !(g.outputs & SIM_OUT_SPECTRUM)) ||
        (signals && signals[i] && !(g.outputs & SIM_OUT_SIGNAL)) ||
        (labels && labels[i] && !(g.outputs & SIM_OUT_LABELS)))
      return SIM_E_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_stream) {
    bool ok = cudaStreamCreateWithFlags(&g_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreate(&g_ev0) == cudaSuccess && cudaEventCreate(&g_ev1) == cudaSuccess &&
              cudaEventCreateWithFlags(&g_fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&g_gemm, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < kBranches && ok; ++k)
      ok = cudaStreamCreateWithFlags(&g_branch[k], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&g_pre[k], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&g_post[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {  // release what was made; a later call tries again
      for (int k = 0; k < kBranches; ++k) {
        if (g_branch[k]) cudaStreamDestroy(g_branch[k]);
        if (g_pre[k]) cudaEventDestroy(g_pre[k]);
        if (g_post[k]) cudaEventDestroy(g_post[k]);
        g_branch[k] = nullptr;
        g_pre[k] = g_post[k] = nullptr;
      }
      for (cudaEvent_t *e : {&g_ev0, &g_ev1, &g_fork, &g_gemm}) {
        if (*e) cudaEventDestroy(*e);
        *e = nullptr;
      }
      if (g_stream) cudaStreamDestroy(g_stream);
      g_stream = nullptr;
      cudaGetLastError();
      return SIM_E_CUDA;
    }
  }
  cudaStream_t s = g_stream;
  const Key key = key_of(n, ctxs, rays);
  auto it = g_plans.find(key);
  BatchPlan *plan = nullptr;
  bool fresh = false;
  if (it == g_plans.end()) {
    if (g_plans.size() >= kMaxPlans) g_plans.erase(g_plans.begin());
    auto np = std::make_unique<BatchPlan>();
    const int rc = build_plan(n, ctxs, rays, *np);
    if (rc != SIM_OK) return rc;
    plan = np.get();
    g_plans[key] = std::move(np);
    fresh = true;
  } else {
    plan = it->second.get();
  }
  // inputs into the plan's buffers
  for (int i = 0; i < n; ++i) {
    const SceneBufs &q = plan->bufs[static_cast<size_t>(i)];
    const size_t un = static_cast<size_t>(rays[i].n);
    if (un == 0) continue;
    uint8_t *b = plan->block;
    cudaMemcpyAsync(b + q.d, rays[i].range_rt_m, 8 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + q.a, rays[i].amplitude, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + q.v, rays[i].radial_velocity_mps, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + q.az, rays[i].azimuth_rad, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + q.el, rays[i].elevation_rad, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + q.p0, rays[i].phase0_rad, 4 * un, cudaMemcpyDefault, s);
    if (plan->gs[static_cast<size_t>(i)].outputs & SIM_OUT_LABELS)
      cudaMemcpyAsync(b + q.obj, meta[i].object_id, 4 * un, cudaMemcpyDefault, s);
  }
  cudaEventRecord(g_ev0, s);
  if (fresh) {
    // first run eagerly (sets kernel attributes, checks the launches), then capture the graph
    plan->kernels = enqueue(*plan, s);
    cudaEventRecord(g_ev1, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return SIM_E_CUDA;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SIM_E_CUDA;
    enqueue(*plan, s);
    if (cudaStreamEndCapture(s, &graph) != cudaSuccess) return SIM_E_CUDA;
    const cudaError_t ie = cudaGraphInstantiate(&plan->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      plan->exec = nullptr;
      return SIM_E_CUDA;
    }
  } else {
    if (cudaGraphLaunch(plan->exec, s) != cudaSuccess) return SIM_E_CUDA;
    cudaEventRecord(g_ev1, s);
  }
  for (int i = 0; i < n; ++i) {
    const SceneBufs &q = plan->bufs[static_cast<size_t>(i)];
    const Derived &g = plan->gs[static_cast<size_t>(i)];
    if (spectra && spectra[i])
      cudaMemcpyAsync(spectra[i], plan->block + q.spec, 8 * static_cast<size_t>(g.n_cell), cudaMemcpyDefault, s);
    if (signals && signals[i])
      cudaMemcpyAsync(signals[i], plan->block + q.sig, 8 * static_cast<size_t>(g.n_sig), cudaMemcpyDefault, s);
    if (labels && labels[i])
      cudaMemcpyAsync(labels[i], plan->block + q.labels, 4 * static_cast<size_t>(g.n_cell), cudaMemcpyDefault, s);
  }
  std::vector<uint32_t> status(static_cast<size_t>(n), 0);
  cudaMemcpyAsync(status.data(), plan->block + plan->status_off, 4 * static_cast<size_t>(n), cudaMemcpyDeviceToHost,
                  s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return SIM_E_CUDA;
  if (device_ms) {
    *device_ms = 0.f;
    cudaEventElapsedTime(device_ms, g_ev0, g_ev1);
  }
  if (kernel_count) *kernel_count = plan->kernels;
  if (!launches_ok()) return SIM_E_CUDA;
  uint32_t any = 0;
  for (uint32_t v : status) any |= v;
  if (any & kStatusBadRay) return SIM_E_INVALID;
  return any ? SIM_E_DEVICE : SIM_OK;
}
