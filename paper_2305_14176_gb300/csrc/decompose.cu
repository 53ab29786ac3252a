// sim_decompose: the radar signal split by ray meta data (arXiv 2305.14176, Sec. II-C, Eq. 5).
//
//   s_IF = sum_h s_IF^h, each part s^h summed over the rays of span h only.
//
// A span is chosen by a filter rule on a ray's meta data: its object (mesh) id, its material
// id and its number of hits, e.g. "any hit on the pedestrian", "more than one hit" (multi-path
// ghosts) or "exactly one hit on object 7" (line of sight).  Every span's part goes through
// the same windowed FFTs, and each cell is labelled with the span whose image is strongest
// there, among the spans whose image passes a relative threshold: the paper's simple binary
// segmentation of each part, with overlaps resolved by energy.
//
// The per-ray prep runs once.  Each span's rays are then packed in ray order (block counts of
// every span, a scan, one read-back of the span sizes, a stable gather) and summed alone
// through the context's ray-sum arithmetic (direct or tensor core): a span costs its own ray
// count, so the spans of a partition cost one scene's ray sums together, and a span's part is
// bit for bit the scene of its rays alone.  Spans run on up to four streams at once, each with
// its own packed prep, workspace and signal; a span's range FFT writes into its spectrum slot,
// where its Doppler and angle FFTs follow in place.  (The Doppler and angle FFTs of all spans as
// one launch each after the sums were measured slower: 5.49 against 5.31 ms per automotive
// decomposition at FP16 hi + lo, since on the lanes they overlap other spans' sums.)
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.h"

using namespace rs;

namespace {

struct RuleDev {
  int32_t object_id, material_id, min_hits, max_hits, exclude;
};

__device__ __forceinline__ bool in_span(const RuleDev &r, const int32_t *obj, const int32_t *mat,
                                        const int32_t *hits, int64_t i) {
  bool in = true;
  if (r.object_id >= 0) in = in && obj && obj[i] == r.object_id;
  if (r.material_id >= 0) in = in && mat && mat[i] == r.material_id;
  if (r.min_hits > 0 || r.max_hits >= 0) {
    const int32_t h = hits ? hits[i] : 1;
    in = in && h >= r.min_hits && (r.max_hits < 0 || h <= r.max_hits);
  }
  return r.exclude ? !in : in;
}

constexpr int kSpanBlock = 1024;  // rays per compaction block (one thread each)
constexpr int kLanes = 4;         // spans summed concurrently (streams)
// Each span's tensor-core sum plans one wave of CTAs (a scene alone plans four): the lanes share
// the GPU, and a span's CTAs then take several times more rays each, with as many fewer split-K
// partials to write and reduce.  Its workspace is sized by the same plan.
constexpr float kSpanWaves = 0.5f;
constexpr int64_t kSpanMinChunk = 8192;

// cnt[h nb + b]: rays of block b in span h (grid nb x n_spans)
__global__ void __launch_bounds__(kSpanBlock) span_count_kernel(const int32_t *__restrict__ obj,
                                                                const int32_t *__restrict__ mat,
                                                                const int32_t *__restrict__ hits, int64_t n,
                                                                const RuleDev *__restrict__ rules, int nb,
                                                                uint32_t *__restrict__ cnt) {
  __shared__ uint32_t wsum[kSpanBlock / 32];
  const int h = blockIdx.y;
  const int64_t i = blockIdx.x * static_cast<int64_t>(kSpanBlock) + threadIdx.x;
  const bool f = i < n && in_span(rules[h], obj, mat, hits, i);
  const uint32_t bal = __ballot_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = __popc(bal);
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t v = wsum[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) cnt[static_cast<int64_t>(h) * nb + blockIdx.x] = v;
  }
}

// per span h (one block each): off[h nb + b] = rays of span h in blocks before b; total[h]
__global__ void __launch_bounds__(kSpanBlock) span_scan_kernel(const uint32_t *__restrict__ cnt, int nb,
                                                               uint32_t *__restrict__ off,
                                                               uint32_t *__restrict__ total) {
  __shared__ uint32_t sh[kSpanBlock];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * nb;
  const int per = (nb + kSpanBlock - 1) / kSpanBlock;
  const int t = threadIdx.x, s0 = t * per;
  uint32_t local = 0;
  for (int k = 0; k < per; ++k)
    if (s0 + k < nb) local += cnt[base + s0 + k];
  sh[t] = local;
  __syncthreads();
  for (int d = 1; d < kSpanBlock; d <<= 1) {  // inclusive scan
    const uint32_t v = t >= d ? sh[t - d] : 0u;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  uint32_t run = sh[t] - local;
  for (int k = 0; k < per; ++k)
    if (s0 + k < nb) {
      off[base + s0 + k] = run;
      run += cnt[base + s0 + k];
    }
  if (t == kSpanBlock - 1) total[blockIdx.x] = sh[t];
}

// The prep words of span h's rays, packed in ray order: ray i of the span goes to
// off_h[block] + (its rank among the span's rays of the block).
__global__ void __launch_bounds__(kSpanBlock) span_gather_kernel(RaysPrep src, RaysPrep dst,
                                                                 const int32_t *__restrict__ obj,
                                                                 const int32_t *__restrict__ mat,
                                                                 const int32_t *__restrict__ hits, int64_t n,
                                                                 const RuleDev *__restrict__ rule,
                                                                 const uint32_t *__restrict__ off_h) {
  __shared__ uint32_t wpre[kSpanBlock / 32];
  const int64_t i = blockIdx.x * static_cast<int64_t>(kSpanBlock) + threadIdx.x;
  const bool f = i < n && in_span(*rule, obj, mat, hits, i);
  const uint32_t bal = __ballot_sync(0xffffffffu, f);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wpre[w] = __popc(bal);
  __syncthreads();
  if (w == 0) {  // exclusive scan of the 32 warp counts
    const uint32_t v = wpre[lane];
    uint32_t x = v;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    wpre[lane] = x - v;
  }
  __syncthreads();
  if (!f) return;
  const int64_t j = off_h[blockIdx.x] + wpre[w] + __popc(bal & ((1u << lane) - 1u));
  dst.carrier[j] = src.carrier[i];
  dst.nu_r[j] = src.nu_r[i];
  dst.nu_d[j] = src.nu_d[i];
  dst.nu_a[j] = src.nu_a[i];
  dst.amp[j] = src.amp[i];
  dst.step_d[j] = src.step_d[i];
  dst.step_r[j] = src.step_r[i];
  dst.nu_tx[j] = src.nu_tx[i];
  if (src.eps) {
    dst.eps[j] = src.eps[i];
    dst.eps_t[j] = src.eps_t[i];
  }
}

// largest |X|^2 over all spans and cells (non-negative floats: bit order is value order)
__global__ void power_max_kernel(const float2 *__restrict__ x, int64_t n, uint32_t *max_bits) {
  uint32_t m = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float2 v = x[i];
    m = max(m, __float_as_uint(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y))));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(max_bits, m);
}

// label[c] = argmax_h |X_h[c]|^2 over spans with |X_h[c]|^2 >= t^2 max; ties to the lower span
__global__ void span_label_kernel(const float2 *__restrict__ spectra, int n_spans, int64_t n_cell, float t2,
                                  const uint32_t *max_bits, int32_t *__restrict__ labels) {
  // powers as (x*x) + (y*y), each operation rounded on its own (no fused multiply-add), so a
  // host can repeat every decision in FP32
  const float floor_p = __fmul_rn(t2, __uint_as_float(*max_bits));
  for (int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; c < n_cell;
       c += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int best = -1;
    float best_p = 0.f;
    for (int h = 0; h < n_spans; ++h) {
      const float2 v = spectra[static_cast<int64_t>(h) * n_cell + c];
      const float p = __fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y));
      if (p >= floor_p && p > 0.f && (best < 0 || p > best_p)) {
        best = h;
        best_p = p;
      }
    }
    labels[c] = best;
  }
}

size_t round256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

}  // namespace

extern "C" SIM_API int sim_decompose(sim_ctx *ctx, const sim_rays *rays, const sim_meta *meta, int32_t n_spans,
                                     const sim_span_rule *rules, void *const *span_spectra, int32_t *span_labels,
                                     float threshold) {
  if (!ctx || !rays || !rules || n_spans < 1 || n_spans > 64) return SIM_E_INVALID;
  launches_begin();
  if (!(threshold >= 0.f && threshold <= 1.f)) return SIM_E_INVALID;
  const Derived &g = ctx->g;
  const int64_t n = rays->n;
  if (n < 0 || n > g.max_rays) return SIM_E_INVALID;
  for (int h = 0; h < n_spans; ++h) {
    const sim_span_rule &r = rules[h];
    if (r.object_id >= 0 && (!meta || !meta->object_id)) return SIM_E_INVALID;
    if (r.material_id >= 0 && (!meta || !meta->material_id)) return SIM_E_INVALID;
    if ((r.min_hits > 0 || r.max_hits >= 0) && (!meta || !meta->n_hits)) return SIM_E_INVALID;
    if (r.max_hits >= 0 && r.max_hits < r.min_hits) return SIM_E_INVALID;
  }
  if (n > 0 && (!rays->range_rt_m || !rays->amplitude || !rays->radial_velocity_mps || !rays->azimuth_rad ||
                !rays->elevation_rad || !rays->phase0_rad))
    return SIM_E_INVALID;

  // device workspace: inputs, meta, prep, compaction counts, spectra, labels (the lanes' blocks
  // follow once the span sizes are known)
  const size_t un = static_cast<size_t>(n), up = (un + 31) / 32 * 32;
  const bool tensor = g.precision != SIM_PREC_FP32_DIRECT;
  const bool exact = g.model == SIM_MODEL_EXACT;
  const int nb = n > 0 ? static_cast<int>((n + kSpanBlock - 1) / kSpanBlock) : 0;
  const size_t ub = static_cast<size_t>(nb) * static_cast<size_t>(n_spans);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += round256(bytes > 0 ? bytes : 1);
    return o;
  };
  const size_t o_d = take(8 * un), o_a = take(4 * un), o_v = take(4 * un), o_az = take(4 * un),
               o_el = take(4 * un), o_p0 = take(4 * un), o_obj = take(4 * un), o_mat = take(4 * un),
               o_hit = take(4 * un);
  const size_t o_car = take(8 * up), o_nur = take(8 * up), o_nud = take(8 * up), o_nua = take(8 * up),
               o_amp = take(4 * up), o_cell = take(4 * up), o_en = take(8 * up), o_sd = take(8 * up),
               o_sr = take(8 * up), o_eps = take(exact ? 8 * up : 0), o_ntx = take(8 * up),
               o_epst = take(exact ? 8 * up : 0);
  const size_t o_rules = take(sizeof(RuleDev) * static_cast<size_t>(n_spans)), o_cnt = take(4 * ub),
               o_off = take(4 * ub), o_tot = take(4 * static_cast<size_t>(n_spans));
  const size_t o_status = take(256), o_max = take(256);
  const size_t o_spec = take(8 * static_cast<size_t>(g.n_cell) * static_cast<size_t>(n_spans));
  const size_t o_lab = take(4 * static_cast<size_t>(g.n_cell));
  // the call's block and the lanes' blocks come from the context's scratch (kept between calls);
  // both leases end after `finish` has waited for every stream
  ScratchLease lease_b, lease_ws;
  uint8_t *b = static_cast<uint8_t *>(lease_b.get(ctx->scratch[kSlotDecompose], off));
  if (!b) return SIM_E_NOMEM;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SIM_E_CUDA;
  void *ws = nullptr;  // the lanes' blocks: packed prep, ray-sum workspace, signal, FFT scratch
  cudaStream_t lane_s[kLanes] = {};
  cudaEvent_t lane_done[kLanes] = {};
  for (int l = 1; l < kLanes; ++l) cudaEventCreateWithFlags(&lane_done[l], cudaEventDisableTiming);
  auto finish = [&](int rc) {
    for (int l = 1; l < kLanes; ++l) {
      if (lane_s[l]) {
        cudaStreamSynchronize(lane_s[l]);
        cudaStreamDestroy(lane_s[l]);
      }
      if (lane_done[l]) cudaEventDestroy(lane_done[l]);
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    cudaGetLastError();
    return rc;
  };
  const int32_t *dobj = nullptr, *dmat = nullptr, *dhit = nullptr;
  if (n > 0) {
    cudaMemcpyAsync(b + o_d, rays->range_rt_m, 8 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + o_a, rays->amplitude, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + o_v, rays->radial_velocity_mps, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + o_az, rays->azimuth_rad, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + o_el, rays->elevation_rad, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + o_p0, rays->phase0_rad, 4 * un, cudaMemcpyDefault, s);
    if (meta && meta->object_id) {
      cudaMemcpyAsync(b + o_obj, meta->object_id, 4 * un, cudaMemcpyDefault, s);
      dobj = reinterpret_cast<const int32_t *>(b + o_obj);
    }
    if (meta && meta->material_id) {
      cudaMemcpyAsync(b + o_mat, meta->material_id, 4 * un, cudaMemcpyDefault, s);
      dmat = reinterpret_cast<const int32_t *>(b + o_mat);
    }
    if (meta && meta->n_hits) {
      cudaMemcpyAsync(b + o_hit, meta->n_hits, 4 * un, cudaMemcpyDefault, s);
      dhit = reinterpret_cast<const int32_t *>(b + o_hit);
    }
  }
  std::vector<RuleDev> hrules(static_cast<size_t>(n_spans));
  for (int h = 0; h < n_spans; ++h)
    hrules[h] = RuleDev{rules[h].object_id, rules[h].material_id, rules[h].min_hits, rules[h].max_hits,
                        rules[h].exclude};
  const RuleDev *drules = reinterpret_cast<const RuleDev *>(b + o_rules);
  cudaMemcpyAsync(b + o_rules, hrules.data(), sizeof(RuleDev) * hrules.size(), cudaMemcpyHostToDevice, s);
  uint32_t *status = reinterpret_cast<uint32_t *>(b + o_status);
  uint32_t *pmax = reinterpret_cast<uint32_t *>(b + o_max);
  cudaMemsetAsync(status, 0, 8, s);  // status bits and route mask
  cudaMemsetAsync(pmax, 0, 4, s);
  RaysIn in{reinterpret_cast<const double *>(b + o_d), reinterpret_cast<const float *>(b + o_a),
            reinterpret_cast<const float *>(b + o_v), reinterpret_cast<const float *>(b + o_az),
            reinterpret_cast<const float *>(b + o_el), reinterpret_cast<const float *>(b + o_p0), dobj};
  RaysPrep rp{reinterpret_cast<uint64_t *>(b + o_car), reinterpret_cast<uint64_t *>(b + o_nur),
              reinterpret_cast<uint64_t *>(b + o_nud), reinterpret_cast<uint64_t *>(b + o_nua),
              reinterpret_cast<float *>(b + o_amp), reinterpret_cast<int32_t *>(b + o_cell),
              reinterpret_cast<uint64_t *>(b + o_en), reinterpret_cast<float2 *>(b + o_sd),
              reinterpret_cast<float2 *>(b + o_sr), exact ? reinterpret_cast<uint64_t *>(b + o_eps) : nullptr,
              reinterpret_cast<uint64_t *>(b + o_ntx), exact ? reinterpret_cast<uint64_t *>(b + o_epst) : nullptr};
  // events: start, after the span sizes, after every span's sum and FFT, after the labels
  std::vector<cudaEvent_t> ev(4, nullptr);
  for (auto &e : ev) cudaEventCreate(&e);
  struct EventsGuard {
    std::vector<cudaEvent_t> &v;
    ~EventsGuard() {
      for (auto &e : v)
        if (e) cudaEventDestroy(e);
    }
  } ev_guard{ev};
  int kernels = 0;
  cudaEventRecord(ev[0], s);
  kernels += launch_prep(g, in, n, rp, status, s);
  // span sizes: block counts of every span, their scan, one read-back of the sizes
  uint32_t *cnt = reinterpret_cast<uint32_t *>(b + o_cnt), *boff = reinterpret_cast<uint32_t *>(b + o_off);
  uint32_t *tot = reinterpret_cast<uint32_t *>(b + o_tot);
  std::vector<uint32_t> sizes(static_cast<size_t>(n_spans), 0u);
  if (n > 0) {
    span_count_kernel<<<dim3(static_cast<unsigned>(nb), static_cast<unsigned>(n_spans)), kSpanBlock, 0, s>>>(
        dobj, dmat, dhit, n, drules, nb, cnt);
    span_scan_kernel<<<static_cast<unsigned>(n_spans), kSpanBlock, 0, s>>>(cnt, nb, boff, tot);
    kernels += 2;
  }
  cudaEventRecord(ev[1], s);
  if (n > 0) cudaMemcpyAsync(sizes.data(), tot, 4 * sizes.size(), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return finish(SIM_E_CUDA);
  // Spans run on up to kLanes streams at once.  Each lane has its own packed prep, ray-sum
  // workspace and signal, so small spans' launches fill each other's gaps on the device while
  // every span's arithmetic stays what it would be alone.
  int live = 0;
  for (uint32_t nh : sizes) live += nh > 0 ? 1 : 0;
  int lanes = std::max(1, std::min(kLanes, live));
  int64_t need = 0;  // ray-sum workspace of the largest span
  for (uint32_t nh : sizes)
    if (nh > 0)
      need = std::max<int64_t>(need, tensor ? umma_workspace_bytes(g, static_cast<int64_t>(nh), kSpanWaves, kSpanMinChunk)
                                            : direct_workspace_bytes(g, static_cast<int64_t>(nh)));
  const size_t l_prep = round256((exact ? 76 : 60) * up), l_ws = round256(static_cast<size_t>(need)),
               l_sig = round256(8 * static_cast<size_t>(g.n_sig));
  const size_t lane_bytes = l_prep + l_ws + l_sig;  // prep, workspace, signal
  ws = lease_ws.get(ctx->scratch[kSlotDecomposeLanes], lane_bytes * static_cast<size_t>(lanes));
  if (!ws && lanes > 1) {
    lanes = 1;
    ws = lease_ws.get(ctx->scratch[kSlotDecomposeLanes], lane_bytes);
  }
  if (!ws) return finish(SIM_E_NOMEM);
  for (int l = 1; l < lanes; ++l) {
    if (cudaStreamCreateWithFlags(&lane_s[l], cudaStreamNonBlocking) != cudaSuccess) return finish(SIM_E_CUDA);
    cudaStreamWaitEvent(lane_s[l], ev[1], 0);  // after prep and the span sizes
  }
  lane_s[0] = s;
  auto lane_prep = [&](int l) {
    uint8_t *pb = static_cast<uint8_t *>(ws) + static_cast<size_t>(l) * lane_bytes;
    RaysPrep q = rp;  // a packed span: its own copies of every word a ray sum reads (cell and
                      // energy stay the scene's, unused)
    q.carrier = reinterpret_cast<uint64_t *>(pb);
    q.nu_r = reinterpret_cast<uint64_t *>(pb + 8 * up);
    q.nu_d = reinterpret_cast<uint64_t *>(pb + 16 * up);
    q.nu_a = reinterpret_cast<uint64_t *>(pb + 24 * up);
    q.nu_tx = reinterpret_cast<uint64_t *>(pb + 32 * up);
    q.step_d = reinterpret_cast<float2 *>(pb + 40 * up);
    q.step_r = reinterpret_cast<float2 *>(pb + 48 * up);
    q.amp = reinterpret_cast<float *>(pb + 56 * up);
    q.eps = exact ? reinterpret_cast<uint64_t *>(pb + 60 * up) : nullptr;
    q.eps_t = exact ? reinterpret_cast<uint64_t *>(pb + 68 * up) : nullptr;
    return q;
  };
  float2 *spectra = reinterpret_cast<float2 *>(b + o_spec);
  // lanes by longest span first, each span to the lane with the fewest rays so far (a span's
  // bits do not depend on its lane)
  std::vector<int> order(static_cast<size_t>(n_spans));
  for (int h = 0; h < n_spans; ++h) order[static_cast<size_t>(h)] = h;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return sizes[x] > sizes[y]; });
  std::vector<int64_t> lane_rays(static_cast<size_t>(lanes), 0);
  for (int h : order) {
    const int64_t nh = sizes[h];
    float2 *x = spectra + static_cast<int64_t>(h) * g.n_cell;
    if (nh > 0) {
      const int l = static_cast<int>(std::min_element(lane_rays.begin(), lane_rays.end()) - lane_rays.begin());
      lane_rays[static_cast<size_t>(l)] += nh;
      cudaStream_t sl = lane_s[l];
      uint8_t *lb = static_cast<uint8_t *>(ws) + static_cast<size_t>(l) * lane_bytes;
      const RaysPrep q = lane_prep(l);
      float2 *lsig = reinterpret_cast<float2 *>(lb + l_prep + l_ws);
      span_gather_kernel<<<static_cast<unsigned>(nb), kSpanBlock, 0, sl>>>(rp, q, dobj, dmat, dhit, n, drules + h,
                                                                           boff + static_cast<int64_t>(h) * nb);
      kernels += 1 + (tensor ? launch_umma_sum(g, q, nh, lsig, lb + l_prep, status, sl, nullptr, kSpanWaves, kSpanMinChunk)
                             : launch_direct_sum(g, q, nh, lsig, lb + l_prep, sl));
      // the range FFT into the span's spectrum slot (the lane's signal is then free for its next
      // span) and the Doppler and angle FFTs in place there, no scratch cube
      kernels += launch_fft_range_into(g, ctx->t, lsig, x, sl);
      kernels += launch_fft_planes(g, ctx->t, x, 1, sl);
      if (span_spectra && span_spectra[h])
        cudaMemcpyAsync(span_spectra[h], x, 8 * static_cast<size_t>(g.n_cell), cudaMemcpyDefault, sl);
    } else {
      cudaMemsetAsync(x, 0, 8 * static_cast<size_t>(g.n_cell), s);  // the FFT of zeros
      if (span_spectra && span_spectra[h])
        cudaMemcpyAsync(span_spectra[h], x, 8 * static_cast<size_t>(g.n_cell), cudaMemcpyDefault, s);
    }
  }
  for (int l = 1; l < lanes; ++l) {  // join the lanes before the labels read every spectrum
    cudaEventRecord(lane_done[l], lane_s[l]);
    cudaStreamWaitEvent(s, lane_done[l], 0);
  }
  cudaEventRecord(ev[2], s);
  if (span_labels) {
    const int64_t all = g.n_cell * n_spans;
    power_max_kernel<<<1024, 256, 0, s>>>(spectra, all, pmax);
    int32_t *dlab = nullptr;
    cudaPointerAttributes at;
    const bool dev_out = handled_call([&] { return cudaPointerGetAttributes(&at, span_labels); }) == cudaSuccess &&
                         (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    if (dev_out) dlab = span_labels;
    else dlab = reinterpret_cast<int32_t *>(b + o_lab);
    const float t2 = threshold * threshold;
    span_label_kernel<<<1024, 256, 0, s>>>(spectra, n_spans, g.n_cell, t2, pmax, dlab);
    kernels += 2;
    if (!dev_out)
      cudaMemcpyAsync(span_labels, dlab, 4 * static_cast<size_t>(g.n_cell), cudaMemcpyDeviceToHost, s);
  }
  cudaEventRecord(ev[3], s);
  uint32_t st[2] = {0, 0};  // status bits, route mask
  cudaMemcpyAsync(st, status, 8, cudaMemcpyDeviceToHost, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  const bool launch_ok = launches_ok();
  if (e != cudaSuccess || !launch_ok) return finish(SIM_E_CUDA);
  if (st[0] & (kStatusBadRay | kStatusModelRange)) return finish(SIM_E_INVALID);
  if (st[0]) return finish(SIM_E_DEVICE);
  // stage times as sim_last_stage_ms reports them: prep (with the span sizes), the spans'
  // packing, ray sums and FFTs together (they overlap on the lanes), labels, and the whole
  // call on the device's clock (with the read-back of the span sizes)
  auto el = [&](int a, int c) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[static_cast<size_t>(a)], ev[static_cast<size_t>(c)]);
    return ms;
  };
  float ms[7] = {0, el(0, 1), el(1, 2), 0, 0, el(2, 3), el(0, 3)};
  record_stage_ms(ctx, ms, kernels, st[1]);
  return finish(SIM_OK);
}
