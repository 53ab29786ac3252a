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
// The per-ray prep runs once; each span reuses it with the amplitudes of the other rays
// zeroed, through the context's ray-sum arithmetic (direct or tensor core).
#include <cuda_runtime.h>

#include <vector>

#include "internal.h"

using namespace rs;

namespace {

struct RuleDev {
  int32_t object_id, material_id, min_hits, max_hits, exclude;
};

__global__ void span_mask_kernel(const float *__restrict__ amp, const int32_t *__restrict__ obj,
                                 const int32_t *__restrict__ mat, const int32_t *__restrict__ hits, int64_t n,
                                 RuleDev r, float *__restrict__ out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  bool in = true;
  if (r.object_id >= 0) in = in && obj && obj[i] == r.object_id;
  if (r.material_id >= 0) in = in && mat && mat[i] == r.material_id;
  if (r.min_hits > 0 || r.max_hits >= 0) {
    const int32_t h = hits ? hits[i] : 1;
    in = in && h >= r.min_hits && (r.max_hits < 0 || h <= r.max_hits);
  }
  if (r.exclude) in = !in;
  out[i] = in ? amp[i] : 0.f;
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

  // device workspace: inputs, meta, prep, masked amplitudes, signal, FFT scratch, spectra
  const size_t un = static_cast<size_t>(n), up = (un + 31) / 32 * 32;
  const bool tensor = g.precision != SIM_PREC_FP32_DIRECT;
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
               o_sr = take(8 * up), o_eps = take(g.model == SIM_MODEL_EXACT ? 8 * up : 0), o_mamp = take(4 * up),
               o_ntx = take(8 * up), o_epst = take(g.model == SIM_MODEL_EXACT ? 8 * up : 0);
  const size_t o_status = take(256), o_max = take(256);
  const size_t o_sig = take(8 * static_cast<size_t>(g.n_sig)), o_tmp = take(8 * static_cast<size_t>(g.n_sig));
  const size_t o_spec = take(8 * static_cast<size_t>(g.n_cell) * static_cast<size_t>(n_spans));
  const size_t o_ws = take(tensor ? static_cast<size_t>(umma_workspace_bytes(g, n)) : 0);
  const size_t o_lab = take(4 * static_cast<size_t>(g.n_cell));
  uint8_t *b = nullptr;
  if (cudaMalloc(&b, off) != cudaSuccess) {
    cudaGetLastError();
    return SIM_E_NOMEM;
  }
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(b);
    return SIM_E_CUDA;
  }
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
  uint32_t *status = reinterpret_cast<uint32_t *>(b + o_status);
  uint32_t *pmax = reinterpret_cast<uint32_t *>(b + o_max);
  cudaMemsetAsync(status, 0, 4, s);
  cudaMemsetAsync(pmax, 0, 4, s);
  RaysIn in{reinterpret_cast<const double *>(b + o_d), reinterpret_cast<const float *>(b + o_a),
            reinterpret_cast<const float *>(b + o_v), reinterpret_cast<const float *>(b + o_az),
            reinterpret_cast<const float *>(b + o_el), reinterpret_cast<const float *>(b + o_p0), dobj};
  RaysPrep rp{reinterpret_cast<uint64_t *>(b + o_car), reinterpret_cast<uint64_t *>(b + o_nur),
              reinterpret_cast<uint64_t *>(b + o_nud), reinterpret_cast<uint64_t *>(b + o_nua),
              reinterpret_cast<float *>(b + o_amp), reinterpret_cast<int32_t *>(b + o_cell),
              reinterpret_cast<uint64_t *>(b + o_en), reinterpret_cast<float2 *>(b + o_sd),
              reinterpret_cast<float2 *>(b + o_sr),
              g.model == SIM_MODEL_EXACT ? reinterpret_cast<uint64_t *>(b + o_eps) : nullptr,
              reinterpret_cast<uint64_t *>(b + o_ntx),
              g.model == SIM_MODEL_EXACT ? reinterpret_cast<uint64_t *>(b + o_epst) : nullptr};
  launch_prep(g, in, n, rp, status, s);
  RaysPrep span = rp;
  span.amp = reinterpret_cast<float *>(b + o_mamp);
  float2 *sig = reinterpret_cast<float2 *>(b + o_sig);
  float2 *spectra = reinterpret_cast<float2 *>(b + o_spec);
  for (int h = 0; h < n_spans; ++h) {
    const sim_span_rule &r = rules[h];
    const RuleDev rd{r.object_id, r.material_id, r.min_hits, r.max_hits, r.exclude};
    if (n > 0)
      span_mask_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(rp.amp, dobj, dmat, dhit, n, rd,
                                                                               span.amp);
    if (tensor) launch_umma_sum(g, span, n, sig, b + o_ws, status, s, nullptr);
    else launch_direct_sum(g, span, n, sig, s);
    float2 *x = spectra + static_cast<int64_t>(h) * g.n_cell;
    launch_fft(g, ctx->t, sig, reinterpret_cast<float2 *>(b + o_tmp), x, s);
    if (span_spectra && span_spectra[h])
      cudaMemcpyAsync(span_spectra[h], x, 8 * static_cast<size_t>(g.n_cell), cudaMemcpyDefault, s);
  }
  if (span_labels) {
    const int64_t all = g.n_cell * n_spans;
    power_max_kernel<<<1024, 256, 0, s>>>(spectra, all, pmax);
    int32_t *dlab = nullptr;
    cudaPointerAttributes at;
    const bool dev_out = cudaPointerGetAttributes(&at, span_labels) == cudaSuccess &&
                         (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (dev_out) dlab = span_labels;
    else dlab = reinterpret_cast<int32_t *>(b + o_lab);
    const float t2 = threshold * threshold;
    span_label_kernel<<<1024, 256, 0, s>>>(spectra, n_spans, g.n_cell, t2, pmax, dlab);
    if (!dev_out)
      cudaMemcpyAsync(span_labels, dlab, 4 * static_cast<size_t>(g.n_cell), cudaMemcpyDeviceToHost, s);
  }
  uint32_t st = 0;
  cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  cudaFree(b);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return SIM_E_CUDA;
  if (st & kStatusBadRay) return SIM_E_INVALID;
  return st ? SIM_E_DEVICE : SIM_OK;
}
