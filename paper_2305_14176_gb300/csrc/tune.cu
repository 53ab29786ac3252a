// Autotuner for the launch shapes of the ray sum and the FFTs (see include/radarsim.h).
//
// For one radar shape and ray count, sim_autotune times on the device, with CUDA events:
//   * the tensor-core ray sum at a handful of split-K counts (the wave-filling heuristic,
//     whole numbers of waves, and twice / half the heuristic), on synthetic rays;
//   * the three FFT passes at different tile widths (points per range block, samples per
//     Doppler strip, positions per angle strip), one parameter at a time;
// and keeps the fastest in a table keyed by (N_v, N_c, N_s, N_a, precision, ceil(log2 R)).
// Every later launch of that shape (single scenes, batches, the allocation-free call) reads
// the table, so a scene's decomposition, and with it its bits, stays the same alone and in
// a batch.  The table can be saved to and loaded from a JSON file.
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace rs {
namespace {

using Key = std::tuple<int, int, int, int, int, int>;  // nv, nc, ns, na, precision, bucket

std::mutex g_tmu;
std::map<Key, Tuning> g_table;

int bucket_of(int64_t n) {
  int b = 0;
  while (b < 62 && (int64_t{1} << b) < n) ++b;
  return b;
}

Key key_of(const Derived &g, int64_t n) { return Key(g.nv, g.nc, g.ns, g.na, g.precision, bucket_of(n)); }

__device__ __forceinline__ uint64_t hash64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// synthetic prepared rays: uniformly random phases, unit amplitudes, matching phasor steps
__global__ void synth_rays(RaysPrep p, int64_t n) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  p.carrier[i] = hash64(4 * i);
  p.nu_r[i] = hash64(4 * i + 1) >> 2;
  p.nu_d[i] = hash64(4 * i + 2);
  p.nu_a[i] = hash64(4 * i + 3);
  p.nu_tx[i] = hash64(4 * i + 3) * 4;
  p.amp[i] = 1.0f;
  p.cell[i] = 0;
  p.energy[i] = 0;
  float s, c;
  sincospif(2.0f * static_cast<float>(static_cast<int64_t>(p.nu_d[i] * 32ull)) * 0x1p-64f, &s, &c);
  p.step_d[i] = make_float2(c, s);
  sincospif(2.0f * static_cast<float>(static_cast<int64_t>(p.nu_r[i] * 32ull)) * 0x1p-64f, &s, &c);
  p.step_r[i] = make_float2(c, s);
}

template <typename F>
float time_min(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, F &&f, int reps = 3) {
  f();  // warm-up
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, s);
    f();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  return best;
}

}  // namespace

bool tuning_lookup(const Derived &g, int64_t n, Tuning *t) {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (n < 0) {  // FFT shape only: any entry of the same radar shape
    for (const auto &kv : g_table) {
      const Key &k = kv.first;
      if (std::get<0>(k) == g.nv && std::get<1>(k) == g.nc && std::get<2>(k) == g.ns && std::get<3>(k) == g.na) {
        *t = kv.second;
        return true;
      }
    }
    return false;
  }
  auto it = g_table.find(key_of(g, n));
  if (it == g_table.end()) return false;
  *t = it->second;
  return true;
}

}  // namespace rs

using namespace rs;

extern "C" SIM_API int sim_autotune(sim_ctx *ctx, int64_t n_rays, sim_tuning *out) {
  if (!ctx || n_rays < 1 || n_rays > ctx->g.max_rays) return SIM_E_INVALID;
  launches_begin();
  const Derived &g = ctx->g;
  const bool tensor = g.precision != SIM_PREC_FP32_DIRECT;
  // the table holds separable-model choices; the exact model's tiles are planned on their own
  if (tensor && g.model == SIM_MODEL_EXACT) return SIM_E_INVALID;
  int cand[16];
  const int nc = tensor ? umma_split_candidates(g, n_rays, cand, 16) : 0;
  int max_splits = tensor ? umma_builtin_splits(g, n_rays) : 1;
  for (int i = 0; i < nc; ++i) max_splits = cand[i] > max_splits ? cand[i] : max_splits;
  const size_t un = static_cast<size_t>((n_rays + 31) / 32 * 32);
  const size_t prep_bytes = un * 72;
  const size_t sig_bytes = 8 * static_cast<size_t>(g.n_sig), spec_bytes = 8 * static_cast<size_t>(g.n_cell);
  const size_t ws_bytes = tensor ? static_cast<size_t>(umma_workspace_bytes_splits(g, max_splits)) : 0;
  const size_t total = prep_bytes + 2 * sig_bytes + spec_bytes + ws_bytes + 256 + 1024;
  uint8_t *b = nullptr;
  if (cudaMalloc(&b, total) != cudaSuccess) {
    cudaGetLastError();
    return SIM_E_NOMEM;
  }
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    uint8_t *p = b + off;
    off += (bytes + 255) & ~static_cast<size_t>(255);
    return p;
  };
  RaysPrep rp;
  rp.carrier = reinterpret_cast<uint64_t *>(take(8 * un));
  rp.nu_r = reinterpret_cast<uint64_t *>(take(8 * un));
  rp.nu_d = reinterpret_cast<uint64_t *>(take(8 * un));
  rp.nu_a = reinterpret_cast<uint64_t *>(take(8 * un));
  rp.amp = reinterpret_cast<float *>(take(4 * un));
  rp.cell = reinterpret_cast<int32_t *>(take(4 * un));
  rp.energy = reinterpret_cast<uint64_t *>(take(8 * un));
  rp.step_d = reinterpret_cast<float2 *>(take(8 * un));
  rp.step_r = reinterpret_cast<float2 *>(take(8 * un));
  rp.eps = nullptr;
  rp.nu_tx = reinterpret_cast<uint64_t *>(take(8 * un));
  rp.eps_t = nullptr;
  float2 *sig = reinterpret_cast<float2 *>(take(sig_bytes));
  float2 *tmp = reinterpret_cast<float2 *>(take(sig_bytes));
  float2 *spec = reinterpret_cast<float2 *>(take(spec_bytes));
  uint32_t *status = reinterpret_cast<uint32_t *>(take(256));
  void *ws = take(ws_bytes > 0 ? ws_bytes : 1);
  synth_rays<<<static_cast<unsigned>((n_rays + 255) / 256), 256, 0, s>>>(rp, n_rays);
  cudaMemsetAsync(status, 0, 4, s);

  Tuning best{};
  float best_sum = 0.f;
  if (tensor) {
    // the built-in plan first (splits = 0 keeps it): a forced count must beat it
    best_sum = time_min(s, e0, e1, [&] { launch_umma_sum_splits(g, rp, n_rays, sig, ws, status, s, 0); });
    for (int i = 0; i < nc; ++i) {
      const int sp = cand[i];
      const float ms = time_min(s, e0, e1, [&] { launch_umma_sum_splits(g, rp, n_rays, sig, ws, status, s, sp); });
      if (ms < best_sum) {
        best_sum = ms;
        best.splits = sp;
      }
    }
  }
  // FFT tiles, one parameter at a time from the built-in choice
  Tuning fcur{};
  auto fft_ms = [&](const Tuning &t) {
    return time_min(s, e0, e1, [&] { launch_fft_with(g, ctx->t, sig, tmp, spec, s, t); });
  };
  float best_fft = fft_ms(fcur);
  for (int pts : {1024, 4096}) {
    Tuning t = fcur;
    t.fft_range_points = pts;
    const float ms = fft_ms(t);
    if (ms < best_fft) { best_fft = ms; fcur = t; }
  }
  for (int tw : {4, 8, 32}) {
    Tuning t = fcur;
    t.fft_doppler_strip = tw;
    const float ms = fft_ms(t);
    if (ms < best_fft) { best_fft = ms; fcur = t; }
  }
  for (int tw : {8, 16}) {
    Tuning t = fcur;
    t.fft_angle_strip = tw;
    const float ms = fft_ms(t);
    if (ms < best_fft) { best_fft = ms; fcur = t; }
  }
  best.fft_range_points = fcur.fft_range_points;
  best.fft_doppler_strip = fcur.fft_doppler_strip;
  best.fft_angle_strip = fcur.fft_angle_strip;

  const cudaError_t err = cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  cudaFree(b);
  if (err != cudaSuccess || !launches_ok()) return SIM_E_CUDA;
  {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_table[key_of(g, n_rays)] = best;
  }
  if (out) {
    out->splits = best.splits;
    out->fft_range_points = best.fft_range_points;
    out->fft_doppler_strip = best.fft_doppler_strip;
    out->fft_angle_strip = best.fft_angle_strip;
    out->ray_sum_ms = best_sum;
    out->fft_ms = best_fft;
  }
  return SIM_OK;
}

extern "C" SIM_API int sim_tuning_save(const char *path) {
  if (!path) return SIM_E_INVALID;
  FILE *f = fopen(path, "w");
  if (!f) return SIM_E_INVALID;
  std::lock_guard<std::mutex> lk(g_tmu);
  fprintf(f, "[\n");
  size_t i = 0;
  for (const auto &kv : g_table) {
    const Key &k = kv.first;
    const Tuning &t = kv.second;
    fprintf(f,
            "  {\"n_virtual\": %d, \"n_chirps\": %d, \"n_samples\": %d, \"n_angle\": %d, \"precision\": %d, "
            "\"ray_bucket\": %d, \"splits\": %d, \"fft_range_points\": %d, \"fft_doppler_strip\": %d, "
            "\"fft_angle_strip\": %d}%s\n",
            std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k), t.splits,
            t.fft_range_points, t.fft_doppler_strip, t.fft_angle_strip, ++i < g_table.size() ? "," : "");
  }
  fprintf(f, "]\n");
  fclose(f);
  return SIM_OK;
}

extern "C" SIM_API int sim_tuning_load(const char *path) {
  if (!path) return SIM_E_INVALID;
  FILE *f = fopen(path, "r");
  if (!f) return SIM_E_INVALID;
  char line[1024];
  int loaded = 0;
  std::lock_guard<std::mutex> lk(g_tmu);
  while (fgets(line, sizeof(line), f)) {
    int nv, nc, ns, na, prec, bucket, sp, rp, dp, ap;
    if (sscanf(line,
               " {\"n_virtual\": %d, \"n_chirps\": %d, \"n_samples\": %d, \"n_angle\": %d, \"precision\": %d, "
               "\"ray_bucket\": %d, \"splits\": %d, \"fft_range_points\": %d, \"fft_doppler_strip\": %d, "
               "\"fft_angle_strip\": %d}",
               &nv, &nc, &ns, &na, &prec, &bucket, &sp, &rp, &dp, &ap) == 10) {
      if (sp < 0 || rp < 0 || dp < 0 || ap < 0 || sp > 65535 || rp > 4096 || dp > 4096 || ap > 4096) continue;
      // FFT tile widths are powers of two (0 = built-in choice)
      auto p2 = [](int x) { return x == 0 || (x & (x - 1)) == 0; };
      if (!p2(rp) || !p2(dp) || !p2(ap)) continue;
      g_table[Key(nv, nc, ns, na, prec, bucket)] = Tuning{sp, rp, dp, ap};
      ++loaded;
    }
  }
  fclose(f);
  return loaded >= 0 ? SIM_OK : SIM_E_INVALID;
}

extern "C" SIM_API int sim_tuning_clear(void) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_table.clear();
  return SIM_OK;
}

extern "C" SIM_API int sim_tuning_count(void) {
  std::lock_guard<std::mutex> lk(g_tmu);
  return static_cast<int>(g_table.size());
}
