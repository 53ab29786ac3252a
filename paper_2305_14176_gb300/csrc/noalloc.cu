// sim_raysum_noalloc: the beat-signal ray sum for callers that cannot allocate device
// memory (see include/radarsim.h).
//
// Everything the call needs beyond the caller's inputs and output lives in one static
// device array of kScratchBytes, which the CUDA runtime reserves on every device that
// loads this library and keeps until the process exits.  Host code never passes the
// array's name to a kernel: the name is only a host-side stand-in for the symbol, so the
// device address is looked up once per device with cudaGetSymbolAddress and cached.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kScratchBytes = size_t{128} << 20;  // 128 MiB
constexpr int64_t kMaxRays = int64_t{1} << 18;       // 262,144 rays per call
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

size_t round256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// device address of the scratch array on the current device (first call: set-up)
int scratch_on_current_device(uint8_t **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SIM_E_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SIM_E_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<uint8_t *>(g_scratch_ptr[dev]);
  return SIM_OK;
}

// device (or managed) memory that the current device's kernels can address: memory of another
// GPU is refused, since without peer access a kernel here would fault on it
bool on_device(const void *p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" SIM_API int sim_raysum_noalloc(const sim_radar_params *params, const sim_rays *rays, void *signal_c64,
                                          void *stream) {
  using namespace rs;
  // an error left by an unrelated earlier call must not be reported as this call's
  cudaGetLastError();
  launches_begin();
  Derived g;
  int rc = derive_radar(params, &g);
  if (rc != SIM_OK) return rc;
  if (!rays || !signal_c64) return SIM_E_INVALID;
  const int64_t n = rays->n;
  if (n < 0 || n > kMaxRays || n > g.max_rays) return SIM_E_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SIM_E_CUDA;
  if (n > 0) {
    const void *arr[6] = {rays->range_rt_m, rays->amplitude, rays->radial_velocity_mps, rays->azimuth_rad,
                          rays->elevation_rad, rays->phase0_rad};
    for (const void *a : arr)
      if (!a || !on_device(a, dev)) return SIM_E_INVALID;
  }
  if (!on_device(signal_c64, dev)) return SIM_E_INVALID;
  uint8_t *scr = nullptr;
  rc = scratch_on_current_device(&scr);
  if (rc != SIM_OK) return rc;

  // carve the scratch: per-ray prep arrays (padded to whole 32-ray stages), status, workspace
  const size_t up = static_cast<size_t>((n + 31) / 32 * 32);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += round256(bytes > 0 ? bytes : 1);
    return scr + o;
  };
  RaysPrep rp;
  rp.carrier = reinterpret_cast<uint64_t *>(take(8 * up));
  rp.nu_r = reinterpret_cast<uint64_t *>(take(8 * up));
  rp.nu_d = reinterpret_cast<uint64_t *>(take(8 * up));
  rp.nu_a = reinterpret_cast<uint64_t *>(take(8 * up));
  rp.amp = reinterpret_cast<float *>(take(4 * up));
  rp.cell = reinterpret_cast<int32_t *>(take(4 * up));
  rp.energy = reinterpret_cast<uint64_t *>(take(8 * up));
  rp.step_d = reinterpret_cast<float2 *>(take(8 * up));
  rp.step_r = reinterpret_cast<float2 *>(take(8 * up));
  rp.eps = g.model == SIM_MODEL_EXACT ? reinterpret_cast<uint64_t *>(take(8 * up)) : nullptr;
  rp.nu_tx = reinterpret_cast<uint64_t *>(take(8 * up));
  rp.eps_t = g.model == SIM_MODEL_EXACT ? reinterpret_cast<uint64_t *>(take(8 * up)) : nullptr;
  uint32_t *status = reinterpret_cast<uint32_t *>(take(256));
  uint8_t *ws = scr + off;
  const int64_t ws_bytes = static_cast<int64_t>(kScratchBytes) - static_cast<int64_t>(off);
  // the tensor-core path needs room for at least one FP32 partial of the whole cube
  const int64_t one_split = 256 + 8 * g.n_sig;
  if (g.precision != SIM_PREC_FP32_DIRECT && one_split > ws_bytes) return SIM_E_INVALID;
  if (g.model == SIM_MODEL_EXACT && g.precision != SIM_PREC_FP32_DIRECT) {
    // the per-chirp exact form used here has no TDM slot term, and its split partials (one
    // FP32 cube each) must fit the scratch left after the per-ray data
    if (g.tslot != 0.0 || exact_workspace_bytes(g, n) > ws_bytes) return SIM_E_INVALID;
  }

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float2 *sig = static_cast<float2 *>(signal_c64);
  cudaMemsetAsync(status, 0, 4, s);  // the array keeps the previous call's contents
  RaysIn in{rays->range_rt_m, rays->amplitude, rays->radial_velocity_mps, rays->azimuth_rad,
            rays->elevation_rad, rays->phase0_rad, nullptr};
  launch_prep(g, in, n, rp, status, s);
  if (g.precision == SIM_PREC_FP32_DIRECT) {
    launch_direct_sum(g, rp, n, sig, direct_workspace_bytes(g, n) <= ws_bytes ? ws : nullptr, s);
  } else if (launch_umma_sum_in(g, rp, n, sig, ws, ws_bytes, status, s) < 0) {
    return SIM_E_INVALID;  // one split of this cube does not fit the scratch array, or the exact
                           // model with TDM slots (no per-chirp form) was asked for
  }
  uint32_t st = 0;
  cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return SIM_E_CUDA;
  if (!launches_ok()) return SIM_E_CUDA;
  if (st & kStatusBadRay) return SIM_E_INVALID;
  return st ? SIM_E_DEVICE : SIM_OK;
}
