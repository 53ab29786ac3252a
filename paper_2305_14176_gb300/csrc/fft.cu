// K_c: windowed range, Doppler and angle FFTs (arXiv 2305.14176, Sec. II-A, Eq. 4).
//
// Eq. 4 names a 2-D DFT over fast time and chirps and leaves windowing and zero
// padding out; here the periodic Hann (or the configured window) is applied on load,
// and a third DFT runs along the virtual channels, zero padded from N_v to N_a.
// Forward, unnormalised, natural bin order.
//
// Each pass stages a tile of lines in shared memory (window fused into the load, in
// bit-reversed order), runs an in-place radix-2 decimation-in-time FFT on all lines of
// the tile, and writes the tile back.  Tiles are chosen so global accesses are
// contiguous runs: whole rows for the range pass, 16-column strips for Doppler and
// 32-column strips of the (m, n) plane for angle.  Twiddles e^{-2 pi i j/N} come from an
// FP64 host table rounded to FP32.
#include "internal.h"

namespace rs {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int bitrev(int t, int log2n) {
  return static_cast<int>(__brev(static_cast<unsigned>(t)) >> (32 - log2n));
}

// In-place radix-2 DIT butterflies over `lines` sequences of length N held at
// x[pt * ps + line * ls], already in bit-reversed order.  LINE_FAST decides whether
// consecutive threads walk lines (column tiles) or points (row tiles).
template <bool LINE_FAST>
__device__ void smem_fft(float2 *x, int N, int log2N, int lines, int ps, int ls,
                         const float2 *__restrict__ tw) {
  const int half_n = N >> 1;
  const int nb = half_n * lines;
  for (int s = 1; s <= log2N; ++s) {
    const int half = 1 << (s - 1);
    const int tws = N >> s;
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      int line, bb;
      if (LINE_FAST) { line = b % lines; bb = b / lines; }
      else { line = b / half_n; bb = b - line * half_n; }
      const int j = bb & (half - 1);
      const int i0 = ((bb >> (s - 1)) << s) + j;
      const int i1 = i0 + half;
      const float2 w = tw[j * tws];
      float2 *p0 = x + i0 * ps + line * ls;
      float2 *p1 = x + i1 * ps + line * ls;
      const float2 a = *p0;
      const float2 t = cmul(w, *p1);
      *p0 = make_float2(a.x + t.x, a.y + t.y);
      *p1 = make_float2(a.x - t.x, a.y - t.y);
    }
  }
  __syncthreads();
}

// range: lines are rows of N_s contiguous samples
__global__ void __launch_bounds__(256) fft_range_kernel(const float2 *__restrict__ in, float2 *out,
                                                        const float *__restrict__ win,
                                                        const float2 *__restrict__ tw, int N, int log2N,
                                                        int lines_per_cta, int64_t total_lines) {
  extern __shared__ float2 sm[];
  const int64_t line0 = static_cast<int64_t>(blockIdx.x) * lines_per_cta;
  const int lines = static_cast<int>(total_lines - line0 < lines_per_cta ? total_lines - line0 : lines_per_cta);
  const float2 *src = in + line0 * N;
  for (int e = threadIdx.x; e < lines * N; e += blockDim.x) {
    const int l = e >> log2N, t = e & (N - 1);
    const float2 v = src[e];
    const float w = win[t];
    sm[l * N + bitrev(t, log2N)] = make_float2(v.x * w, v.y * w);
  }
  smem_fft<false>(sm, N, log2N, lines, 1, N, tw);
  float2 *dst = out + line0 * N;
  for (int e = threadIdx.x; e < lines * N; e += blockDim.x) dst[e] = sm[e];
}

// Doppler: a strip of TW consecutive samples n of one channel, all N_c chirps (in place)
__global__ void __launch_bounds__(256) fft_doppler_kernel(float2 *data, const float *__restrict__ win,
                                                          const float2 *__restrict__ tw, int Nc, int log2Nc,
                                                          int Ns, int TW) {
  extern __shared__ float2 sm[];
  float2 *base = data + static_cast<int64_t>(blockIdx.y) * Nc * Ns + static_cast<int64_t>(blockIdx.x) * TW;
  for (int e = threadIdx.x; e < Nc * TW; e += blockDim.x) {
    const int m = e / TW, c = e - m * TW;
    const float2 v = base[static_cast<int64_t>(m) * Ns + c];
    const float w = win[m];
    sm[bitrev(m, log2Nc) * TW + c] = make_float2(v.x * w, v.y * w);
  }
  smem_fft<true>(sm, Nc, log2Nc, TW, TW, 1, tw);
  for (int e = threadIdx.x; e < Nc * TW; e += blockDim.x) {
    const int m = e / TW, c = e - m * TW;
    base[static_cast<int64_t>(m) * Ns + c] = sm[e];
  }
}

// angle: a strip of TW consecutive (m, n) positions, channels k < N_v, zero padded to N_a
__global__ void __launch_bounds__(256) fft_angle_kernel(const float2 *__restrict__ in, float2 *__restrict__ out,
                                                        const float *__restrict__ win,
                                                        const float2 *__restrict__ tw, int Nv, int Na,
                                                        int log2Na, int64_t plane, int TW) {
  extern __shared__ float2 sm[];
  const int64_t f0 = static_cast<int64_t>(blockIdx.x) * TW;
  for (int e = threadIdx.x; e < Na * TW; e += blockDim.x) {
    const int k = e / TW, c = e - k * TW;
    float2 v = make_float2(0.f, 0.f);
    if (k < Nv) {
      const float2 x = in[static_cast<int64_t>(k) * plane + f0 + c];
      const float w = win[k];
      v = make_float2(x.x * w, x.y * w);
    }
    sm[bitrev(k, log2Na) * TW + c] = v;
  }
  smem_fft<true>(sm, Na, log2Na, TW, TW, 1, tw);
  for (int e = threadIdx.x; e < Na * TW; e += blockDim.x) {
    const int a = e / TW, c = e - a * TW;
    out[static_cast<int64_t>(a) * plane + f0 + c] = sm[e];
  }
}

bool g_attr_done = false;

}  // namespace

int launch_fft(const Derived &g, const Tables &t, const float2 *sig, float2 *tmp, float2 *spec, cudaStream_t s) {
  Tuning tu{};
  const bool have = tuning_lookup(g, -1, &tu);
  if (!have) tu = Tuning{};
  return launch_fft_with(g, t, sig, tmp, spec, s, tu);
}

int launch_fft_with(const Derived &g, const Tables &t, const float2 *sig, float2 *tmp, float2 *spec,
                    cudaStream_t s, const Tuning &tu) {
  if (!g_attr_done) {
    cudaFuncSetAttribute(fft_range_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(fft_doppler_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(fft_angle_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    g_attr_done = true;
  }
  // range: rows of N_s, about 2048 points per block
  const int64_t rows = static_cast<int64_t>(g.nv) * g.nc;
  int points = tu.fft_range_points > 0 ? tu.fft_range_points : 2048;
  if (points > 4096) points = 4096;
  const int lpc = g.ns >= points ? 1 : points / g.ns;
  const int64_t rb = (rows + lpc - 1) / lpc;
  fft_range_kernel<<<static_cast<unsigned>(rb), 256, sizeof(float2) * lpc * g.ns, s>>>(
      sig, tmp, t.win_r, t.tw_r, g.ns, g.log2_ns, lpc, rows);
  // Doppler: strips of TW samples, N_c * TW * 8 bytes <= 64 KB
  int twd = 8192 / g.nc;
  const int twd_pref = tu.fft_doppler_strip > 0 ? tu.fft_doppler_strip : 16;
  if (twd > twd_pref) twd = twd_pref;
  if (twd > g.ns) twd = g.ns;
  dim3 gd(g.ns / twd, g.nv);
  fft_doppler_kernel<<<gd, 256, sizeof(float2) * g.nc * twd, s>>>(tmp, t.win_d, t.tw_d, g.nc, g.log2_nc, g.ns, twd);
  // angle: strips of TW positions of the (m, n) plane
  const int64_t plane = static_cast<int64_t>(g.nc) * g.ns;
  int twa = 8192 / g.na;
  const int twa_pref = tu.fft_angle_strip > 0 ? tu.fft_angle_strip : 32;
  if (twa > twa_pref) twa = twa_pref;
  const int64_t ab = plane / twa;
  fft_angle_kernel<<<static_cast<unsigned>(ab), 256, sizeof(float2) * g.na * twa, s>>>(
      tmp, spec, t.win_a, t.tw_a, g.nv, g.na, g.log2_na, plane, twa);
  return 3;
}

}  // namespace rs
