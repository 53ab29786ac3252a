// K_c: windowed range, Doppler and angle FFTs (arXiv 2305.14176, Sec. II-A, Eq. 4).
//
// Eq. 4 names a 2-D DFT over fast time and chirps and leaves windowing and zero
// padding out; here the periodic Hann (or the configured window) is applied on load,
// and a third DFT runs along the virtual channels, zero padded from N_v to N_a.
// Forward, unnormalised, natural bin order.
//
// Each pass stages a tile of lines in shared memory (window fused into the load, in
// bit-reversed order; 16-byte global loads and stores, two complex samples each), runs an
// in-place decimation-in-time FFT on all lines of the tile (radix-4 stages, one radix-2
// stage for an odd log2 N), and writes the tile back.  Tiles are chosen so global accesses are
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

// In-place radix-2 DIT FFT over `lines` sequences of length N held at x[pt * ps + line * ls],
// already in bit-reversed order.  Stages go two at a time as radix-4 (2^2) butterflies: the
// four points (base + t half), t = 0..3, of stages s and s + 1 stay in registers, with the
// radix-2 twiddles of both stages (the same table entries and operations as one stage at a
// time, so the same bits); an odd log2 N starts with one radix-2 stage.  LINE_FAST decides
// whether consecutive threads walk lines (column tiles) or points (row tiles).  PAD (row tiles,
// ps = 1) places point i of a line at i + i / 16: the bit-reversed scatter and the short
// butterfly strides would otherwise put most of a warp's accesses in one shared-memory bank.
template <bool LINE_FAST, bool PAD = false>
__device__ __forceinline__ float2 *pt(float2 *x, int line, int idx, int ps, int ls) {
  return x + line * ls + (PAD ? idx + (idx >> 4) : idx * ps);
}

template <bool LINE_FAST, bool PAD = false>
__device__ void smem_fft(float2 *x, int N, int log2N, int lines, int ps, int ls,
                         const float2 *__restrict__ tw) {
  int s = 1;
  if (log2N & 1) {  // stage 1: pairs (2i, 2i + 1), twiddle tw[0] = 1
    const int nb = (N >> 1) * lines;
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      int line, bb;
      if (LINE_FAST) { line = b % lines; bb = b / lines; }
      else { line = b / (N >> 1); bb = b - line * (N >> 1); }
      float2 *p0 = pt<LINE_FAST, PAD>(x, line, 2 * bb, ps, ls);
      float2 *p1 = pt<LINE_FAST, PAD>(x, line, 2 * bb + 1, ps, ls);
      const float2 a = *p0;
      const float2 t = cmul(tw[0], *p1);
      *p0 = make_float2(a.x + t.x, a.y + t.y);
      *p1 = make_float2(a.x - t.x, a.y - t.y);
    }
    s = 2;
  }
  const int quarter = N >> 2;
  const int ng = quarter * lines;
  for (; s < log2N; s += 2) {
    const int half = 1 << (s - 1);
    const int tws = N >> s, tws1 = N >> (s + 1);
    __syncthreads();
    for (int b = threadIdx.x; b < ng; b += blockDim.x) {
      int line, gq;
      if (LINE_FAST) { line = b % lines; gq = b / lines; }
      else { line = b / quarter; gq = b - line * quarter; }
      const int j = gq & (half - 1);
      const int i0 = ((gq >> (s - 1)) << (s + 1)) + j;
      float2 *p0 = pt<LINE_FAST, PAD>(x, line, i0, ps, ls), *p1 = pt<LINE_FAST, PAD>(x, line, i0 + half, ps, ls);
      float2 *p2 = pt<LINE_FAST, PAD>(x, line, i0 + 2 * half, ps, ls);
      float2 *p3 = pt<LINE_FAST, PAD>(x, line, i0 + 3 * half, ps, ls);
      const float2 w = tw[j * tws];                // stage s, both pairs
      const float2 u = tw[j * tws1];               // stage s + 1, pair (0, 2)
      const float2 v = tw[(j + half) * tws1];      // stage s + 1, pair (1, 3)
      const float2 a0 = *p0, a2 = *p2;
      const float2 t1 = cmul(w, *p1), t3 = cmul(w, *p3);
      const float2 b0 = make_float2(a0.x + t1.x, a0.y + t1.y), b1 = make_float2(a0.x - t1.x, a0.y - t1.y);
      const float2 b2 = make_float2(a2.x + t3.x, a2.y + t3.y), b3 = make_float2(a2.x - t3.x, a2.y - t3.y);
      const float2 t2 = cmul(u, b2), t4 = cmul(v, b3);
      *p0 = make_float2(b0.x + t2.x, b0.y + t2.y);
      *p2 = make_float2(b0.x - t2.x, b0.y - t2.y);
      *p1 = make_float2(b1.x + t4.x, b1.y + t4.y);
      *p3 = make_float2(b1.x - t4.x, b1.y - t4.y);
    }
  }
  __syncthreads();
}

// range: lines are rows of N_s contiguous samples; 16-byte loads and stores (two samples); a
// line takes N + N / 16 points of shared memory (the padded layout of smem_fft)
__host__ __device__ constexpr int range_line_stride(int N) { return N + N / 16; }

__global__ void __launch_bounds__(256) fft_range_kernel(const float2 *__restrict__ in, float2 *out,
                                                        const float *__restrict__ win,
                                                        const float2 *__restrict__ tw, int N, int log2N,
                                                        int lines_per_cta, int64_t total_lines) {
  extern __shared__ float2 sm[];
  const int LS = range_line_stride(N);
  const int64_t line0 = static_cast<int64_t>(blockIdx.x) * lines_per_cta;
  const int lines = static_cast<int>(total_lines - line0 < lines_per_cta ? total_lines - line0 : lines_per_cta);
  const float4 *src = reinterpret_cast<const float4 *>(in + line0 * N);
  for (int e = threadIdx.x; e < lines * N / 2; e += blockDim.x) {
    const int i = 2 * e, l = i >> log2N, t = i & (N - 1);
    const float4 v = src[e];
    const float w0 = win[t], w1 = win[t + 1];
    *pt<false, true>(sm, l, bitrev(t, log2N), 1, LS) = make_float2(v.x * w0, v.y * w0);
    *pt<false, true>(sm, l, bitrev(t + 1, log2N), 1, LS) = make_float2(v.z * w1, v.w * w1);
  }
  smem_fft<false, true>(sm, N, log2N, lines, 1, LS, tw);
  float4 *dst = reinterpret_cast<float4 *>(out + line0 * N);
  for (int e = threadIdx.x; e < lines * N / 2; e += blockDim.x) {
    const int i = 2 * e, l = i >> log2N, t = i & (N - 1);
    const float2 a = *pt<false, true>(sm, l, t, 1, LS), b = *pt<false, true>(sm, l, t + 1, 1, LS);
    dst[e] = make_float4(a.x, a.y, b.x, b.y);
  }
}

// Doppler: a strip of TW (even) consecutive samples n of one channel, all N_c chirps (in place);
// 16-byte accesses cover two neighbouring samples.  Cube blockIdx.z starts at data + z cube.
__global__ void __launch_bounds__(256) fft_doppler_kernel(float2 *data, const float *__restrict__ win,
                                                          const float2 *__restrict__ tw, int Nc, int log2Nc,
                                                          int Ns, int TW, int64_t cube) {
  extern __shared__ float2 sm[];
  float2 *base = data + static_cast<int64_t>(blockIdx.z) * cube + static_cast<int64_t>(blockIdx.y) * Nc * Ns +
                 static_cast<int64_t>(blockIdx.x) * TW;
  for (int e = threadIdx.x; e < Nc * TW / 2; e += blockDim.x) {
    const int i = 2 * e, m = i / TW, c = i - m * TW;
    const float4 v = *reinterpret_cast<const float4 *>(base + static_cast<int64_t>(m) * Ns + c);
    const float w = win[m];
    float2 *d = sm + bitrev(m, log2Nc) * TW + c;
    d[0] = make_float2(v.x * w, v.y * w);
    d[1] = make_float2(v.z * w, v.w * w);
  }
  smem_fft<true>(sm, Nc, log2Nc, TW, TW, 1, tw);
  for (int e = threadIdx.x; e < Nc * TW / 2; e += blockDim.x) {
    const int i = 2 * e, m = i / TW, c = i - m * TW;
    const float2 a = sm[i], b = sm[i + 1];
    *reinterpret_cast<float4 *>(base + static_cast<int64_t>(m) * Ns + c) = make_float4(a.x, a.y, b.x, b.y);
  }
}

// angle: a strip of TW (even) consecutive (m, n) positions, channels k < N_v, zero padded to N_a.
// Cube blockIdx.y reads from in + y cube and writes to out + y cube.  in may equal out: a block
// reads its whole strip into shared memory before it writes any of it, and no other block
// touches the strip's positions.
__global__ void __launch_bounds__(256) fft_angle_kernel(const float2 *in, float2 *out, const float *__restrict__ win,
                                                        const float2 *__restrict__ tw, int Nv, int Na,
                                                        int log2Na, int64_t plane, int TW, int64_t cube) {
  extern __shared__ float2 sm[];
  const int64_t f0 = static_cast<int64_t>(blockIdx.x) * TW;
  in += static_cast<int64_t>(blockIdx.y) * cube;
  out += static_cast<int64_t>(blockIdx.y) * cube;
  for (int e = threadIdx.x; e < Na * TW / 2; e += blockDim.x) {
    const int i = 2 * e, k = i / TW, c = i - k * TW;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < Nv) {
      const float4 x = *reinterpret_cast<const float4 *>(in + static_cast<int64_t>(k) * plane + f0 + c);
      const float w = win[k];
      v = make_float4(x.x * w, x.y * w, x.z * w, x.w * w);
    }
    float2 *d = sm + bitrev(k, log2Na) * TW + c;
    d[0] = make_float2(v.x, v.y);
    d[1] = make_float2(v.z, v.w);
  }
  smem_fft<true>(sm, Na, log2Na, TW, TW, 1, tw);
  for (int e = threadIdx.x; e < Na * TW / 2; e += blockDim.x) {
    const int i = 2 * e, a = i / TW, c = i - a * TW;
    const float2 p = sm[i], q = sm[i + 1];
    *reinterpret_cast<float4 *>(out + static_cast<int64_t>(a) * plane + f0 + c) = make_float4(p.x, p.y, q.x, q.y);
  }
}

// the largest power of two <= x, at least 2
int pow2_floor_min2(int x) {
  int p = 2;
  while (p * 2 <= x) p *= 2;
  return p;
}

}  // namespace

int launch_fft(const Derived &g, const Tables &t, const float2 *sig, float2 *tmp, float2 *spec, cudaStream_t s) {
  Tuning tu{};
  const bool have = tuning_lookup(g, -1, &tu);
  if (!have) tu = Tuning{};
  return launch_fft_with(g, t, sig, tmp, spec, s, tu);
}

namespace {

void fft_attrs() {
  static std::atomic<uint64_t> done{0};
  once_per_device(done, [] {
    note_launch(cudaFuncSetAttribute(fft_range_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    note_launch(cudaFuncSetAttribute(fft_doppler_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    note_launch(cudaFuncSetAttribute(fft_angle_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
  });
}

// range: rows of N_s, about 2048 points per block; sig (N_v N_c rows) into out
void range_pass(const Derived &g, const Tables &t, const float2 *sig, float2 *out, cudaStream_t s, const Tuning &tu) {
  const int64_t rows = static_cast<int64_t>(g.nv) * g.nc;
  int points = tu.fft_range_points > 0 ? tu.fft_range_points : 2048;
  if (points > 4096) points = 4096;
  const int lpc = g.ns >= points ? 1 : points / g.ns;
  const int64_t rb = (rows + lpc - 1) / lpc;
  fft_range_kernel<<<static_cast<unsigned>(rb), 256, sizeof(float2) * lpc * range_line_stride(g.ns), s>>>(
      sig, out, t.win_r, t.tw_r, g.ns, g.log2_ns, lpc, rows);
}

// Doppler in place on `count` cubes of N_v channels starting `cube` elements apart: strips of
// TW samples, N_c * TW * 8 bytes <= 64 KB; TW a power of two >= 2 (the 16-byte accesses cover
// two samples)
void doppler_pass(const Derived &g, const Tables &t, float2 *data, int count, int64_t cube, cudaStream_t s,
                  const Tuning &tu) {
  int twd = 8192 / g.nc;
  const int twd_pref = tu.fft_doppler_strip > 0 ? tu.fft_doppler_strip : 16;
  if (twd > twd_pref) twd = twd_pref;
  if (twd > g.ns) twd = g.ns;
  twd = pow2_floor_min2(twd);
  const dim3 gd(static_cast<unsigned>(g.ns / twd), static_cast<unsigned>(g.nv), static_cast<unsigned>(count));
  fft_doppler_kernel<<<gd, 256, sizeof(float2) * g.nc * twd, s>>>(data, t.win_d, t.tw_d, g.nc, g.log2_nc, g.ns, twd,
                                                                   cube);
}

// angle on `count` cubes: strips of TW positions of the (m, n) plane, in + c cube -> out + c cube
void angle_pass(const Derived &g, const Tables &t, const float2 *in, float2 *out, int count, int64_t cube,
                cudaStream_t s, const Tuning &tu) {
  const int64_t plane = static_cast<int64_t>(g.nc) * g.ns;
  int twa = 8192 / g.na;
  const int twa_pref = tu.fft_angle_strip > 0 ? tu.fft_angle_strip : 32;
  if (twa > twa_pref) twa = twa_pref;
  twa = pow2_floor_min2(twa);
  const dim3 ga(static_cast<unsigned>(plane / twa), static_cast<unsigned>(count));
  fft_angle_kernel<<<ga, 256, sizeof(float2) * g.na * twa, s>>>(in, out, t.win_a, t.tw_a, g.nv, g.na, g.log2_na,
                                                                plane, twa, cube);
}

Tuning fft_tuning(const Derived &g) {
  Tuning tu{};
  if (!tuning_lookup(g, -1, &tu)) tu = Tuning{};
  return tu;
}

}  // namespace

int launch_fft_with(const Derived &g, const Tables &t, const float2 *sig, float2 *tmp, float2 *spec,
                    cudaStream_t s, const Tuning &tu) {
  fft_attrs();
  range_pass(g, t, sig, tmp, s, tu);
  doppler_pass(g, t, tmp, 1, 0, s, tu);
  angle_pass(g, t, tmp, spec, 1, 0, s, tu);
  return 3;
}

int launch_fft_range_into(const Derived &g, const Tables &t, const float2 *sig, float2 *slot, cudaStream_t s) {
  fft_attrs();
  range_pass(g, t, sig, slot, s, fft_tuning(g));
  return 1;
}

int launch_fft_planes(const Derived &g, const Tables &t, float2 *slots, int count, cudaStream_t s) {
  if (count <= 0) return 0;
  fft_attrs();
  const Tuning tu = fft_tuning(g);
  doppler_pass(g, t, slots, count, g.n_cell, s, tu);
  angle_pass(g, t, slots, slots, count, g.n_cell, s, tu);
  return 2;
}

}  // namespace rs
