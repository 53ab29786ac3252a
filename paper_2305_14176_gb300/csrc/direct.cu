// K_b0: the plain direct ray sum (arXiv 2305.14176, Sec. II-A, Eq. 2).
//
//   s[k][m][n] = sum_i a_i exp(2 pi j (carrier_i + k nu_a,i + m nu_d,i + n nu_r,i))
//
// One FP32 sine and cosine per ray and output sample.  The phase is accumulated
// exactly in Q0.64 integers (wrap = one cycle) and only its top 23 bits are turned into
// an FP32 angle in [-pi, pi), so the hardware sin/cos sees a small argument.
//
// A block owns one (k, m) row and all N_s samples; rays stream through shared memory
// in chunks, and each chunk is summed into a per-thread partial before it is added
// to the running total (two-level summation keeps FP32 rounding at ~1e-6 of the
// cube norm for 10^6 rays).
#include "internal.h"

namespace rs {
namespace {

constexpr int kChunk = 256;

// Top 23 bits of a Q0.64 phase turned into an angle in [-pi, pi) without an integer-to-float
// conversion: with u' = u + 2^31 (mod 2^32), (u' >> 9) | 0x3F800000 is the float 1 + u'/2^32
// in [1, 2), and (that - 1.5) = u/2^32 - k for the integer k that lands it in [-1/2, 1/2).
__device__ __forceinline__ float q64_to_rad(uint64_t p) {
  const uint32_t u = static_cast<uint32_t>(p >> 32) ^ 0x80000000u;
  const float f = __uint_as_float((u >> 9) | 0x3F800000u);
  return (f - 1.5f) * 6.28318530717958647692f;
}

// Add one staged chunk of rays to the thread's samples n = t + j T (j < NPT): phase words
// (base of the row, per-sample step) and amplitudes in shared memory.
template <int NPT>
__device__ __forceinline__ void sum_chunk(const ulonglong2 *s_ph, const float *s_amp, int cnt, int t, uint64_t T,
                                          float (&re)[NPT], float (&im)[NPT]) {
#pragma unroll 2
  for (int i = 0; i < cnt; ++i) {
    const ulonglong2 q = s_ph[i];
    const float a = s_amp[i];
    uint64_t ph = q.x + static_cast<uint64_t>(t) * q.y;
    const uint64_t step = T * q.y;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      float sn, cs;
      __sincosf(q64_to_rad(ph), &sn, &cs);
      re[j] = fmaf(a, cs, re[j]);
      im[j] = fmaf(a, sn, im[j]);
      ph += step;
    }
  }
}

// One block per (k, m) row: thread t owns samples n = t + j * T (j < NPT).
template <int NPT>
__global__ void __launch_bounds__(128) direct_sum_kernel(RaysPrep p, int64_t n_rays, int nc, int ns,
                                                         int nrx, float2 *__restrict__ sig) {
  __shared__ ulonglong2 s_ph[kChunk];  // (base phase of this row, range step)
  __shared__ float s_amp[kChunk];
  const int row = blockIdx.x;
  const uint64_t k = static_cast<uint64_t>(row / nc);
  const uint64_t m = static_cast<uint64_t>(row % nc);
  const uint64_t tx = k / static_cast<uint64_t>(nrx), rx = k - tx * static_cast<uint64_t>(nrx);
  const int t = threadIdx.x;
  const uint64_t T = blockDim.x;
  float tot_re[NPT], tot_im[NPT];
#pragma unroll
  for (int j = 0; j < NPT; ++j) { tot_re[j] = 0.f; tot_im[j] = 0.f; }

  for (int64_t c0 = 0; c0 < n_rays; c0 += kChunk) {
    const int cnt = static_cast<int>(n_rays - c0 < kChunk ? n_rays - c0 : kChunk);
    __syncthreads();
    for (int i = t; i < cnt; i += blockDim.x) {
      const int64_t r = c0 + i;
      // exact Eq. 2 adds n (m eps + tx eps_t): on row (tx, m) the per-sample increment grows by that
      const uint64_t nur = p.eps ? p.nu_r[r] + m * p.eps[r] + tx * p.eps_t[r] : p.nu_r[r];
      // channel k = tx N_rx + rx: phase tx nu_tx + rx nu_a (= k nu_a without TDM slots)
      s_ph[i] = make_ulonglong2(p.carrier[r] + tx * p.nu_tx[r] + rx * p.nu_a[r] + m * p.nu_d[r], nur);
      s_amp[i] = p.amp[r];
    }
    __syncthreads();
    // per-chunk partial sums, then added to the totals (two-level summation)
    float re[NPT], im[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) { re[j] = 0.f; im[j] = 0.f; }
    sum_chunk<NPT>(s_ph, s_amp, cnt, t, T, re, im);
#pragma unroll
    for (int j = 0; j < NPT; ++j) { tot_re[j] += re[j]; tot_im[j] += im[j]; }
  }
  float2 *o = sig + static_cast<int64_t>(row) * ns;
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int n = t + j * blockDim.x;
    if (n < ns) o[n] = make_float2(tot_re[j], tot_im[j]);
  }
}

// The same sum with phase words per (ray, chirp, transmitter) and (ray, chirp, receiver):
// row (k = tx N_rx + rx, m) takes base = wt.x + wr.x and step = wt.y + wr.y, wt =
// w_tx[(m N_tx + tx) stride + i], wr = w_rx[(m N_rx + rx) stride + i] (Q0.64, wrap-exact
// sums).  With `accumulate` the row is added to what sig holds (rays in several chunks).
template <int NPT>
__global__ void __launch_bounds__(128) pair_sum_kernel(const ulonglong2 *__restrict__ w_tx,
                                                       const ulonglong2 *__restrict__ w_rx,
                                                       const float *__restrict__ amp, int64_t n_rays, int64_t stride,
                                                       int nc, int ns, int ntx, int nrx, int accumulate,
                                                       float2 *__restrict__ sig) {
  __shared__ ulonglong2 s_ph[kChunk];
  __shared__ float s_amp[kChunk];
  const int row = blockIdx.x;
  const int k = row / nc, m = row % nc;
  const int tx = k / nrx, rx = k - tx * nrx;
  const ulonglong2 *wt = w_tx + (static_cast<int64_t>(m) * ntx + tx) * stride;
  const ulonglong2 *wr = w_rx + (static_cast<int64_t>(m) * nrx + rx) * stride;
  const int t = threadIdx.x;
  const uint64_t T = blockDim.x;
  float tot_re[NPT], tot_im[NPT];
#pragma unroll
  for (int j = 0; j < NPT; ++j) { tot_re[j] = 0.f; tot_im[j] = 0.f; }
  for (int64_t c0 = 0; c0 < n_rays; c0 += kChunk) {
    const int cnt = static_cast<int>(n_rays - c0 < kChunk ? n_rays - c0 : kChunk);
    __syncthreads();
    for (int i = t; i < cnt; i += blockDim.x) {
      const ulonglong2 a = wt[c0 + i], b = wr[c0 + i];
      s_ph[i] = make_ulonglong2(a.x + b.x, a.y + b.y);
      s_amp[i] = amp[c0 + i];
    }
    __syncthreads();
    float re[NPT], im[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) { re[j] = 0.f; im[j] = 0.f; }
    sum_chunk<NPT>(s_ph, s_amp, cnt, t, T, re, im);
#pragma unroll
    for (int j = 0; j < NPT; ++j) { tot_re[j] += re[j]; tot_im[j] += im[j]; }
  }
  float2 *o = sig + static_cast<int64_t>(row) * ns;
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int n = t + j * blockDim.x;
    if (n < ns) {
      if (accumulate) {
        const float2 v = o[n];
        o[n] = make_float2(v.x + tot_re[j], v.y + tot_im[j]);
      } else {
        o[n] = make_float2(tot_re[j], tot_im[j]);
      }
    }
  }
}

}  // namespace

int launch_direct_sum(const Derived &g, RaysPrep p, int64_t n, float2 *sig, cudaStream_t s) {
  const int rows = g.nv * g.nc;
  const int threads = g.ns < 128 ? g.ns : 128;
  const int npt = g.ns / threads;  // N_s is a power of two >= 16
  switch (npt) {
    case 1: direct_sum_kernel<1><<<rows, threads, 0, s>>>(p, n, g.nc, g.ns, g.nrx, sig); break;
    case 2: direct_sum_kernel<2><<<rows, threads, 0, s>>>(p, n, g.nc, g.ns, g.nrx, sig); break;
    case 4: direct_sum_kernel<4><<<rows, threads, 0, s>>>(p, n, g.nc, g.ns, g.nrx, sig); break;
    case 8: direct_sum_kernel<8><<<rows, threads, 0, s>>>(p, n, g.nc, g.ns, g.nrx, sig); break;
    case 16: direct_sum_kernel<16><<<rows, threads, 0, s>>>(p, n, g.nc, g.ns, g.nrx, sig); break;
    default: direct_sum_kernel<32><<<rows, threads, 0, s>>>(p, n, g.nc, g.ns, g.nrx, sig); break;
  }
  return 1;
}

int launch_pair_sum(const Derived &g, const ulonglong2 *w_tx, const ulonglong2 *w_rx, const float *amp, int64_t n,
                    int64_t stride, bool accumulate, float2 *sig, cudaStream_t s) {
  const int rows = g.nv * g.nc;
  const int threads = g.ns < 128 ? g.ns : 128;
  const int npt = g.ns / threads;
  const int acc = accumulate ? 1 : 0;
#define RS_PAIR(N) pair_sum_kernel<N><<<rows, threads, 0, s>>>(w_tx, w_rx, amp, n, stride, g.nc, g.ns, g.ntx, g.nrx, acc, sig)
  switch (npt) {
    case 1: RS_PAIR(1); break;
    case 2: RS_PAIR(2); break;
    case 4: RS_PAIR(4); break;
    case 8: RS_PAIR(8); break;
    case 16: RS_PAIR(16); break;
    default: RS_PAIR(32); break;
  }
#undef RS_PAIR
  return 1;
}

}  // namespace rs
