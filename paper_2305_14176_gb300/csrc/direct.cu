// K_b0: the plain direct ray sum (arXiv 2305.14176, Sec. II-A, Eq. 2).
//
//   s[k][m][n] = sum_i a_i exp(2 pi j (carrier_i + k nu_a,i + m nu_d,i + n nu_r,i))
//
// A thread owns the samples n = t + j T of a row (T threads, j < NPT).  For each ray it takes
// one FP32 sine and cosine of the exact Q0.64 phase of its first sample (only the top 23 bits
// become an FP32 angle in [-pi, pi), so the hardware sin/cos sees a small argument) and steps
// to the others by complex multiplication with e^{2 pi j T nu_r}: one sin/cos per NPT
// contributions, the rest on the FMA pipe.
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

// e^{2 pi j q 2^-64} for a Q0.64 phase q, from the signed cycle count in FP32 (relative
// precision 2^-24 of a value in [-1/2, 1/2)), for the phasor steps of the recurrence below
__device__ __forceinline__ float2 phasor_of(uint64_t q) {
  const float f = static_cast<float>(static_cast<int64_t>(q)) * 0x1p-64f;
  float sn, cs;
  sincospif(2.0f * f, &sn, &cs);
  return make_float2(cs, sn);
}

// Two FP32 lanes in one 64-bit register: element-wise f32x2 arithmetic, one instruction for a
// pair of rays
using f2 = unsigned long long;
__device__ __forceinline__ f2 pack2(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float sum_lanes(f2 x) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
  return a + b;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// A staged chunk of rays: per ray its phase words (base of the row, per-sample step), its
// amplitude and the T-sample step phasor e^{2 pi j T step} = (w_r, w_i), kept with -w_i.
// An odd chunk is padded with one silent ray so rays go in pairs.
struct Staged {
  ulonglong2 ph[kChunk];
  __align__(16) float amp[kChunk];
  __align__(16) float wr[kChunk];
  __align__(16) float wi[kChunk];
  __align__(16) float nwi[kChunk];
};

__device__ __forceinline__ void stage_ray(Staged &st, int i, uint64_t base, uint64_t step, float amp, uint64_t T) {
  st.ph[i] = make_ulonglong2(base, step);
  st.amp[i] = amp;
  const float2 w = phasor_of(T * step);
  st.wr[i] = w.x;
  st.wi[i] = w.y;
  st.nwi[i] = -w.y;
}

__device__ __forceinline__ void stage_pad(Staged &st, int cnt) {
  if (cnt & 1) {
    st.ph[cnt] = make_ulonglong2(0, 0);
    st.amp[cnt] = 0.f;
    st.wr[cnt] = 1.f;
    st.wi[cnt] = 0.f;
    st.nwi[cnt] = 0.f;
  }
}

// Add one staged chunk to the thread's samples n = t + j T (j < NPT), two rays at a time in
// the lanes of f32x2 registers.  The first sample of each ray takes one sine and cosine of its
// exact Q0.64 phase; the next NPT - 1 follow by complex multiplication with its step phasor
// (FP32 error growing by about one rounding per step).  The two lanes are added at the end.
template <int NPT>
__device__ __forceinline__ void sum_chunk(const Staged &st, int cnt, int t, float (&re)[NPT], float (&im)[NPT]) {
  f2 accr[NPT], acci[NPT];
#pragma unroll
  for (int j = 0; j < NPT; ++j) { accr[j] = 0ull; acci[j] = 0ull; }
  const uint64_t tt = static_cast<uint64_t>(t);
#pragma unroll 2
  for (int i = 0; i < cnt; i += 2) {
    const ulonglong2 q0 = st.ph[i], q1 = st.ph[i + 1];
    float s0, c0, s1, c1;
    __sincosf(q64_to_rad(q0.x + tt * q0.y), &s0, &c0);
    __sincosf(q64_to_rad(q1.x + tt * q1.y), &s1, &c1);
    const f2 a = *reinterpret_cast<const f2 *>(st.amp + i);
    f2 zr = mul2(a, pack2(c0, c1)), zi = mul2(a, pack2(s0, s1));
    accr[0] = add2(accr[0], zr);
    acci[0] = add2(acci[0], zi);
    if constexpr (NPT > 1) {
      const f2 wr = *reinterpret_cast<const f2 *>(st.wr + i);
      const f2 wi = *reinterpret_cast<const f2 *>(st.wi + i);
      const f2 nwi = *reinterpret_cast<const f2 *>(st.nwi + i);
#pragma unroll
      for (int j = 1; j < NPT; ++j) {
        const f2 nr = fma2(zi, nwi, mul2(zr, wr));  // zr w_r - zi w_i
        const f2 ni = fma2(zr, wi, mul2(zi, wr));   // zi w_r + zr w_i
        zr = nr;
        zi = ni;
        accr[j] = add2(accr[j], zr);
        acci[j] = add2(acci[j], zi);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    re[j] += sum_lanes(accr[j]);
    im[j] += sum_lanes(acci[j]);
  }
}

// One block per ((k, m) row, ray part): thread t owns samples n = t + j * T (j < NPT) and sums
// the rays of part blockIdx.y, [ray_lo + y part_len, ...) below ray_hi; part 0 writes sig,
// part y > 0 writes parts[(y - 1) n_sig + ...] (added in order afterwards).
template <int NPT>
__global__ void __launch_bounds__(128) direct_sum_kernel(RaysPrep p, int64_t n_rays, int64_t part_len, int nc,
                                                         int ns, int nrx, float2 *__restrict__ sig,
                                                         float2 *__restrict__ parts, int64_t n_sig) {
  __shared__ Staged st;
  const int row = blockIdx.x;
  const uint64_t k = static_cast<uint64_t>(row / nc);
  const uint64_t m = static_cast<uint64_t>(row % nc);
  const uint64_t tx = k / static_cast<uint64_t>(nrx), rx = k - tx * static_cast<uint64_t>(nrx);
  const int t = threadIdx.x;
  const uint64_t T = blockDim.x;
  float tot_re[NPT], tot_im[NPT];
#pragma unroll
  for (int j = 0; j < NPT; ++j) { tot_re[j] = 0.f; tot_im[j] = 0.f; }

  const int64_t lo = static_cast<int64_t>(blockIdx.y) * part_len;
  const int64_t hi = lo + part_len < n_rays ? lo + part_len : n_rays;
  for (int64_t c0 = lo; c0 < hi; c0 += kChunk) {
    const int cnt = static_cast<int>(hi - c0 < kChunk ? hi - c0 : kChunk);
    __syncthreads();
    for (int i = t; i < cnt; i += blockDim.x) {
      const int64_t r = c0 + i;
      // exact Eq. 2 adds n (m eps + tx eps_t): on row (tx, m) the per-sample increment grows by that
      const uint64_t nur = p.eps ? p.nu_r[r] + m * p.eps[r] + tx * p.eps_t[r] : p.nu_r[r];
      // channel k = tx N_rx + rx: phase tx nu_tx + rx nu_a (= k nu_a without TDM slots)
      stage_ray(st, i, p.carrier[r] + tx * p.nu_tx[r] + rx * p.nu_a[r] + m * p.nu_d[r], nur, p.amp[r], T);
    }
    if (t == 0) stage_pad(st, cnt);
    __syncthreads();
    // per-chunk partial sums, then added to the totals (two-level summation)
    float re[NPT], im[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) { re[j] = 0.f; im[j] = 0.f; }
    sum_chunk<NPT>(st, cnt, t, re, im);
#pragma unroll
    for (int j = 0; j < NPT; ++j) { tot_re[j] += re[j]; tot_im[j] += im[j]; }
  }
  float2 *o = (blockIdx.y == 0 ? sig : parts + (static_cast<int64_t>(blockIdx.y) - 1) * n_sig) +
              static_cast<int64_t>(row) * ns;
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int n = t + j * blockDim.x;
    if (n < ns) o[n] = make_float2(tot_re[j], tot_im[j]);
  }
}

// gate (may be null) holding a term count: a tensor-core expansion computed the chunk instead
__device__ __forceinline__ bool gated_off(const uint32_t *gate) {
  if (!gate) return false;
  return expansion_terms(*gate);
}

// sig += parts[0] + parts[1] + ... in part order
__global__ void add_parts_kernel(float2 *__restrict__ sig, const float2 *__restrict__ parts, int extra,
                                 int64_t n_sig, const uint32_t *gate) {
  if (gated_off(gate)) return;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_sig;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float2 v = sig[i];
    for (int q = 0; q < extra; ++q) {
      const float2 w = parts[q * n_sig + i];
      v = make_float2(v.x + w.x, v.y + w.y);
    }
    sig[i] = v;
  }
}

// The same sum with phase words per (ray, chirp, transmitter) and (ray, chirp, receiver):
// row (k = tx N_rx + rx, m) takes base = wt.x + wr.x and step = wt.y + wr.y, wt =
// w_tx[(m N_tx + tx) stride + i], wr = w_rx[(m N_rx + rx) stride + i] (Q0.32, wrap-exact
// sums, staged as the upper halves of Q0.64 phases).  With `accumulate` the row is added to what sig holds (rays in several chunks).  Ray
// part blockIdx.y > 0 (rays [y part_len, ...)) writes its row to parts[(y - 1) n_sig + ...]
// instead, added in order afterwards.
template <int NPT>
__global__ void __launch_bounds__(128) pair_sum_kernel(const uint2 *__restrict__ w_tx,
                                                       const uint2 *__restrict__ w_rx,
                                                       const float *__restrict__ amp, int64_t n_rays, int64_t stride,
                                                       int64_t part_len, int nc, int ns, int ntx, int nrx,
                                                       int accumulate, float2 *__restrict__ sig,
                                                       float2 *__restrict__ parts, int64_t n_sig,
                                                       const uint32_t *gate) {
  if (gated_off(gate)) return;  // the tensor-core expansion owns this chunk
  __shared__ Staged st;
  const int row = blockIdx.x;
  const int k = row / nc, m = row % nc;
  const int tx = k / nrx, rx = k - tx * nrx;
  const uint2 *wt = w_tx + (static_cast<int64_t>(m) * ntx + tx) * stride;
  const uint2 *wr = w_rx + (static_cast<int64_t>(m) * nrx + rx) * stride;
  const int t = threadIdx.x;
  const uint64_t T = blockDim.x;
  float tot_re[NPT], tot_im[NPT];
#pragma unroll
  for (int j = 0; j < NPT; ++j) { tot_re[j] = 0.f; tot_im[j] = 0.f; }
  const int64_t lo = static_cast<int64_t>(blockIdx.y) * part_len;
  const int64_t hi = lo + part_len < n_rays ? lo + part_len : n_rays;
  for (int64_t c0 = lo; c0 < hi; c0 += kChunk) {
    const int cnt = static_cast<int>(hi - c0 < kChunk ? hi - c0 : kChunk);
    __syncthreads();
    for (int i = t; i < cnt; i += blockDim.x) {
      const uint2 a = wt[c0 + i], b = wr[c0 + i];
      stage_ray(st, i, static_cast<uint64_t>(a.x + b.x) << 32, static_cast<uint64_t>(a.y + b.y) << 32, amp[c0 + i], T);
    }
    if (t == 0) stage_pad(st, cnt);
    __syncthreads();
    float re[NPT], im[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) { re[j] = 0.f; im[j] = 0.f; }
    sum_chunk<NPT>(st, cnt, t, re, im);
#pragma unroll
    for (int j = 0; j < NPT; ++j) { tot_re[j] += re[j]; tot_im[j] += im[j]; }
  }
  const bool to_sig = blockIdx.y == 0;
  float2 *o = (to_sig ? sig : parts + (static_cast<int64_t>(blockIdx.y) - 1) * n_sig) + static_cast<int64_t>(row) * ns;
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int n = t + j * blockDim.x;
    if (n < ns) {
      if (accumulate && to_sig) {
        const float2 v = o[n];
        o[n] = make_float2(v.x + tot_re[j], v.y + tot_im[j]);
      } else {
        o[n] = make_float2(tot_re[j], tot_im[j]);
      }
    }
  }
}

// Threads per row, N_s a power of two in 16 .. 4096 (samples per thread 1, 2, .., 32).
// Separable sum: one warp with up to 32 samples each, N_s > 1024 taking N_s / 32 threads (the
// per-ray start of a phasor chain, one sin/cos and a 64-bit phase product, is shared by more
// samples: 80.5 -> 76.1 ms per automotive frame against two warps).  Snapshot sum: two warps,
// whose staging (two phase words and a sin/cos per ray) needs the wider block (one warp:
// 76.9 -> 78.9 ms).
int row_threads(int ns) { return ns <= 32 ? ns : (ns / 32 > 32 ? ns / 32 : 32); }
int pair_row_threads(int ns) { return ns <= 64 ? ns : (ns / 32 > 64 ? ns / 32 : 64); }

}  // namespace

// Ray parts of the separable direct sum: one block per (row, part), so a frame whose rows are
// too few for the resident blocks (3072 automotive rows at 16 blocks per SM: 1.26 waves) fills
// the SMs; the smallest part count giving at least three waves, at most 4, at least 512 rays
// per part.  The part signals are added in fixed order afterwards.
namespace {
template <int NPT>
int resident_blocks(int threads) {
  static const int per_sm = [threads] {
    int r = 0;
    return handled_call([&] {
             return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, direct_sum_kernel<NPT>, threads, 0);
           }) == cudaSuccess && r > 0
               ? r
               : 1;
  }();
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
  return per_sm * sms;
}

int resident_for(const Derived &g) {
  const int threads = row_threads(g.ns);
  switch (g.ns / threads) {
    case 1: return resident_blocks<1>(threads);
    case 2: return resident_blocks<2>(threads);
    case 4: return resident_blocks<4>(threads);
    case 8: return resident_blocks<8>(threads);
    case 16: return resident_blocks<16>(threads);
    default: return resident_blocks<32>(threads);
  }
}
}  // namespace

int direct_parts(const Derived &g, int64_t n) {
  const int64_t rows = static_cast<int64_t>(g.nv) * g.nc;
  const int64_t resident = resident_for(g);
  int parts = 1;
  while (parts < 4 && rows * parts < 3 * resident && n / (parts + 1) >= 512) ++parts;
  return parts;
}

int64_t direct_workspace_bytes(const Derived &g, int64_t n) {
  return static_cast<int64_t>(direct_parts(g, n) - 1) * 8 * g.n_sig;
}

int launch_direct_sum(const Derived &g, RaysPrep p, int64_t n, float2 *sig, void *workspace, cudaStream_t s) {
  const int rows = g.nv * g.nc;
  const int threads = row_threads(g.ns);
  const int P = workspace ? direct_parts(g, n) : 1;
  int64_t part_len = (n + P - 1) / P;
  part_len = (part_len + 1) / 2 * 2;  // whole ray pairs per part
  if (part_len < 2) part_len = 2;
  float2 *parts = static_cast<float2 *>(workspace);
  const dim3 grid(static_cast<unsigned>(rows), static_cast<unsigned>(P));
#define RS_DIRECT(N) \
  direct_sum_kernel<N><<<grid, threads, 0, s>>>(p, n, part_len, g.nc, g.ns, g.nrx, sig, parts, g.n_sig)
  switch (g.ns / threads) {
    case 1: RS_DIRECT(1); break;
    case 2: RS_DIRECT(2); break;
    case 4: RS_DIRECT(4); break;
    case 8: RS_DIRECT(8); break;
    case 16: RS_DIRECT(16); break;
    case 32: RS_DIRECT(32); break;
    default: return 0;
  }
#undef RS_DIRECT
  if (P > 1) {
    add_parts_kernel<<<4 * 152, 256, 0, s>>>(sig, parts, P - 1, g.n_sig, nullptr);
    return 2;
  }
  return 1;
}

int pair_parts(const Derived &g, int64_t n) {
  const int64_t rows = static_cast<int64_t>(g.nv) * g.nc;
  const int threads = pair_row_threads(g.ns);
  int per_sm = 0;
  handled_call([&] {
    switch (g.ns / threads) {  // resident blocks of the instance this shape launches
      case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_sum_kernel<1>, threads, 0);
      case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_sum_kernel<2>, threads, 0);
      case 4: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_sum_kernel<4>, threads, 0);
      case 8: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_sum_kernel<8>, threads, 0);
      case 16: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_sum_kernel<16>, threads, 0);
      default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_sum_kernel<32>, threads, 0);
    }
  });
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
  const int64_t resident = static_cast<int64_t>(per_sm > 0 ? per_sm : 1) * sms;
  int parts = 1;
  while (parts < 4 && rows * parts < 3 * resident && n / (parts + 1) >= 512) ++parts;
  return parts;
}

int64_t pair_workspace_bytes(const Derived &g, int64_t n) {
  return static_cast<int64_t>(pair_parts(g, n) - 1) * 8 * g.n_sig;
}

int launch_pair_sum(const Derived &g, const uint2 *w_tx, const uint2 *w_rx, const float *amp, int64_t n,
                    int64_t stride, bool accumulate, float2 *sig, void *workspace, const uint32_t *gate,
                    cudaStream_t s) {
  const int rows = g.nv * g.nc;
  const int threads = pair_row_threads(g.ns);
  const int acc = accumulate ? 1 : 0;
  const int P = workspace ? pair_parts(g, n) : 1;
  int64_t part_len = (n + P - 1) / P;
  part_len = (part_len + 1) / 2 * 2;
  if (part_len < 2) part_len = 2;
  float2 *parts = static_cast<float2 *>(workspace);
  const dim3 grid(static_cast<unsigned>(rows), static_cast<unsigned>(P));
#define RS_PAIR(N)                                                                                                 \
  pair_sum_kernel<N><<<grid, threads, 0, s>>>(w_tx, w_rx, amp, n, stride, part_len, g.nc, g.ns, g.ntx, g.nrx, acc, \
                                              sig, parts, g.n_sig, gate)
  switch (g.ns / threads) {
    case 1: RS_PAIR(1); break;
    case 2: RS_PAIR(2); break;
    case 4: RS_PAIR(4); break;
    case 8: RS_PAIR(8); break;
    case 16: RS_PAIR(16); break;
    case 32: RS_PAIR(32); break;
    default: return 0;
  }
#undef RS_PAIR
  if (P > 1) {
    add_parts_kernel<<<4 * 152, 256, 0, s>>>(sig, parts, P - 1, g.n_sig, gate);
    return 2;
  }
  return 1;
}

}  // namespace rs
