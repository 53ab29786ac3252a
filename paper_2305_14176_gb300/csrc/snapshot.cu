// Virtual snapshots and antenna displacement (arXiv 2305.14176, Sec. II-D Eq. 6, Sec. II-E Eq. 7).
//
// A ray is traced once, at the first chirp, between one transmitter and one receiver; it keeps
// its hits as (triangle, u, v).  At chirp j each hit sits at (1 - u - v) v1 + u v2 + v v3 of its
// triangle's vertices at that snapshot (Eq. 6), and the path to transmitter t and receiver r is
// the traced length with both antenna legs replaced (Eq. 7) and the stretch between the first
// and the last hit measured again at snapshot j:
//
//   l(j, t, r) = d + [inner(j) - inner(0)] + |p_f(j) - x_t| - |p_f(0) - x_ref,tx|
//                  + |p_l(j) - x_r| - |p_l(0) - x_ref,rx|          = A_t(j) + B_r(j).
//
// Each path enters Eq. 2 with tau = l / c in both the beat and the carrier term, so the sum is
// not separable over chirps and channels: it runs on the direct-sum path (FP32) or, at the
// tensor-core precisions, through the per-tile expansion of umma_taylor.cu with each row's own
// phase words (the direct sum remains that path's fallback, gated on the device).  One thread per
// (ray, chirp) computes A_t and B_r and stores them as phase words (carrier f_c l / c plus the
// start phase, per-sample step B l / (c N_s)); the row (k = t N_rx + r, m) of the sum adds the
// transmitter's and the receiver's word.  The words are formed in Q0.64 and stored rounded to
// Q0.32 (a uint2 per word): a row's phase at sample n is off by at most n 2^-32 cycles from
// the two roundings of its step (7.5e-7 rad at n = 512, 6e-6 at n = 4096, against the carrier
// phase's own FP32 resolution of ~2^-25 cycles), and half the bytes are read and written.  The
// words of all chirps and antennas take N_c (N_tx + N_rx) 8 bytes per ray, so rays go through
// in chunks that keep them within 3 GiB (224,512 rays at the automotive size: 200,000 rays in
// one chunk).  The chunk size was measured (automotive frame, 200,000 rays): FP16 hi + lo 20.43
// ms with 1 GiB chunks, 20.14 with 1.5, 20.12 with 2 and 19.82 with 3 GiB; single pass 10.45,
// 10.25, 10.23 and 10.01 ms.  With 16-byte Q0.64 words the same frame took 25.4 ms at best
// (3 GiB chunks, two of them) and 27.8 ms in one 5.3 GiB chunk: smaller chunks keep the words
// one split of rays carries, which the four column tiles of a row tile all read, closer to the
// L2's size; larger ones pay the per-chunk statistics, term choice and reduction fewer times.
//
// The reference paths need ~48 bits (f_c l / c is ~10^4 cycles, wanted to ~10^-9): the hit
// positions, the legs to the two reference antennas s = |p - x_ref| and the reference phase
// words are carried per chirp as float-float numbers (hi + lo FP32), since this GPU's FP64 rate
// is 1/64 of its FP32 rate; FP64 is used once per call (the vertices, split into float-float
// relative to the reference transmitter) and once per ray (the snapshot-0 terms of Eq. 7).  An
// antenna at x_ref + e differs from the reference leg by |u - e| - |u| = (|e|^2 - 2 u.e) /
// (|u - e| + |u|), u = p - x_ref, a few centimetres for a compact array: that difference is
// taken in FP32, by its series in (|e|^2 - 2 u.e) / |u|^2 where that is small (relative error
// ~2^-22, so ~5 nm for e = 2 cm, 8e-6 rad of carrier phase), and added to the words in Q0.64
// before their rounding.
#include <cuda_runtime.h>

#include <math.h>

#include <vector>

#include "internal.h"

using namespace rs;

namespace {

constexpr double kInv2Pi = 0x1.45f306dc9c883p-3;
constexpr size_t kWordBudget = size_t{3} << 30;

// Float-float numbers x = hi + lo with |lo| <= ulp(hi) / 2, about 48 significant bits
struct ff {
  float hi, lo;
};

struct GeomDev {
  const double *vert;  // [N_c][V][3]
  const float2 *vff;   // [N_c][V][3]: the vertices minus ref_tx as float-float (hi, lo)
  const int32_t *tri;  // [T][3]
  const float4 *tx;    // [n_tx]: (e, |e|^2) with e = x_t - ref_tx
  const float4 *rx;    // [n_rx]: (e, |e|^2) with e = x_r - ref_rx
  double ref_tx[3], ref_rx[3];
  ff t2r[3];           // ref_tx - ref_rx
  const int64_t *off;  // [n + 1]
  const int32_t *htri;
  const float *hu, *hv;
  int64_t n_vert, n_tri, n_hits;
};

struct PhaseConst {
  ff fc;  // f_c / c: carrier cycles per metre of path
  ff sp;  // B / (c N_s): beat cycles per sample per metre of path
  int nc, ntx, nrx;
  int tc, rc;  // the tensor expansion's reference antennas (records below)
};

// x mod 1 as a Q0.64 phase, from the bits of x: x = +-m 2^(e - 1075) with m the 53-bit
// significand, so x 2^64 mod 2^64 = +-m 2^(e - 1011) mod 2^64 (rounded to nearest when the
// shift is to the right; zero, subnormal and non-finite x give 0)
__device__ __forceinline__ uint64_t frac_q64(double x) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
  const int e = static_cast<int>((b >> 52) & 0x7ff);
  if (e == 0 || e == 0x7ff) return 0;
  const uint64_t m = (b & 0xfffffffffffffull) | (uint64_t{1} << 52);
  const int sh = e - 1011;
  uint64_t q = 0;
  if (sh >= 0) {
    if (sh < 64) q = m << sh;
  } else if (sh > -64) {
    q = (m + (uint64_t{1} << (-sh - 1))) >> -sh;
  }
  return (b >> 63) ? uint64_t{0} - q : q;
}

// x to FP64 by its bits (exact); zero, subnormal and non-finite x through the instruction
__device__ __forceinline__ double f64_of(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t e = (u >> 23) & 0xff;
  if (e == 0 || e == 0xff) return static_cast<double>(x);
  return __longlong_as_double(static_cast<long long>((static_cast<uint64_t>(u & 0x80000000u) << 32) |
                                                     (static_cast<uint64_t>(e + 896) << 52) |
                                                     (static_cast<uint64_t>(u & 0x7fffffu) << 29)));
}

// ---- float-float arithmetic.  This GPU's FP64 pipe runs at 1/64 of its FP32 rate, so the
// per-chirp path lengths are carried as unevaluated sums of two floats, using the error-free
// transformations of Knuth (two-sum), Dekker (fast two-sum) and the fma product error.  Every
// operand here is a length of at most ~10^3 m (or one times a cycles-per-metre constant), and
// the sums below err by ~2^-47 of their operands, so a path stays within ~10^-12 m of its FP64
// value.  Products that must be rounded use __fmul_rn, which is never fused into an fma.
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ ff ff_fast(float a, float b) {  // a + b, |a| >= |b| or a = 0
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff_fast(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  const ff s = ff_two_sum(a.hi, b);
  return ff_fast(s.hi, s.lo + a.lo);
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, {-b.hi, -b.lo}); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  return ff_fast(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p))));
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  const float p = __fmul_rn(a.hi, b);
  return ff_fast(p, fmaf(a.lo, b, fmaf(a.hi, b, -p)));
}

__device__ __forceinline__ ff ff_sqr(ff a) {
  const float p = __fmul_rn(a.hi, a.hi);
  return ff_fast(p, fmaf(2.f * a.hi, a.lo, fmaf(a.hi, a.hi, -p)));
}

// sqrt(x), x >= 0: the FP32 root s0 and one Newton (Heron) step s0 + (x - s0^2) / (2 s0), the
// residual formed exactly to first order (x.hi - s0^2 is exact by Sterbenz's lemma)
__device__ __forceinline__ ff ff_sqrt(ff x) {
  if (!(x.hi > 0.f)) return {0.f, 0.f};
  const float s0 = sqrtf(x.hi);
  const float p = __fmul_rn(s0, s0);
  const float r = ((x.hi - p) - fmaf(s0, s0, -p)) + x.lo;
  return ff_fast(s0, __fdividef(r, s0 + s0));
}

__device__ __forceinline__ ff ff_norm(const ff u[3]) {
  return ff_sqrt(ff_add(ff_add(ff_sqr(u[0]), ff_sqr(u[1])), ff_sqr(u[2])));
}

// a cycle count x (any float) mod 1 as a Q0.64 phase: f = x - rint(x) is exact and within
// +-1/2; f 2^64 is taken as h 2^33 + l 2^2 with h = rint(f 2^31) and l = rint((f 2^31 - h) 2^31),
// both exact 31-bit conversions
__device__ __forceinline__ uint64_t q64_of(float x) {
  const float y = (x - rintf(x)) * 2147483648.0f;
  const float h = rintf(y);
  return (static_cast<uint64_t>(static_cast<int64_t>(__float2int_rn(h))) << 33) +
         (static_cast<uint64_t>(static_cast<int64_t>(__float2int_rn((y - h) * 2147483648.0f))) << 2);
}

// (a K) mod 1 as a Q0.64 phase for a length a and a cycles-per-metre constant K, both
// float-float: the rounded product p, and its error plus the cross terms t (~2^-9 for a 10^4-cycle
// path), each reduced on its own and added as integers
__device__ __forceinline__ uint64_t q64_prod(ff a, ff K) {
  const float p = __fmul_rn(a.hi, K.hi);
  const float t = fmaf(a.hi, K.lo, fmaf(a.lo, K.hi, fmaf(a.hi, K.hi, -p)));
  return q64_of(p) + q64_of(t);
}

// hit h at snapshot j (Eq. 6); false when its triangle or one of the vertex indices is out of range
__device__ __forceinline__ bool hit_tri(const GeomDev &g, int64_t h, int32_t &a, int32_t &b, int32_t &c) {
  const int32_t tr = g.htri[h];
  if (tr < 0 || tr >= g.n_tri) return false;
  a = g.tri[3 * static_cast<int64_t>(tr)];
  b = g.tri[3 * static_cast<int64_t>(tr) + 1];
  c = g.tri[3 * static_cast<int64_t>(tr) + 2];
  return a >= 0 && a < g.n_vert && b >= 0 && b < g.n_vert && c >= 0 && c < g.n_vert;
}

__device__ bool hit_at(const GeomDev &g, int64_t j, int64_t h, double p[3]) {
  int32_t a, b, c;
  if (!hit_tri(g, h, a, b, c)) return false;
  const double *V = g.vert + j * g.n_vert * 3;
  const double u = static_cast<double>(g.hu[h]), v = static_cast<double>(g.hv[h]);
  const double w = 1.0 - u - v;
#pragma unroll
  for (int q = 0; q < 3; ++q) p[q] = w * V[3 * a + q] + u * V[3 * b + q] + v * V[3 * c + q];
  return true;
}

// the same in float-float, relative to ref_tx
__device__ bool hit_at_ff(const GeomDev &g, int64_t j, int64_t h, ff p[3]) {
  int32_t a, b, c;
  if (!hit_tri(g, h, a, b, c)) return false;
  const float2 *V = g.vff + j * g.n_vert * 3;
  const float u = g.hu[h], v = g.hv[h];
  const ff w = ff_add_f(ff_two_sum(1.f, -u), -v);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float2 va = V[3 * a + q], vb = V[3 * b + q], vc = V[3 * c + q];
    p[q] = ff_add(ff_add(ff_mul(w, {va.x, va.y}), ff_mul_f({vb.x, vb.y}, u)), ff_mul_f({vc.x, vc.y}, v));
  }
  return true;
}

__device__ __forceinline__ double dist3(const double *a, const double *b) {
  const double x = a[0] - b[0], y = a[1] - b[1], z = a[2] - b[2];
  return sqrt(x * x + y * y + z * z);
}

// Hits of ray i at snapshot j: first and last position and the length between them; false
// when the hit list or an index is out of range (nothing is read past it).  P is double (FP64,
// absolute positions) or ff (float-float, relative to ref_tx).
__device__ __forceinline__ bool hit_pos(const GeomDev &g, int64_t j, int64_t h, double p[3]) {
  return hit_at(g, j, h, p);
}
__device__ __forceinline__ bool hit_pos(const GeomDev &g, int64_t j, int64_t h, ff p[3]) {
  return hit_at_ff(g, j, h, p);
}
__device__ __forceinline__ void leg_add(double &s, const double *a, const double *b) { s += dist3(a, b); }
__device__ __forceinline__ void leg_add(ff &s, const ff *a, const ff *b) {
  const ff d[3] = {ff_sub(a[0], b[0]), ff_sub(a[1], b[1]), ff_sub(a[2], b[2])};
  s = ff_add(s, ff_norm(d));
}

template <typename P>
__device__ bool ray_hits(const GeomDev &g, int64_t i, int64_t j, P pf[3], P pl[3], P &inner) {
  const int64_t h0 = g.off[i], h1 = g.off[i + 1];
  if (!(h0 >= 0 && h1 > h0 && h1 <= g.n_hits)) return false;
  if (!hit_pos(g, j, h0, pf)) return false;
#pragma unroll
  for (int q = 0; q < 3; ++q) pl[q] = pf[q];
  for (int64_t h = h0 + 1; h < h1; ++h) {
    P c[3];
    if (!hit_pos(g, j, h, c)) return false;
    leg_add(inner, pl, c);
#pragma unroll
    for (int q = 0; q < 3; ++q) pl[q] = c[q];
  }
  return true;
}

__device__ __forceinline__ float4 ff_pair(double a, double b) {
  const float ah = static_cast<float>(a), bh = static_cast<float>(b);
  return make_float4(ah, static_cast<float>(a - static_cast<double>(ah)), bh,
                     static_cast<float>(b - static_cast<double>(bh)));
}

// Per ray, in FP64: snapshot 0 of Eq. 7, base0 = (d - inner(0) - |p_f(0) - ref_tx|,
// -|p_l(0) - ref_rx|) as two float-float numbers, and the start phase phi0 / 2 pi as Q0.64
__global__ void __launch_bounds__(128) snapshot0_kernel(GeomDev g, const double *__restrict__ d,
                                                        const float *__restrict__ p0, int64_t n,
                                                        float4 *__restrict__ base0, uint64_t *__restrict__ q0,
                                                        uint32_t *status) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  q0[i] = frac_q64(static_cast<double>(p0[i]) * kInv2Pi);
  double pf[3] = {0, 0, 0}, pl[3] = {0, 0, 0}, inner = 0.0;
  if (!ray_hits(g, i, 0, pf, pl, inner)) {
    atomicOr(status, kStatusBadGeometry);
    base0[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  base0[i] = ff_pair(d[i] - inner - dist3(pf, g.ref_tx), -dist3(pl, g.ref_rx));
}

// The vertices of every snapshot minus ref_tx, split into float-float (FP64, once per call)
__global__ void split_vertices_kernel(const double *__restrict__ v, int64_t n_val, double r0, double r1, double r2,
                                      float2 *__restrict__ out) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n_val;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int q = static_cast<int>(e % 3);
    const double x = v[e] - (q == 0 ? r0 : (q == 1 ? r1 : r2));
    const float hi = static_cast<float>(x);
    out[e] = make_float2(hi, static_cast<float>(x - static_cast<double>(hi)));
  }
}

// |u - e| - |u| for an antenna offset e from the reference (see the file comment), FP32, with
// s = |u| and inv_s = 1 / s.  With num = |e|^2 - 2 u.e and x = num / s^2 it is
// s (sqrt(1 + x) - 1) = num / (2 s) (1 - x/4 + x^2/8 - 5 x^3/64 + 7 x^4/128 - ...), whose
// truncation after x^4 is below 1.4e-8 of the result for |x| <= 1/20 (a compact array: |x| is
// about 2 |e| / s, 0.01 for 1.6 cm at 3 m); beyond that the rationalised form num / (|u - e| + s).
__device__ __forceinline__ float leg_offset(const ff u[3], float s, float inv_s, float4 e) {
  const float num = fmaf(-2.f, fmaf(u[0].hi, e.x, fmaf(u[1].hi, e.y, u[2].hi * e.z)), e.w);
  const float h = 0.5f * num * inv_s, x = num * inv_s * inv_s;
  if (fabsf(x) <= 0.05f) {
    float p = fmaf(x, 7.f / 128.f, -5.f / 64.f);
    p = fmaf(p, x, 1.f / 8.f);
    p = fmaf(p, x, -0.25f);
    p = fmaf(p, x, 1.f);
    return h * p;
  }
  return num / (sqrtf(fmaf(s, s, num)) + s);
}

// a small cycle count as a Q0.32 phase: only x - rint(x), exact and within +-1/2, counts, so a
// 32-bit conversion of it times 2^32 gives the word (f 2^32 is exact, its rounding the only one)
__device__ __forceinline__ uint32_t q32_small(float x) {
  const float f = x - rintf(x);
  return static_cast<uint32_t>(__float2int_rn(f * 4294967296.0f));
}

// a signed offset sum kept within int32 (antennas far enough apart to reach it give a bound the
// expansion refuses)
__device__ __forceinline__ int32_t sat32(int64_t x) {
  return static_cast<int32_t>(x > INT32_MAX ? INT32_MAX : (x < -INT32_MAX ? -INT32_MAX : x));
}

// a Q0.64 phase rounded to the nearest Q0.32 word (modulo one cycle)
__device__ __forceinline__ uint32_t q32_of(uint64_t q) {
  return static_cast<uint32_t>((q + (uint64_t{1} << 31)) >> 32);
}

// One thread per (ray li of the chunk starting at i0, snapshot j = blockIdx.y), in float-float
// and FP32 only.  paths != null: l(j, t, r) into paths[(i N_c + j) N_v + t N_rx + r]; else the
// phase words of A_t and B_r, and, when rec_s != null, the record of (li, j) at j stride + li:
// the step word S(j, t_c, r_c) of the reference antennas and the largest and smallest
// S(j, t, r) - S(j, t_c, r_c), the sum of the transmitter's and the receiver's extremes.
__global__ void __launch_bounds__(128) snapshot_kernel(GeomDev g, const float4 *__restrict__ base0,
                                                       const uint64_t *__restrict__ q0s, int64_t i0, int64_t cnt,
                                                       PhaseConst k, double *__restrict__ paths,
                                                       uint2 *__restrict__ w_tx, uint2 *__restrict__ w_rx,
                                                       int64_t stride, uint32_t *__restrict__ rec_s,
                                                       int32_t *__restrict__ rec_hi, int32_t *__restrict__ rec_lo,
                                                       uint32_t *status) {
  const int64_t li = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (li >= cnt) return;
  const int64_t i = i0 + li;
  ff ut[3] = {}, pl[3] = {}, inner = {0.f, 0.f};
  const bool ok = ray_hits(g, i, j, ut, pl, inner);  // positions relative to ref_tx: ut = p_f - ref_tx
  if (!ok) atomicOr(status, kStatusBadGeometry);
  const ff ur[3] = {ff_add(pl[0], g.t2r[0]), ff_add(pl[1], g.t2r[1]), ff_add(pl[2], g.t2r[2])};
  const ff st = ff_norm(ut), sr = ff_norm(ur);
  const float inv_st = 1.f / st.hi, inv_sr = 1.f / sr.hi;
  const float4 b0 = base0[i];
  // Eq. 7 with the reference antennas: the traced length without its snapshot-0 antenna legs,
  // the stretch between the hits re-measured, and the two reference legs at snapshot j
  const ff a_ref = ff_add(ff_add({b0.x, b0.y}, inner), st);
  const ff b_ref = ff_add({b0.z, b0.w}, sr);
  if (paths) {
    const int nv = k.ntx * k.nrx;
    double *o = paths + (i * k.nc + j) * nv;
    for (int t = 0; t < k.ntx; ++t) {
      const ff a = ff_add_f(a_ref, leg_offset(ut, st.hi, inv_st, g.tx[t]));
      for (int r = 0; r < k.nrx; ++r) {
        const ff l = ff_add(a, ff_add_f(b_ref, leg_offset(ur, sr.hi, inv_sr, g.rx[r])));
        o[t * k.nrx + r] = ok ? f64_of(l.hi) + f64_of(l.lo) : 0.0;
      }
    }
    return;
  }
  // the four reference words rounded once: an antenna's offset is a whole number of Q0.32
  // units (q32_small), so its word is the rounded reference plus that offset, exactly
  const uint32_t at_c = q32_of(q64_prod(a_ref, k.fc) + q0s[i]), at_s = q32_of(q64_prod(a_ref, k.sp));
  const uint32_t br_c = q32_of(q64_prod(b_ref, k.fc)), br_s = q32_of(q64_prod(b_ref, k.sp));
  const float fc_f = k.fc.hi, sp_f = k.sp.hi;
  // step offsets of the antennas relative to antenna 0 (their extremes, and the reference
  // antenna's, give the records' offsets from the reference)
  uint32_t ot0 = 0, or0 = 0;
  int32_t dt_hi = 0, dt_lo = 0, dt_c = 0, dr_hi = 0, dr_lo = 0, dr_c = 0;
  uint2 *wt = w_tx + j * k.ntx * stride + li;
  for (int t = 0; t < k.ntx; ++t, wt += stride) {
    const float e = leg_offset(ut, st.hi, inv_st, g.tx[t]);
    const uint32_t os = q32_small(e * sp_f);
    if (t == 0) ot0 = os;
    const int32_t d = static_cast<int32_t>(os - ot0);
    dt_hi = max(dt_hi, d);
    dt_lo = min(dt_lo, d);
    if (t == k.tc) dt_c = d;
    *wt = ok ? make_uint2(at_c + q32_small(e * fc_f), at_s + os) : make_uint2(0u, 0u);
  }
  uint2 *wr = w_rx + j * k.nrx * stride + li;
  for (int r = 0; r < k.nrx; ++r, wr += stride) {
    const float e = leg_offset(ur, sr.hi, inv_sr, g.rx[r]);
    const uint32_t os = q32_small(e * sp_f);
    if (r == 0) or0 = os;
    const int32_t d = static_cast<int32_t>(os - or0);
    dr_hi = max(dr_hi, d);
    dr_lo = min(dr_lo, d);
    if (r == k.rc) dr_c = d;
    *wr = ok ? make_uint2(br_c + q32_small(e * fc_f), br_s + os) : make_uint2(0u, 0u);
  }
  if (rec_s) {
    // the words' own units: S(m, t, r) - S(m, t_c, r_c) of the stored words is exactly the
    // recorded D, and s(m) is the stored reference pair's sum
    const int64_t at = j * stride + li;
    rec_s[at] = ok ? (at_s + ot0 + static_cast<uint32_t>(dt_c)) + (br_s + or0 + static_cast<uint32_t>(dr_c)) : 0u;
    rec_hi[at] = ok ? sat32(static_cast<int64_t>(dt_hi) - dt_c + static_cast<int64_t>(dr_hi) - dr_c) : 0;
    rec_lo[at] = ok ? sat32(static_cast<int64_t>(dt_lo) - dt_c + static_cast<int64_t>(dr_lo) - dr_c) : 0;
  }
}

ff ff_host(double x) {
  const float hi = static_cast<float>(x);
  return {hi, static_cast<float>(x - static_cast<double>(hi))};
}

size_t round256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

bool finite3(const double *p) { return isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]); }

bool device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// One call's device block: the rays, hits and mesh copied in, per-ray prep, and the outputs.
struct SnapRun {
  const Derived *g = nullptr;
  int64_t n = 0, H = 0, chunk = 0;
  uint8_t *b = nullptr;
  cudaStream_t s = nullptr;
  GeomDev gd{};
  size_t o_d = 0, o_a = 0, o_v = 0, o_az = 0, o_el = 0, o_p0 = 0, o_obj = 0;
  size_t o_car = 0, o_nur = 0, o_nud = 0, o_nua = 0, o_amp = 0, o_cell = 0, o_en = 0, o_sd = 0, o_sr = 0, o_ntx = 0;
  size_t o_base0 = 0, o_q0 = 0, o_vff = 0, o_status = 0, o_wt = 0, o_wr = 0, o_sig = 0, o_tmp = 0, o_spec = 0, o_lab = 0, o_paths = 0;
  size_t o_pk = 0, o_pe = 0, o_ck = 0, o_cm = 0, o_co = 0, o_pw = 0, o_tw = 0, o_rec = 0;
  int64_t cap = 0;
  uint32_t route = 0;  // the route mask read back by snap_finish
  ScratchLease lease;  // b: the context's snapshot scratch (kept between calls) or this call's own
  ~SnapRun() {
    if (s) {
      cudaStreamSynchronize(s);  // nothing may still use b when the lease ends
      cudaStreamDestroy(s);
    }
  }
};

// Checks the arguments, sizes and fills the device block.  mode 0: path lengths only;
// mode 1: signal (+ spectrum, + labels).
int snap_setup(SnapRun &R, sim_ctx *ctx, const sim_rays *rays, const sim_meta *meta, const sim_hits *hits,
               const sim_geometry *geom, int mode, bool want_spec, bool want_labels, bool paths_on_device) {
  if (!ctx || !rays || !hits || !geom) return SIM_E_INVALID;
  launches_begin();
  const Derived &g = ctx->g;
  R.g = &g;
  if (g.tslot != 0.0) return SIM_E_INVALID;  // snapshots exist at j T_d only
  const int64_t n = rays->n;
  if (n < 0 || n > g.max_rays) return SIM_E_INVALID;
  if (geom->n_vertices < 1 || geom->n_vertices > (int64_t{1} << 31) || geom->n_triangles < 1 ||
      geom->n_triangles > (int64_t{1} << 31))
    return SIM_E_INVALID;
  if (!geom->vertices || !geom->triangles || !geom->tx_pos || !geom->rx_pos || !hits->offset) return SIM_E_INVALID;
  if (!finite3(geom->ref_tx) || !finite3(geom->ref_rx)) return SIM_E_INVALID;
  if (n > 0 && (!rays->range_rt_m || !rays->amplitude || !rays->radial_velocity_mps || !rays->azimuth_rad ||
                !rays->elevation_rad || !rays->phase0_rad || !hits->triangle || !hits->u || !hits->v))
    return SIM_E_INVALID;
  if (want_labels && (!meta || !meta->object_id)) return SIM_E_INVALID;
  // antenna positions and the hit count are read on the host
  std::vector<double> txp(3 * static_cast<size_t>(g.ntx)), rxp(3 * static_cast<size_t>(g.nrx));
  int64_t off0 = 0, H = 0;
  if (cudaMemcpy(txp.data(), geom->tx_pos, 8 * txp.size(), cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(rxp.data(), geom->rx_pos, 8 * rxp.size(), cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(&off0, hits->offset, 8, cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(&H, hits->offset + n, 8, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return SIM_E_INVALID;
  }
  for (int t = 0; t < g.ntx; ++t)
    if (!finite3(&txp[3 * t])) return SIM_E_INVALID;
  for (int r = 0; r < g.nrx; ++r)
    if (!finite3(&rxp[3 * r])) return SIM_E_INVALID;
  if (off0 != 0 || H < n || H > (int64_t{1} << 32)) return SIM_E_INVALID;
  R.n = n;
  R.H = H;

  const size_t un = static_cast<size_t>(n), up = (un + 31) / 32 * 32, uh = static_cast<size_t>(H);
  const size_t per_ray_words = 8 * static_cast<size_t>(g.nc) * static_cast<size_t>(g.ntx + g.nrx);
  int64_t chunk = 0;
  if (mode == 1 && n > 0) {
    chunk = static_cast<int64_t>(kWordBudget / per_ray_words) / 256 * 256;
    if (chunk < 256) chunk = 256;
    if (chunk > n) chunk = (n + 3) / 4 * 4;  // row strides of four: 16-byte word pairs, record quads
  }
  R.chunk = chunk;
  const size_t vbytes = 24 * static_cast<size_t>(g.nc) * static_cast<size_t>(geom->n_vertices);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += round256(bytes > 0 ? bytes : 1);
    return o;
  };
  R.o_d = take(8 * un); R.o_a = take(4 * un); R.o_v = take(4 * un); R.o_az = take(4 * un);
  R.o_el = take(4 * un); R.o_p0 = take(4 * un); R.o_obj = take(want_labels ? 4 * un : 0);
  const size_t o_off = take(8 * (un + 1)), o_ht = take(4 * uh), o_hu = take(4 * uh), o_hv = take(4 * uh);
  const size_t o_vert = take(vbytes), o_tri = take(12 * static_cast<size_t>(geom->n_triangles));
  const size_t o_tx = take(16 * static_cast<size_t>(g.ntx)), o_rx = take(16 * static_cast<size_t>(g.nrx));
  R.o_base0 = take(16 * un);
  R.o_q0 = take(8 * un);
  R.o_vff = take(vbytes);
  R.o_car = take(8 * up); R.o_nur = take(8 * up); R.o_nud = take(8 * up); R.o_nua = take(8 * up);
  R.o_amp = take(4 * up); R.o_cell = take(4 * up); R.o_en = take(8 * up); R.o_sd = take(8 * up);
  R.o_sr = take(8 * up); R.o_ntx = take(8 * up);
  R.o_status = take(256);
  R.o_wt = take(mode == 1 ? 8 * static_cast<size_t>(chunk) * g.nc * g.ntx : 0);
  R.o_wr = take(mode == 1 ? 8 * static_cast<size_t>(chunk) * g.nc * g.nrx : 0);
  R.o_sig = take(mode == 1 ? 8 * static_cast<size_t>(g.n_sig) : 0);
  R.o_pw = take(mode == 1 && chunk > 0 ? static_cast<size_t>(pair_workspace_bytes(g, chunk)) : 0);  // ray parts
  // tensor-core precisions: the expansion's header and split-K partials
  R.o_tw = take(mode == 1 && chunk > 0 && g.precision != SIM_PREC_FP32_DIRECT
                    ? static_cast<size_t>(snap_tensor_workspace_bytes(g, chunk))
                    : 0);
  // tensor-core precisions: the per-(ray, chirp) records that bound the expansion
  R.o_rec = take(mode == 1 && chunk > 0 && g.precision != SIM_PREC_FP32_DIRECT
                     ? 12 * static_cast<size_t>(chunk) * static_cast<size_t>(g.nc)
                     : 0);
  R.o_tmp = take(mode == 1 && want_spec ? 8 * static_cast<size_t>(g.n_sig) : 0);
  R.o_spec = take(mode == 1 && want_spec ? 8 * static_cast<size_t>(g.n_cell) : 0);
  R.o_lab = take(want_labels ? 4 * static_cast<size_t>(g.n_cell) : 0);
  R.cap = want_labels ? label_capacity(n) : 0;
  const size_t cap = static_cast<size_t>(R.cap);
  R.o_pk = take(8 * cap); R.o_pe = take(8 * cap); R.o_ck = take(4 * cap); R.o_cm = take(8 * cap);
  R.o_co = take(4 * cap);
  R.o_paths = take(mode == 0 && !paths_on_device ? 8 * un * g.nc * g.nv : 0);
  R.b = static_cast<uint8_t *>(R.lease.get(ctx->scratch[kSlotSnapshot], off));
  if (!R.b) return SIM_E_NOMEM;
  if (cudaStreamCreateWithFlags(&R.s, cudaStreamNonBlocking) != cudaSuccess) {
    R.s = nullptr;
    return SIM_E_CUDA;
  }
  uint8_t *b = R.b;
  cudaStream_t s = R.s;
  if (n > 0) {
    cudaMemcpyAsync(b + R.o_d, rays->range_rt_m, 8 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + R.o_a, rays->amplitude, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + R.o_v, rays->radial_velocity_mps, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + R.o_az, rays->azimuth_rad, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + R.o_el, rays->elevation_rad, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + R.o_p0, rays->phase0_rad, 4 * un, cudaMemcpyDefault, s);
    if (want_labels) cudaMemcpyAsync(b + R.o_obj, meta->object_id, 4 * un, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + o_ht, hits->triangle, 4 * uh, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + o_hu, hits->u, 4 * uh, cudaMemcpyDefault, s);
    cudaMemcpyAsync(b + o_hv, hits->v, 4 * uh, cudaMemcpyDefault, s);
  }
  cudaMemcpyAsync(b + o_off, hits->offset, 8 * (un + 1), cudaMemcpyDefault, s);
  cudaMemcpyAsync(b + o_vert, geom->vertices, vbytes, cudaMemcpyDefault, s);
  cudaMemcpyAsync(b + o_tri, geom->triangles, 12 * static_cast<size_t>(geom->n_triangles), cudaMemcpyDefault, s);
  // antenna offsets from the reference antennas, FP32 with their squared length
  std::vector<float> etx(4 * static_cast<size_t>(g.ntx)), erx(4 * static_cast<size_t>(g.nrx));
  auto offsets = [](const std::vector<double> &x, const double *ref, std::vector<float> &e) {
    for (size_t a = 0; a < e.size() / 4; ++a) {
      double n2 = 0.0;
      for (int q = 0; q < 3; ++q) {
        const double d = x[3 * a + q] - ref[q];
        e[4 * a + q] = static_cast<float>(d);
        n2 += d * d;
      }
      e[4 * a + 3] = static_cast<float>(n2);
    }
  };
  offsets(txp, geom->ref_tx, etx);
  offsets(rxp, geom->ref_rx, erx);
  cudaMemcpyAsync(b + o_tx, etx.data(), 4 * etx.size(), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(b + o_rx, erx.data(), 4 * erx.size(), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(b + R.o_status, 0, 8, s);  // status bits and route mask
  GeomDev &gd = R.gd;
  gd.vert = reinterpret_cast<const double *>(b + o_vert);
  gd.vff = reinterpret_cast<const float2 *>(b + R.o_vff);
  gd.tri = reinterpret_cast<const int32_t *>(b + o_tri);
  gd.tx = reinterpret_cast<const float4 *>(b + o_tx);
  gd.rx = reinterpret_cast<const float4 *>(b + o_rx);
  for (int q = 0; q < 3; ++q) {
    gd.ref_tx[q] = geom->ref_tx[q];
    gd.ref_rx[q] = geom->ref_rx[q];
    gd.t2r[q] = ff_host(geom->ref_tx[q] - geom->ref_rx[q]);
  }
  gd.off = reinterpret_cast<const int64_t *>(b + o_off);
  gd.htri = reinterpret_cast<const int32_t *>(b + o_ht);
  gd.hu = reinterpret_cast<const float *>(b + o_hu);
  gd.hv = reinterpret_cast<const float *>(b + o_hv);
  gd.n_vert = geom->n_vertices;
  gd.n_tri = geom->n_triangles;
  gd.n_hits = H;
  // the host copies of the antenna offsets must outlive the copies above
  if (cudaStreamSynchronize(s) != cudaSuccess) return SIM_E_CUDA;
  return SIM_OK;
}

// the snapshot-0 terms of every ray (after snap_setup, on its stream); returns kernels launched
// the float-float vertices and the per-ray snapshot-0 terms
int launch_snapshot0(SnapRun &R) {
  if (R.n <= 0) return 0;
  const int64_t n_val = 3 * static_cast<int64_t>(R.g->nc) * R.gd.n_vert;
  const int64_t blocks = (n_val + 255) / 256 < 4096 ? (n_val + 255) / 256 : 4096;
  split_vertices_kernel<<<static_cast<unsigned>(blocks), 256, 0, R.s>>>(
      R.gd.vert, n_val, R.gd.ref_tx[0], R.gd.ref_tx[1], R.gd.ref_tx[2], reinterpret_cast<float2 *>(R.b + R.o_vff));
  snapshot0_kernel<<<static_cast<unsigned>((R.n + 127) / 128), 128, 0, R.s>>>(
      R.gd, reinterpret_cast<const double *>(R.b + R.o_d), reinterpret_cast<const float *>(R.b + R.o_p0), R.n,
      reinterpret_cast<float4 *>(R.b + R.o_base0), reinterpret_cast<uint64_t *>(R.b + R.o_q0),
      reinterpret_cast<uint32_t *>(R.b + R.o_status));
  return 2;
}

PhaseConst phase_const(const Derived &g) {
  PhaseConst k;
  k.fc = ff_host(g.fc / kC);
  k.sp = ff_host(g.bw / (kC * static_cast<double>(g.ns)));
  k.nc = g.nc;
  k.ntx = g.ntx;
  k.nrx = g.nrx;
  k.tc = snap_ref_tx(g);
  k.rc = snap_ref_rx(g);
  return k;
}

int snap_finish(SnapRun &R) {
  uint32_t st[2] = {0, 0};  // status bits, route mask
  cudaMemcpyAsync(st, R.b + R.o_status, 8, cudaMemcpyDeviceToHost, R.s);
  const cudaError_t e = cudaStreamSynchronize(R.s);
  if (e != cudaSuccess || !launches_ok()) return SIM_E_CUDA;
  if (st[0] & (kStatusBadRay | kStatusBadGeometry)) return SIM_E_INVALID;
  R.route = st[1];
  return st[0] ? SIM_E_DEVICE : SIM_OK;
}

}  // namespace

extern "C" SIM_API int sim_snapshot_paths(sim_ctx *ctx, const sim_rays *rays, const sim_hits *hits,
                                          const sim_geometry *geom, double *paths) {
  if (!paths) return SIM_E_INVALID;
  SnapRun R;
  const bool dev = device_ptr(paths);
  int rc = snap_setup(R, ctx, rays, nullptr, hits, geom, 0, false, false, dev);
  if (rc != SIM_OK) return rc;
  const Derived &g = *R.g;
  launch_snapshot0(R);
  if (R.n > 0) {
    double *out = dev ? paths : reinterpret_cast<double *>(R.b + R.o_paths);
    const dim3 grid(static_cast<unsigned>((R.n + 127) / 128), static_cast<unsigned>(g.nc));
    snapshot_kernel<<<grid, 128, 0, R.s>>>(R.gd, reinterpret_cast<const float4 *>(R.b + R.o_base0),
                                           reinterpret_cast<const uint64_t *>(R.b + R.o_q0), 0, R.n, phase_const(g),
                                           out, nullptr, nullptr, 0, nullptr, nullptr, nullptr,
                                           reinterpret_cast<uint32_t *>(R.b + R.o_status));
    if (!dev)
      cudaMemcpyAsync(paths, out, 8 * static_cast<size_t>(R.n) * g.nc * g.nv, cudaMemcpyDeviceToHost, R.s);
  }
  return snap_finish(R);
}

extern "C" SIM_API int sim_snapshot_run(sim_ctx *ctx, const sim_rays *rays, const sim_meta *meta,
                                        const sim_hits *hits, const sim_geometry *geom, void *spectrum,
                                        void *signal, int32_t *labels) {
  if (!ctx || (!spectrum && !signal && !labels)) return SIM_E_INVALID;
  if ((spectrum && !(ctx->g.outputs & SIM_OUT_SPECTRUM)) || (labels && !(ctx->g.outputs & SIM_OUT_LABELS)))
    return SIM_E_INVALID;
  SnapRun R;
  int rc = snap_setup(R, ctx, rays, meta, hits, geom, 1, spectrum != nullptr, labels != nullptr, false);
  if (rc != SIM_OK) return rc;
  const Derived &g = *R.g;
  uint8_t *b = R.b;
  cudaStream_t s = R.s;
  uint32_t *status = reinterpret_cast<uint32_t *>(b + R.o_status);
  RaysIn in{reinterpret_cast<const double *>(b + R.o_d), reinterpret_cast<const float *>(b + R.o_a),
            reinterpret_cast<const float *>(b + R.o_v), reinterpret_cast<const float *>(b + R.o_az),
            reinterpret_cast<const float *>(b + R.o_el), reinterpret_cast<const float *>(b + R.o_p0),
            labels ? reinterpret_cast<const int32_t *>(b + R.o_obj) : nullptr};
  RaysPrep rp{reinterpret_cast<uint64_t *>(b + R.o_car), reinterpret_cast<uint64_t *>(b + R.o_nur),
              reinterpret_cast<uint64_t *>(b + R.o_nud), reinterpret_cast<uint64_t *>(b + R.o_nua),
              reinterpret_cast<float *>(b + R.o_amp), reinterpret_cast<int32_t *>(b + R.o_cell),
              reinterpret_cast<uint64_t *>(b + R.o_en), reinterpret_cast<float2 *>(b + R.o_sd),
              reinterpret_cast<float2 *>(b + R.o_sr), nullptr, reinterpret_cast<uint64_t *>(b + R.o_ntx), nullptr};
  // events around every stage: prep, per chunk (phase words | direct sum), FFTs, labels
  const int64_t n_chunks = R.chunk > 0 ? (R.n + R.chunk - 1) / R.chunk : 0;
  std::vector<cudaEvent_t> ev(static_cast<size_t>(2 * n_chunks + 5), nullptr);
  for (auto &e : ev) cudaEventCreate(&e);
  int kernels = 0, ei = 0;
  cudaEventRecord(ev[ei++], s);
  // per-ray validation, antenna-pattern amplitudes, label cells and energies
  kernels += launch_prep(g, in, R.n, rp, status, s);
  kernels += launch_snapshot0(R);
  cudaEventRecord(ev[ei++], s);
  float2 *sig = reinterpret_cast<float2 *>(b + R.o_sig);
  if (R.n == 0) cudaMemsetAsync(sig, 0, 8 * static_cast<size_t>(g.n_sig), s);
  uint2 *wt = reinterpret_cast<uint2 *>(b + R.o_wt), *wr = reinterpret_cast<uint2 *>(b + R.o_wr);
  const PhaseConst k = phase_const(g);
  const bool tensor = g.precision != SIM_PREC_FP32_DIRECT;
  const size_t rec_n = static_cast<size_t>(R.chunk) * static_cast<size_t>(g.nc);
  uint32_t *rec_s = tensor ? reinterpret_cast<uint32_t *>(b + R.o_rec) : nullptr;
  int32_t *rec_hi = tensor ? reinterpret_cast<int32_t *>(b + R.o_rec) + rec_n : nullptr;
  int32_t *rec_lo = tensor ? reinterpret_cast<int32_t *>(b + R.o_rec) + 2 * rec_n : nullptr;
  for (int64_t i0 = 0; i0 < R.n; i0 += R.chunk) {
    const int64_t cnt = R.n - i0 < R.chunk ? R.n - i0 : R.chunk;
    const dim3 grid(static_cast<unsigned>((cnt + 127) / 128), static_cast<unsigned>(g.nc));
    snapshot_kernel<<<grid, 128, 0, s>>>(R.gd, reinterpret_cast<const float4 *>(b + R.o_base0),
                                         reinterpret_cast<const uint64_t *>(b + R.o_q0), i0, cnt, k,
                                         nullptr, wt, wr, R.chunk, rec_s, rec_hi, rec_lo, status);
    cudaEventRecord(ev[ei++], s);
    if (g.precision == SIM_PREC_FP32_DIRECT)
      kernels += 1 + launch_pair_sum(g, wt, wr, rp.amp + i0, cnt, R.chunk, i0 > 0, sig, b + R.o_pw, nullptr, s);
    else
      kernels += 1 + launch_snap_tensor(g, wt, wr, SnapRec{rec_s, rec_hi, rec_lo}, R.chunk, rp.amp + i0, cnt, i0 > 0,
                                        sig, b + R.o_tw, b + R.o_pw, status, s);
    cudaEventRecord(ev[ei++], s);
  }
  if (signal) cudaMemcpyAsync(signal, sig, 8 * static_cast<size_t>(g.n_sig), cudaMemcpyDefault, s);
  if (spectrum) {
    float2 *spec = reinterpret_cast<float2 *>(b + R.o_spec);
    kernels += launch_fft(g, ctx->t, sig, reinterpret_cast<float2 *>(b + R.o_tmp), spec, s);
    cudaMemcpyAsync(spectrum, spec, 8 * static_cast<size_t>(g.n_cell), cudaMemcpyDefault, s);
  }
  cudaEventRecord(ev[ei++], s);
  if (labels) {
    LabelScratch sc{reinterpret_cast<uint64_t *>(b + R.o_pk), reinterpret_cast<uint64_t *>(b + R.o_pe),
                    reinterpret_cast<uint32_t *>(b + R.o_ck), reinterpret_cast<uint64_t *>(b + R.o_cm),
                    reinterpret_cast<uint32_t *>(b + R.o_co), R.cap};
    int32_t *dlab = reinterpret_cast<int32_t *>(b + R.o_lab);
    kernels += launch_labels(g, rp, in.obj, R.n, sc, dlab, status, s);
    cudaMemcpyAsync(labels, dlab, 4 * static_cast<size_t>(g.n_cell), cudaMemcpyDefault, s);
  }
  cudaEventRecord(ev[ei++], s);
  rc = snap_finish(R);
  if (rc == SIM_OK) {
    auto span = [&](int a, int b2) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[static_cast<size_t>(a)], ev[static_cast<size_t>(b2)]);
      return ms;
    };
    float ms[7] = {0, span(0, 1), 0, 0, 0, 0, 0};
    int prev = 1;
    for (int64_t c = 0; c < n_chunks; ++c) {
      ms[1] += span(prev, prev + 1);      // phase words of the chunk
      ms[2] += span(prev + 1, prev + 2);  // its direct sum
      prev += 2;
    }
    ms[4] = span(prev, prev + 1);
    ms[5] = span(prev + 1, prev + 2);
    ms[6] = span(0, prev + 2);
    record_stage_ms(ctx, ms, kernels, R.route);
  }
  for (auto &e : ev) cudaEventDestroy(e);
  return rc;
}
