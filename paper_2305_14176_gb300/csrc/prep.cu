// K_a: per-ray prep in FP64 (arXiv 2305.14176, Sec. II-A Eqs. 1-3, Sec. II-E Eq. 7).
//
// For every ray: validate it, range-reduce its phase increments to Q0.64 fixed point
// (the one step whose accuracy needs FP64: f_c d / c is up to ~1e5 cycles; the reduction mod 1
// works on the FP64 product's bits), and compute its label cell and fixed-point energy.  All FP64 arithmetic uses explicit _rn
// intrinsics so no multiply-add is contracted: the bin coordinates follow a fixed
// operation order and are reproducible bit for bit.
#include <math.h>

#include "internal.h"

namespace rs {
namespace {

// pi/2 as a sum of two doubles (Cody-Waite), and 2/pi, each the nearest double
__device__ constexpr double kP1 = 0x1.921fb54442d18p+0;
__device__ constexpr double kP2 = 0x1.1a62633145c07p-54;
__device__ constexpr double kTwoOverPi = 0x1.45f306dc9c883p-1;
__device__ constexpr double kInv2Pi = 0x1.45f306dc9c883p-3;  // 1 / (2 pi)

// Taylor series of sin on [-pi/4, pi/4] through r^17, Horner in r^2 with fused multiply-adds
__device__ __forceinline__ double poly_sin(double r) {
  const double z = __dmul_rn(r, r);
  double p = 1.0 / 355687428096000.0;
  p = __fma_rn(p, z, -1.0 / 1307674368000.0);
  p = __fma_rn(p, z, 1.0 / 6227020800.0);
  p = __fma_rn(p, z, -1.0 / 39916800.0);
  p = __fma_rn(p, z, 1.0 / 362880.0);
  p = __fma_rn(p, z, -1.0 / 5040.0);
  p = __fma_rn(p, z, 1.0 / 120.0);
  p = __fma_rn(p, z, -1.0 / 6.0);
  return __fma_rn(__dmul_rn(r, z), p, r);
}

// Taylor series of cos on [-pi/4, pi/4] through r^18
__device__ __forceinline__ double poly_cos(double r) {
  const double z = __dmul_rn(r, r);
  double q = -1.0 / 6402373705728000.0;
  q = __fma_rn(q, z, 1.0 / 20922789888000.0);
  q = __fma_rn(q, z, -1.0 / 87178291200.0);
  q = __fma_rn(q, z, 1.0 / 479001600.0);
  q = __fma_rn(q, z, -1.0 / 3628800.0);
  q = __fma_rn(q, z, 1.0 / 40320.0);
  q = __fma_rn(q, z, -1.0 / 720.0);
  q = __fma_rn(q, z, 1.0 / 24.0);
  q = __fma_rn(q, z, -1.0 / 2.0);
  return __fma_rn(z, q, 1.0);
}

// sin (want_cos = false) or cos of x, |x| <= fl32(pi): quadrant k = rint(x 2/pi) in -2..2,
// r = (x - k P1) - k P2 (the first subtraction is exact), then the series by quadrant.
__device__ __forceinline__ double sin_or_cos(double x, bool want_cos) {
  const double k = rint(__dmul_rn(x, kTwoOverPi));
  const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(k, kP1)), __dmul_rn(k, kP2));
  const int q = (static_cast<int>(k) + (want_cos ? 1 : 0)) & 3;
  switch (q) {
    case 0: return poly_sin(r);
    case 1: return poly_cos(r);
    case 2: return -poly_sin(r);
    default: return -poly_cos(r);
  }
}

// x mod 1 as a Q0.64 phase, from the bits of x on the integer pipes (this GPU's FP64 pipe is
// the prep's limit): x = +-m 2^(e - 1075) with m the 53-bit significand, so x 2^64 mod 2^64 =
// +-m 2^(e - 1011) mod 2^64, rounded to nearest when the shift is to the right; zero,
// subnormal and non-finite x give 0 (the validated inputs give none of those but zero).
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

// e^{2 pi j 32 q} for a Q0.64 phase increment q.  The exact Q0.64 product p = 32 q splits into
// a 24-bit head h (signed cycles in [-1/2, 1/2), exact in FP32) and a remainder r < 2^-24
// cycles: e^{2 pi j p} = e^{2 pi j h} (1 + 2 pi j r) to within (2 pi r)^2 / 2 < 7e-14, below FP32
// resolution.  The FP32 sin/cos of the head keeps the phasor within ~1.5 ulp, which the tensor
// kernels' recurrences (at most 7 steps per chain) turn into < 3e-7 relative error, against
// ~4e-6 for their hi + lo arithmetic; FP64 sin/cos here cost ~40 % of this FP64-bound kernel.
__device__ __forceinline__ float2 step32(uint64_t q) {
  const uint64_t p = q * 32ull;
  const int32_t head24 = static_cast<int32_t>(static_cast<uint32_t>(p >> 40) << 8) >> 8;  // sign-extended
  const float h = static_cast<float>(head24) * 0x1p-24f;
  const float r = static_cast<float>(static_cast<uint32_t>(p >> 8)) * 0x1p-56f;  // bits 8..39: [0, 2^-24)
  float s, c;
  sincospif(2.0f * h, &s, &c);
  const float d = 6.28318530717958648f * r;  // 2 pi r radians
  return make_float2(c - s * d, s + c * d);
}

// floor(x + 1/2) modulo n (Euclidean); n is a power of two, so the remainder is a mask of the
// two's-complement value
__device__ __forceinline__ int64_t bin_of(double x, int64_t n) {
  const int64_t q = static_cast<int64_t>(floor(__dadd_rn(x, 0.5)));
  return q & (n - 1);
}

struct PrepConst {
  int pattern_exp;
  double fc, bw, td, tslot, nc_d, ka;
  // phase-word constants (no bin depends on them): f_c / c, 2 f_c T_slot / c, and the
  // range-migration words' 2 B T_d / (c N_s) and 2 B T_slot / (c N_s), each one FP64 product
  // per ray instead of a division
  double fc_c, nut_v, eps_v, epst_v;
  uint64_t nrx;
  double inv_ns, inv_nc, inv_na;
  int64_t ns, nc, na;
  int want_labels;
};

__global__ void __launch_bounds__(256) prep_kernel(PrepConst k, RaysIn in, int64_t n, RaysPrep out,
                                                   uint32_t *status) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const double d = in.d[i];
  const float a = in.a[i], v = in.v[i], az = in.az[i], el = in.el[i], p0 = in.p0[i];
  const int32_t obj = k.want_labels ? in.obj[i] : 0;
  // validation: NaN fails every comparison below
  const bool ok = (d >= 0.0 && d <= 1.0e7) && (a >= 0.0f && a <= 3.0e38f) &&
                  (fabsf(v) <= 1.0e5f) && (fabsf(az) <= 3.14159274f) && (fabsf(el) <= 1.57079637f) &&
                  (fabsf(p0) <= 1.0e6f) && (obj >= 0);
  if (!ok) {
    atomicOr(status, kStatusBadRay);
    out.carrier[i] = 0; out.nu_r[i] = 0; out.nu_d[i] = 0; out.nu_a[i] = 0;
    out.amp[i] = 0.0f; out.cell[i] = -1; out.energy[i] = 0;
    out.step_d[i] = make_float2(1.f, 0.f); out.step_r[i] = make_float2(1.f, 0.f);
    if (out.eps) out.eps[i] = 0;
    out.nu_tx[i] = 0;
    if (out.eps_t) out.eps_t[i] = 0;
    return;
  }
  const double vd = static_cast<double>(v);
  // analytic bin coordinates (fixed order, no contraction)
  const double x_r = __ddiv_rn(__dmul_rn(k.bw, d), kC);
  const double x_d = __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(2.0, vd), k.fc), k.td), k.nc_d), kC);
  const double cos_el = sin_or_cos(static_cast<double>(el), true);
  const double x_a = __dmul_rn(k.ka, __dmul_rn(sin_or_cos(static_cast<double>(az), false), cos_el));
  // antenna pattern A(az, el) = (cos(az) cos(el))^q (Eq. 2), q products in order
  double aa = static_cast<double>(a);
  if (k.pattern_exp > 0) {
    const double c = __dmul_rn(sin_or_cos(static_cast<double>(az), true), cos_el);
    for (int e = 0; e < k.pattern_exp; ++e) aa = __dmul_rn(aa, c);
  }
  // phase increments per sample / chirp / channel: x_x / N_x (exact scaling by a power of two)
  const uint64_t nu_r = frac_q64(__dmul_rn(x_r, k.inv_ns));
  const uint64_t nu_d = frac_q64(__dmul_rn(x_d, k.inv_nc));
  out.nu_r[i] = nu_r;
  out.nu_d[i] = nu_d;
  out.step_r[i] = step32(nu_r);
  out.step_d[i] = step32(nu_d);
  const uint64_t nu_a = frac_q64(__dmul_rn(x_a, k.inv_na));
  out.nu_a[i] = nu_a;
  // TDM-MIMO: transmitter t fires chirp j at j T_d + t T_slot, so its phase gains t nu_t with
  // nu_t = 2 v f_c T_slot / c; channel k = t N_rx + r then has phase t (N_rx nu_a + nu_t) + r nu_a
  const uint64_t nu_t = k.tslot > 0.0 ? frac_q64(__dmul_rn(vd, k.nut_v)) : 0ull;
  out.nu_tx[i] = k.nrx * nu_a + nu_t;
  if (out.eps) {
    // exact Eq. 2: mu t_n (tau_i(j) - tau_i(0)) = n j B (2 v T_d) / (c N_s) cycles
    out.eps[i] = frac_q64(__dmul_rn(vd, k.eps_v));
    // and with TDM slots n t B (2 v T_slot) / (c N_s)
    out.eps_t[i] = frac_q64(__dmul_rn(vd, k.epst_v));
  }
  // carrier phase f_c tau (Eq. 1, Eq. 2) plus the ray's start phase
  out.carrier[i] = frac_q64(__dmul_rn(d, k.fc_c)) + frac_q64(__dmul_rn(static_cast<double>(p0), kInv2Pi));
  out.amp[i] = static_cast<float>(aa);
  const int64_t cell = (bin_of(x_a, k.na) * k.nc + bin_of(x_d, k.nc)) * k.ns + bin_of(x_r, k.ns);
  out.cell[i] = static_cast<int32_t>(cell);
  double e = rint(ldexp(__dmul_rn(aa, aa), 32));
  if (e > 2199023255552.0) e = 2199023255552.0;  // 2^41
  out.energy[i] = static_cast<uint64_t>(e);
}

}  // namespace

// device-resident caller arrays into the scene's block: one launch for all seven arrays
__global__ void __launch_bounds__(256) ingest_kernel(IngestArgs x, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    x.dst_d[i] = x.d[i];
    x.dst_a[i] = x.a[i];
    x.dst_v[i] = x.v[i];
    x.dst_az[i] = x.az[i];
    x.dst_el[i] = x.el[i];
    x.dst_p0[i] = x.p0[i];
    if (x.obj) x.dst_obj[i] = x.obj[i];
  }
}

int launch_ingest(const IngestArgs &x, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  const int64_t blocks = (n + 255) / 256;
  ingest_kernel<<<static_cast<unsigned>(blocks < 1216 ? blocks : 1216), 256, 0, s>>>(x, n);
  return 1;
}

int launch_prep(const Derived &g, RaysIn in, int64_t n, RaysPrep out, uint32_t *status, cudaStream_t s) {
  if (n <= 0) return 0;
  PrepConst k;
  k.pattern_exp = g.pattern_exp;
  k.tslot = g.tslot;
  k.nrx = static_cast<uint64_t>(g.nrx);
  k.fc = g.fc;
  k.bw = g.bw;
  k.td = g.td;
  k.nc_d = static_cast<double>(g.nc);
  k.ka = g.ka;
  k.fc_c = g.fc / kC;
  k.nut_v = 2.0 * g.fc * g.tslot / kC;
  k.eps_v = 2.0 * g.bw * g.td / (kC * g.ns);
  k.epst_v = 2.0 * g.bw * g.tslot / (kC * g.ns);
  k.inv_ns = 1.0 / g.ns;
  k.inv_nc = 1.0 / g.nc;
  k.inv_na = 1.0 / g.na;
  k.ns = g.ns;
  k.nc = g.nc;
  k.na = g.na;
  k.want_labels = in.obj != nullptr;
  const int64_t blocks = (n + 255) / 256;
  prep_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(k, in, n, out, status);
  return 1;
}

}  // namespace rs
