// K_b1x: the exact signal model on tensor cores by a per-tile expansion of the range-migration
// phase (arXiv 2305.14176, Sec. II-A, Eq. 2 with mu t (tau_i(j) - tau_i(0)) kept).
//
// The exact phase of ray i at channel k = (t, r), chirp m and sample n is
//   phi_i + t nu_tx,i + r nu_a,i + m nu_d,i + n nu_r,i + n m eps_i.
// Inside one output tile write m = m_c + m' and n = n_c + n' about the tile's centre:
//   n m eps = n_c m' eps + n m_c eps + n' m' eps.
// The first two terms are exact per-tile shifts of the chirp and sample frequencies; only
// e^{2 pi j n' m' eps} still couples rows and columns, and over a tile |m'| <= m_h, |n'| <= n_h
// are small, so e^{j x t}, x = 2 pi eps m' n_h (row) and t = n' / n_h in [-1, 1) (column), is
// replaced by a separable series of P terms: Taylor,
//   e^{j x t} = sum_{p<P} (j x)^p / p! t^p + R,   |R| <= |x|^P / P!,
// or Chebyshev (Jacobi-Anger, see chebyshev_series_terms), eps_p j^p J_p(x) times T_p(t), whose
// remainder is 2^(P-1) times smaller.  The tile is one complex product over K = P x rays:
//   S[row, n] = sum_{i, p} A_p[row, i] B_p[i, n]
//   A_p[row, i] = a_i e^{2 pi j (phi + t nu_tx + r nu_a + m nu_d + n_c m' eps)} c_p(x_row,i)
//   B_p[i, n]   = e^{2 pi j n (nu_r + m_c eps)} b_p(n' / n_h),      x_row,i = 2 pi eps_i m' n_h
// with c_p(x) = (j x)^p / p!, b_p(t) = t^p (Taylor) or c_p(x) = eps_p j^p J_p(x), b_p = T_p.
// Rows are chirp-major (row = m N_v + k), so a 256-row tile spans only about 256 / N_v chirps,
// and each synthesised value serves a whole 256 x NC tile instead of N_v channels.
// With TDM slot offsets the phase also holds n t eps_t (transmitter t); with t = t_c + t' it
// joins the coupling the same way: the shifts take n_c t' eps_t (rows) and n t_c eps_t
// (columns), and x = 2 pi n' (m' eps + t' eps_t).
//
// The device takes four Taylor terms when their bound theta^4 / 4!, theta = 2 pi n_h (max|eps|
// m_h + max|eps_t| t_h), is at most 1e-6 at the hi + lo precisions (1e-5 single pass, whose
// operand rounding is ~3e-4), else the fewest Chebyshev terms (4, 6, 8) that meet it; a device
// kernel takes theta from the scene's largest |eps|, so no host round trip is needed.  When even
// eight terms would not meet the bound (velocities far beyond road traffic), P = 0 is written and the
// per-chirp kernel of umma_exact.cu, launched behind this one, computes the scene instead: each
// of the two kernels (and its reduction) returns at once when the other one owns the scene.
// The per-chirp form has no slot term, so with TDM slots P = 0 is an error instead (a status
// bit reported as invalid rays).
//
// At the hi + lo precisions the second 16-slot K step of every stage holds only terms of order
// p >= P / 2 (at P = 6 term 3 of the stage's first ray falls in the first K step and keeps its
// lo operands), each at most theta^(P/2) / (P/2)! of the ray's amplitude (Chebyshev: 2 (theta /
// 2)^(P/2) / (P/2)!), so single-pass operand rounding (<= 2u relative, u = 2^-11 FP16, 2^-8
// BF16) adds at most that times 2u; when
// the device finds this below 2e-6 that K step skips its lo operands and the hi x lo MMAs (8
// MMA units per stage instead of 12).
//
// Pipeline, tensor-core issue and drain are those of the separable kernel's two-SM form: CTA
// pairs (cta_group::2, M = 256), planar K (Re S += A_re B_re - A_im B_im, Im S += A_re B_im +
// A_im B_re, split precision adds the hi / lo cross terms), FP32 running sum in tensor memory
// every 512 K slots at split precision, FP32 partials per ray chunk added by a second kernel.
// A stage holds 32 K slots: RS = floor(32 / P) rays times P terms, slot = p RS + q, and at P = 6
// two zero slots (5 rays: 0.8 K steps of MMAs per ray against 1.0 at P = 8).  Every mbarrier
// wait is bounded; a wait that runs out sets a status bit and the CTA drains and returns.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "tcgen05.cuh"

namespace rs {
namespace {

constexpr int TBM = 128;               // rows per CTA (TMEM lanes); a CTA pair covers 256
constexpr int TKS = 32;                // K slots per stage
constexpr int TGSIZE = 128;            // producer threads per group (one A row each)
constexpr int TMAX_GROUPS = 4;
constexpr int TNDRAIN = 128;
// producer groups: four for single pass; three at split precision, whose 96 registers per
// thread a fourth group would cut to 80 with spills (measured: 4 groups 6.69 -> 6.40 ms single
// pass, 15.07 -> 15.49 ms FP16 hi + lo per automotive frame)
template <bool SPLIT>
__host__ __device__ constexpr int t_groups() {
  return SPLIT ? 3 : 4;
}
// Stages per accumulation chain at split precision.  The tensor core's accumulate is not
// round-to-nearest, so a chain is folded into the FP32 running sum after a bounded number of
// MMAs into its accumulator: 192, as in the separable kernel's 512-ray chains.  A stage adds 12
// MMAs to each accumulator block when every term keeps its lo operands (16 stages) and 8 when
// the high-order terms go single pass (24 stages); each fold stalls the tensor pipe.
constexpr int TSUBST_SPLIT = 16;
constexpr int TSUBST_SPLIT_LOW = 24;
constexpr uint32_t TSUM_COL = 256;     // TMEM column of the running sum
constexpr int TMAX_RAYS = 8;           // rays per stage at P = 4 (5 at P = 6, 4 at P = 8)
// workspace header: amplitude maximum (u32 bits), P (u32), largest |eps| (u64), whether the
// high-order K step keeps its lo operands (u32), largest |eps_t| (u64), the expansion's form
// (u32: 0 Taylor, 1 Chebyshev)
constexpr size_t kOffTerms = 4, kOffEpsMax = 8, kOffLoHigh = 16, kOffEpsTMax = 24, kOffForm = 32, kHeader = 256;

// what the rows and columns are synthesised from
constexpr int kExact = 0;     // exact Eq. 2: per-ray words of the prep kernel
constexpr int kExactTdm = 1;  // the same with TDM slot offsets
constexpr int kSnap = 2;      // virtual snapshots: per-(ray, chirp, antenna) phase words

// Snapshot mode at split precision folds the MMA issuer into the first drain warp: 16 warps,
// so 128 registers a thread and no spills (measured 36.6 -> 34.4 ms per automotive snapshot
// frame at FP16 hi + lo).  The other kernels keep a warp of their own for it, which measured
// faster for them (the exact model at FP16 hi + lo 14.8 against 15.6 ms).
template <bool SPLIT, int MODE>
__host__ __device__ constexpr bool t_merged() {
  return SPLIT && MODE == kSnap;
}
template <bool SPLIT, int MODE>
__host__ __device__ constexpr int t_threads() {
  return t_groups<SPLIT>() * TGSIZE + (t_merged<SPLIT, MODE>() ? 0 : 32) + TNDRAIN;
}

struct TArgs {
  RaysPrep p;
  // kSnap: Q0.32 phase words (base, per-sample step) w_tx[(m N_tx + t) stride + i],
  // w_rx[(m N_rx + r) stride + i] of the chunk's rays, their amplitudes, the reference antennas
  const uint2 *w_tx, *w_rx;
  int64_t stride;
  const float *samp;
  int ntx, r_c;
  int64_t n_rays, chunk;  // rays, rays per split (multiple of 8)
  int nc, ns, nv, nrx, m_rows;
  int t_c;                // centre transmitter of the slot term
  int bn;                 // real columns per tile, 2 NC
  int mt2, nt;            // 256-row tiles, column tiles
  float *partials;        // [split][M chirp-major rows][2 N_s], each tile as (Re block | Im block)
  const uint32_t *amax_bits;
  const uint32_t *terms;  // P chosen on the device; 0: the per-chirp kernel owns the scene
  const uint32_t *lo_high;  // split precision: 0 when the terms p >= P/2 go single pass
  const uint32_t *form;     // 0: Taylor terms, 1: Chebyshev (Jacobi-Anger) terms
  uint32_t *status;
};

// per-ray words of one stage (at most 8 rays)
struct TStage {
  uint64_t car[TMAX_RAYS], nua[TMAX_RAYS], nud[TMAX_RAYS], nutx[TMAX_RAYS], nur[TMAX_RAYS], eps[TMAX_RAYS];
  uint64_t epst[TMAX_RAYS];
  float amp[TMAX_RAYS];
};

struct TWords {
  uint64_t car, nua, nud, nutx, nur, eps, epst;
  float amp;
};

// thread gt < rays of the stage fetches its ray's words (rays past the chunk read as 0).
// kSnap: the ray's reference per-sample step (the tile's centre chirp m_c, antennas t_c, r_c),
// a Q0.32 word kept in the low half of `nur`, and its amplitude.
template <int MODE>
__device__ __forceinline__ TWords tfetch(const TArgs &g, int64_t ray0, int rays, int64_t k_hi, int gt, int m_c) {
  TWords w{0, 0, 0, 0, 0, 0, 0, 0.f};
  const int64_t ray = ray0 + gt;
  if constexpr (MODE == kSnap) {
    if (gt < rays && ray < k_hi) {
      w.nur = g.w_tx[(static_cast<int64_t>(m_c) * g.ntx + g.t_c) * g.stride + ray].y +
              g.w_rx[(static_cast<int64_t>(m_c) * g.nrx + g.r_c) * g.stride + ray].y;  // modulo 2^32
      w.amp = g.samp[ray];
    }
    return w;
  }
  if (gt < rays && ray < k_hi) {
    w.car = g.p.carrier[ray];
    w.nua = g.p.nu_a[ray];
    w.nud = g.p.nu_d[ray];
    w.nutx = g.p.nu_tx[ray];
    w.nur = g.p.nu_r[ray];
    w.eps = g.p.eps[ray];
    if constexpr (MODE == kExactTdm) w.epst = g.p.eps_t[ray];
    w.amp = g.p.amp[ray];
  }
  return w;
}

template <int MODE>
__device__ __forceinline__ void tstore(TStage &s, int gt, const TWords &w) {
  if constexpr (MODE == kSnap) {
    if (gt < TMAX_RAYS) {
      s.nur[gt] = w.nur;
      s.amp[gt] = w.amp;
    }
    return;
  }
  if (gt < TMAX_RAYS) {
    s.car[gt] = w.car;
    s.nua[gt] = w.nua;
    s.nud[gt] = w.nud;
    s.nutx[gt] = w.nutx;
    s.nur[gt] = w.nur;
    s.eps[gt] = w.eps;
    if constexpr (MODE == kExactTdm) s.epst[gt] = w.epst;
    s.amp[gt] = w.amp;
  }
}

__device__ __forceinline__ void tgroup_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(TGSIZE) : "memory");
}

// What one producer thread needs of its A row and B columns for a whole unit.
struct RowCtx {
  uint32_t tx, rx, m;       // channel (t, r), chirp
  int32_t ncm, nct;         // n_c m', n_c t' (|n_c m'| < 2^23)
  float xm, xt;             // 2 pi m' n_h 2^-64, 2 pi t' n_h 2^-64: x = xm eps_i + xt eps_t,i (words)
  bool valid;
  // kSnap: the row's phase-word rows, n_c, and 2 pi n_h 2^-32 (x = xs delta_i, Q0.32 words)
  const uint2 *wt, *wr;
  uint32_t n_c;
  float xs;
};
struct ColCtx {
  uint32_t n, nmc, ntc;     // sample index, n m_c, n t_c (< 2^26)
  float u;                  // n' / n_h
  int c;                    // column in this CTA's B block
  uint32_t octets;          // bit o: this thread writes K chunk o of the column
  bool active;
};

// Chebyshev form of the coupling factor (Jacobi-Anger): for real x and t in [-1, 1],
//   e^{j x t} = J_0(x) + 2 sum_{p>=1} j^p J_p(x) T_p(t),
// truncated after P terms with remainder at most 2 sum_{p>=P} |J_p(x)| <= 2 (|x|/2)^P / P! /
// (1 - |x| / (2 (P + 1))), using |J_p(x)| <= (|x|/2)^p / p!.  That is 2^(P-1) times below the
// Taylor bound, so a given tolerance is met with fewer terms.  Rows take eps_p j^p J_p(x),
// columns T_p(n' / n_h).  J_p(x) = (x/2)^p / p! S_p(-x^2/4), S_p(w) = sum_k w^k / (k! (p+1)_k),
// summed to k = K: K = 2, 4, 6 for P = 4, 6, 8 leaves < 5e-8 of the largest J_p at the largest
// x each P is chosen for (0.21, 0.78, 1.62 at the single-pass tolerance).
__host__ __device__ constexpr int chebyshev_series_terms(int P) { return P <= 4 ? 2 : (P <= 6 ? 4 : 6); }
__host__ __device__ constexpr float ja_coef(int p, int k) {
  double c = 1.0;
  for (int i = 1; i <= k; ++i) c /= static_cast<double>(i) * static_cast<double>(p + i);
  return static_cast<float>(c);
}
template <int K>
__device__ __forceinline__ float ja_series(int p, float w) {  // S_p(w) by Horner; p compile-time after unrolling
  float s = ja_coef(p, K);
#pragma unroll
  for (int k = K - 1; k >= 0; --k) s = fmaf(s, w, ja_coef(p, k));
  return s;
}
__device__ __forceinline__ float2 rot_i(float2 v, int p) {  // v j^p
  switch (p & 3) {
    case 0: return v;
    case 1: return make_float2(-v.y, v.x);
    case 2: return make_float2(-v.x, -v.y);
    default: return make_float2(v.y, -v.x);
  }
}
__device__ __forceinline__ float chebyshev_t(int p, float u) {  // T_p(u) by the three-term recurrence
  float t0 = 1.f, t1 = u;
  if (p == 0) return 1.f;
  for (int k = 1; k < p; ++k) {
    const float t2 = 2.f * u * t1 - t0;
    t0 = t1;
    t1 = t2;
  }
  return t1;
}

// One stage of operands: A row gt (all 32 slots) and this thread's B column octets, in the
// no-swizzle K-major core-matrix layout of the separable kernel (octet o = K chunk o).
// Slot s = p RS + q holds term p of the stage's ray q; with RS = floor(32 / P) rays per stage the
// slots from P RS on (two at P = 6) are zero on both sides.
// kSnap: rays li0 + q, q < valid, of the chunk are present; the rest read as silent.
template <bool F16, bool SPLIT, int MODE, int P, bool CH>
__device__ __forceinline__ void produce_taylor(const TStage &sr, uint8_t *stage, int gt, int ncb, const RowCtx &rc,
                                               const ColCtx &cc, float scale, bool lo_high, int64_t li0,
                                               int valid) {
  constexpr bool TDM = MODE == kExactTdm;
  constexpr int RS = TKS / P;   // rays per stage
  static_assert(RS <= TMAX_RAYS && P * RS <= TKS, "stage slots");
  const uint32_t a_half = TBM * TKS * 2;
  const uint32_t x_half = static_cast<uint32_t>(ncb) * TKS * 2;
  const uint32_t lo = SPLIT ? 2 * a_half + 2 * x_half : 0;
  uint8_t *a_re = stage, *a_im = stage + a_half, *x_re = stage + 2 * a_half, *x_im = x_re + x_half;
  {
    float2 t[RS];
    float x[RS];
    float h[RS];  // CH: eps_p (x / 2)^p / p! of the current term
    // kSnap: the row's words of the stage's rays, two rays per 16-byte load when RS is even (the
    // stage's first ray is then even and the row stride is even, so each pair is aligned; a pair
    // whose first ray is present lies inside the row, its second ray is masked below if absent)
    uint2 wa[RS], wb[RS];
    if constexpr (MODE == kSnap) {
      if constexpr (RS % 2 == 0) {
#pragma unroll
        for (int q = 0; q < RS; q += 2) {
          uint4 u = make_uint4(0u, 0u, 0u, 0u), v = make_uint4(0u, 0u, 0u, 0u);
          if (rc.valid && q < valid) {
            u = *reinterpret_cast<const uint4 *>(rc.wt + li0 + q);
            v = *reinterpret_cast<const uint4 *>(rc.wr + li0 + q);
          }
          wa[q] = make_uint2(u.x, u.y);
          wa[q + 1] = make_uint2(u.z, u.w);
          wb[q] = make_uint2(v.x, v.y);
          wb[q + 1] = make_uint2(v.z, v.w);
        }
      } else {
#pragma unroll
        for (int q = 0; q < RS; ++q) {
          const bool live = rc.valid && q < valid;
          wa[q] = live ? rc.wt[li0 + q] : make_uint2(0u, 0u);
          wb[q] = live ? rc.wr[li0 + q] : make_uint2(0u, 0u);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < RS; ++q) {
      float sn, cs;
      if constexpr (MODE == kSnap) {
        // base C and per-sample step S of this row's path, delta = S - S_ref (a small signed
        // word): phase C + n_c delta, expansion variable x = 2 pi n_h delta (Q0.32, wrapping)
        const bool live = rc.valid && q < valid;
        uint32_t c = 0, d = 0;
        if (live) {
          c = wa[q].x + wb[q].x;
          d = wa[q].y + wb[q].y - static_cast<uint32_t>(sr.nur[q]);
        }
        __sincosf(q32_to_rad(c + rc.n_c * d), &sn, &cs);
        const float am = live ? sr.amp[q] * scale : 0.f;
        t[q] = make_float2(am * cs, am * sn);
        x[q] = rc.xs * static_cast<float>(static_cast<int32_t>(d));
      } else {
        uint64_t ph = sr.car[q] + static_cast<uint64_t>(rc.tx) * sr.nutx[q] + static_cast<uint64_t>(rc.rx) * sr.nua[q] +
                      static_cast<uint64_t>(rc.m) * sr.nud[q] +
                      static_cast<uint64_t>(static_cast<int64_t>(rc.ncm)) * sr.eps[q];
        if constexpr (TDM) ph += static_cast<uint64_t>(static_cast<int64_t>(rc.nct)) * sr.epst[q];
        __sincosf(q64_to_rad(ph), &sn, &cs);
        const float am = rc.valid ? sr.amp[q] * scale : 0.f;
        t[q] = make_float2(am * cs, am * sn);
        x[q] = rc.xm * s64_to_f32(sr.eps[q]);
        if constexpr (TDM) x[q] += rc.xt * s64_to_f32(sr.epst[q]);
      }
    }
    if constexpr (CH) {
#pragma unroll
      for (int q = 0; q < RS; ++q) h[q] = 1.f;
    }
    uint32_t off = (gt >> 3) * 128 + (gt & 7) * 16;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      float2 z[OCT];
#pragma unroll
      for (int e = 0; e < OCT; ++e) {
        const int sl = o * OCT + e, p = sl / RS, q = sl % RS;  // compile-time after unrolling
        if constexpr (CH) {
          // t i^p eps_p J_p(x), J_p(x) = (x / 2)^p / p! S_p(-x^2 / 4)
          if (p < P) {
            const float c = h[q] * ja_series<chebyshev_series_terms(P)>(p, -0.25f * x[q] * x[q]);
            const float2 v = rot_i(t[q], p);
            z[e] = make_float2(v.x * c, v.y * c);
          } else {
            z[e] = make_float2(0.f, 0.f);
          }
          if (q == RS - 1 && p + 1 < P) {
            const float f = (p == 0 ? 1.f : 0.5f) / static_cast<float>(p + 1);  // eps_{p+1} / eps_p / 2 / (p + 1)
#pragma unroll
            for (int r = 0; r < RS; ++r) h[r] *= x[r] * f;
          }
        } else {
          z[e] = p < P ? t[q] : make_float2(0.f, 0.f);
          if (q == RS - 1 && p + 1 < P) {
            const float inv = 1.f / static_cast<float>(p + 1);
#pragma unroll
            for (int r = 0; r < RS; ++r) {
              const float f = x[r] * inv;  // t <- t (j x) / (p + 1): term p + 1
              t[r] = make_float2(-t[r].y * f, t[r].x * f);
            }
          }
        }
      }
      if (o < 2 || lo_high) put_octet<F16, SPLIT>(z, a_re + off, a_im + off, a_re + lo + off, a_im + lo + off);
      else put_octet<F16, false>(z, a_re + off, a_im + off, a_re + off, a_im + off);
      off += TBM * 16;
    }
  }
  if (cc.active) {
    float2 b[RS];
#pragma unroll
    for (int q = 0; q < RS; ++q) {
      float sn, cs;
      if constexpr (MODE == kSnap) {
        __sincosf(q32_to_rad(cc.n * static_cast<uint32_t>(sr.nur[q])), &sn, &cs);  // the ray's reference step
      } else {
        uint64_t ph = static_cast<uint64_t>(cc.n) * sr.nur[q] + static_cast<uint64_t>(cc.nmc) * sr.eps[q];
        if constexpr (TDM) ph += static_cast<uint64_t>(cc.ntc) * sr.epst[q];
        __sincosf(q64_to_rad(ph), &sn, &cs);
      }
      b[q] = make_float2(cs, sn);
    }
    const uint32_t off0 = (cc.c >> 3) * 128 + (cc.c & 7) * 16;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      if (!((cc.octets >> o) & 1)) continue;
      float2 z[OCT];
#pragma unroll
      for (int e = 0; e < OCT; ++e) {
        const int sl = o * OCT + e, p = sl / RS, q = sl % RS;
        float u = 1.f;  // Taylor: (n' / n_h)^p; CH: T_p(n' / n_h) (a compile-time count of steps)
        if constexpr (CH) {
          u = chebyshev_t(p, cc.u);
        } else {
#pragma unroll
          for (int k = 0; k < p; ++k) u *= cc.u;
        }
        z[e] = p < P ? make_float2(b[q].x * u, b[q].y * u) : make_float2(0.f, 0.f);
      }
      const uint32_t off = o * static_cast<uint32_t>(ncb) * 16 + off0;
      if (o < 2 || lo_high) put_octet<F16, SPLIT>(z, x_re + off, x_im + off, x_re + lo + off, x_im + lo + off);
      else put_octet<F16, false>(z, x_re + off, x_im + off, x_re + off, x_im + off);
    }
  }
}

template <bool SPLIT>
__host__ __device__ constexpr int t_stages() {
  return SPLIT ? 4 : 6;
}
// bytes of one stage: A (Re, Im) 128 x 32 slots and this CTA's B (Re, Im) bn/4 x 32, x2 for lo
template <bool SPLIT>
__host__ __device__ constexpr uint32_t t_stage_bytes(int bn) {
  return static_cast<uint32_t>(TBM * TKS * 2 * 2 + (bn / 4) * TKS * 2 * 2) * (SPLIT ? 2u : 1u);
}

// The MMAs of one stage for both CTAs of the pair: Re and Im of the M = 256 x N product over
// the stage's 32 K slots, with the lo operand products at split precision (all K steps, or
// only the first when the high-order terms go single pass).
struct TIssue {
  uint32_t idesc, ineg, lbo_a, lbo_x, a_half, x_half, lo, t_re, t_im;
};
template <bool SPLIT>
__device__ __forceinline__ void t_issue_stage(const TIssue &w, uint32_t sb, bool first, bool lo_high) {
  const uint32_t ar = sb, ai = sb + w.a_half, xr = sb + 2 * w.a_half, xi = xr + w.x_half;
#pragma unroll
  for (int kh = 0; kh < TKS / 16; ++kh) {
    const uint32_t acc = (!first || kh > 0) ? 1u : 0u;
    const uint32_t oa = kh * 2 * w.lbo_a, ox = kh * 2 * w.lbo_x;
    const uint64_t dar = make_sdesc(ar + oa, w.lbo_a, 128), dai = make_sdesc(ai + oa, w.lbo_a, 128);
    const uint64_t dxr = make_sdesc(xr + ox, w.lbo_x, 128), dxi = make_sdesc(xi + ox, w.lbo_x, 128);
    mma_f16<true>(w.t_re, dar, dxr, w.idesc, acc);
    mma_f16<true>(w.t_re, dai, dxi, w.ineg, 1u);
    mma_f16<true>(w.t_im, dar, dxi, w.idesc, acc);
    mma_f16<true>(w.t_im, dai, dxr, w.idesc, 1u);
    if (SPLIT && (kh == 0 || lo_high)) {
      const uint32_t lo = w.lo;
      const uint64_t lar = make_sdesc(ar + lo + oa, w.lbo_a, 128), lai = make_sdesc(ai + lo + oa, w.lbo_a, 128);
      const uint64_t lxr = make_sdesc(xr + lo + ox, w.lbo_x, 128), lxi = make_sdesc(xi + lo + ox, w.lbo_x, 128);
      mma_f16<true>(w.t_re, dar, lxr, w.idesc, 1u);
      mma_f16<true>(w.t_re, lar, dxr, w.idesc, 1u);
      mma_f16<true>(w.t_re, dai, lxi, w.ineg, 1u);
      mma_f16<true>(w.t_re, lai, dxi, w.ineg, 1u);
      mma_f16<true>(w.t_im, dar, lxi, w.idesc, 1u);
      mma_f16<true>(w.t_im, lar, dxi, w.idesc, 1u);
      mma_f16<true>(w.t_im, dai, lxr, w.idesc, 1u);
      mma_f16<true>(w.t_im, lai, dxr, w.idesc, 1u);
    }
  }
}

// Launched as clusters of two CTAs; cluster u takes unit u = (split, tile_n, tile_m), the even
// CTA holding rows 0..127 of the 256-row tile and issuing the M = 256 MMAs.
// PT, CH: the term count and form (Taylor, Chebyshev) this instance is built for (it returns at
// once for another choice), or PT = 0 for every choice behind a branch per stage.  Split
// precision launches one instance per choice, whose producers then fit their registers without
// spills (exact model, FP16 hi + lo automotive frame: 13.95 ms against 14.53 with the branch);
// single pass keeps the branch (5.8 against 6.0 ms).  The chooser takes Taylor terms only at
// P = 4 (fewer operations per slot than Chebyshev terms at the same count) and Chebyshev terms
// wherever they need fewer terms than Taylor's.
template <bool F16, bool SPLIT, int MODE, int PT, bool CH>
__global__ void __launch_bounds__(t_threads<SPLIT, MODE>(), 1) taylor_sum_kernel(TArgs g) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int TGROUPS = t_groups<SPLIT>();
  constexpr int TMMA_WARP = TGROUPS * TGSIZE / 32;
  __shared__ TStage s_rays[TMAX_GROUPS];
  const uint32_t P = *g.terms;
  const bool cheb = *g.form != 0u;
  // another instance, or the per-chirp kernel, owns this scene (both CTAs return)
  if (PT == 0 ? (!expansion_terms(P) || cheb != CH) : (P != static_cast<uint32_t>(PT) || cheb != CH)) return;
  const bool lo_high = !SPLIT || *g.lo_high != 0u;
  constexpr int NST = t_stages<SPLIT>();
  constexpr uint32_t TMEM_COLS = 512;
  // a stage is signalled by one thread of each CTA's group after the group's barrier, at every
  // precision (at split precision against every producer thread arriving on its own: exact
  // model 14.19 -> 14.11 ms, snapshots 29.34 -> 28.87 ms per FP16 hi+lo frame)
  constexpr bool ONE_ARRIVE = true;
  const uint32_t stage_bytes = t_stage_bytes<SPLIT>(g.bn);
  const uint32_t rank = cluster_rank();
  uint8_t *base = smem;
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + NST * stage_bytes);
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + 2 * NST + 3);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + NST);
  const uint32_t accf = smem_u32(bars + 2 * NST), acce = smem_u32(bars + 2 * NST + 1);
  const uint32_t done = smem_u32(bars + 2 * NST + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0_c = cluster_addr(full0, 0);
  const uint32_t acce_c = cluster_addr(acce, 0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(full0 + 8 * s, (ONE_ARRIVE ? 1 : TGSIZE) * 2);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, 2 * TNDRAIN);
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == TMMA_WARP) tmem_alloc<true>(smem_u32(tmem_holder), TMEM_COLS);
  tc_fence_before();
  cluster_sync();  // both CTAs' barriers exist before any remote arrival
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  const int u = static_cast<int>(blockIdx.x >> 1);
  const int per = g.mt2 * g.nt;
  const int split = u / per;
  const int tile_n = (u - split * per) / g.mt2;
  const int tile_m = u - split * per - tile_n * g.mt2;
  const int bn = g.bn, NC = bn >> 1, ncb = bn >> 2;
  const int r0 = tile_m * 2 * TBM;                    // first row of the pair's tile
  const int row0 = r0 + static_cast<int>(rank) * TBM;  // this CTA's rows
  const int col0 = tile_n * bn;                        // real column; complex n0 = col0 / 2
  const int n0 = tile_n * NC;
  // tile centre: chirp and sample (kSnap: a chirp that exists, its reference words are read)
  const int m_c = MODE == kSnap ? min((r0 + TBM) / g.nv, g.nc - 1) : (r0 + TBM) / g.nv;
  const int n_c = n0 + NC / 2, n_h = NC / 2;
  const int RS = TKS / static_cast<int>(P);
  const int64_t k_lo = static_cast<int64_t>(split) * g.chunk;
  const int64_t k_hi = k_lo + g.chunk < g.n_rays ? k_lo + g.chunk : g.n_rays;
  const int n_stages = k_hi > k_lo ? static_cast<int>((k_hi - k_lo + RS - 1) / RS) : 0;
  const int SUBST = SPLIT ? (lo_high ? TSUBST_SPLIT : TSUBST_SPLIT_LOW) : (n_stages > 0 ? n_stages : 1);
  const int n_sub = (n_stages + SUBST - 1) / SUBST;
  bool failed = false;

  if (warp < TMMA_WARP) {
    // ---------------- producers: group grp builds stages grp, grp + TGROUPS, ...
    const int grp = warp / (TGSIZE / 32), gt = threadIdx.x % TGSIZE;
    const float scale = amp_scale<F16>(g.amax_bits);
    RowCtx rc;
    {
      const int r = row0 + gt;
      rc.valid = r < g.m_rows;
      const int m = r / g.nv, k = r - m * g.nv;
      const int t = k / g.nrx;
      rc.tx = static_cast<uint32_t>(t);
      rc.rx = static_cast<uint32_t>(k - t * g.nrx);
      rc.m = static_cast<uint32_t>(m);
      const int mp = m - m_c;
      rc.ncm = n_c * mp;
      rc.xm = static_cast<float>(mp) * static_cast<float>(n_h) * 3.40612158008655459e-19f;  // 2 pi 2^-64
      const int tp = t - g.t_c;
      rc.nct = n_c * tp;
      rc.xt = static_cast<float>(tp) * static_cast<float>(n_h) * 3.40612158008655459e-19f;
      rc.n_c = static_cast<uint32_t>(n_c);
      rc.xs = static_cast<float>(n_h) * 1.46291807926715968e-09f;  // 2 pi 2^-32
      rc.wt = rc.wr = nullptr;
      if (MODE == kSnap && rc.valid) {
        rc.wt = g.w_tx + (static_cast<int64_t>(m) * g.ntx + t) * g.stride;
        rc.wr = g.w_rx + (static_cast<int64_t>(m) * g.nrx + (k - t * g.nrx)) * g.stride;
      }
    }
    ColCtx cc;
    {
      // ncb <= 128 columns: tpc threads share a column, thread h of them takes octets h, h + tpc, ...
      const int tpc = TGSIZE / ncb, h = gt / ncb;
      cc.c = gt % ncb;
      cc.octets = 0;
      for (int o = h; o < 4; o += tpc) cc.octets |= 1u << o;
      cc.active = cc.octets != 0;
      const int n = n0 + static_cast<int>(rank) * ncb + cc.c;
      cc.n = static_cast<uint32_t>(n);
      cc.nmc = static_cast<uint32_t>(n) * static_cast<uint32_t>(m_c);
      cc.ntc = static_cast<uint32_t>(n) * static_cast<uint32_t>(g.t_c);
      cc.u = static_cast<float>(n - n_c) / static_cast<float>(n_h);  // n_h is a power of two
    }
    TWords nxt{0, 0, 0, 0, 0, 0, 0, 0.f};
    if (grp < n_stages) nxt = tfetch<MODE>(g, k_lo + static_cast<int64_t>(grp) * RS, RS, k_hi, gt, m_c);
    for (int st = grp; st < n_stages; st += TGROUPS) {
      const int s = st % NST;
      const int64_t ray0 = k_lo + static_cast<int64_t>(st) * RS;
      tstore<MODE>(s_rays[grp], gt, nxt);
      if (st + TGROUPS < n_stages) nxt = tfetch<MODE>(g, ray0 + TGROUPS * RS, RS, k_hi, gt, m_c);
      // kSnap: this row's words of the group's stage after next (one line each, inside the row
      // since that stage's first ray is below k_hi), pulled into L2 two group rounds ahead
      if (MODE == kSnap && rc.valid && st + 2 * TGROUPS < n_stages) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(rc.wt + ray0 + 2 * TGROUPS * RS));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(rc.wr + ray0 + 2 * TGROUPS * RS));
      }
      const int valid = static_cast<int>(k_hi - ray0 < RS ? k_hi - ray0 : RS);
      // the stage slot is free, and the group's ray words are visible; a wait that ran out in
      // any thread takes the whole group out of the loop
      const bool slot_ok = st < NST || mbar_wait(empty0 + 8 * s, ((st / NST) - 1) & 1);
      if (bar_any(grp + 1, TGSIZE, !slot_ok)) {
        failed = true;
        break;
      }
      uint8_t *st_base = base + s * stage_bytes;
      if constexpr (PT != 0)
        produce_taylor<F16, SPLIT, MODE, (PT != 0 ? PT : 4), CH>(s_rays[grp], st_base, gt, ncb, rc, cc, scale, lo_high,
                                                                 ray0, valid);
      else if (P == 4u)
        produce_taylor<F16, SPLIT, MODE, 4, CH>(s_rays[grp], st_base, gt, ncb, rc, cc, scale, lo_high, ray0, valid);
      else if (P == 6u)
        produce_taylor<F16, SPLIT, MODE, 6, CH>(s_rays[grp], st_base, gt, ncb, rc, cc, scale, lo_high, ray0, valid);
      else
        produce_taylor<F16, SPLIT, MODE, 8, CH>(s_rays[grp], st_base, gt, ncb, rc, cc, scale, lo_high, ray0, valid);
      fence_proxy_async();  // this thread's stores, visible to the tensor core
      if constexpr (ONE_ARRIVE) {
        tgroup_sync(grp);  // the group's stores are done and s_rays[grp] is free again
        if (gt == 0) mbar_arrive_cluster(full0_c + 8 * s);
      } else {
        mbar_arrive_cluster(full0_c + 8 * s);
        tgroup_sync(grp);  // s_rays[grp] is rewritten next round
      }
    }
  } else {
    constexpr bool MERGED = t_merged<SPLIT, MODE>();
    TIssue iw{};
    iw.idesc = make_idesc(F16, 2 * TBM, NC);
    iw.ineg = iw.idesc | (1u << 14);  // negate B: Re S -= A_im B_im
    iw.lbo_a = TBM * 16;
    iw.lbo_x = static_cast<uint32_t>(ncb) * 16;
    iw.a_half = TBM * TKS * 2;
    iw.x_half = static_cast<uint32_t>(ncb) * TKS * 2;
    iw.lo = 2 * iw.a_half + 2 * iw.x_half;
    iw.t_re = tmem;
    iw.t_im = tmem + static_cast<uint32_t>(NC);
    const uint32_t sbase = smem_u32(base);
    if (!MERGED && warp == TMMA_WARP) {
      // ---------------- MMA issuer warp (CTA 0 issues for both; CTA 1 only waits for the end)
      if (lane == 0 && rank != 0) {
        if (!mbar_wait(done, 0)) failed = true;
      } else if (lane == 0) {
        bool open = false;
        for (int st = 0; st < n_stages; ++st) {
          const int s = st % NST;
          const int gc = st / SUBST;
          const bool first = (st % SUBST) == 0;
          if (first && gc > 0 && !mbar_wait(acce, (gc - 1) & 1)) {
            failed = true;
            break;
          }
          if (!mbar_wait(full0 + 8 * s, (st / NST) & 1)) {
            failed = true;
            break;
          }
          tc_fence_after();
          t_issue_stage<SPLIT>(iw, sbase + s * stage_bytes, first, lo_high);
          open = true;
          mma_commit<true>(empty0 + 8 * s);
          if ((st % SUBST) == SUBST - 1 || st == n_stages - 1) {
            mma_commit<true>(accf);
            open = false;
          }
        }
        if (open) mma_commit<true>(accf);
        mma_commit<true>(done);  // fires in both CTAs once every issued MMA has completed
        if (!mbar_wait(done, 0)) failed = true;
      }
    } else {
      // ---------------- drain: TMEM lane quarter warp % 4; each finished chain is added in FP32
      // to the running sum in tensor memory, the last one goes to this split's partial.  MERGED:
      // lane 0 of the first drain warp in CTA 0 is the issuer; it issues each chain before its
      // warp drains it (the next chain's first MMAs wait for the drain in either layout).
      const bool issuer = MERGED && warp == TMMA_WARP && lane == 0 && rank == 0;
      const int q = warp & 3;
      const int grow = row0 + q * 32 + lane;
      float *dst = g.partials + (static_cast<int64_t>(split) * g.m_rows + grow) * (2 * g.ns) + col0;
      const uint32_t trow = tmem + (static_cast<uint32_t>(q * 32) << 16);
      if (n_stages == 0 && grow < g.m_rows) {
        for (int c = 0; c < bn; c += 4) *reinterpret_cast<float4 *>(dst + c) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      int st = 0;  // the merged issuer's next stage
      for (int sub = 0; sub < n_sub; ++sub) {
        if constexpr (MERGED) {
          if (issuer && !failed) {
            const int st_end = min(n_stages, (sub + 1) * SUBST);
            for (; st < st_end; ++st) {
              const int s = st % NST;
              const bool first = (st % SUBST) == 0;
              if (first && sub > 0 && !mbar_wait(acce, (sub - 1) & 1)) {
                failed = true;
                break;
              }
              if (!mbar_wait(full0 + 8 * s, (st / NST) & 1)) {
                failed = true;
                break;
              }
              tc_fence_after();
              t_issue_stage<SPLIT>(iw, sbase + s * stage_bytes, first, lo_high);
              mma_commit<true>(empty0 + 8 * s);
            }
            // complete once these MMAs are (after a failed wait too, so the drains end at once)
            mma_commit<true>(accf);
          }
          __syncwarp();  // the tensor-memory loads below are warp-collective
        }
        if (!mbar_wait_sleep(accf, sub & 1)) {
          failed = true;
          break;
        }
        tc_fence_after();
        const bool last = sub == n_sub - 1;
        // 32 columns per load pair and wait where the tile allows (the tensor pipe waits while
        // a chain drains), 16 at the tail
        for (int c = 0; c < bn;) {
          if (c + 32 <= bn) {
            uint32_t h[32];
            if (sub > 0) {
              uint32_t r[32];
              tmem_ld32x2(trow + static_cast<uint32_t>(c), trow + TSUM_COL + static_cast<uint32_t>(c), h, r);
#pragma unroll
              for (int x = 0; x < 32; ++x) h[x] = __float_as_uint(__uint_as_float(h[x]) + __uint_as_float(r[x]));
            } else {
              tmem_ld32(trow + static_cast<uint32_t>(c), h);
            }
            if (!last) {
              tmem_st32(trow + TSUM_COL + static_cast<uint32_t>(c), h);
            } else if (grow < g.m_rows) {
#pragma unroll
              for (int x = 0; x < 32; x += 4)
                *reinterpret_cast<float4 *>(dst + c + x) =
                    make_float4(__uint_as_float(h[x]), __uint_as_float(h[x + 1]), __uint_as_float(h[x + 2]),
                                __uint_as_float(h[x + 3]));
            }
            c += 32;
          } else {
            uint32_t h[16];
            tmem_ld16(trow + static_cast<uint32_t>(c), h);
            if (sub > 0) {
              uint32_t r[16];
              tmem_ld16(trow + TSUM_COL + static_cast<uint32_t>(c), r);
#pragma unroll
              for (int x = 0; x < 16; ++x) h[x] = __float_as_uint(__uint_as_float(h[x]) + __uint_as_float(r[x]));
            }
            if (!last) {
              tmem_st16(trow + TSUM_COL + static_cast<uint32_t>(c), h);
            } else if (grow < g.m_rows) {
#pragma unroll
              for (int x = 0; x < 16; x += 4)
                *reinterpret_cast<float4 *>(dst + c + x) =
                    make_float4(__uint_as_float(h[x]), __uint_as_float(h[x + 1]), __uint_as_float(h[x + 2]),
                                __uint_as_float(h[x + 3]));
            }
            c += 16;
          }
        }
        if (!last) tmem_wait_st();
        tc_fence_before();
        mbar_arrive_cluster(acce_c);
      }
      if (MERGED && warp == TMMA_WARP && lane == 0) {
        if (issuer) mma_commit<true>(done);  // fires in both CTAs once every issued MMA has completed
        if (!mbar_wait(done, 0)) failed = true;
      }
    }
  }
  if (failed) atomicOr(g.status, kStatusWaitLimit);
  tc_fence_before();
  // neither CTA leaves while the other may still arrive on its barriers or the issuer's MMAs may
  // still read its shared memory
  cluster_sync();
  if (warp == TMMA_WARP) {
    tc_fence_after();
    tmem_dealloc<true>(tmem, TMEM_COLS);
  }
}

// Partials of the chirp-major rows -> the signal in channel-major order:
//   sig[k][m][n] = sum_s (P_s[m N_v + k][t bn + nl], P_s[m N_v + k][t bn + bn/2 + nl]) / scale,
// t = n / (bn/2), nl = n % (bn/2); four samples per thread, splits added in order.
// With `accumulate` the result is added to what sig holds (snapshot rays in several chunks).
template <bool F16>
__global__ void taylor_reduce(const float *__restrict__ part, int splits, int nv, int nc, int ns, int bn,
                              float2 *__restrict__ sig, const uint32_t *amax_bits, const uint32_t *terms,
                              int accumulate) {
  if (!expansion_terms(*terms)) return;
  const float inv = F16 ? 1.f / amp_scale<true>(amax_bits) : 1.f;
  const int64_t m_rows = static_cast<int64_t>(nv) * nc;
  const int64_t n_q = m_rows * ns / 4;
  const int64_t plane = m_rows * 2 * ns;
  const int half = bn / 2, ns4 = ns / 4;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_q;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t row = i / ns4;  // k N_c + m
    const int n = static_cast<int>(i - row * ns4) * 4;
    const int k = static_cast<int>(row / nc), m = static_cast<int>(row - static_cast<int64_t>(k) * nc);
    const int64_t prow = static_cast<int64_t>(m) * nv + k;
    const int t = n / half, nl = n - t * half;
    const float *p = part + prow * 2 * ns + t * bn + nl;
    float4 re = *reinterpret_cast<const float4 *>(p), im = *reinterpret_cast<const float4 *>(p + half);
#pragma unroll 6
    for (int s = 1; s < splits; ++s) {
      const float4 a = *reinterpret_cast<const float4 *>(p + s * plane);
      const float4 b = *reinterpret_cast<const float4 *>(p + s * plane + half);
      re.x += a.x; re.y += a.y; re.z += a.z; re.w += a.w;
      im.x += b.x; im.y += b.y; im.z += b.z; im.w += b.w;
    }
    float4 *o = reinterpret_cast<float4 *>(sig + row * ns + n);
    float4 v0 = make_float4(re.x * inv, im.x * inv, re.y * inv, im.y * inv);
    float4 v1 = make_float4(re.z * inv, im.z * inv, re.w * inv, im.w * inv);
    if (accumulate) {
      const float4 a0 = o[0], a1 = o[1];
      v0 = make_float4(a0.x + v0.x, a0.y + v0.y, a0.z + v0.z, a0.w + v0.w);
      v1 = make_float4(a1.x + v1.x, a1.y + v1.y, a1.z + v1.z, a1.w + v1.w);
    }
    o[0] = v0;
    o[1] = v1;
  }
}

__device__ __forceinline__ unsigned long long signed_mag(uint64_t e) {
  return static_cast<int64_t>(e) < 0 ? ~e + 1ull : e;  // |signed Q0.64 word|
}
__device__ __forceinline__ uint32_t signed_mag32(uint32_t e) {
  return static_cast<int32_t>(e) < 0 ? ~e + 1u : e;  // |signed Q0.32 word|
}

// amplitude maximum (FP16 scaling) and largest |eps| and |eps_t| of the scene
__global__ void exact_stats(const float *__restrict__ amp, const uint64_t *__restrict__ eps,
                            const uint64_t *__restrict__ eps_t, int64_t n, bool want_amax, uint32_t *amax_bits,
                            unsigned long long *eps_max, unsigned long long *eps_t_max) {
  uint32_t ma = 0;
  unsigned long long me = 0, mt = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (want_amax) ma = max(ma, __float_as_uint(amp[i]));  // amplitudes are >= 0
    me = max(me, signed_mag(eps[i]));
    mt = max(mt, signed_mag(eps_t[i]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    ma = max(ma, __shfl_xor_sync(0xffffffffu, ma, o));
    me = max(me, __shfl_xor_sync(0xffffffffu, me, o));
    mt = max(mt, __shfl_xor_sync(0xffffffffu, mt, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (want_amax) atomicMax(amax_bits, ma);
    atomicMax(eps_max, me);
    atomicMax(eps_t_max, mt);
  }
}

// P from the truncation bound theta^P / P! <= tol, theta = 2 pi n_h (max|eps| m_h + max|eps_t| t_h)
// (xs_m, xs_t: the factors of the two word maxima); at split precision (two_u = twice the unit
// roundoff) the terms p >= P/2 drop their lo operands when theta^(P/2) / (P/2)! * two_u <= tol_lo.
// With TDM slots there is no per-chirp fallback: P = 0 raises the model-range status bit.
// bound of the Chebyshev remainder after P terms at |x| <= th (see chebyshev_series_terms)
__device__ double chebyshev_bound(double th, int P) {
  double b = 2.0;
  for (int p = 1; p <= P; ++p) b *= 0.5 * th / p;
  const double g = 1.0 - th / (2.0 * (P + 1));
  return g > 0.0 ? b / g : 1e300;
}
// The expansion: Taylor terms when four of them meet tol, else the fewest Chebyshev terms (4, 6,
// 8) that do, else none (P = 0).  lo_high: whether the second K step, which holds only terms of
// order >= P/2, keeps its lo operands (its largest term times 2u above tol_lo).
__global__ void choose_terms(const unsigned long long *eps_max, const unsigned long long *eps_t_max, uint32_t *terms,
                             uint32_t *form, uint32_t *lo_high, double xs_m, double xs_t, double tol, double two_u,
                             double tol_lo, bool tdm, uint32_t *status) {
  const double th = static_cast<double>(*eps_max) * xs_m + static_cast<double>(*eps_t_max) * xs_t;
  const double t2 = th * th, t4 = t2 * t2;
  uint32_t P = 0, ch = 0;
  if (t4 / 24.0 <= tol) {
    P = 4;
  } else {
    for (int c = 4; c <= 8 && P == 0; c += 2)
      if (chebyshev_bound(th, c) <= tol) {
        P = static_cast<uint32_t>(c);
        ch = 1;
      }
  }
  *terms = P;
  *form = ch;
  // largest term of the second K step: Taylor th^2 / 2 at P = 4; Chebyshev 2 (th/2)^(P/2) /
  // (P/2)! (at P = 6 slot 15, term 3 of the stage's first ray, sits in the first K step and keeps
  // its lo operands)
  double high = t2 / 2.0;
  if (ch) {
    high = 2.0;
    for (uint32_t p = 1; p <= P / 2; ++p) high *= 0.5 * th / p;
  }
  *lo_high = (two_u > 0.0 && high * two_u > tol_lo) ? 1u : 0u;
  if (P == 0 && tdm) atomicOr(status, kStatusModelRange);
  // the route mask read back at fetch: bit P (Taylor), bit 16 + P (Chebyshev), bit 0 (none)
  atomicOr(status + 1, P ? (1u << (P + (ch ? 16u : 0u))) : 1u);
}

// Virtual snapshots: a bound on the largest |S - S_ref| over the chunk's rays and every row, S
// the per-sample step of row (m, k = t N_rx + r) and S_ref the ray's reference step of that
// row's 256-row tile (chirp m_c, antennas t_c, r_c), from the signed Q0.32 words, returned in
// Q0.64 units with 2^33 (two word units) added as a margin; and the amplitude maximum (FP16
// scaling).  It reads the phase-word kernel's record of each (ray, chirp):
// s(m) = S(m, t_c, r_c) and the largest and smallest D(m, t, r) = S(m, t, r) - s(m) over the
// antennas, which splits as D = D_tx(t) + D_rx(r), so its extremes are those of the two parts.
// For a tile holding chirp m, S - S_ref = (s(m) - s(m_c)) + D lies between (s(m) - s(m_c)) plus
// the smallest and plus the largest D; the bound is exact for chirps whose rows all fall in one
// tile and at most the rest of their antennas' offsets above it for the others.  Chirps stride
// over the grid's y, groups of four rays over its x (16-byte loads: the stride and the chunk's
// first ray are multiples of four; lanes past cnt are masked), so no thread divides to find its
// chirp.
__global__ void snap_stats(SnapRec rec, int64_t stride, const float *__restrict__ amp, int64_t cnt, int nc, int nv,
                           bool want_amax, uint32_t *amax_bits, unsigned long long *d_max) {
  uint32_t ma = 0, md = 0;
  const int64_t quads = (cnt + 3) / 4;
  const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int m = blockIdx.y; m < nc; m += gridDim.y) {
    const int t0 = (m * nv) >> 8, t1 = (m * nv + nv - 1) >> 8;
    const uint4 *srow = reinterpret_cast<const uint4 *>(rec.s + static_cast<int64_t>(m) * stride);
    const uint4 *hrow = reinterpret_cast<const uint4 *>(rec.d_hi + static_cast<int64_t>(m) * stride);
    const uint4 *lrow = reinterpret_cast<const uint4 *>(rec.d_lo + static_cast<int64_t>(m) * stride);
    for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < quads; q += step) {
      const int64_t live = cnt - 4 * q;  // lanes e < live hold rays
      const uint4 s4 = srow[q], h4 = hrow[q], l4 = lrow[q];
      const uint32_t sm[4] = {s4.x, s4.y, s4.z, s4.w}, hi[4] = {h4.x, h4.y, h4.z, h4.w},
                     lo[4] = {l4.x, l4.y, l4.z, l4.w};
      if (want_amax && m == 0) {
        const uint4 a4 = reinterpret_cast<const uint4 *>(amp)[q];  // amplitudes are >= 0
        const uint32_t av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (e < live) ma = max(ma, av[e]);
      }
      for (int tile = t0; tile <= t1; ++tile) {
        const int mc = min((tile * 256 + 128) / nv, nc - 1);
        const uint4 c4 = reinterpret_cast<const uint4 *>(rec.s + static_cast<int64_t>(mc) * stride)[q];
        const uint32_t sc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const uint32_t base = sm[e] - sc[e];
          if (e < live) md = max(md, max(signed_mag32(base + hi[e]), signed_mag32(base + lo[e])));
        }
      }
    }
  }
  unsigned long long md64 = (static_cast<unsigned long long>(md) << 32) + (1ull << 33);  // Q0.64 units
  for (int o = 16; o > 0; o >>= 1) {
    ma = max(ma, __shfl_xor_sync(0xffffffffu, ma, o));
    md64 = max(md64, __shfl_xor_sync(0xffffffffu, md64, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (want_amax) atomicMax(amax_bits, ma);
    atomicMax(d_max, md64);
  }
}

int sms_t() {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    return cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0 ? n : 148;
  }();
  return sms;
}

struct TShape {
  int bn, mt2, nt, splits, mh;
  int64_t chunk;
};

// Pair tiles of 256 chirp-major rows x bn real columns (512 single pass, 256 split); rays split
// into chunks so that the CTA pairs fill whole waves (at least four) as evenly as possible.
TShape plan_taylor(const Derived &g, int64_t n) {
  TShape s{};
  const bool split = g.precision == SIM_PREC_BF16_SPLIT || g.precision == SIM_PREC_FP16_SPLIT;
  const int cap = split ? 256 : 512;
  s.bn = 2 * g.ns < cap ? 2 * g.ns : cap;
  const int M = g.nv * g.nc;
  s.mt2 = (M + 2 * TBM - 1) / (2 * TBM);
  s.nt = 2 * g.ns / s.bn;
  s.mh = TBM / g.nv + 1;  // |m - m_c| over a 256-row tile
  const int64_t wave = sms_t() / 2;  // CTA pairs per wave
  const int64_t tiles = static_cast<int64_t>(s.mt2) * s.nt;
  const int64_t lo = std::max<int64_t>(1, (4 * wave + tiles - 1) / tiles);
  int64_t best = lo, best_waste = -1, best_slots = 1;
  for (int64_t sp = lo; sp <= 3 * lo; ++sp) {
    const int64_t ctas = tiles * sp, slots = (ctas + wave - 1) / wave * wave, waste = slots - ctas;
    if (best_waste < 0 || waste * best_slots < best_waste * slots) {
      best = sp;
      best_waste = waste;
      best_slots = slots;
    }
  }
  const int64_t max_splits = std::max<int64_t>(1, (n + TMAX_RAYS - 1) / TMAX_RAYS);
  int64_t splits = std::max<int64_t>(1, std::min<int64_t>(best, max_splits));
  int64_t chunk = (n + splits - 1) / splits;
  chunk = std::max<int64_t>(TMAX_RAYS, (chunk + TMAX_RAYS - 1) / TMAX_RAYS * TMAX_RAYS);
  s.chunk = chunk;
  s.splits = static_cast<int>(std::max<int64_t>(1, (n + chunk - 1) / chunk));
  return s;
}

// the expansion needs two-SM tiles of at least 32 complex columns
bool taylor_eligible(const Derived &g) { return g.ns >= 32; }

// dynamic shared memory of a launch: the stages of tiles bn columns wide and the barriers
template <bool SPLIT>
constexpr size_t t_smem(int bn) {
  return t_stages<SPLIT>() * static_cast<size_t>(t_stage_bytes<SPLIT>(bn)) + 8 * (2 * t_stages<SPLIT>() + 3) + 16;
}

template <bool F16, bool SPLIT, int MODE, int PT, bool CH>
void launch_taylor_p(const TShape &sh, const TArgs &a, cudaStream_t s) {
  const size_t smem = t_smem<SPLIT>(sh.bn);
  static std::atomic<uint64_t> done{0};
  once_per_device(done, [] {
    // the widest tile's need (plan_taylor caps bn at 256 split, 512 single pass)
    note_launch(cudaFuncSetAttribute(taylor_sum_kernel<F16, SPLIT, MODE, PT, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(t_smem<SPLIT>(SPLIT ? 256 : 512))));
  });
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(2u * static_cast<unsigned>(sh.mt2 * sh.nt * sh.splits));
  cfg.blockDim = dim3(t_threads<SPLIT, MODE>());
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  note_launch(cudaLaunchKernelEx(&cfg, taylor_sum_kernel<F16, SPLIT, MODE, PT, CH>, a));
}

// the instances of one precision and mode; returns the number of launches
template <bool F16, bool SPLIT, int MODE>
int launch_taylor(const TShape &sh, const TArgs &a, cudaStream_t s) {
  if constexpr (SPLIT) {
    launch_taylor_p<F16, SPLIT, MODE, 4, false>(sh, a, s);
    launch_taylor_p<F16, SPLIT, MODE, 4, true>(sh, a, s);
    launch_taylor_p<F16, SPLIT, MODE, 6, true>(sh, a, s);
    launch_taylor_p<F16, SPLIT, MODE, 8, true>(sh, a, s);
    return 4;
  } else {
    launch_taylor_p<F16, SPLIT, MODE, 0, false>(sh, a, s);  // Taylor terms
    launch_taylor_p<F16, SPLIT, MODE, 0, true>(sh, a, s);   // Chebyshev terms
    return 2;
  }
}

template <int MODE>
int launch_taylor_mode(bool f16, bool split, const TShape &sh, const TArgs &a, cudaStream_t s) {
  if (f16) return split ? launch_taylor<true, true, MODE>(sh, a, s) : launch_taylor<true, false, MODE>(sh, a, s);
  return split ? launch_taylor<false, true, MODE>(sh, a, s) : launch_taylor<false, false, MODE>(sh, a, s);
}

}  // namespace

int64_t exact_tensor_workspace_bytes(const Derived &g, int64_t n) {
  const int64_t chirp = exact_workspace_bytes(g, n);
  if (!taylor_eligible(g)) return chirp;
  const TShape t = plan_taylor(g, n);
  const int64_t tb = static_cast<int64_t>(kHeader) + static_cast<int64_t>(t.splits) * g.nv * g.nc * 2 * g.ns * 4;
  return std::max(chirp, tb);
}

int launch_exact_tensor(const Derived &g, RaysPrep p, int64_t n, float2 *sig, void *workspace, uint32_t *status,
                        cudaStream_t s, cudaEvent_t after_main) {
  if (!taylor_eligible(g) || n <= 0) return launch_exact_sum(g, p, n, sig, workspace, status, s, after_main);
  const TShape sh = plan_taylor(g, n);
  const bool f16 = g.precision == SIM_PREC_FP16 || g.precision == SIM_PREC_FP16_SPLIT;
  const bool split = g.precision == SIM_PREC_BF16_SPLIT || g.precision == SIM_PREC_FP16_SPLIT;
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  uint32_t *amax = reinterpret_cast<uint32_t *>(ws);
  uint32_t *terms = reinterpret_cast<uint32_t *>(ws + kOffTerms);
  unsigned long long *eps_max = reinterpret_cast<unsigned long long *>(ws + kOffEpsMax);
  uint32_t *lo_high = reinterpret_cast<uint32_t *>(ws + kOffLoHigh);
  uint32_t *form = reinterpret_cast<uint32_t *>(ws + kOffForm);
  unsigned long long *eps_t_max = reinterpret_cast<unsigned long long *>(ws + kOffEpsTMax);
  const bool tdm = g.tslot != 0.0;
  const int t_c = g.ntx / 2, t_h = std::max(t_c, g.ntx - 1 - t_c);  // |t - t_c| <= t_h
  int kernels = 0;
  cudaMemsetAsync(ws, 0, 64, s);
  exact_stats<<<2 * sms_t(), 256, 0, s>>>(p.amp, p.eps, p.eps_t, n, f16, amax, eps_max, eps_t_max);
  // theta = 2 pi n_h (max|eps| m_h + max|eps_t| t_h) with eps in cycles (the word times 2^-64)
  const double xs = 6.283185307179586 * (sh.bn / 4) * 5.421010862427522e-20;
  // unit roundoff 2^-11 (FP16), 2^-8 (BF16); single pass has no lo operands to drop
  const double two_u = split ? (f16 ? 9.765625e-4 : 7.8125e-3) : 0.0;
  choose_terms<<<1, 1, 0, s>>>(eps_max, eps_t_max, terms, form, lo_high, xs * sh.mh, xs * t_h, split ? 1e-6 : 1e-5,
                               two_u, 2e-6, tdm, status);
  kernels += 2;
  TArgs a{};
  a.p = p;
  a.n_rays = n;
  a.chunk = sh.chunk;
  a.nc = g.nc;
  a.ns = g.ns;
  a.nv = g.nv;
  a.nrx = g.nrx;
  a.m_rows = g.nv * g.nc;
  a.t_c = t_c;
  a.bn = sh.bn;
  a.mt2 = sh.mt2;
  a.nt = sh.nt;
  a.partials = reinterpret_cast<float *>(ws + kHeader);
  a.amax_bits = amax;
  a.terms = terms;
  a.lo_high = lo_high;
  a.form = form;
  a.status = status;
  kernels += tdm ? launch_taylor_mode<kExactTdm>(f16, split, sh, a, s) : launch_taylor_mode<kExact>(f16, split, sh, a, s);
  // the per-chirp kernel, which returns at once unless P = 0 (it has no slot term: not with TDM)
  if (!tdm) kernels += launch_exact_main(g, p, n, workspace, status, s, terms);
  if (after_main) cudaEventRecord(after_main, s);
  const int rb = 4 * sms_t();
  if (f16)
    taylor_reduce<true><<<rb, 256, 0, s>>>(a.partials, sh.splits, g.nv, g.nc, g.ns, sh.bn, sig, amax, terms, 0);
  else
    taylor_reduce<false><<<rb, 256, 0, s>>>(a.partials, sh.splits, g.nv, g.nc, g.ns, sh.bn, sig, amax, terms, 0);
  ++kernels;
  if (!tdm) kernels += launch_exact_reduce(g, n, sig, workspace, s, terms);
  return kernels;
}

int64_t snap_tensor_workspace_bytes(const Derived &g, int64_t chunk) {
  if (!taylor_eligible(g) || chunk <= 0) return 0;
  const TShape t = plan_taylor(g, chunk);
  return static_cast<int64_t>(kHeader) + static_cast<int64_t>(t.splits) * g.nv * g.nc * 2 * g.ns * 4;
}

// Virtual snapshots on tensor cores, one chunk of rays: the same per-tile expansion with each
// row's exact phase words, S_ref the ray's step at the tile's centre chirp and antennas,
//   A_p[row, i] = a_i e^{2 pi j (C_row,i + n_c delta)} (j 2 pi n_h delta)^p / p!,
//   B_p[i, n]   = e^{2 pi j n S_ref,i} (n' / n_h)^p,      delta = S_row,i - S_ref,i,
// P from the chunk's largest |delta|; beyond the bound the direct pair sum runs instead (both
// are launched, each returns at once when the other owns the chunk).  Adds to sig when
// `accumulate`.
int launch_snap_tensor(const Derived &g, const uint2 *w_tx, const uint2 *w_rx, SnapRec rec, int64_t stride,
                       const float *amp, int64_t cnt, bool accumulate, float2 *sig, void *workspace, void *pair_ws,
                       uint32_t *status, cudaStream_t s) {
  if (!taylor_eligible(g) || cnt <= 0)
    return launch_pair_sum(g, w_tx, w_rx, amp, cnt, stride, accumulate, sig, pair_ws, nullptr, s);
  const TShape sh = plan_taylor(g, cnt);
  const bool f16 = g.precision == SIM_PREC_FP16 || g.precision == SIM_PREC_FP16_SPLIT;
  const bool split = g.precision == SIM_PREC_BF16_SPLIT || g.precision == SIM_PREC_FP16_SPLIT;
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  uint32_t *amax = reinterpret_cast<uint32_t *>(ws);
  uint32_t *terms = reinterpret_cast<uint32_t *>(ws + kOffTerms);
  unsigned long long *d_max = reinterpret_cast<unsigned long long *>(ws + kOffEpsMax);
  uint32_t *lo_high = reinterpret_cast<uint32_t *>(ws + kOffLoHigh);
  uint32_t *form = reinterpret_cast<uint32_t *>(ws + kOffForm);
  unsigned long long *none = reinterpret_cast<unsigned long long *>(ws + kOffEpsTMax);  // stays 0
  const int t_c = snap_ref_tx(g), r_c = snap_ref_rx(g);
  int kernels = 0;
  cudaMemsetAsync(ws, 0, 64, s);
  snap_stats<<<dim3(2u * static_cast<unsigned>(sms_t()), static_cast<unsigned>(std::min(g.nc, 4))), 256, 0, s>>>(
      rec, stride, amp, cnt, g.nc, g.nv, f16, amax, d_max);
  // theta = 2 pi n_h max|delta|, delta in cycles per sample (the word times 2^-64)
  const double xs = 6.283185307179586 * (sh.bn / 4) * 5.421010862427522e-20;
  const double two_u = split ? (f16 ? 9.765625e-4 : 7.8125e-3) : 0.0;
  choose_terms<<<1, 1, 0, s>>>(d_max, none, terms, form, lo_high, xs, 0.0, split ? 1e-6 : 1e-5, two_u, 2e-6, false,
                               status);
  kernels += 2;
  TArgs a{};
  a.w_tx = w_tx;
  a.w_rx = w_rx;
  a.stride = stride;
  a.samp = amp;
  a.ntx = g.ntx;
  a.r_c = r_c;
  a.n_rays = cnt;
  a.chunk = sh.chunk;
  a.nc = g.nc;
  a.ns = g.ns;
  a.nv = g.nv;
  a.nrx = g.nrx;
  a.m_rows = g.nv * g.nc;
  a.t_c = t_c;
  a.bn = sh.bn;
  a.mt2 = sh.mt2;
  a.nt = sh.nt;
  a.partials = reinterpret_cast<float *>(ws + kHeader);
  a.amax_bits = amax;
  a.terms = terms;
  a.lo_high = lo_high;
  a.form = form;
  a.status = status;
  kernels += launch_taylor_mode<kSnap>(f16, split, sh, a, s);
  const int rb = 4 * sms_t();
  if (f16)
    taylor_reduce<true><<<rb, 256, 0, s>>>(a.partials, sh.splits, g.nv, g.nc, g.ns, sh.bn, sig, amax, terms,
                                           accumulate ? 1 : 0);
  else
    taylor_reduce<false><<<rb, 256, 0, s>>>(a.partials, sh.splits, g.nv, g.nc, g.ns, sh.bn, sig, amax, terms,
                                            accumulate ? 1 : 0);
  ++kernels;
  // the direct pair sum, which returns at once unless P = 0
  kernels += launch_pair_sum(g, w_tx, w_rx, amp, cnt, stride, accumulate, sig, pair_ws, terms, s);
  return kernels;
}

}  // namespace rs
