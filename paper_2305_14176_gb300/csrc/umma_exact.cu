// The exact signal model on tensor cores (arXiv 2305.14176, Sec. II-A, Eq. 2 with the
// range-migration product mu t (tau_i(j) - tau_i(0)) kept).
//
// The exact phase adds n m eps_i to the separable one, so the cube is no longer one product
// over rays; for a fixed chirp m it still is, with the samples as rows and the channels as
// columns:
//   s[k][m][n] = sum_i X_m[n, i] C_m[i, k]
//   X_m[n, i] = exp(2 pi j n (nu_r,i + m eps_i))                 (samples x rays)
//   C_m[i, k] = a_i exp(2 pi j (carrier_i + k nu_a,i + m nu_d,i))  (rays x channels)
// One work unit is (chirp m, 128-sample tile, channel tile of NT <= 64 columns, ray chunk):
// M = 128 samples, N = NT channels (a multiple of 16; columns past N_v are zero), planar K
// order as in the separable kernel (Re D += X_re C_re - X_im C_im, Im D += X_re C_im + X_im C_re,
// split precision adds the hi / lo cross terms).  Producer warps synthesise both operands in
// shared memory: X along the samples by 32-sample complex steps whose phasor e^{2 pi j 32
// (nu_r + m eps)} is taken once per ray and stage, C per channel from its exact Q0.64 phase.
// Drain warps keep the FP32 running sum of split precision in tensor memory, as in the
// separable kernel, and store each unit's FP32 partial; a second kernel adds the partials.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "tcgen05.cuh"

namespace rs {
namespace {

constexpr int XM = 128;                 // sample rows per tile (TMEM lanes)
constexpr int XK = 32;                  // rays per stage
constexpr int XNPROD = 384;             // producer threads: 3 groups of 128
constexpr int XGROUPS = 3;
constexpr int XGSIZE = XNPROD / XGROUPS;
constexpr int XMMA_WARP = XNPROD / 32;
constexpr int XNDRAIN = 128;
constexpr int XTHREADS = XNPROD + 32 + XNDRAIN;
constexpr int XMAX_ST = 6;              // barrier slots (stages in flight at most)
constexpr int XSUBST_SPLIT = 16;        // stages per tensor-core accumulation chain (split)
constexpr uint32_t XSUM_COL = 256;      // TMEM column of the running sum
constexpr int kMaxDynSmemX = 232448 - 8192;

struct XArgs {
  RaysPrep p;
  int64_t n_rays, chunk;
  int nc, ns, nv, nrx;
  int nt;                   // channel columns per tile (multiple of 16, <= 64)
  int mtiles, ktiles;       // sample tiles, channel tiles
  int nst;                  // pipeline stages
  uint32_t stage_bytes;
  float *partials;          // [split][N_v][N_c][N_s] complex64
  const uint32_t *amax_bits;
  uint32_t *status;
  const uint32_t *gate;     // may be null; when it holds a term count the expanded kernel owns the scene
};

// the expanded tensor-core kernel (umma_taylor.cu) has taken the scene
__device__ __forceinline__ bool gated_off(const uint32_t *gate) {
  if (!gate) return false;
  return expansion_terms(*gate);
}

struct XStage {               // per-ray words of one stage
  uint64_t car[XK], nur[XK], nua[XK], nutx[XK];
  float2 w[XK];               // e^{2 pi j 32 (nu_r + m eps)}
  float amp[XK];
};

__device__ __forceinline__ void xgroup_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(XGSIZE) : "memory");
}

// The per-ray words of one stage for chirp m, fetched by 32 threads of the group (one ray
// each) one stage ahead of their use; rays past the chunk read as silent.
struct XWords {
  uint64_t car, nur, nua, nutx;
  float amp;
};

__device__ __forceinline__ XWords xfetch(const XArgs &g, int64_t ray0, int64_t k_hi, int gt, uint64_t m) {
  XWords w{0, 0, 0, 0, 0.f};
  const int64_t ray = ray0 + gt;
  if (gt < XK && ray < k_hi) {
    w.car = g.p.carrier[ray] + m * g.p.nu_d[ray];
    w.nur = g.p.nu_r[ray] + m * g.p.eps[ray];
    w.nua = g.p.nu_a[ray];
    w.nutx = g.p.nu_tx[ray];
    w.amp = g.p.amp[ray];
  }
  return w;
}

__device__ __forceinline__ void xstore(XStage &sr, int gt, const XWords &w) {
  if (gt >= XK) return;
  sr.car[gt] = w.car;
  sr.nur[gt] = w.nur;
  sr.nua[gt] = w.nua;
  sr.nutx[gt] = w.nutx;
  sr.amp[gt] = w.amp;
  const float f = static_cast<float>(static_cast<int64_t>(w.nur * 32ull)) * 0x1p-64f;  // cycles in [-1/2, 1/2)
  float sn, cs;
  sincospif(2.0f * f, &sn, &cs);
  sr.w[gt] = make_float2(cs, sn);
}

// One stage of operands: X_re | X_im (128 sample rows x 32 rays) | C_re | C_im (NT channel
// rows) | the same for lo.  Thread (octet o = t / 32, lane j = t % 32): samples j + 32 l and
// channels j + 32 l below NT.
template <bool F16, bool SPLIT>
__device__ __forceinline__ void xproduce(const XArgs &g, const XStage &sr, uint8_t *stage, int gt, int n0, int k0,
                                         float scale) {
  const int NT = g.nt;
  const uint32_t x_half = XM * XK * 2, c_half = static_cast<uint32_t>(NT) * XK * 2;
  const uint32_t lo = SPLIT ? 2 * x_half + 2 * c_half : 0;
  uint8_t *x_re = stage, *x_im = stage + x_half, *c_re = stage + 2 * x_half, *c_im = c_re + c_half;
  const int o = gt >> 5, j = gt & 31;
  {
    // ---- X: samples n0 + j + 32 l
    uint32_t off = o * (XM * 16) + (j >> 3) * 128 + (j & 7) * 16;
    float2 z[OCT], w[OCT];
    const uint64_t n = static_cast<uint64_t>(n0 + j);
#pragma unroll
    for (int q = 0; q < OCT; ++q) {
      const int i = o * OCT + q;
      float sn, cs;
      __sincosf(q64_to_rad(n * sr.nur[i]), &sn, &cs);
      z[q] = make_float2(cs, sn);
      w[q] = sr.w[i];
    }
#pragma unroll 1
    for (int l = 0; l < XM / 32; ++l) {
      if (l > 0) {
#pragma unroll
        for (int q = 0; q < OCT; ++q) z[q] = cmulf(z[q], w[q]);  // 32 samples on
      }
      if (n0 + j + 32 * l >= g.ns) {
#pragma unroll
        for (int q = 0; q < OCT; ++q) z[q] = make_float2(0.f, 0.f);
      }
      put_octet<F16, SPLIT>(z, x_re + off, x_im + off, x_re + lo + off, x_im + lo + off);
      off += 512;
    }
  }
  // ---- C: channels k0 + c for c = j, j + 32, .. below NT (zero past N_v)
  for (int c = j; c < NT; c += 32) {
    const uint32_t off = o * static_cast<uint32_t>(NT * 16) + (c >> 3) * 128 + (c & 7) * 16;
    const int k = k0 + c;
    float2 z[OCT];
    if (k < g.nv) {
      const uint64_t tq = static_cast<uint64_t>(k / g.nrx), rq = static_cast<uint64_t>(k % g.nrx);
#pragma unroll
      for (int q = 0; q < OCT; ++q) {
        const int i = o * OCT + q;
        float sn, cs;
        __sincosf(q64_to_rad(sr.car[i] + tq * sr.nutx[i] + rq * sr.nua[i]), &sn, &cs);
        const float am = sr.amp[i] * scale;
        z[q] = make_float2(am * cs, am * sn);
      }
    } else {
#pragma unroll
      for (int q = 0; q < OCT; ++q) z[q] = make_float2(0.f, 0.f);
    }
    put_octet<F16, SPLIT>(z, c_re + off, c_im + off, c_re + lo + off, c_im + lo + off);
  }
}

template <bool F16, bool SPLIT>
__global__ void __launch_bounds__(XTHREADS, 1) exact_sum_kernel(XArgs g) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ XStage s_rays[XGROUPS];
  __shared__ uint64_t bars[2 * XMAX_ST + 3];
  __shared__ uint32_t tmem_holder;
  if (gated_off(g.gate)) return;  // uniform over the grid, before any barrier or allocation
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nst = g.nst;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + XMAX_ST);
  const uint32_t accf = smem_u32(bars + 2 * XMAX_ST), acce = smem_u32(bars + 2 * XMAX_ST + 1);
  const uint32_t done = smem_u32(bars + 2 * XMAX_ST + 2);
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(full0 + 8 * s, XGSIZE);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, XNDRAIN);
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == XMMA_WARP) tmem_alloc<false>(smem_u32(&tmem_holder), 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_holder;

  // unit = ((split * N_c + m) * ktiles + kt) * mtiles + mt
  int u = static_cast<int>(blockIdx.x);
  const int mt = u % g.mtiles;
  u /= g.mtiles;
  const int kt = u % g.ktiles;
  u /= g.ktiles;
  const int m = u % g.nc;
  const int split = u / g.nc;
  const int n0 = mt * XM, k0 = kt * g.nt;
  const int64_t k_lo = static_cast<int64_t>(split) * g.chunk;
  const int64_t k_hi = k_lo + g.chunk < g.n_rays ? k_lo + g.chunk : g.n_rays;
  const int n_stages = k_hi > k_lo ? static_cast<int>((k_hi - k_lo + XK - 1) / XK) : 0;
  const int SUBST = SPLIT ? XSUBST_SPLIT : (n_stages > 0 ? n_stages : 1);
  const int n_sub = (n_stages + SUBST - 1) / SUBST;
  bool failed = false;
  uint8_t *base = smem;

  if (warp < XMMA_WARP) {
    // ---------------- producers: group grp builds stages grp, grp + 3, ...
    const int grp = warp / (XGSIZE / 32), gt = threadIdx.x % XGSIZE;
    const float scale = amp_scale<F16>(g.amax_bits);
    const uint64_t mu = static_cast<uint64_t>(m);
    XWords nxt = xfetch(g, k_lo + static_cast<int64_t>(grp) * XK, k_hi, gt, mu);
    for (int st = grp; st < n_stages; st += XGROUPS) {
      const int s = st % nst;
      xstore(s_rays[grp], gt, nxt);
      if (st + XGROUPS < n_stages) nxt = xfetch(g, k_lo + static_cast<int64_t>(st + XGROUPS) * XK, k_hi, gt, mu);
      // the stage slot is free, and the group's ray words are visible; a wait that ran out in
      // any thread takes the whole group out of the loop
      const bool slot_ok = st < nst || mbar_wait(empty0 + 8 * s, ((st / nst) - 1) & 1);
      if (bar_any(grp + 1, XGSIZE, !slot_ok)) {
        failed = true;
        break;
      }
      xproduce<F16, SPLIT>(g, s_rays[grp], base + s * g.stage_bytes, gt, n0, k0, scale);
      fence_proxy_async();
      mbar_arrive(full0 + 8 * s);
      xgroup_sync(grp);  // s_rays[grp] is rewritten next round
    }
  } else if (warp == XMMA_WARP) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t sbase = smem_u32(base);
      const int NT = g.nt;
      const uint32_t idesc = make_idesc(F16, XM, NT);
      const uint32_t ineg = idesc | (1u << 14);
      const uint32_t lbo_x = XM * 16, lbo_c = static_cast<uint32_t>(NT) * 16;
      const uint32_t x_half = XM * XK * 2, c_half = static_cast<uint32_t>(NT) * XK * 2;
      const uint32_t lo = 2 * x_half + 2 * c_half;
      // K step kh accumulates into set kh (Re at 2 NT kh, Im at 2 NT kh + NT): the MMAs of a
      // stage form four independent chains instead of two; the drain adds the sets
      const uint32_t t_re0 = tmem, t_im0 = tmem + static_cast<uint32_t>(NT);
      bool open = false;
      for (int st = 0; st < n_stages; ++st) {
        const int s = st % nst;
        const int gc = st / SUBST;
        const bool first = (st % SUBST) == 0;
        if (first && gc > 0 && !mbar_wait(acce, (gc - 1) & 1)) {
          failed = true;
          break;
        }
        if (!mbar_wait(full0 + 8 * s, (st / nst) & 1)) {
          failed = true;
          break;
        }
        tc_fence_after();
        const uint32_t sb = sbase + s * g.stage_bytes;
        const uint32_t xr = sb, xi = sb + x_half, cr = sb + 2 * x_half, ci = cr + c_half;
#pragma unroll
        for (int kh = 0; kh < XK / 16; ++kh) {
          const uint32_t acc = first ? 0u : 1u;
          const uint32_t t_re = t_re0 + 2 * NT * kh, t_im = t_im0 + 2 * NT * kh;
          const uint32_t ox = kh * 2 * lbo_x, oc = kh * 2 * lbo_c;
          const uint64_t dxr = make_sdesc(xr + ox, lbo_x, 128), dxi = make_sdesc(xi + ox, lbo_x, 128);
          const uint64_t dcr = make_sdesc(cr + oc, lbo_c, 128), dci = make_sdesc(ci + oc, lbo_c, 128);
          mma_f16<false>(t_re, dxr, dcr, idesc, acc);
          mma_f16<false>(t_im, dxr, dci, idesc, acc);
          mma_f16<false>(t_re, dxi, dci, ineg, 1u);
          mma_f16<false>(t_im, dxi, dcr, idesc, 1u);
          if constexpr (SPLIT) {
            const uint64_t lxr = make_sdesc(xr + lo + ox, lbo_x, 128), lxi = make_sdesc(xi + lo + ox, lbo_x, 128);
            const uint64_t lcr = make_sdesc(cr + lo + oc, lbo_c, 128), lci = make_sdesc(ci + lo + oc, lbo_c, 128);
            mma_f16<false>(t_re, dxr, lcr, idesc, 1u);
            mma_f16<false>(t_im, dxr, lci, idesc, 1u);
            mma_f16<false>(t_re, lxr, dcr, idesc, 1u);
            mma_f16<false>(t_im, lxr, dci, idesc, 1u);
            mma_f16<false>(t_re, dxi, lci, ineg, 1u);
            mma_f16<false>(t_im, dxi, lcr, idesc, 1u);
            mma_f16<false>(t_re, lxi, dci, ineg, 1u);
            mma_f16<false>(t_im, lxi, dcr, idesc, 1u);
          }
        }
        open = true;
        mma_commit<false>(empty0 + 8 * s);
        if ((st % SUBST) == SUBST - 1 || st == n_stages - 1) {
          mma_commit<false>(accf);
          open = false;
        }
      }
      if (open) mma_commit<false>(accf);
      mma_commit<false>(done);
      if (!mbar_wait(done, 0)) failed = true;
    }
  } else {
    // ---------------- drain: TMEM lane quarter (warp % 4) = samples; columns = channels
    const int q = warp & 3;
    const int n = n0 + q * 32 + lane;
    const uint32_t trow = tmem + (static_cast<uint32_t>(q * 32) << 16);
    const int NT = g.nt;
    const int kmax = NT < g.nv - k0 ? NT : g.nv - k0;
    float2 *dst = reinterpret_cast<float2 *>(g.partials) +
                  ((static_cast<int64_t>(split) * g.nv + k0) * g.nc + m) * g.ns + n;
    const int64_t kstride = static_cast<int64_t>(g.nc) * g.ns;
    if (n_stages == 0 && n < g.ns)
      for (int c = 0; c < kmax; ++c) dst[c * kstride] = make_float2(0.f, 0.f);
    for (int sub = 0; sub < n_sub; ++sub) {
      if (!mbar_wait_sleep(accf, sub & 1)) {
        failed = true;
        break;
      }
      tc_fence_after();
      const bool last = sub == n_sub - 1;
      for (int c0 = 0; c0 < NT; c0 += 16) {
        uint32_t re[16], im[16], re1[16], im1[16];
        tmem_ld16(trow + static_cast<uint32_t>(c0), re);
        tmem_ld16(trow + static_cast<uint32_t>(NT + c0), im);
        tmem_ld16(trow + static_cast<uint32_t>(2 * NT + c0), re1);
        tmem_ld16(trow + static_cast<uint32_t>(3 * NT + c0), im1);
#pragma unroll
        for (int x = 0; x < 16; ++x) {
          re[x] = __float_as_uint(__uint_as_float(re[x]) + __uint_as_float(re1[x]));
          im[x] = __float_as_uint(__uint_as_float(im[x]) + __uint_as_float(im1[x]));
        }
        if (sub > 0) {
          uint32_t r1[16], r2[16];
          tmem_ld16(trow + XSUM_COL + static_cast<uint32_t>(c0), r1);
          tmem_ld16(trow + XSUM_COL + static_cast<uint32_t>(NT + c0), r2);
#pragma unroll
          for (int x = 0; x < 16; ++x) {
            re[x] = __float_as_uint(__uint_as_float(re[x]) + __uint_as_float(r1[x]));
            im[x] = __float_as_uint(__uint_as_float(im[x]) + __uint_as_float(r2[x]));
          }
        }
        if (!last) {
          tmem_st16(trow + XSUM_COL + static_cast<uint32_t>(c0), re);
          tmem_st16(trow + XSUM_COL + static_cast<uint32_t>(NT + c0), im);
        } else if (n < g.ns) {
#pragma unroll
          for (int x = 0; x < 16; ++x)
            if (c0 + x < kmax)
              dst[(c0 + x) * kstride] = make_float2(__uint_as_float(re[x]), __uint_as_float(im[x]));
        }
      }
      if (!last) tmem_wait_st();
      tc_fence_before();
      mbar_arrive(acce);
    }
  }
  if (failed) atomicOr(g.status, kStatusWaitLimit);
  tc_fence_before();
  __syncthreads();
  if (warp == XMMA_WARP) {
    tc_fence_after();
    tmem_dealloc<false>(tmem, 512);
  }
}

// sig[i] = sum_s P_s[i] / scale, splits in order
template <bool F16>
__global__ void exact_reduce(const float2 *__restrict__ part, int splits, int64_t n_sig, float2 *__restrict__ sig,
                             const uint32_t *amax_bits, const uint32_t *gate) {
  if (gated_off(gate)) return;
  const float inv = F16 ? 1.f / amp_scale<true>(amax_bits) : 1.f;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_sig;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float2 v = part[i];
    for (int s = 1; s < splits; ++s) {
      const float2 p = part[s * n_sig + i];
      v.x += p.x;
      v.y += p.y;
    }
    sig[i] = make_float2(v.x * inv, v.y * inv);
  }
}

__global__ void exact_amax(const float *__restrict__ amp, int64_t n, uint32_t *amax_bits) {
  uint32_t mx = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    mx = max(mx, __float_as_uint(amp[i]));
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax_bits, mx);
}

int sms_count() {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    return cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0 ? n : 148;
  }();
  return sms;
}

struct XShape {
  int nt, mtiles, ktiles, splits, nst;
  int64_t chunk;
  uint32_t stage_bytes;
};

XShape plan_exact(const Derived &g, int64_t n) {
  XShape s{};
  const bool split = g.precision == SIM_PREC_BF16_SPLIT || g.precision == SIM_PREC_FP16_SPLIT;
  int nt = (g.nv + 15) / 16 * 16;
  s.nt = nt < 64 ? nt : 64;  // two accumulator sets of 2 NT columns below the running sum
  s.mtiles = (g.ns + XM - 1) / XM;
  s.ktiles = (g.nv + s.nt - 1) / s.nt;
  s.stage_bytes = static_cast<uint32_t>(XM * XK * 4 + s.nt * XK * 4) * (split ? 2u : 1u);
  s.nst = std::min<int>(XMAX_ST, static_cast<int>((kMaxDynSmemX - 1024) / s.stage_bytes));
  const int sms = sms_count();
  const int64_t tiles = static_cast<int64_t>(g.nc) * s.mtiles * s.ktiles;
  const int64_t max_splits = std::max<int64_t>(1, (n + XK - 1) / XK);
  // enough units for four waves, split counts that fill the last wave best
  const int64_t lo = std::max<int64_t>(1, (4 * sms + tiles - 1) / tiles);
  int64_t best = lo, best_waste = -1, best_slots = 1;
  for (int64_t sp = lo; sp <= 3 * lo; ++sp) {
    const int64_t ctas = tiles * sp, slots = (ctas + sms - 1) / sms * sms, waste = slots - ctas;
    if (best_waste < 0 || waste * best_slots < best_waste * slots) {
      best = sp;
      best_waste = waste;
      best_slots = slots;
    }
  }
  int64_t splits = std::min<int64_t>(best, max_splits);
  int64_t chunk = (n + splits - 1) / splits;
  chunk = std::max<int64_t>(XK, (chunk + XK - 1) / XK * XK);
  s.chunk = chunk;
  s.splits = static_cast<int>(std::max<int64_t>(1, (n + chunk - 1) / chunk));
  return s;
}

}  // namespace

int64_t exact_workspace_bytes(const Derived &g, int64_t n) {
  const XShape s = plan_exact(g, n);
  return 256 + static_cast<int64_t>(s.splits) * g.n_sig * 8;
}

int launch_exact_main(const Derived &g, RaysPrep p, int64_t n, void *workspace, uint32_t *status, cudaStream_t s,
                      const uint32_t *gate) {
  const XShape sh = plan_exact(g, n);
  const bool f16 = g.precision == SIM_PREC_FP16 || g.precision == SIM_PREC_FP16_SPLIT;
  const bool split = g.precision == SIM_PREC_BF16_SPLIT || g.precision == SIM_PREC_FP16_SPLIT;
  XArgs a{};
  a.p = p;
  a.n_rays = n;
  a.chunk = sh.chunk;
  a.nc = g.nc;
  a.ns = g.ns;
  a.nv = g.nv;
  a.nrx = g.nrx;
  a.nt = sh.nt;
  a.mtiles = sh.mtiles;
  a.ktiles = sh.ktiles;
  a.nst = sh.nst;
  a.stage_bytes = sh.stage_bytes;
  a.partials = reinterpret_cast<float *>(static_cast<uint8_t *>(workspace) + 256);
  a.amax_bits = static_cast<uint32_t *>(workspace);
  a.status = status;
  a.gate = gate;
  const size_t smem = static_cast<size_t>(sh.nst) * sh.stage_bytes;
  const unsigned grid = static_cast<unsigned>(static_cast<int64_t>(g.nc) * sh.mtiles * sh.ktiles * sh.splits);
#define RS_EXACT(F, SP)                                                                                      \
  do {                                                                                                       \
    note_launch(cudaFuncSetAttribute(exact_sum_kernel<F, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                     kMaxDynSmemX));                                                       \
    exact_sum_kernel<F, SP><<<grid, XTHREADS, smem, s>>>(a);                                                 \
  } while (0)
  if (f16) {
    if (split) RS_EXACT(true, true);
    else RS_EXACT(true, false);
  } else {
    if (split) RS_EXACT(false, true);
    else RS_EXACT(false, false);
  }
#undef RS_EXACT
  return 1;
}

int launch_exact_reduce(const Derived &g, int64_t n, float2 *sig, void *workspace, cudaStream_t s,
                        const uint32_t *gate) {
  const XShape sh = plan_exact(g, n);
  const bool f16 = g.precision == SIM_PREC_FP16 || g.precision == SIM_PREC_FP16_SPLIT;
  const uint32_t *amax = static_cast<uint32_t *>(workspace);
  const float2 *partials = reinterpret_cast<const float2 *>(static_cast<uint8_t *>(workspace) + 256);
  const int rb = 4 * sms_count();
  if (f16) exact_reduce<true><<<rb, 256, 0, s>>>(partials, sh.splits, g.n_sig, sig, amax, gate);
  else exact_reduce<false><<<rb, 256, 0, s>>>(partials, sh.splits, g.n_sig, sig, amax, gate);
  return 1;
}

int launch_exact_sum(const Derived &g, RaysPrep p, int64_t n, float2 *sig, void *workspace, uint32_t *status,
                     cudaStream_t s, cudaEvent_t after_main) {
  const bool f16 = g.precision == SIM_PREC_FP16 || g.precision == SIM_PREC_FP16_SPLIT;
  uint32_t *amax = static_cast<uint32_t *>(workspace);
  int kernels = 0;
  cudaMemsetAsync(amax, 0, 4, s);
  if (f16 && n > 0) {
    exact_amax<<<2 * sms_count(), 256, 0, s>>>(p.amp, n, amax);
    ++kernels;
  }
  kernels += launch_exact_main(g, p, n, workspace, status, s, nullptr);
  if (after_main) cudaEventRecord(after_main, s);
  kernels += launch_exact_reduce(g, n, sig, workspace, s, nullptr);
  return kernels;
}

}  // namespace rs
