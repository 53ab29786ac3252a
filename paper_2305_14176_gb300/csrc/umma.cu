// K_b1: the ray sum as a tensor-core GEMM (arXiv 2305.14176, Sec. II-A, Eq. 2).
//
// With the separable phase, the beat cube is a complex product over rays:
//   S[row, n] = sum_i A[row, i] B[i, n],   row = (k, m) = k N_c + m, k = t N_rx + r
//   A[row, i] = a_i exp(2 pi j (carrier_i + t nu_tx,i + r nu_a,i + m nu_d,i))
//   B[i, n]   = exp(2 pi j n nu_r,i)
// computed in planar form: per 16-ray K step, four real MMAs of N = NC complex columns,
//   Re S += A_re B_re - A_im B_im   (the minus by the instruction descriptor's negate-B bit)
//   Im S += A_re B_im + A_im B_re
// into two TMEM accumulator blocks (Re, Im).  Split precision adds the cross terms
// A_hi B_lo + A_lo B_hi of each product: twelve MMAs per K step.
//
// Operands are never stored in HBM: three groups of producer warps synthesise the A and B
// tiles of a stage of 32 rays straight into shared memory (Q0.64 phases from the prep
// kernel, one FP32 sin/cos per phasor chain, then FP32 complex steps of 32 chirps or 32
// samples with the prep kernel's step phasors (exact Q0.64 phase, ~1.5 ulp), rounded to BF16 or FP16 and
// optionally split into hi + lo), in the no-swizzle K-major core-matrix layout.  One thread
// issues tcgen05.mma (kind::f16, FP32 accumulation in tensor memory).  Four drain warps add
// each finished accumulation chain (at most 16 stages, 512 rays, for split precision: the
// tensor core's accumulate is not round-to-nearest, so long chains lose accuracy) to an FP32
// running sum kept in tensor memory, and store the sum when the unit ends.
//
// Work is split over rays (split-K): each unit sums one chunk of rays for one 128-row x
// BN-column tile and writes an FP32 partial; a second kernel adds the partials in chunk
// order.  The decomposition depends only on the scene's own shape, so a scene gives the
// same bits alone or beside others.  In the persistent form a CTA takes units from an
// atomic work list (batches of scenes).
//
// Every mbarrier wait is bounded; a wait that runs out sets a status bit, the CTA stops
// issuing work, drains what it issued, frees its tensor memory and returns.
#include <algorithm>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "tcgen05.cuh"

namespace rs {
namespace {

constexpr int BM = 128;          // tile rows (TMEM lanes)
constexpr int KS = 32;           // rays per pipeline stage (K = 2 KS real elements)
constexpr int KELEM = 2 * KS;    // K elements per stage
constexpr int NPROD = 384;       // producer threads (12 warps, 3 groups)
// ------------------------------------------------------------------ kernel
constexpr int NDRAIN = 128;            // drain threads: one TMEM lane each
constexpr int MMA_WARP = NPROD / 32;   // the warp after the producers
constexpr int NTHREADS_ALL = NPROD + 32 + NDRAIN;
// Stages (of KS rays) per tensor-core accumulation chain before it is folded into the FP32
// running sum: the tensor core's accumulate is not IEEE round-to-nearest and its error grows
// with the chain, so split precision folds every 512 rays; single precision (whose operand
// rounding is ~1e-3) folds only at the end of its chunk.  Each fold stalls the tensor pipe
// (about 3 us per chain); 1024-ray chains were measured 3.5 % faster but gave 1.14e-5 on a
// 1,500-ray scene at FP16 hi + lo, whose whole sum is one chain.
constexpr int SUBST_SPLIT = 16;
constexpr uint32_t kSumCol = 256;      // TMEM column of the FP32 running sum
constexpr int NGROUP = 3;              // producer groups; group g builds stages g, g + 3, ...
constexpr int GSIZE = NPROD / NGROUP;  // 128 threads (4 warps) per group

struct Args {
  RaysPrep p;
  int64_t n_rays;
  int64_t chunk;       // rays per split (multiple of KS)
  int nc, ns, m_rows;  // N_c, N_s, M = N_v N_c
  int nrx;             // N_rx: channel k = tx N_rx + rx
  int bn;              // MMA N (real columns per tile) = min(256, 2 N_s)
  float *partials;     // [splits][M][2 N_s], each bn-column tile as (Re block, Im block)
  const uint32_t *amax_bits;  // scene amplitude maximum (FP16 scaling), may be null
  uint32_t *status;
  // self-test mode: operands copied from row-major global matrices instead of synthesised
  const uint16_t *test_a;  // [M][K] 16-bit
  const uint16_t *test_b;  // [2 N_s][K] 16-bit
  int64_t test_k;
  int test_negate_b;       // self-test: set the instruction descriptor's negate-B bit
};

// Per-ray inputs of one stage, staged in shared memory by the producer group that builds it.
// base = carrier + t0 nu_tx + r0 nu_a + m0 nu_d is the phase at the tile's first row
// (k0 = t0 N_rx + r0, m0).
// The fields every producer thread reads for each ray sit in one record per operand, so that a
// ray costs three 16-byte loads (broadcast to the warp) instead of six narrow ones.
struct __align__(16) RayA {  // A rows of the fast path
  uint64_t base, nud;        // phase at the tile's first row, phase step per chirp
  float2 wd;                 // e^{2 pi j 32 nu_d}
  float amp, pad;
};
struct __align__(16) RayB {  // B columns
  uint64_t nur;              // phase step per sample
  float2 wr;                 // e^{2 pi j 32 nu_r}
};
struct StageRays {
  RayA a[KS];
  RayB b[KS];
  uint64_t car[KS], nua[KS], nutx[KS];  // carrier, channel and transmitter steps (general path)
};

__device__ __forceinline__ RayA load_ray_a(const StageRays &sr, int i) {
  const uint4 v0 = *reinterpret_cast<const uint4 *>(&sr.a[i]);
  const uint4 v1 = *(reinterpret_cast<const uint4 *>(&sr.a[i]) + 1);
  RayA r;
  r.base = static_cast<uint64_t>(v0.x) | (static_cast<uint64_t>(v0.y) << 32);
  r.nud = static_cast<uint64_t>(v0.z) | (static_cast<uint64_t>(v0.w) << 32);
  r.wd = make_float2(__uint_as_float(v1.x), __uint_as_float(v1.y));
  r.amp = __uint_as_float(v1.z);
  r.pad = 0.f;
  return r;
}
__device__ __forceinline__ RayB load_ray_b(const StageRays &sr, int i) {
  const uint4 v = *reinterpret_cast<const uint4 *>(&sr.b[i]);
  RayB r;
  r.nur = static_cast<uint64_t>(v.x) | (static_cast<uint64_t>(v.y) << 32);
  r.wr = make_float2(__uint_as_float(v.z), __uint_as_float(v.w));
  return r;
}

// Group threads fetch the stage's per-ray words one group-stage ahead: thread (f, q) with
// f = gt / 32 takes field set f of ray q.  Rays past the chunk read as 0.
struct RayWords {
  uint64_t v0, v1, v2, v3;
};

__device__ __forceinline__ RayWords fetch_ray_words(const Args &g, int64_t ray0, int64_t k_hi, int gt) {
  const int f = gt >> 5, q = gt & 31;
  const int64_t ray = ray0 + q;
  RayWords w{0, 0, 0, 0};
  if (ray < k_hi) {
    if (f == 0) {
      w.v0 = g.p.carrier[ray];
      w.v1 = g.p.nu_a[ray];
      w.v2 = g.p.nu_d[ray];
      w.v3 = g.p.nu_tx[ray];
    } else if (f == 1) {
      w.v0 = g.p.nu_r[ray];
      w.v1 = *reinterpret_cast<const uint64_t *>(g.p.step_r + ray);
      w.v2 = __float_as_uint(g.p.amp[ray]);
      w.v3 = *reinterpret_cast<const uint64_t *>(g.p.step_d + ray);
    }
  }
  return w;
}

__device__ __forceinline__ void store_ray_words(StageRays &sr, int gt, const RayWords &w, uint64_t t0, uint64_t r0,
                                                uint64_t m0) {
  const int f = gt >> 5, q = gt & 31;
  if (f == 0) {
    sr.car[q] = w.v0;
    sr.nua[q] = w.v1;
    sr.a[q].nud = w.v2;
    sr.nutx[q] = w.v3;
    sr.a[q].base = w.v0 + t0 * w.v3 + r0 * w.v1 + m0 * w.v2;
  } else if (f == 1) {
    sr.b[q].nur = w.v0;
    sr.b[q].wr = *reinterpret_cast<const float2 *>(&w.v1);
    sr.a[q].amp = __uint_as_float(static_cast<uint32_t>(w.v2));
    sr.a[q].wd = *reinterpret_cast<const float2 *>(&w.v3);
  }
}

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(GSIZE) : "memory");
}

// Synthesise one stage of operands in planar K order: within each 16-ray K step, the first
// K chunk of the A tile holds Re A of eight rays and the next Im A, likewise for B.
//   Shared layout of a stage: A_re | A_im (128 rows x 32 rays each, core matrices of 8 rows x
//   8 rays, 2048 bytes per K chunk) | B_re | B_im (NC rows each) | the same four for lo.
//   Every thread of the group takes ray octet o = t / 32 (one warp per octet) and lane
//   j = t % 32: A rows j, j + 32, j + 64, j + 96 and B columns j, j + 32, ... below NC, so the
//   work is even across the group and each warp's 16-byte stores cover 512 contiguous bytes.
//   Each phasor chain starts from one hardware sin/cos of its exact Q0.64 phase and steps 32
//   chirps / 32 samples per complex multiply with the prep kernel's e^{2 pi j 32 nu} (from the
//   exact Q0.64 product, within ~1.5 ulp).
//   PAIR: this CTA holds B for its half of the tile's complex columns (NC = bn / 4 of them).
// bytes of the hi A planes (A_re | A_im) of one stage; split precision stores the lo planes next
__host__ __device__ constexpr uint32_t hi_bytes_a() {
  return 2u * BM * KS * 2;
}

// Eight B phasors of eight rays -> the window rows of one column: B_re at +nc16, B_im at
// +2 nc16 and -B_im (exact sign flips of the same hi and lo values) at +0; the lo block at +lo.
template <bool F16>
__device__ __forceinline__ void put_octet_window(const float2 (&z)[OCT], uint8_t *p, uint32_t nc16, uint32_t lo) {
  constexpr uint32_t kSign = 0x80008000u;
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) encode<F16, true>(z[2 * q].x, z[2 * q + 1].x, h[q], l[q]);
  sts128(p + nc16, h[0], h[1], h[2], h[3]);
  sts128(p + nc16 + lo, l[0], l[1], l[2], l[3]);
#pragma unroll
  for (int q = 0; q < 4; ++q) encode<F16, true>(z[2 * q].y, z[2 * q + 1].y, h[q], l[q]);
  sts128(p + 2 * nc16, h[0], h[1], h[2], h[3]);
  sts128(p + 2 * nc16 + lo, l[0], l[1], l[2], l[3]);
  sts128(p, h[0] ^ kSign, h[1] ^ kSign, h[2] ^ kSign, h[3] ^ kSign);
  sts128(p + lo, l[0] ^ kSign, l[1] ^ kSign, l[2] ^ kSign, l[3] ^ kSign);
}

template <bool F16, bool SPLIT, bool FAST, bool PAIR>
__device__ __forceinline__ void produce_planar(const Args &g, const StageRays &sr, uint8_t *stage, int gt, int row0,
                                               int col0, float scale, int rank) {
  const int NC = PAIR ? g.bn >> 2 : g.bn >> 1;         // complex B columns held here
  const uint32_t a_half = BM * KS * 2;                 // bytes of A_re (or A_im)
  const uint32_t x_half = static_cast<uint32_t>(NC) * KS * 2;
  const uint32_t hi_bytes = 2 * a_half + 2 * x_half;
  uint8_t *a_re = stage, *a_im = stage + a_half, *x_re = stage + 2 * a_half, *x_im = x_re + x_half;
  // A lo planes: after all hi planes, or (window form) right after the A hi planes
  const uint32_t lo = SPLIT ? (PAIR ? 2 * a_half : hi_bytes) : 0;
  const int o = gt >> 5, j = gt & 31;
  {
    // ---- A: rows j + 32 l
    uint32_t off = o * (BM * 16) + (j >> 3) * 128 + (j & 7) * 16;
    float2 z[OCT], w[OCT];
    int grow = row0 + j;
    int kq = grow / g.nc, mq = grow - kq * g.nc;
    auto start = [&]() {  // exact phases of row (kq, mq), kq = tq N_rx + rq
      const int tq = kq / g.nrx, rq = kq - tq * g.nrx;
#pragma unroll 2
      for (int q = 0; q < OCT; ++q) {
        const int i = o * OCT + q;
        float sn, cs;
        const RayA ra = load_ray_a(sr, i);
        __sincosf(q64_to_rad(sr.car[i] + static_cast<uint64_t>(tq) * sr.nutx[i] + static_cast<uint64_t>(rq) * sr.nua[i] +
                             static_cast<uint64_t>(mq) * ra.nud),
                  &sn, &cs);
        const float am = ra.amp * scale;
        z[q] = make_float2(am * cs, am * sn);
      }
    };
    if constexpr (FAST) {
      // the tile's rows share channel k0 and rows are m0 + r: phase = base + r nu_d
#pragma unroll
      for (int q = 0; q < OCT; ++q) {
        const RayA ra = load_ray_a(sr, o * OCT + q);
        float sn, cs;
        __sincosf(q64_to_rad(ra.base + static_cast<uint64_t>(j) * ra.nud), &sn, &cs);
        const float am = ra.amp * scale;
        z[q] = make_float2(am * cs, am * sn);
        w[q] = ra.wd;
      }
    } else {
      start();
#pragma unroll
      for (int q = 0; q < OCT; ++q) w[q] = sr.a[o * OCT + q].wd;
    }
#pragma unroll 1
    for (int l = 0; l < BM / 32; ++l) {
      if (l > 0) {
        if constexpr (FAST) {
#pragma unroll
          for (int q = 0; q < OCT; ++q) z[q] = cmulf(z[q], w[q]);  // 32 chirps on
        } else {
          grow += 32;
          mq += 32;
          if (mq >= g.nc) {  // crossed into another channel: restart from the exact phases
            kq = grow / g.nc;
            mq = grow - kq * g.nc;
            start();
          } else {
#pragma unroll
            for (int q = 0; q < OCT; ++q) z[q] = cmulf(z[q], w[q]);
          }
        }
      }
      if (!FAST && grow >= g.m_rows) {
#pragma unroll
        for (int q = 0; q < OCT; ++q) z[q] = make_float2(0.f, 0.f);
      }
      put_octet<F16, SPLIT>(z, a_re + off, a_im + off, a_re + lo + off, a_im + lo + off);
      off += 512;
    }
  }
  if constexpr (PAIR && SPLIT) {
    // ---- B, window form: per K chunk this CTA's rows are [-B_im | B_re | B_im] (NC rows each)
    // so that one MMA takes A_re against [B_re | B_im] and one takes A_im against [-B_im | B_re]
    if (j < NC) {
      const uint32_t nc16 = static_cast<uint32_t>(NC * 16);
      uint8_t *xb = stage + 2 * hi_bytes_a();
      const uint32_t lo_b = 3 * nc16 * (KS / OCT);  // the lo block follows the hi block
      uint32_t off = o * 3 * nc16 + (j >> 3) * 128 + (j & 7) * 16;
      float2 z[OCT], w[OCT];
#pragma unroll
      for (int q = 0; q < OCT; ++q) {
        const int i = o * OCT + q;
        const RayB rb = load_ray_b(sr, i);
        float sn, cs;
        __sincosf(q64_to_rad(static_cast<uint64_t>(col0 / 2 + rank * NC + j) * rb.nur), &sn, &cs);
        z[q] = make_float2(cs, sn);
        w[q] = rb.wr;
      }
#pragma unroll 1
      for (int c = j; c < NC; c += 32) {
        if (c > j) {
#pragma unroll
          for (int q = 0; q < OCT; ++q) z[q] = cmulf(z[q], w[q]);  // 32 samples on
        }
        put_octet_window<F16>(z, xb + off, nc16, lo_b);
        off += 512;
      }
    }
  } else if (j < NC) {
    // ---- B: columns j + 32 l below NC
    uint32_t off = o * static_cast<uint32_t>(NC * 16) + (j >> 3) * 128 + (j & 7) * 16;
    float2 z[OCT], w[OCT];
#pragma unroll
    for (int q = 0; q < OCT; ++q) {
      const int i = o * OCT + q;
      float sn, cs;
      const RayB rb = load_ray_b(sr, i);
      __sincosf(q64_to_rad(static_cast<uint64_t>(col0 / 2 + (PAIR ? rank * NC : 0) + j) * rb.nur), &sn, &cs);
      z[q] = make_float2(cs, sn);
      w[q] = rb.wr;
    }
#pragma unroll 1
    for (int c = j; c < NC; c += 32) {
      if (c > j) {
#pragma unroll
        for (int q = 0; q < OCT; ++q) z[q] = cmulf(z[q], w[q]);  // 32 samples on
      }
      put_octet<F16, SPLIT>(z, x_re + off, x_im + off, x_re + lo + off, x_im + lo + off);
      off += 512;
    }
  }
}

// Copy one stage of operands from row-major 16-bit matrices (self-test), in the interleaved
// layout: 128 rows x 64 K of A, then bn rows x 64 K of B.
__device__ __forceinline__ void copy_stage(const Args &g, uint8_t *a_hi, uint8_t *b_hi, int64_t ray0, int row0,
                                           int col0, int gt) {
  const int bn = g.bn;
  const uint32_t lbo_a = BM * 16, lbo_b = static_cast<uint32_t>(bn) * 16;
  for (int item = gt; item < BM * (KELEM / 8); item += GSIZE) {
    const int r = item % BM, kc = item / BM;
    const int grow = row0 + r;
    uint32_t v[4];
    for (int q = 0; q < 4; ++q) {
      const int64_t kk = 2 * ray0 + kc * 8 + 2 * q;
      v[q] = 0;
      if (grow < g.m_rows && kk < g.test_k) {
        const uint16_t *src = g.test_a + static_cast<int64_t>(grow) * g.test_k + kk;
        v[q] = static_cast<uint32_t>(src[0]) | (static_cast<uint32_t>(src[1]) << 16);
      }
    }
    *reinterpret_cast<uint4 *>(a_hi + kc * lbo_a + r * 16) = make_uint4(v[0], v[1], v[2], v[3]);
  }
  for (int item = gt; item < bn * (KELEM / 8); item += GSIZE) {
    const int r = item % bn, kc = item / bn;
    const int gcol = col0 + r;
    uint32_t v[4];
    for (int q = 0; q < 4; ++q) {
      const int64_t kk = 2 * ray0 + kc * 8 + 2 * q;
      v[q] = 0;
      if (kk < g.test_k) {
        const uint16_t *src = g.test_b + static_cast<int64_t>(gcol) * g.test_k + kk;
        v[q] = static_cast<uint32_t>(src[0]) | (static_cast<uint32_t>(src[1]) << 16);
      }
    }
    *reinterpret_cast<uint4 *>(b_hi + kc * lbo_b + r * 16) = make_uint4(v[0], v[1], v[2], v[3]);
  }
}

// One work unit: a 128-row x bn-column tile of one scene summed over one chunk of its rays.
// One work unit: one tile of one scene summed over rays [k_lo, k_hi) into partial `split`.
struct Unit {
  int scene, tile_m, tile_n, split;
  int64_t k_lo, k_hi;
};

// Stream-K plan of a scene (split precision): its T tiles x S stages of rays form W = T S
// stage-units in tile order (tile t = tile_n mt + tile_m); program c of C takes the contiguous
// range [c W / C, (c + 1) W / C), cut at tile boundaries into pieces.  Piece slot = c minus the
// program holding the tile's first stage, so a tile's pieces are slots 0 .. p_t - 1 in ray
// order.  The plan depends only on the scene's own shape and the program count.
struct StreamK {
  int64_t w, s;  // stage-units and stages per tile; w = 0: no stream-K plan
  int c, mt;     // programs, tile rows (the tile order's stride)
};

// program holding stage-unit x: the largest j with floor(j W / C) <= x
__host__ __device__ inline int64_t sk_program_of(const StreamK &k, int64_t x) {
  return ((x + 1) * k.c + k.w - 1) / k.w - 1;
}
// pieces of tile t
__host__ __device__ inline int sk_pieces(const StreamK &k, int64_t t) {
  return static_cast<int>(sk_program_of(k, (t + 1) * k.s - 1) - sk_program_of(k, t * k.s) + 1);
}
// piece `idx` of program c (tile, ray range, slot); false once the program has no more
__host__ __device__ inline bool sk_piece(const StreamK &k, int64_t n_rays, int c, int idx, Unit &u) {
  int64_t pos = static_cast<int64_t>(c) * k.w / k.c;
  const int64_t end = static_cast<int64_t>(c + 1) * k.w / k.c;
  for (int q = 0; q < idx && pos < end; ++q) pos = (pos / k.s + 1) * k.s < end ? (pos / k.s + 1) * k.s : end;
  if (pos >= end) return false;
  const int64_t t = pos / k.s;
  const int64_t hi = (t + 1) * k.s < end ? (t + 1) * k.s : end;
  u.scene = 0;
  u.split = static_cast<int>(c - sk_program_of(k, t * k.s));
  u.tile_n = static_cast<int>(t / k.mt);
  u.tile_m = static_cast<int>(t - static_cast<int64_t>(u.tile_n) * k.mt);
  u.k_lo = (pos - t * k.s) * KS;
  u.k_hi = (hi - t * k.s) * KS < n_rays ? (hi - t * k.s) * KS : n_rays;
  return true;
}

// A launch of the ray-sum kernel: one scene whose units are decoded from the CTA index (one
// split unit per CTA, or with a stream-K plan the pieces of one program per CTA), or a
// persistent batch whose CTAs take units from a work list (longest first) through an atomic
// counter.
struct Launch {
  Args inline_scene;     // used when `scenes` is null
  const Args *scenes;    // per-scene arguments in device memory, or null
  const Unit *units;     // work list in device memory, or null (decode from inline_scene)
  int n_units;
  int mt, nt;            // tiles of the inline scene (for decoding)
  StreamK sk;            // the inline scene's stream-K plan (sk.w = 0: split units)
  unsigned *counter;     // persistent mode: next unit to take (zeroed before the launch)
  int bn_layout;         // B rows the shared-memory stages are laid out for (max bn)
};

template <bool SPLIT, bool TEST, bool PAIR>
__host__ __device__ constexpr int num_stages() {
  return TEST ? 4 : (PAIR ? (SPLIT ? 3 : 6) : (SPLIT ? 3 : 6));
}

// bytes of one pipeline stage (PAIR: B for half the tile's columns)
template <bool SPLIT, bool TEST, bool PAIR>
__host__ __device__ constexpr uint32_t stage_size(int bn) {
  // split precision on two-SM tiles (window form): A_re | A_im, hi then lo, then per hi and lo
  // block KS / 8 K chunks of 3 x bn / 4 B rows ([-B_im | B_re | B_im] for this CTA's columns)
  return TEST ? static_cast<uint32_t>(BM * KELEM * 2 + bn * KELEM * 2)
              : (PAIR && SPLIT ? 2 * hi_bytes_a() + 2u * (KS / OCT) * 3u * static_cast<uint32_t>(bn / 4) * 16u
                               : static_cast<uint32_t>(BM * KELEM * 2 + (PAIR ? bn / 2 : bn) * KS * 2) * (SPLIT ? 2u : 1u));
}

// PAIR: launched as clusters of two CTAs; each cluster takes one unit of 256 rows, the even
// CTA (rank 0) holding rows 0..127 and issuing the M = 256 MMAs, the odd CTA rows 128..255.
// Each CTA builds A for its rows and B for its half of the columns; every pipeline barrier the
// issuer waits on lives in CTA 0 and counts both CTAs' arrivals.  One unit per cluster.
template <bool F16, bool SPLIT, bool TEST, bool FAST, bool PAIR>
__global__ void __launch_bounds__(NTHREADS_ALL, 1) umma_sum_kernel(Launch L) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ Args s_args;
  __shared__ Unit s_unit;
  __shared__ int s_abort;
  __shared__ int s_next, s_peer_abort;  // PAIR work list: the pair's next unit, the odd CTA's abort
  __shared__ StageRays s_rays[NGROUP];
  constexpr int NST = num_stages<SPLIT, TEST, PAIR>();
  constexpr uint32_t TMEM_COLS = 512;  // accumulator (0..255) and running sum (256..511)
  const uint32_t stage_bytes = stage_size<SPLIT, TEST, PAIR>(L.bn_layout);
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  // How producers signal a finished stage: single pass, whose stages are short, gains from one
  // arrival per group after the group barrier; split precision (MMA-bound) from every thread
  // arriving as soon as its own stores are done (same-box timing of both schemes).
  constexpr bool ONE_ARRIVE = !SPLIT && !TEST;
  uint8_t *base = smem;
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + NST * stage_bytes);
  // barriers: full[NST], empty[NST], acc_full, acc_empty, mma_done
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + 2 * NST + 3);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + NST);
  const uint32_t accf = smem_u32(bars + 2 * NST), acce = smem_u32(bars + 2 * NST + 1);
  const uint32_t done = smem_u32(bars + 2 * NST + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // the issuer's barriers (in CTA 0) as every thread of the pair addresses them
  const uint32_t full0_c = PAIR ? cluster_addr(full0, 0) : full0;
  const uint32_t acce_c = PAIR ? cluster_addr(acce, 0) : acce;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(full0 + 8 * s, (ONE_ARRIVE ? 1 : GSIZE) * (PAIR ? 2 : 1));
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, PAIR ? 2 * NDRAIN : NDRAIN);
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
    s_next = 0;
    s_peer_abort = 0;
  }
  if (warp == MMA_WARP) tmem_alloc<PAIR>(smem_u32(tmem_holder), TMEM_COLS);
  tc_fence_before();
  if constexpr (PAIR) cluster_sync();  // both CTAs' barriers exist before any remote arrival
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;

  // running counters shared by every role: pipeline stages, accumulation chains, units
  int gst = 0, gsub = 0, gunit = 0;
  int u = static_cast<int>(PAIR ? blockIdx.x >> 1 : blockIdx.x);
  // PAIR with a work list: CTA 0 takes the pair's next unit (or stops the pair when either CTA
  // has aborted) and writes it into both CTAs' s_next; every thread of both CTAs calls this
  auto pair_next = [&]() -> int {
    if (rank != 0 && threadIdx.x == 0 && s_abort) st_cluster_u32(cluster_addr(smem_u32(&s_peer_abort), 0), 1u);
    cluster_sync();
    if (rank == 0 && threadIdx.x == 0) {
      const int v = (s_abort || s_peer_abort) ? L.n_units : static_cast<int>(atomicAdd(L.counter, 1u));
      s_next = v;
      st_cluster_u32(cluster_addr(smem_u32(&s_next), 1), static_cast<uint32_t>(v));
    }
    cluster_sync();
    return s_next;
  };
  if (L.counter) {
    if constexpr (PAIR) {
      u = pair_next();
    } else {
      if (threadIdx.x == 0) s_unit.scene = static_cast<int>(atomicAdd(L.counter, 1u));
      __syncthreads();
      u = s_unit.scene;
      __syncthreads();
    }
  }
  // inline stream-K: this CTA (pair) is program `prog` and runs its pieces 0, 1, ...
  const int prog = u;
  if (!L.units && L.sk.w > 0) u = 0;
  while (u < L.n_units) {
    if (threadIdx.x == 0) {
      if (L.units) {
        s_unit = L.units[u];
      } else if (L.sk.w > 0) {
        const int64_t kt = TEST ? L.inline_scene.test_k / 2 : L.inline_scene.n_rays;
        if (!sk_piece(L.sk, kt, prog, u, s_unit)) s_unit.scene = -1;
      } else {
        const int per = L.mt * L.nt;
        const Args &a = L.inline_scene;
        const int64_t kt = TEST ? a.test_k / 2 : a.n_rays;
        s_unit.scene = 0;
        s_unit.split = u / per;
        s_unit.tile_n = (u - s_unit.split * per) / L.mt;
        s_unit.tile_m = u - s_unit.split * per - s_unit.tile_n * L.mt;
        s_unit.k_lo = static_cast<int64_t>(s_unit.split) * a.chunk;
        s_unit.k_hi = s_unit.k_lo + a.chunk < kt ? s_unit.k_lo + a.chunk : kt;
      }
      if (s_unit.scene >= 0) s_args = L.scenes ? L.scenes[s_unit.scene] : L.inline_scene;
    }
    __syncthreads();
    if (s_unit.scene < 0) break;  // the program's pieces are done (uniform across the CTA pair)
    const Args &g = s_args;
    const int bn = g.bn;
    const int NC = bn >> 1;
    const int row0 = (PAIR ? 2 * s_unit.tile_m + static_cast<int>(rank) : s_unit.tile_m) * BM;
    const int col0 = s_unit.tile_n * bn;  // real column; complex n0 = col0 / 2
    const int split = s_unit.split;
    const int64_t k_lo = s_unit.k_lo, k_hi = s_unit.k_hi;
    const int n_stages = k_hi > k_lo ? static_cast<int>((k_hi - k_lo + KS - 1) / KS) : 0;
    const int SUBST = SPLIT ? SUBST_SPLIT : (n_stages > 0 ? n_stages : 1);
    const int n_sub = (n_stages + SUBST - 1) / SUBST;
    bool failed = false;

    if (warp < MMA_WARP) {
      // ---------------- producers: group grp builds stages grp, grp + NGROUP, ...
      const int grp = warp / (GSIZE / 32), gt = threadIdx.x % GSIZE;
      const float scale = TEST ? 1.f : amp_scale<F16>(g.amax_bits);
      const uint64_t k0 = static_cast<uint64_t>(row0 / g.nc), m0 = static_cast<uint64_t>(row0 % g.nc);
      const uint64_t t0 = k0 / static_cast<uint64_t>(g.nrx), r0 = k0 - t0 * static_cast<uint64_t>(g.nrx);
      RayWords nxt{0, 0, 0, 0};
      if (!TEST && grp < n_stages) nxt = fetch_ray_words(g, k_lo + static_cast<int64_t>(grp) * KS, k_hi, gt);
      for (int st = grp; st < n_stages; st += NGROUP) {
        const int gs = gst + st;
        const int s = gs % NST;
        const int64_t ray0 = k_lo + static_cast<int64_t>(st) * KS;
        if constexpr (!TEST) {
          store_ray_words(s_rays[grp], gt, nxt, t0, r0, m0);
          if (st + NGROUP < n_stages) nxt = fetch_ray_words(g, ray0 + NGROUP * KS, k_hi, gt);
        }
        // the stage slot is free, and the group's ray words are visible; a wait that ran out
        // in any thread takes the whole group out of the loop
        const bool slot_ok = gs < NST || mbar_wait(empty0 + 8 * s, ((gs / NST) - 1) & 1);
        if (bar_any(grp + 1, GSIZE, !slot_ok)) {
          failed = true;
          break;
        }
        uint8_t *st_base = base + s * stage_bytes;
        if constexpr (TEST) {
          copy_stage(g, st_base, st_base + BM * KELEM * 2, ray0, row0, col0, gt);
        } else {
          produce_planar<F16, SPLIT, FAST, PAIR>(g, s_rays[grp], st_base, gt, row0, col0, scale,
                                                 static_cast<int>(rank));
        }
        fence_proxy_async();  // this thread's stores, visible to the tensor core
        if constexpr (ONE_ARRIVE) {
          // the whole group's stores are done (and s_rays[grp] is free for the next round):
          // one thread signals the stage
          group_sync(grp);
          if (gt == 0) {
            if constexpr (PAIR) mbar_arrive_cluster(full0_c + 8 * s);
            else mbar_arrive(full0 + 8 * s);
          }
        } else {
          if constexpr (PAIR) mbar_arrive_cluster(full0_c + 8 * s);
          else mbar_arrive(full0 + 8 * s);
          if constexpr (!TEST) group_sync(grp);  // s_rays[grp] is rewritten next round
        }
      }
    } else if (warp == MMA_WARP) {
      // ---------------- MMA issuer (PAIR: CTA 0 issues for both; CTA 1 only waits for the end)
      if (lane == 0 && PAIR && rank != 0) {
        if (!mbar_wait(done, gunit & 1)) failed = true;
      } else if (lane == 0) {
        const uint32_t sbase = smem_u32(base);
        bool open = false;  // issued MMAs not yet committed to acc_full
        const uint32_t tmem = tmem_base;
        for (int st = 0; st < n_stages; ++st) {
          const int gs = gst + st;
          const int s = gs % NST;
          const int gc = gsub + st / SUBST;  // this chain's index across the CTA's life
          const bool first = (st % SUBST) == 0;
          if (first && gc > 0 && !mbar_wait(acce, (gc - 1) & 1)) {
            failed = true;
            break;
          }
          if (!mbar_wait(full0 + 8 * s, (gs / NST) & 1)) {
            failed = true;
            break;
          }
          tc_fence_after();
          const uint32_t sb = sbase + s * stage_bytes;
          if constexpr (TEST && !PAIR) {
            // interleaved layout: D = A B^T over 4 K steps of 16
            const uint32_t idesc = make_idesc(F16, BM, bn) | (g.test_negate_b ? (1u << 14) : 0u);
            const uint32_t lbo_a = BM * 16, lbo_b = static_cast<uint32_t>(bn) * 16;
            const uint32_t b0 = sb + BM * KELEM * 2;
#pragma unroll
            for (int kk = 0; kk < KELEM / 16; ++kk)
              mma_f16<false>(tmem, make_sdesc(sb + kk * 2 * lbo_a, lbo_a, 128),
                             make_sdesc(b0 + kk * 2 * lbo_b, lbo_b, 128), idesc, (!first || kk > 0) ? 1u : 0u);
          } else if constexpr (PAIR && SPLIT) {
            // window form: per 16-ray K step, [Re | Im] += A_re [B_re | B_im] + A_im [-B_im | B_re]
            // as two MMAs of N = 2 NC (CTA 0's window rows give accumulator columns 0 .. NC - 1,
            // CTA 1's the rest: [Re | Im] of each CTA's NC / 2 columns), for hi x hi, hi x lo and
            // lo x hi: six MMAs, each A plane read once per complex product
            const uint32_t idesc = make_idesc(F16, 2 * BM, 2 * NC);
            const uint32_t h = static_cast<uint32_t>(NC / 2);  // complex columns of this CTA
            const uint32_t lbo_a = BM * 16, lbo_x = 3 * h * 16;
            const uint32_t a_half = BM * KS * 2;
            const uint32_t ar = sb, ai = sb + a_half, alo = 2 * a_half;
            const uint32_t xb = sb + 4 * a_half, xlo = (KS / OCT) * lbo_x;
            const uint32_t w1 = h * 16;  // window [B_re | B_im] starts after the -B_im rows
#pragma unroll
            for (int kh = 0; kh < KS / 16; ++kh) {
              const uint32_t acc = (!first || kh > 0) ? 1u : 0u;
              const uint32_t oa = kh * 2 * lbo_a, ox = kh * 2 * lbo_x;
              const uint64_t dar = make_sdesc(ar + oa, lbo_a, 128), dai = make_sdesc(ai + oa, lbo_a, 128);
              const uint64_t lar = make_sdesc(ar + alo + oa, lbo_a, 128), lai = make_sdesc(ai + alo + oa, lbo_a, 128);
              const uint64_t w1h = make_sdesc(xb + ox + w1, lbo_x, 128), w2h = make_sdesc(xb + ox, lbo_x, 128);
              const uint64_t w1l = make_sdesc(xb + xlo + ox + w1, lbo_x, 128), w2l = make_sdesc(xb + xlo + ox, lbo_x, 128);
              mma_f16<true>(tmem, dar, w1h, idesc, acc);
              mma_f16<true>(tmem, dai, w2h, idesc, 1u);
              mma_f16<true>(tmem, dar, w1l, idesc, 1u);
              mma_f16<true>(tmem, dai, w2l, idesc, 1u);
              mma_f16<true>(tmem, lar, w1h, idesc, 1u);
              mma_f16<true>(tmem, lai, w2h, idesc, 1u);
            }
          } else {
            // planar layout: per 16-ray K step, Re S += A_re B_re - A_im B_im and
            // Im S += A_re B_im + A_im B_re (the minus by the descriptor's negate-B bit).
            // PAIR: M = 256 over both CTAs, each CTA's B blocks hold NC / 2 of the NC columns.
            const uint32_t idesc = make_idesc(F16, PAIR ? 2 * BM : BM, NC);
            const uint32_t ineg = idesc | (1u << 14);
            const uint32_t ncx = static_cast<uint32_t>(PAIR ? NC / 2 : NC);
            const uint32_t lbo_a = BM * 16, lbo_x = ncx * 16;
            const uint32_t a_half = BM * KS * 2, x_half = ncx * KS * 2;
            const uint32_t ar = sb, ai = sb + a_half, xr = sb + 2 * a_half, xi = xr + x_half;
            const uint32_t lo = 2 * a_half + 2 * x_half;
            const uint32_t t_re = tmem, t_im = tmem + static_cast<uint32_t>(NC);
#pragma unroll
            for (int kh = 0; kh < KS / 16; ++kh) {
              const uint32_t acc = (!first || kh > 0) ? 1u : 0u;
              const uint32_t oa = kh * 2 * lbo_a, ox = kh * 2 * lbo_x;
              const uint64_t dar = make_sdesc(ar + oa, lbo_a, 128), dai = make_sdesc(ai + oa, lbo_a, 128);
              const uint64_t dxr = make_sdesc(xr + ox, lbo_x, 128), dxi = make_sdesc(xi + ox, lbo_x, 128);
              mma_f16<PAIR>(t_re, dar, dxr, idesc, acc);
              mma_f16<PAIR>(t_re, dai, dxi, ineg, 1u);
              mma_f16<PAIR>(t_im, dar, dxi, idesc, acc);
              mma_f16<PAIR>(t_im, dai, dxr, idesc, 1u);
              if constexpr (SPLIT) {
                const uint64_t lar = make_sdesc(ar + lo + oa, lbo_a, 128), lai = make_sdesc(ai + lo + oa, lbo_a, 128);
                const uint64_t lxr = make_sdesc(xr + lo + ox, lbo_x, 128), lxi = make_sdesc(xi + lo + ox, lbo_x, 128);
                mma_f16<PAIR>(t_re, dar, lxr, idesc, 1u);
                mma_f16<PAIR>(t_re, lar, dxr, idesc, 1u);
                mma_f16<PAIR>(t_re, dai, lxi, ineg, 1u);
                mma_f16<PAIR>(t_re, lai, dxi, ineg, 1u);
                mma_f16<PAIR>(t_im, dar, lxi, idesc, 1u);
                mma_f16<PAIR>(t_im, lar, dxi, idesc, 1u);
                mma_f16<PAIR>(t_im, dai, lxr, idesc, 1u);
                mma_f16<PAIR>(t_im, lai, dxr, idesc, 1u);
              }
            }
          }
          open = true;
          mma_commit<PAIR>(empty0 + 8 * s);
          if ((st % SUBST) == SUBST - 1 || st == n_stages - 1) {
            mma_commit<PAIR>(accf);
            open = false;
          }
        }
        if (open) mma_commit<PAIR>(accf);
        // every issued MMA of this unit has completed once `done` fires (in both CTAs)
        mma_commit<PAIR>(done);
        if (!mbar_wait(done, gunit & 1)) failed = true;
      }
    } else {
      // ---------------- drain: TMEM lane quarter (warp % 4).  Each finished chain is added in
      // FP32 (round to nearest) to the running sum kept in tensor memory, 32 columns per load
      // pair and wait (the tensor pipe waits while a chain drains); after the last chain the sum
      // goes to this split's partial in global memory.
      const int q = warp & 3;
      const int grow = row0 + q * 32 + lane;
      float *dst = g.partials + (static_cast<int64_t>(split) * g.m_rows + grow) * (2 * g.ns) + col0;
      const uint32_t trow = tmem_base + (static_cast<uint32_t>(q * 32) << 16);
      // 16 accumulator columns from column c to the partial (window form: accumulator columns
      // [Re | Im] of CTA 0's columns, then of CTA 1's, in blocks of bn / 4; the partial keeps
      // the tile as [Re block | Im block])
      auto put16 = [&](int c, const uint32_t *v) {
        int dc = c;
        if constexpr (PAIR && SPLIT) {
          const int hq = bn >> 2;
          if (c >= hq && c < 2 * hq) dc = c + hq;
          else if (c >= 2 * hq && c < 3 * hq) dc = c - hq;
        }
#pragma unroll
        for (int x = 0; x < 16; x += 4)
          *reinterpret_cast<float4 *>(dst + dc + x) =
              make_float4(__uint_as_float(v[x]), __uint_as_float(v[x + 1]), __uint_as_float(v[x + 2]),
                          __uint_as_float(v[x + 3]));
      };
      if (n_stages == 0 && grow < g.m_rows) {
        for (int c = 0; c < bn; c += 4) *reinterpret_cast<float4 *>(dst + c) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      for (int sub = 0; sub < n_sub; ++sub) {
        if (!mbar_wait_sleep(accf, (gsub + sub) & 1)) {
          failed = true;
          break;
        }
        tc_fence_after();
        const bool last = sub == n_sub - 1;
        for (int c = 0; c < bn;) {
          if (c + 32 <= bn) {
            uint32_t h[32];
            if (sub > 0) {
              uint32_t r[32];
              tmem_ld32x2(trow + static_cast<uint32_t>(c), trow + kSumCol + static_cast<uint32_t>(c), h, r);
#pragma unroll
              for (int x = 0; x < 32; ++x) h[x] = __float_as_uint(__uint_as_float(h[x]) + __uint_as_float(r[x]));
            } else {
              tmem_ld32(trow + static_cast<uint32_t>(c), h);
            }
            if (!last) {
              tmem_st32(trow + kSumCol + static_cast<uint32_t>(c), h);
            } else if (grow < g.m_rows) {
              put16(c, h);
              put16(c + 16, h + 16);
            }
            c += 32;
          } else {
            uint32_t h[16];
            tmem_ld16(trow + static_cast<uint32_t>(c), h);
            if (sub > 0) {
              uint32_t r[16];
              tmem_ld16(trow + kSumCol + static_cast<uint32_t>(c), r);
#pragma unroll
              for (int x = 0; x < 16; ++x) h[x] = __float_as_uint(__uint_as_float(h[x]) + __uint_as_float(r[x]));
            }
            if (!last) tmem_st16(trow + kSumCol + static_cast<uint32_t>(c), h);
            else if (grow < g.m_rows) put16(c, h);
            c += 16;
          }
        }
        if (!last) tmem_wait_st();
        tc_fence_before();
        if constexpr (PAIR) mbar_arrive_cluster(acce_c);
        else mbar_arrive(acce);
      }
    }
    if (failed) {
      atomicOr(g.status, kStatusWaitLimit);
      s_abort = 1;
    }
    gst += n_stages;
    gsub += n_sub;
    ++gunit;
    tc_fence_before();
    __syncthreads();  // every role is done with this unit (and with s_args)
    tc_fence_after();
    if (!L.counter) {
      if (L.units || L.sk.w == 0) break;
      // the program's next piece; a CTA pair stops together when either CTA has aborted
      if constexpr (PAIR) {
        if (rank != 0 && threadIdx.x == 0 && s_abort) st_cluster_u32(cluster_addr(smem_u32(&s_peer_abort), 0), 1u);
        cluster_sync();
        if (rank == 0 && threadIdx.x == 0) {
          const int v = (s_abort || s_peer_abort) ? 1 : 0;
          s_next = v;
          st_cluster_u32(cluster_addr(smem_u32(&s_next), 1), static_cast<uint32_t>(v));
        }
        cluster_sync();
        if (s_next) break;
      } else {
        if (s_abort) break;
      }
      ++u;
      continue;
    }
    if constexpr (PAIR) {
      u = pair_next();  // both CTAs stop together
    } else {
      if (s_abort) break;
      if (threadIdx.x == 0) s_unit.scene = static_cast<int>(atomicAdd(L.counter, 1u));
      __syncthreads();
      u = s_unit.scene;
      __syncthreads();
    }
  }
  tc_fence_before();
  // PAIR: neither CTA leaves while the other may still arrive on its barriers or the issuer's
  // MMAs may still read its shared memory
  if constexpr (PAIR) cluster_sync();
  else __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    tmem_dealloc<PAIR>(tmem_base, TMEM_COLS);
  }
}

// Sum the split partials in split order and interleave each tile's (Re block, Im block):
//   sig[row][n] = sum_s (P_s[row][t bn + nl], P_s[row][t bn + bn/2 + nl]) / scale,
//   t = n / (bn/2), nl = n % (bn/2).
// A thread takes four consecutive samples (16-byte loads; bn / 2 and N_s are multiples of 16).
// With a stream-K plan (sk.w > 0) tile t has sk_pieces(t) partials instead of `splits`;
// tile_rows is the rows of a tile (256 for two-SM tiles).
template <bool F16>
__global__ void reduce_partials(const float *__restrict__ part, int splits, int64_t m_rows, int ns, int bn,
                                float2 *__restrict__ sig, const uint32_t *amax_bits, StreamK sk, int tile_rows) {
  const float inv = F16 ? 1.f / amp_scale<true>(amax_bits) : 1.f;
  const int64_t n_q = m_rows * ns / 4;
  const int64_t plane = m_rows * 2 * ns;
  const int half = bn / 2, ns4 = ns / 4;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_q;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t row = i / ns4;
    const int n = static_cast<int>(i - row * ns4) * 4;
    const int t = n / half, nl = n - t * half;
    const float *p = part + row * 2 * ns + t * bn + nl;
    float4 re = *reinterpret_cast<const float4 *>(p), im = *reinterpret_cast<const float4 *>(p + half);
    const int n_split = sk.w > 0 ? sk_pieces(sk, static_cast<int64_t>(t) * sk.mt + row / tile_rows) : splits;
#pragma unroll 6
    for (int s = 1; s < n_split; ++s) {
      const float4 a = *reinterpret_cast<const float4 *>(p + s * plane);
      const float4 b = *reinterpret_cast<const float4 *>(p + s * plane + half);
      re.x += a.x; re.y += a.y; re.z += a.z; re.w += a.w;
      im.x += b.x; im.y += b.y; im.z += b.z; im.w += b.w;
    }
    float4 *o = reinterpret_cast<float4 *>(sig + row * ns + n);
    o[0] = make_float4(re.x * inv, im.x * inv, re.y * inv, im.y * inv);
    o[1] = make_float4(re.z * inv, im.z * inv, re.w * inv, im.w * inv);
  }
}

__global__ void amax_kernel(const float *__restrict__ amp, int64_t n, uint32_t *amax_bits) {
  uint32_t m = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    m = max(m, __float_as_uint(amp[i]));  // amplitudes are >= 0: bit order is value order
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax_bits, m);
}

struct Shape {
  int mt, nt, splits, bn;  // splits: partials per tile (with stream-K the most any tile has)
  int64_t chunk;
  StreamK sk;              // sk.w > 0: stream-K plan
};

int num_sms() {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    return cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0 ? n : 148;
  }();
  return sms;
}

// Tiles of 128 rows x bn columns; the rays split into `splits` chunks so that the CTAs fill
// whole waves of the SMs (at least `waves`, four for a scene that has the GPU to itself) as
// evenly as possible.  Depends only on the scene's own shape and ray count.
Shape plan_shape_forced(const Derived &g, int64_t n, int forced_splits, float waves = 4.f, int64_t min_chunk = 0);

// Two-SM tiles (M = 256 over a CTA pair, each CTA building B for half the columns) when the
// tile has at least 32 complex columns; the split-K chunks are those of the one-SM tiling.
bool use_pair(const Shape &sh) { return sh.bn >= 64; }

// Split precision on a GPU to itself: one program per SM (pair), each summing a contiguous run
// of the scene's (tile, ray stage) work, at least one accumulation chain long.  A tile then
// has at most a few partials (three on the automotive frame, against 19 split units), and a
// CTA switches tiles once or twice instead of once per split.
Shape with_stream_k(Shape s, int64_t n) {
  const bool pair = use_pair(s);
  const int mtp = pair ? (s.mt + 1) / 2 : s.mt;
  const int64_t tiles = static_cast<int64_t>(mtp) * s.nt;
  const int64_t stages = (n + KS - 1) / KS;
  const int64_t w = tiles * stages;
  const int64_t programs = pair ? num_sms() / 2 : num_sms();
  StreamK k{w, stages, static_cast<int>(std::max<int64_t>(1, std::min(programs, w / SUBST_SPLIT))), mtp};
  int pmax = 1;
  for (int64_t t = 0; t < tiles; ++t) pmax = std::max(pmax, sk_pieces(k, t));
  s.sk = k;
  s.splits = pmax;
  s.chunk = stages * KS;
  return s;
}

// allow_sk: a scene planned for the whole GPU with split precision and no tuned entry takes the
// stream-K plan
Shape plan_shape(const Derived &g, int64_t n, float waves = 4.f, int64_t min_chunk = 0, bool allow_sk = true) {
  Tuning tu{};
  if (waves == 4.f && min_chunk == 0 && tuning_lookup(g, n, &tu) && tu.splits > 0) return plan_shape_forced(g, n, tu.splits);
  const Shape s = plan_shape_forced(g, n, 0, waves, min_chunk);
  const bool split = g.precision == SIM_PREC_BF16_SPLIT || g.precision == SIM_PREC_FP16_SPLIT;
  if (allow_sk && split && waves == 4.f && min_chunk == 0 && n > 0) return with_stream_k(s, n);
  return s;
}

// forced_splits > 0 replaces the wave-filling choice (autotuned tables, tuner trials)
Shape plan_shape_forced(const Derived &g, int64_t n, int forced_splits, float waves, int64_t min_chunk) {
  Shape s{};
  const int M = g.nv * g.nc;
  // single pass keeps no running sum in tensor memory, so its tiles can take 256 complex columns
  // (Re and Im blocks fill all 512 TMEM columns); split precision tiles take 128
  const bool split = g.precision == SIM_PREC_BF16_SPLIT || g.precision == SIM_PREC_FP16_SPLIT;
  const int bn_cap = split ? 256 : 512;
  s.bn = 2 * g.ns < bn_cap ? 2 * g.ns : bn_cap;
  s.mt = (M + BM - 1) / BM;
  s.nt = 2 * g.ns / s.bn;
  const int sms = num_sms();
  const int64_t tiles = static_cast<int64_t>(s.mt) * s.nt;
  const int64_t max_splits = (n + KS - 1) / KS > 0 ? (n + KS - 1) / KS : 1;
  const int64_t target = static_cast<int64_t>(waves * static_cast<float>(sms) + 0.5f);
  const int64_t lo = std::max<int64_t>(1, (target + tiles - 1) / tiles);
  // idle fraction of the last wave, waste / (ctas + waste); smallest wins, ties to fewer splits
  int64_t best = lo, best_waste = -1, best_slots = 1;
  for (int64_t sp = lo; sp <= 3 * lo; ++sp) {
    const int64_t ctas = tiles * sp;
    const int64_t slots = ((ctas + sms - 1) / sms) * sms;
    const int64_t waste = slots - ctas;
    if (best_waste < 0 || waste * best_slots < best_waste * slots) {
      best = sp;
      best_waste = waste;
      best_slots = slots;
    }
  }
  int64_t splits = forced_splits > 0 ? forced_splits : best;
  if (forced_splits <= 0 && min_chunk > 0 && splits > std::max<int64_t>(1, n / min_chunk))
    splits = std::max<int64_t>(1, n / min_chunk);
  if (splits > max_splits) splits = max_splits;
  if (splits > 65535) splits = 65535;
  if (splits < 1) splits = 1;
  int64_t chunk = (n + splits - 1) / splits;
  chunk = (chunk + KS - 1) / KS * KS;
  if (chunk < KS) chunk = KS;
  s.chunk = chunk;
  s.splits = static_cast<int>((n + chunk - 1) / chunk);
  if (s.splits < 1) s.splits = 1;
  return s;
}

size_t smem_bytes(bool split, int bn, bool pair = false) {
  const int nst = pair ? (split ? num_stages<true, false, true>() : num_stages<false, false, true>())
                       : (split ? num_stages<true, false, false>() : num_stages<false, false, false>());
  const size_t stage = pair ? (split ? stage_size<true, false, true>(bn) : stage_size<false, false, true>(bn))
                            : (split ? stage_size<true, false, false>(bn) : stage_size<false, false, false>(bn));
  return nst * stage + 8 * (2 * nst + 3) + 16;
}

constexpr int kMaxDynSmem = 232448 - 8192;  // 227 KB per block, less the kernel's static shared memory

template <bool F16, bool SPLIT, bool TEST, bool FAST, bool PAIR>
void set_smem_attr() {
  static std::atomic<uint64_t> done{0};
  once_per_device(done, [] {
    note_launch(cudaFuncSetAttribute(umma_sum_kernel<F16, SPLIT, TEST, FAST, PAIR>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     TEST ? kMaxDynSmem : static_cast<int>(smem_bytes(SPLIT, SPLIT || !PAIR ? 256 : 512, PAIR))));
  });
}

// one scene, one unit per CTA (PAIR: per cluster of two CTAs, units of 256 rows)
template <bool F16, bool SPLIT, bool TEST, bool FAST, bool PAIR>
void launch_gemm(const Shape &sh, const Args &a, cudaStream_t s) {
  // the self-test reserves the whole shared memory so that every descriptor it builds
  // points inside the allocation
  const size_t sm = TEST ? kMaxDynSmem : smem_bytes(SPLIT, sh.bn, PAIR);
  set_smem_attr<F16, SPLIT, TEST, FAST, PAIR>();
  Launch L{};
  L.inline_scene = a;
  L.mt = PAIR ? (sh.mt + 1) / 2 : sh.mt;
  L.nt = sh.nt;
  L.n_units = L.mt * sh.nt * sh.splits;
  L.bn_layout = sh.bn;
  L.sk = sh.sk;
  // stream-K: one CTA (pair) per program, each running its pieces; n_units only bounds the loop
  const unsigned ctas = sh.sk.w > 0 ? static_cast<unsigned>(sh.sk.c) : static_cast<unsigned>(L.n_units);
  if (sh.sk.w > 0) L.n_units = 0x7fffffff;
  if constexpr (PAIR) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2u * ctas);
    cfg.blockDim = dim3(NTHREADS_ALL);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    note_launch(cudaLaunchKernelEx(&cfg, umma_sum_kernel<F16, SPLIT, TEST, FAST, PAIR>, L));
  } else {
    umma_sum_kernel<F16, SPLIT, TEST, FAST, PAIR><<<ctas, NTHREADS_ALL, sm, s>>>(L);
  }
}

// FAST: every tile's 128 rows lie in one channel (N_c a multiple of 128); the general kernel
// gives the same bits on such scenes, only with more work per row
template <bool PAIR>
void launch_gemm_dispatch_p(bool f16, bool split, bool fast, const Shape &sh, const Args &a, cudaStream_t s) {
  if (f16) {
    if (split) fast ? launch_gemm<true, true, false, true, PAIR>(sh, a, s) : launch_gemm<true, true, false, false, PAIR>(sh, a, s);
    else fast ? launch_gemm<true, false, false, true, PAIR>(sh, a, s) : launch_gemm<true, false, false, false, PAIR>(sh, a, s);
  } else {
    if (split) fast ? launch_gemm<false, true, false, true, PAIR>(sh, a, s) : launch_gemm<false, true, false, false, PAIR>(sh, a, s);
    else fast ? launch_gemm<false, false, false, true, PAIR>(sh, a, s) : launch_gemm<false, false, false, false, PAIR>(sh, a, s);
  }
}

void launch_gemm_dispatch(bool f16, bool split, bool fast, const Shape &sh, const Args &a, cudaStream_t s) {
  if (use_pair(sh)) launch_gemm_dispatch_p<true>(f16, split, fast, sh, a, s);
  else launch_gemm_dispatch_p<false>(f16, split, fast, sh, a, s);
}

}  // namespace

int64_t umma_workspace_bytes(const Derived &g, int64_t n, float waves, int64_t min_chunk) {
  if (g.model == SIM_MODEL_EXACT) return exact_tensor_workspace_bytes(g, n);
  const Shape sh = plan_shape(g, n, waves, min_chunk);
  return 256 + static_cast<int64_t>(sh.splits) * g.nv * g.nc * 2 * g.ns * 4;
}

int launch_umma_sum(const Derived &g, RaysPrep p, int64_t n, float2 *sig, void *workspace, uint32_t *status,
                    cudaStream_t s, cudaEvent_t after_main, float waves, int64_t min_chunk) {
  if (g.model == SIM_MODEL_EXACT) return launch_exact_tensor(g, p, n, sig, workspace, status, s, after_main);
  const Shape sh = plan_shape(g, n, waves, min_chunk);
  uint32_t *amax = static_cast<uint32_t *>(workspace);
  float *partials = reinterpret_cast<float *>(static_cast<uint8_t *>(workspace) + 256);
  const bool f16 = g.precision == SIM_PREC_FP16 || g.precision == SIM_PREC_FP16_SPLIT;
  const bool split = g.precision == SIM_PREC_BF16_SPLIT || g.precision == SIM_PREC_FP16_SPLIT;
  int kernels = 0;
  cudaMemsetAsync(amax, 0, 4, s);
  if (f16 && n > 0) {
    amax_kernel<<<2 * num_sms(), 256, 0, s>>>(p.amp, n, amax);
    ++kernels;
  }
  Args a{};
  a.p = p;
  a.n_rays = n;
  a.chunk = sh.chunk;
  a.nc = g.nc;
  a.ns = g.ns;
  a.m_rows = g.nv * g.nc;
  a.nrx = g.nrx;
  a.bn = sh.bn;
  a.partials = partials;
  a.amax_bits = amax;
  a.status = status;
  launch_gemm_dispatch(f16, split, (g.nc % BM) == 0, sh, a, s);
  ++kernels;
  if (after_main) cudaEventRecord(after_main, s);
  const int rb = 4 * num_sms();
  const int64_t m_rows = static_cast<int64_t>(g.nv) * g.nc;
  if (f16) reduce_partials<true><<<rb, 256, 0, s>>>(partials, sh.splits, m_rows, g.ns, sh.bn, sig, amax, sh.sk,
                                                    use_pair(sh) ? 2 * BM : BM);
  else reduce_partials<false><<<rb, 256, 0, s>>>(partials, sh.splits, m_rows, g.ns, sh.bn, sig, amax, sh.sk,
                                                     use_pair(sh) ? 2 * BM : BM);
  ++kernels;
  return kernels;
}

// ---- autotuner hooks
int umma_split_candidates(const Derived &g, int64_t n, int *out, int max_out) {
  const Shape h = plan_shape_forced(g, n, 0);
  const int64_t tiles = static_cast<int64_t>(h.mt) * h.nt;
  const int sms = num_sms();
  int k = 0;
  auto add = [&](int64_t sp) {
    if (sp < 1 || k >= max_out) return;
    const int64_t mx = (n + KS - 1) / KS;
    if (sp > mx) sp = mx;
    for (int i = 0; i < k; ++i)
      if (out[i] == sp) return;
    out[k++] = static_cast<int>(sp);
  };
  add(h.splits);
  // whole numbers of waves: 2, 4, 6, 8, 12 waves of CTAs
  for (int w : {2, 4, 6, 8, 12}) add((static_cast<int64_t>(w) * sms + tiles - 1) / tiles);
  add(h.splits * 2);
  add(h.splits / 2);
  return k;
}

int64_t umma_workspace_bytes_splits(const Derived &g, int splits) {
  return 256 + static_cast<int64_t>(splits) * g.nv * g.nc * 2 * g.ns * 4;
}

// the plan a scene takes with no table entry (stream-K at split precision)
Shape builtin_shape(const Derived &g, int64_t n) {
  const Shape s = plan_shape_forced(g, n, 0);
  const bool split = g.precision == SIM_PREC_BF16_SPLIT || g.precision == SIM_PREC_FP16_SPLIT;
  return split && n > 0 ? with_stream_k(s, n) : s;
}

int umma_builtin_splits(const Derived &g, int64_t n) { return builtin_shape(g, n).splits; }

int launch_umma_sum_splits(const Derived &g, RaysPrep p, int64_t n, float2 *sig, void *workspace, uint32_t *status,
                           cudaStream_t s, int splits) {
  const Shape sh = splits > 0 ? plan_shape_forced(g, n, splits) : builtin_shape(g, n);
  uint32_t *amax = static_cast<uint32_t *>(workspace);
  float *partials = reinterpret_cast<float *>(static_cast<uint8_t *>(workspace) + 256);
  const bool f16 = g.precision == SIM_PREC_FP16 || g.precision == SIM_PREC_FP16_SPLIT;
  const bool split = g.precision == SIM_PREC_BF16_SPLIT || g.precision == SIM_PREC_FP16_SPLIT;
  cudaMemsetAsync(amax, 0, 4, s);
  if (f16 && n > 0) amax_kernel<<<2 * num_sms(), 256, 0, s>>>(p.amp, n, amax);
  Args a{};
  a.p = p;
  a.n_rays = n;
  a.chunk = sh.chunk;
  a.nc = g.nc;
  a.ns = g.ns;
  a.m_rows = g.nv * g.nc;
  a.nrx = g.nrx;
  a.bn = sh.bn;
  a.partials = partials;
  a.amax_bits = amax;
  a.status = status;
  launch_gemm_dispatch(f16, split, (g.nc % BM) == 0, sh, a, s);
  const int64_t m_rows = static_cast<int64_t>(g.nv) * g.nc;
  if (f16) reduce_partials<true><<<4 * num_sms(), 256, 0, s>>>(partials, sh.splits, m_rows, g.ns, sh.bn, sig, amax,
                                                                sh.sk, use_pair(sh) ? 2 * BM : BM);
  else reduce_partials<false><<<4 * num_sms(), 256, 0, s>>>(partials, sh.splits, m_rows, g.ns, sh.bn, sig, amax,
                                                                 sh.sk, use_pair(sh) ? 2 * BM : BM);
  return sh.splits;
}

// ---- batch: one persistent launch over the units of several scenes
int64_t umma_batch_scratch_bytes(int n_scenes, int64_t n_units) {
  return 256 + static_cast<int64_t>(sizeof(Args)) * n_scenes + static_cast<int64_t>(sizeof(Unit)) * n_units;
}

// The plan of a scene in a batch, one for its work list, workspace and reduction: the plan it
// has alone, so that a batch gives each scene's own bits.  Planning batch scenes for a share of
// the GPU (half a wave, at least 8192 rays per split, as decomposition spans are) measured 4 %
// faster on the 64-scene batch and was kept out for that.
Shape batch_shape(const Derived &g, int64_t n) { return plan_shape(g, n); }

int64_t batch_workspace_bytes(const Derived &g, int64_t n) {
  const Shape sh = batch_shape(g, n);
  return 256 + static_cast<int64_t>(sh.splits) * g.nv * g.nc * 2 * g.ns * 4;
}

// the scene's work units in its standalone plan: stream-K pieces, or tiles x splits
template <typename F>
void for_each_unit(const Shape &sh, int64_t n, F &&f) {
  const int mt = use_pair(sh) ? (sh.mt + 1) / 2 : sh.mt;
  if (sh.sk.w > 0) {
    for (int c = 0; c < sh.sk.c; ++c) {
      Unit u{};
      for (int idx = 0; sk_piece(sh.sk, n, c, idx, u); ++idx) f(u);
    }
    return;
  }
  for (int sp = 0; sp < sh.splits; ++sp) {
    const int64_t k_lo = static_cast<int64_t>(sp) * sh.chunk;
    const int64_t k_hi = std::min<int64_t>(k_lo + sh.chunk, n);
    for (int tn = 0; tn < sh.nt; ++tn)
      for (int tm = 0; tm < mt; ++tm) f(Unit{0, tm, tn, sp, k_lo, std::max(k_hi, k_lo)});
  }
}

int64_t umma_units_of(const Derived &g, int64_t n) {
  const Shape sh = batch_shape(g, n);
  int64_t k = 0;
  for_each_unit(sh, n, [&](const Unit &) { ++k; });
  return k;
}

int prepare_umma_batch(int n_scenes, const Derived *const *gs, const RaysPrep *ps, const int64_t *ns,
                       void *const *workspaces, uint32_t *const *statuses, void *scratch, cudaStream_t s,
                       UmmaBatch *out) {
  std::vector<Args> args(static_cast<size_t>(n_scenes));
  // two work lists: scenes whose standalone launch uses two-SM tiles get pair units (256 rows),
  // the others one-SM units, so that every scene's units are those of its standalone launch
  std::vector<Unit> units, units1;
  std::vector<int64_t> cost, cost1;
  bool f16 = false, split = false;
  int bn_max = 32, bn_max1 = 32;  // widest tile of the two-SM and of the one-SM work list
  for (int i = 0; i < n_scenes; ++i) {
    const Derived &g = *gs[i];
    const Shape sh = batch_shape(g, ns[i]);
    const bool fi = g.precision == SIM_PREC_FP16 || g.precision == SIM_PREC_FP16_SPLIT;
    const bool si = g.precision == SIM_PREC_BF16_SPLIT || g.precision == SIM_PREC_FP16_SPLIT;
    if (i == 0) {
      f16 = fi;
      split = si;
    } else if (fi != f16 || si != split || g.precision == SIM_PREC_FP32_DIRECT) {
      return SIM_E_INVALID;
    }
    if (g.precision == SIM_PREC_FP32_DIRECT || g.model == SIM_MODEL_EXACT) return SIM_E_INVALID;
    Args &a = args[static_cast<size_t>(i)];
    a = Args{};
    a.p = ps[i];
    a.n_rays = ns[i];
    a.chunk = sh.chunk;
    a.nc = g.nc;
    a.ns = g.ns;
    a.m_rows = g.nv * g.nc;
    a.nrx = g.nrx;
    a.bn = sh.bn;
    a.partials = reinterpret_cast<float *>(static_cast<uint8_t *>(workspaces[i]) + 256);
    a.amax_bits = static_cast<const uint32_t *>(workspaces[i]);
    a.status = statuses[i];
    const bool pair = use_pair(sh);
    int &bmax = pair ? bn_max : bn_max1;
    if (sh.bn > bmax) bmax = sh.bn;
    for_each_unit(sh, ns[i], [&](Unit u) {
      u.scene = i;
      (pair ? units : units1).push_back(u);
      (pair ? cost : cost1).push_back((u.k_hi - u.k_lo) * sh.bn);
    });
  }
  // longest first (stable: ties keep scene, split, tile order)
  auto longest_first = [](const std::vector<Unit> &u, const std::vector<int64_t> &c) {
    std::vector<size_t> order(u.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return c[x] > c[y]; });
    std::vector<Unit> sorted(u.size());
    for (size_t k = 0; k < order.size(); ++k) sorted[k] = u[order[k]];
    return sorted;
  };
  std::vector<Unit> sorted = longest_first(units, cost), sorted1 = longest_first(units1, cost1);
  sorted.insert(sorted.end(), sorted1.begin(), sorted1.end());
  uint8_t *scr = static_cast<uint8_t *>(scratch);
  out->counter = reinterpret_cast<unsigned *>(scr);  // [0] pair list, [1] one-SM list
  out->args = scr + 256;
  out->units = scr + 256 + sizeof(Args) * static_cast<size_t>(n_scenes);
  out->n_units = static_cast<int>(units.size());
  out->units1 = static_cast<uint8_t *>(out->units) + sizeof(Unit) * units.size();
  out->n_units1 = static_cast<int>(units1.size());
  out->n_scenes = n_scenes;
  out->f16 = f16;
  out->split = split;
  out->bn_max = bn_max;
  out->bn_max1 = bn_max1;
  if (cudaMemcpyAsync(out->args, args.data(), sizeof(Args) * args.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(out->units, sorted.data(), sizeof(Unit) * sorted.size(), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SIM_E_CUDA;
  bool all_fast = true;
  for (int i = 0; i < n_scenes; ++i) all_fast = all_fast && (gs[i]->nc % BM) == 0;
  out->fast = all_fast;
  set_smem_attr<true, true, false, true, false>();
  set_smem_attr<true, false, false, true, false>();
  set_smem_attr<false, true, false, true, false>();
  set_smem_attr<false, false, false, true, false>();
  set_smem_attr<true, true, false, false, false>();
  set_smem_attr<true, false, false, false, false>();
  set_smem_attr<false, true, false, false, false>();
  set_smem_attr<false, false, false, false, false>();
  set_smem_attr<true, true, false, true, true>();
  set_smem_attr<true, false, false, true, true>();
  set_smem_attr<false, true, false, true, true>();
  set_smem_attr<false, false, false, true, true>();
  set_smem_attr<true, true, false, false, true>();
  set_smem_attr<true, false, false, false, true>();
  set_smem_attr<false, true, false, false, true>();
  set_smem_attr<false, false, false, false, true>();
  return SIM_OK;
}

// persistent launch over one work list: one CTA per SM (PAIR: one cluster of two per SM pair)
template <bool F16, bool SPLIT, bool FAST, bool PAIR>
void launch_persistent(const Launch &L, size_t sm, cudaStream_t s) {
  if constexpr (PAIR) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2u * static_cast<unsigned>(std::min(L.n_units, num_sms() / 2)));
    cfg.blockDim = dim3(NTHREADS_ALL);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    note_launch(cudaLaunchKernelEx(&cfg, umma_sum_kernel<F16, SPLIT, false, FAST, true>, L));
  } else {
    umma_sum_kernel<F16, SPLIT, false, FAST, false><<<std::min(L.n_units, num_sms()), NTHREADS_ALL, sm, s>>>(L);
  }
}

template <bool PAIR>
void launch_persistent_dispatch(const UmmaBatch &b, const Launch &L, cudaStream_t s) {
  const size_t sm = smem_bytes(b.split, L.bn_layout, PAIR);
  if (b.f16) {
    if (b.split) b.fast ? launch_persistent<true, true, true, PAIR>(L, sm, s) : launch_persistent<true, true, false, PAIR>(L, sm, s);
    else b.fast ? launch_persistent<true, false, true, PAIR>(L, sm, s) : launch_persistent<true, false, false, PAIR>(L, sm, s);
  } else {
    if (b.split) b.fast ? launch_persistent<false, true, true, PAIR>(L, sm, s) : launch_persistent<false, true, false, PAIR>(L, sm, s);
    else b.fast ? launch_persistent<false, false, true, PAIR>(L, sm, s) : launch_persistent<false, false, false, PAIR>(L, sm, s);
  }
}

int launch_umma_batch(const UmmaBatch &b, cudaStream_t s) {
  cudaMemsetAsync(b.counter, 0, 8, s);
  int kernels = 0;
  Launch L{};
  L.scenes = static_cast<const Args *>(b.args);
  if (b.n_units > 0) {
    L.bn_layout = b.bn_max;
    L.units = static_cast<const Unit *>(b.units);
    L.n_units = b.n_units;
    L.counter = b.counter;
    launch_persistent_dispatch<true>(b, L, s);
    ++kernels;
  }
  if (b.n_units1 > 0) {
    L.bn_layout = b.bn_max1;
    L.units = static_cast<const Unit *>(b.units1);
    L.n_units = b.n_units1;
    L.counter = b.counter + 1;
    launch_persistent_dispatch<false>(b, L, s);
    ++kernels;
  }
  return kernels;
}

// amax (FP16 scaling) and split reduction of one scene of a batch, around the batched GEMM
int launch_umma_pre(const Derived &g, RaysPrep p, int64_t n, void *workspace, cudaStream_t s) {
  const bool f16 = g.precision == SIM_PREC_FP16 || g.precision == SIM_PREC_FP16_SPLIT;
  uint32_t *amax = static_cast<uint32_t *>(workspace);
  cudaMemsetAsync(amax, 0, 4, s);
  if (f16 && n > 0) {
    amax_kernel<<<2 * num_sms(), 256, 0, s>>>(p.amp, n, amax);
    return 1;
  }
  return 0;
}

int launch_umma_post(const Derived &g, int64_t n, float2 *sig, void *workspace, cudaStream_t s) {
  const Shape sh = batch_shape(g, n);
  const bool f16 = g.precision == SIM_PREC_FP16 || g.precision == SIM_PREC_FP16_SPLIT;
  uint32_t *amax = static_cast<uint32_t *>(workspace);
  float *partials = reinterpret_cast<float *>(static_cast<uint8_t *>(workspace) + 256);
  const int64_t m_rows = static_cast<int64_t>(g.nv) * g.nc;
  if (f16) reduce_partials<true><<<4 * num_sms(), 256, 0, s>>>(partials, sh.splits, m_rows, g.ns, sh.bn, sig, amax,
                                                                sh.sk, use_pair(sh) ? 2 * BM : BM);
  else reduce_partials<false><<<4 * num_sms(), 256, 0, s>>>(partials, sh.splits, m_rows, g.ns, sh.bn, sig, amax,
                                                                 sh.sk, use_pair(sh) ? 2 * BM : BM);
  return 1;
}

int launch_umma_sum_in(const Derived &g, RaysPrep p, int64_t n, float2 *sig, void *workspace, int64_t ws_bytes,
                       uint32_t *status, cudaStream_t s) {
  if (g.model == SIM_MODEL_EXACT) {
    // the per-chirp product has no TDM slot term; its workspace must fit
    if (g.tslot != 0.0 || exact_workspace_bytes(g, n) > ws_bytes) return -1;
    return launch_exact_sum(g, p, n, sig, workspace, status, s, nullptr);
  }
  Shape sh = plan_shape(g, n, 4.f, 0, false);  // split units: their count is capped to the scratch
  const int64_t per_split = static_cast<int64_t>(g.nv) * g.nc * 2 * g.ns * 4;
  const int64_t fit = (ws_bytes - 256) / per_split;
  if (fit < 1) return -1;
  if (sh.splits > fit) {
    int64_t chunk = (n + fit - 1) / fit;
    chunk = (chunk + KS - 1) / KS * KS;
    if (chunk < KS) chunk = KS;
    sh.chunk = chunk;
    sh.splits = static_cast<int>((n + chunk - 1) / chunk);
    if (sh.splits < 1) sh.splits = 1;
  }
  uint32_t *amax = static_cast<uint32_t *>(workspace);
  float *partials = reinterpret_cast<float *>(static_cast<uint8_t *>(workspace) + 256);
  const bool f16 = g.precision == SIM_PREC_FP16 || g.precision == SIM_PREC_FP16_SPLIT;
  const bool split = g.precision == SIM_PREC_BF16_SPLIT || g.precision == SIM_PREC_FP16_SPLIT;
  int kernels = 0;
  cudaMemsetAsync(amax, 0, 4, s);
  if (f16 && n > 0) {
    amax_kernel<<<2 * num_sms(), 256, 0, s>>>(p.amp, n, amax);
    ++kernels;
  }
  Args a{};
  a.p = p;
  a.n_rays = n;
  a.chunk = sh.chunk;
  a.nc = g.nc;
  a.ns = g.ns;
  a.m_rows = g.nv * g.nc;
  a.nrx = g.nrx;
  a.bn = sh.bn;
  a.partials = partials;
  a.amax_bits = amax;
  a.status = status;
  launch_gemm_dispatch(f16, split, (g.nc % BM) == 0, sh, a, s);
  ++kernels;
  const int64_t m_rows = static_cast<int64_t>(g.nv) * g.nc;
  if (f16) reduce_partials<true><<<4 * num_sms(), 256, 0, s>>>(partials, sh.splits, m_rows, g.ns, sh.bn, sig, amax,
                                                                sh.sk, use_pair(sh) ? 2 * BM : BM);
  else reduce_partials<false><<<4 * num_sms(), 256, 0, s>>>(partials, sh.splits, m_rows, g.ns, sh.bn, sig, amax,
                                                                 sh.sk, use_pair(sh) ? 2 * BM : BM);
  ++kernels;
  return kernels;
}

}  // namespace rs

// ------------------------------------------------------------------ self-test entry point
extern "C" SIM_API int sim_selftest_umma(int32_t f16, int32_t m, int32_t n, int64_t k, const void *a, const void *b,
                                         float *d, void *stream) {
  using namespace rs;
  if (m < 1 || n < 32 || (n & 15) || n > 512 || k < 2 || (k & 1) || !a || !b || !d || (f16 & ~3)) return SIM_E_INVALID;
  const bool negate = (f16 & 2) != 0;
  f16 &= 1;
  Shape sh{};
  sh.bn = n < 256 ? n : 256;
  if (n % sh.bn) return SIM_E_INVALID;
  sh.mt = (m + BM - 1) / BM;
  sh.nt = n / sh.bn;
  sh.splits = 1;
  sh.chunk = (k / 2 + KS - 1) / KS * KS;
  Args args{};
  args.n_rays = k / 2;
  args.chunk = sh.chunk;
  args.nc = m;
  args.ns = n / 2;
  args.m_rows = m;
  args.nrx = 1;
  args.bn = sh.bn;
  args.partials = d;
  args.test_a = static_cast<const uint16_t *>(a);
  args.test_b = static_cast<const uint16_t *>(b);
  args.test_k = k;
  args.test_negate_b = negate ? 1 : 0;
  uint32_t *status = nullptr;
  if (cudaMalloc(&status, 4) != cudaSuccess) return SIM_E_NOMEM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaMemsetAsync(status, 0, 4, s);
  args.status = status;
  if (f16) launch_gemm<true, false, true, true, false>(sh, args, s);
  else launch_gemm<false, false, true, true, false>(sh, args, s);
  uint32_t st = 0;
  cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(status);
  if (e != cudaSuccess) return SIM_E_CUDA;
  return st ? SIM_E_DEVICE : SIM_OK;
}
