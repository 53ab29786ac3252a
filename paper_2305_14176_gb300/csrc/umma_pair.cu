// Self-test of the two-SM tensor-core tile: a CTA pair (a cluster of two) computes
// D[256][N] = A[256][K] B[N][K]^T with one tcgen05.mma.cta_group::2 per 16-deep K step.
//
// Each CTA of the pair holds its own 128 rows of A and its own N/2 rows of B (columns of
// D) in shared memory at the same offsets, in the no-swizzle K-major core-matrix layout of
// the single-SM path; the even CTA issues the MMAs, the product lands in both CTAs'
// tensor memory (each its 128 rows, all N columns).  Readiness crosses the pair through
// mbarriers: every thread of both CTAs arrives on the issuing CTA's barrier once its part of
// a stage is in shared memory (remote arrivals through the cluster shared window), and the
// MMA commit arrives on the barriers of both CTAs (multicast).  All waits are bounded.
#include <cuda_runtime.h>

#include "internal.h"

namespace {

constexpr int PT = 128;                 // threads per CTA
constexpr int PK = 64;                  // K elements per stage (four MMA K steps)
constexpr uint64_t kPairWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t su32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// this CTA's shared address `a` as seen in the shared window of cluster CTA `rank`
__device__ __forceinline__ uint32_t peer_addr(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void bar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
// arrive on a barrier of any CTA of the cluster (cluster-scope release)
__device__ __forceinline__ void bar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(a), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool bar_wait(uint32_t a, uint32_t parity) {
  const uint64_t t0 = now_ns();
  while (!bar_try(a, parity))
    if (now_ns() - t0 > kPairWaitNs) return false;
  return true;
}
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__host__ __device__ constexpr uint32_t idesc_f16(bool f16, int m, int n) {
  return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(m >> 4) << 24);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PT, 1)
    pair_tile_kernel(const uint16_t *__restrict__ A, const uint16_t *__restrict__ B, float *__restrict__ D, int n,
                     int64_t k, int f16, uint32_t *status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[3];  // ready (issuing CTA), consumed, done
  __shared__ uint32_t tmem_holder;
  const uint32_t rank = cluster_rank();
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int nh = n / 2;                          // B rows (D columns) this CTA holds
  const uint32_t lbo_a = 128 * 16, lbo_b = static_cast<uint32_t>(nh) * 16;
  uint8_t *sa = smem, *sb = smem + 128 * PK * 2;
  const uint32_t ready = su32(&bars[0]), consumed = su32(&bars[1]), done = su32(&bars[2]);
  const uint32_t ready_leader = peer_addr(ready, 0);
  if (t == 0) {
    bar_init(ready, 2 * PT);
    bar_init(consumed, 1);
    bar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_holder)),
                 "r"(256u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_holder;
  bool failed = false;
  const int n_st = static_cast<int>((k + PK - 1) / PK);
  for (int st = 0; st < n_st && !failed; ++st) {
    if (st > 0 && !bar_wait(consumed, (st - 1) & 1)) {
      failed = true;
      break;
    }
    // this CTA's 128 rows of A and n/2 rows of B for K elements [st PK, st PK + PK)
    for (int item = t; item < 128 * (PK / 8); item += PT) {
      const int r = item % 128, kc = item / 128;
      const int64_t row = static_cast<int64_t>(rank) * 128 + r;
      uint32_t v[4];
      for (int q = 0; q < 4; ++q) {
        const int64_t kk = static_cast<int64_t>(st) * PK + kc * 8 + 2 * q;
        v[q] = 0;
        if (kk < k) v[q] = static_cast<uint32_t>(A[row * k + kk]) | (static_cast<uint32_t>(A[row * k + kk + 1]) << 16);
      }
      *reinterpret_cast<uint4 *>(sa + kc * lbo_a + r * 16) = make_uint4(v[0], v[1], v[2], v[3]);
    }
    for (int item = t; item < nh * (PK / 8); item += PT) {
      const int r = item % nh, kc = item / nh;
      const int64_t col = static_cast<int64_t>(rank) * nh + r;
      uint32_t v[4];
      for (int q = 0; q < 4; ++q) {
        const int64_t kk = static_cast<int64_t>(st) * PK + kc * 8 + 2 * q;
        v[q] = 0;
        if (kk < k) v[q] = static_cast<uint32_t>(B[col * k + kk]) | (static_cast<uint32_t>(B[col * k + kk + 1]) << 16);
      }
      *reinterpret_cast<uint4 *>(sb + kc * lbo_b + r * 16) = make_uint4(v[0], v[1], v[2], v[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    bar_arrive_cluster(ready_leader);
    if (rank == 0 && t == 0) {
      if (!bar_wait(ready, st & 1)) {
        failed = true;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t id = idesc_f16(f16 != 0, 256, n);
        for (int kk = 0; kk < PK / 16; ++kk) {
          const uint64_t da = sdesc(su32(sa) + kk * 2 * lbo_a, lbo_a, 128);
          const uint64_t db = sdesc(su32(sb) + kk * 2 * lbo_b, lbo_b, 128);
          const uint32_t acc = (st > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(da), "l"(db), "r"(id), "r"(acc)
              : "memory");
        }
        // the stage's shared memory is free in both CTAs once these MMAs complete
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                consumed),
            "h"(static_cast<uint16_t>(3))
            : "memory");
      }
    }
  }
  if (rank == 0 && t == 0) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            done),
        "h"(static_cast<uint16_t>(3))
        : "memory");
  }
  if (!bar_wait(done, 0)) failed = true;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!failed) {
    // warp w reads TMEM lanes 32 w .. 32 w + 31: rows rank * 128 + 32 w + lane
    const int64_t row = static_cast<int64_t>(rank) * 128 + warp * 32 + lane;
    const uint32_t trow = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    for (int c = 0; c < n; c += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(trow + static_cast<uint32_t>(c))
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      for (int x = 0; x < 16; ++x) D[row * n + c + x] = __uint_as_float(r[x]);
    }
  } else if (t == 0) {
    atomicOr(status, rs::kStatusWaitLimit);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u) : "memory");
}

}  // namespace

extern "C" SIM_API int sim_selftest_umma_pair(int32_t f16, int32_t n, int64_t k, const void *a, const void *b,
                                              float *d, void *stream) {
  if (n < 32 || n > 256 || (n & 15) || k < 2 || (k & 1) || !a || !b || !d || (f16 & ~1)) return SIM_E_INVALID;
  uint32_t *status = nullptr;
  if (cudaMalloc(&status, 4) != cudaSuccess) return SIM_E_NOMEM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaMemsetAsync(status, 0, 4, s);
  rs::launches_begin();
  const size_t smem = static_cast<size_t>(128 * PK * 2 + (n / 2) * PK * 2);
  rs::note_launch(cudaFuncSetAttribute(pair_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  pair_tile_kernel<<<2, PT, smem, s>>>(static_cast<const uint16_t *>(a), static_cast<const uint16_t *>(b), d, n, k,
                                       f16, status);
  const bool launched = rs::launches_ok();
  uint32_t st = 0;
  cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(status);
  if (!launched || e != cudaSuccess) return SIM_E_CUDA;
  return st ? SIM_E_DEVICE : SIM_OK;
}
