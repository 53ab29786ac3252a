// K_d: automatic annotation from ray meta data (arXiv 2305.14176, Sec. II-C).
//
// Eq. 5 splits the signal into parts by ray meta data; here the part of each object id
// is scored per range/Doppler/angle cell by the energy its rays deposit at their
// analytic cell, and the cell is labelled with the strongest object.
//
//   E[cell, obj] = sum over rays i with cell_i = cell and obj_i = obj of q_i   (int64)
//   label[cell]  = argmax_obj E[cell, obj], ties to the smallest id; -1 if no ray
//
// Integer atomics make every pass order independent, so the labels are bit exact
// whatever the schedule.  Pairs (cell, obj) and cells live in two open-addressing hash
// tables of at least twice the ray count (load <= 1/2), probed linearly with a hard
// probe limit that sets a status bit instead of looping.
#include "internal.h"

namespace rs {

int64_t label_capacity(int64_t n_rays) {
  int64_t c = 1024;
  while (c < 2 * n_rays) c <<= 1;
  return c;
}

namespace {

constexpr uint64_t kEmpty64 = ~0ull;
constexpr uint32_t kEmpty32 = ~0u;
constexpr int kMaxProbe = 1 << 16;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // MurmurHash3 finalizer
  z ^= z >> 33;
  z *= 0xff51afd7ed558ccdull;
  z ^= z >> 33;
  z *= 0xc4ceb9fe1a85ec53ull;
  z ^= z >> 33;
  return z;
}

// slot of `key` in the pair table, inserting it if absent; -1 past the probe limit
__device__ int64_t pair_slot(uint64_t *keys, int64_t mask, uint64_t key) {
  int64_t h = static_cast<int64_t>(mix64(key) & static_cast<uint64_t>(mask));
  for (int probe = 0; probe < kMaxProbe; ++probe) {
    const unsigned long long prev =
        atomicCAS(reinterpret_cast<unsigned long long *>(keys + h), kEmpty64, key);
    if (prev == kEmpty64 || prev == key) return h;
    h = (h + 1) & mask;
  }
  return -1;
}

__device__ int64_t cell_slot(uint32_t *keys, int64_t mask, uint32_t key, bool insert) {
  int64_t h = static_cast<int64_t>(mix64(key) & static_cast<uint64_t>(mask));
  for (int probe = 0; probe < kMaxProbe; ++probe) {
    uint32_t prev;
    if (insert) prev = atomicCAS(keys + h, kEmpty32, key);
    else prev = keys[h];
    if (prev == key) return h;
    if (prev == kEmpty32) return insert ? h : -1;
    h = (h + 1) & mask;
  }
  return -1;
}

// pass 1: per ray, add its energy to its (cell, object) pair
__global__ void label_accumulate(RaysPrep p, const int32_t *__restrict__ obj, int64_t n, LabelScratch sc,
                                 uint32_t *status) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const int32_t cell = p.cell[i];
  if (cell < 0) return;  // invalid ray
  const uint64_t key = (static_cast<uint64_t>(cell) << 32) | static_cast<uint32_t>(obj[i]);
  const int64_t h = pair_slot(sc.pair_key, sc.capacity - 1, key);
  if (h < 0) { atomicOr(status, kStatusHashFull); return; }
  atomicAdd(reinterpret_cast<unsigned long long *>(sc.pair_energy + h),
            static_cast<unsigned long long>(p.energy[i]));
}

// pass 2: per pair, raise its cell's maximum energy
__global__ void label_cell_max(LabelScratch sc, uint32_t *status) {
  const int64_t h = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (h >= sc.capacity) return;
  const uint64_t key = sc.pair_key[h];
  if (key == kEmpty64) return;
  const int64_t c = cell_slot(sc.cell_key, sc.capacity - 1, static_cast<uint32_t>(key >> 32), true);
  if (c < 0) { atomicOr(status, kStatusHashFull); return; }
  atomicMax(reinterpret_cast<unsigned long long *>(sc.cell_max + c),
            static_cast<unsigned long long>(sc.pair_energy[h]));
}

// pass 3: per pair holding its cell's maximum, lower the cell's object id
__global__ void label_argmin_id(LabelScratch sc, uint32_t *status) {
  const int64_t h = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (h >= sc.capacity) return;
  const uint64_t key = sc.pair_key[h];
  if (key == kEmpty64) return;
  const int64_t c = cell_slot(sc.cell_key, sc.capacity - 1, static_cast<uint32_t>(key >> 32), false);
  if (c < 0) { atomicOr(status, kStatusHashFull); return; }
  if (sc.pair_energy[h] == sc.cell_max[c])
    atomicMin(sc.cell_obj + c, static_cast<uint32_t>(key & 0xffffffffu));  // ids are >= 0
}

// pass 4: write each occupied cell's label
__global__ void label_write(LabelScratch sc, int32_t *labels) {
  const int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (c >= sc.capacity) return;
  const uint32_t cell = sc.cell_key[c];
  if (cell == kEmpty32) return;
  labels[cell] = static_cast<int32_t>(sc.cell_obj[c]);
}

}  // namespace

int launch_labels(const Derived &g, RaysPrep p, const int32_t *obj, int64_t n, LabelScratch sc,
                  int32_t *labels, uint32_t *status, cudaStream_t s) {
  const size_t cap = static_cast<size_t>(sc.capacity);
  cudaMemsetAsync(labels, 0xff, sizeof(int32_t) * static_cast<size_t>(g.n_cell), s);
  if (n <= 0) return 0;
  cudaMemsetAsync(sc.pair_key, 0xff, sizeof(uint64_t) * cap, s);
  cudaMemsetAsync(sc.pair_energy, 0, sizeof(uint64_t) * cap, s);
  cudaMemsetAsync(sc.cell_key, 0xff, sizeof(uint32_t) * cap, s);
  cudaMemsetAsync(sc.cell_max, 0, sizeof(uint64_t) * cap, s);
  cudaMemsetAsync(sc.cell_obj, 0xff, sizeof(uint32_t) * cap, s);
  const unsigned rb = static_cast<unsigned>((n + 255) / 256);
  const unsigned cb = static_cast<unsigned>((sc.capacity + 255) / 256);
  label_accumulate<<<rb, 256, 0, s>>>(p, obj, n, sc, status);
  label_cell_max<<<cb, 256, 0, s>>>(sc, status);
  label_argmin_id<<<cb, 256, 0, s>>>(sc, status);
  label_write<<<cb, 256, 0, s>>>(sc, labels);
  return 4;
}

}  // namespace rs
