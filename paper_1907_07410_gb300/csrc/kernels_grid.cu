// Activity-quantile cut of one side of the rating matrix, on the device.
//
// The paper cuts X into equal blocks (Section 3, Eq. "datax"). On
// long-tailed data that leaves a few blocks holding most ratings, so the
// batched form orders the ids of one side (users or items) by their number
// of training ratings, busiest first and lower id first on ties, and cuts
// that order where the running count of ratings first reaches g / parts of
// all ratings: bound g is the smallest position j with
// parts * C_j >= g * nnz in exact integers, C_j being the ratings of the
// first j ids in the order. Each block row (column) then holds about the
// same number of ratings.
//
//   1. k_qhist: ratings per id (32-bit atomics; nnz < 2^32). With at most
//      kQSmemBins ids (the item side) each CTA counts into a shared-memory
//      histogram and adds its nonzero bins to the global counts, since
//      popular ids make global atomics contend (1.4 ms for the 17,770 items
//      of the large workload against 0.5 ms for its 480,189 users).
//   2. k_qkeys: one 64-bit key per id, (2^32 - 1 - count) << 32 | id, so
//      ascending keys are the order above. Keys are distinct. The array is
//      padded to a power of two with all-ones keys, which sort last.
//   3. Bitonic sort of the keys: passes with a partner distance of 2048 or
//      more run one global pass per launch (k_qbitonic_global); the rest of
//      each merge stage runs in shared memory on tiles of 4096 keys
//      (k_qbitonic_shared). The result does not depend on scheduling.
//   4. k_qperm: perm[id] = position.
//   5. k_qtile, k_qcum: C_j for j = 0 .. size: per 4096-position tile the
//      tile's total, then each tile adds the totals before it and scans its
//      own positions (integer sums: exact in any order).
//   6. k_qbounds: bound g by binary search on C (non-decreasing).
#include "kernels.h"

namespace bsvd {

namespace {

constexpr int kTile = 4096;        // keys per shared-memory bitonic tile
constexpr int kTileThreads = 1024;

__global__ void k_qhist(const int32_t *__restrict__ ids, int64_t nnz,
                        int64_t size, unsigned int *__restrict__ counts,
                        int32_t *err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += stride) {
    const int32_t v = ids[e];
    if (v < 0 || v >= size) {
      atomicOr(err, kErrIndex);
      continue;
    }
    atomicAdd(&counts[v], 1u);
  }
}

constexpr int kQSmemBins = 24576;  // 96 KiB of shared counts

__global__ void __launch_bounds__(1024)
k_qhist_smem(const int32_t *__restrict__ ids, int64_t nnz, int32_t size,
             unsigned int *__restrict__ counts, int32_t *err) {
  extern __shared__ unsigned int sc[];
  for (int b = threadIdx.x; b < size; b += blockDim.x) sc[b] = 0;
  __syncthreads();
  int32_t bad = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += stride) {
    const int32_t v = ids[e];
    if (v < 0 || v >= size) {
      bad = kErrIndex;
      continue;
    }
    atomicAdd(&sc[v], 1u);
  }
  if (bad) atomicOr(err, bad);
  __syncthreads();
  for (int b = threadIdx.x; b < size; b += blockDim.x)
    if (sc[b]) atomicAdd(&counts[b], sc[b]);
}

__global__ void k_qkeys(const unsigned int *__restrict__ counts, int64_t size,
                        int64_t padded, unsigned long long *__restrict__ keys) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
       j < padded; j += stride) {
    keys[j] = j < size ? ((unsigned long long)(0xFFFFFFFFu - counts[j]) << 32) |
                             (unsigned long long)j
                       : ~0ull;
  }
}

// One bitonic compare-exchange pass over the whole array: element i and its
// partner i ^ j, ascending where (i & k) == 0.
__global__ void k_qbitonic_global(unsigned long long *keys, int64_t padded,
                                  int64_t k, int64_t j) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
       i < padded; i += stride) {
    const int64_t l = i ^ j;
    if (l <= i) continue;
    const unsigned long long a = keys[i], b = keys[l];
    const bool up = (i & k) == 0;
    if ((a > b) == up) {
      keys[i] = b;
      keys[l] = a;
    }
  }
}

// The passes j = j0, j0 / 2, ..., 1 of merge stage k on one tile of kTile
// keys (j0 < kTile). With k < kTile this also runs every earlier stage,
// sorting the tile from scratch.
__global__ void __launch_bounds__(kTileThreads)
k_qbitonic_shared(unsigned long long *keys, int64_t k_stage, int64_t j0,
                  int full) {
  __shared__ unsigned long long s[kTile];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  for (int t = threadIdx.x; t < kTile; t += blockDim.x) s[t] = keys[base + t];
  __syncthreads();
  auto pass = [&](int64_t k, int64_t j) {
    for (int t = threadIdx.x; t < kTile; t += blockDim.x) {
      const int l = t ^ (int)j;
      if (l > t) {
        const unsigned long long a = s[t], b = s[l];
        const bool up = ((base + t) & k) == 0;
        if ((a > b) == up) {
          s[t] = b;
          s[l] = a;
        }
      }
    }
    __syncthreads();
  };
  if (full) {
    for (int64_t k = 2; k <= kTile; k <<= 1)
      for (int64_t j = k >> 1; j > 0; j >>= 1) pass(k, j);
  } else {
    for (int64_t j = j0; j > 0; j >>= 1) pass(k_stage, j);
  }
  for (int t = threadIdx.x; t < kTile; t += blockDim.x) keys[base + t] = s[t];
}

__global__ void k_qperm(const unsigned long long *__restrict__ keys,
                        int64_t size, int32_t *__restrict__ perm) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
       pos < size; pos += stride)
    perm[keys[pos] & 0xFFFFFFFFull] = (int32_t)pos;
}

// The count of the id at sorted position j, from its key.
__device__ __forceinline__ long long key_count(unsigned long long key) {
  return (long long)(0xFFFFFFFFu - (unsigned int)(key >> 32));
}

// Total of each 4096-position tile (less than 2^32: nnz < 2^32).
__global__ void __launch_bounds__(1024)
k_qtile(const unsigned long long *__restrict__ keys, int64_t size,
        unsigned int *__restrict__ tile_sum) {
  __shared__ long long part[32];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  long long v = 0;
  for (int j = threadIdx.x; j < kTile; j += blockDim.x)
    if (base + j < size) v += key_count(keys[base + j]);
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < 32; ++w) t += part[w];
    tile_sum[blockIdx.x] = (unsigned int)t;
  }
}

// C_0 = 0, C_{j+1} = C_j + count at position j: tile b adds the totals of
// tiles 0 .. b-1, then scans its 4096 positions (4 per thread, a shared
// Hillis-Steele scan of the 1024 thread sums).
__global__ void __launch_bounds__(1024)
k_qcum(const unsigned long long *__restrict__ keys, int64_t size,
       const unsigned int *__restrict__ tile_sum,
       long long *__restrict__ cum) {
  __shared__ long long part[1024];
  __shared__ long long s_off;
  const int t = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * kTile;
  if (t < 32) {
    long long o = 0;
    for (int b = t; b < (int)blockIdx.x; b += 32) o += tile_sum[b];
    for (int d = 16; d > 0; d >>= 1) o += __shfl_xor_sync(0xffffffffu, o, d);
    if (t == 0) s_off = o;
  }
  long long c[4];
  long long sum = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t j = base + 4 * t + q;
    c[q] = j < size ? key_count(keys[j]) : 0;
    sum += c[q];
  }
  part[t] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const long long v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  long long run = s_off + (t > 0 ? part[t - 1] : 0);
  if (blockIdx.x == 0 && t == 0) cum[0] = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t j = base + 4 * t + q;
    run += c[q];
    if (j < size) cum[j + 1] = run;
  }
}

__global__ void k_qbounds(const long long *__restrict__ cum, int64_t size,
                          int32_t parts, long long total,
                          int64_t *__restrict__ bounds) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g > parts) return;
  if (g == 0) { bounds[0] = 0; return; }
  if (g == parts) { bounds[parts] = size; return; }
  // smallest j in [0, size] with parts * C_j >= g * total
  const long long want = (long long)g * total;
  int64_t lo = 0, hi = size;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if ((long long)parts * cum[mid] >= want) hi = mid;
    else lo = mid + 1;
  }
  bounds[g] = lo;
}

int grid_of(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

int64_t quantile_cut_padded(int64_t size) {
  int64_t p = kTile;
  while (p < size) p <<= 1;
  return p;
}

cudaError_t launch_quantile_cut(const int32_t *ids, int64_t nnz, int64_t size,
                                int32_t parts, unsigned int *counts,
                                unsigned long long *keys, long long *cum,
                                int32_t *perm, int64_t *bounds, int32_t *err,
                                int64_t *launches, cudaStream_t st) {
  const int64_t padded = quantile_cut_padded(size);
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned int) * size, st);
  if (e != cudaSuccess) return e;
  int64_t n = 0;
  if (nnz > 0) {
    if (size <= kQSmemBins) {
      const size_t sm = sizeof(unsigned int) * (size_t)size;
      e = cudaFuncSetAttribute(k_qhist_smem,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(sizeof(unsigned int) * kQSmemBins));
      if (e != cudaSuccess) return e;
      int g = (int)((nnz + 1023) / 1024);
      if (g > 152 * 2) g = 152 * 2;
      k_qhist_smem<<<g, 1024, sm, st>>>(ids, nnz, (int32_t)size, counts, err);
    } else {
      k_qhist<<<grid_of(nnz), 256, 0, st>>>(ids, nnz, size, counts, err);
    }
    ++n;
  }
  k_qkeys<<<grid_of(padded), 256, 0, st>>>(counts, size, padded, keys);
  ++n;
  const int tiles = (int)(padded / kTile);
  k_qbitonic_shared<<<tiles, kTileThreads, 0, st>>>(keys, 0, 0, 1);
  ++n;
  for (int64_t k = 2 * kTile; k <= padded; k <<= 1) {
    int64_t j = k >> 1;
    for (; j >= kTile; j >>= 1) {
      k_qbitonic_global<<<grid_of(padded), 256, 0, st>>>(keys, padded, k, j);
      ++n;
    }
    k_qbitonic_shared<<<tiles, kTileThreads, 0, st>>>(keys, k, j, 0);
    ++n;
  }
  k_qperm<<<grid_of(size), 256, 0, st>>>(keys, size, perm);
  // the counts are in the keys now: their array holds the tile totals
  const int ctiles = (int)((size + kTile - 1) / kTile);
  if (ctiles > 0) {
    k_qtile<<<ctiles, 1024, 0, st>>>(keys, size, counts);
    k_qcum<<<ctiles, 1024, 0, st>>>(keys, size, (const unsigned int *)counts,
                                    cum);
    n += 2;
  } else {
    e = cudaMemsetAsync(cum, 0, sizeof(long long), st);
    if (e != cudaSuccess) return e;
  }
  k_qbounds<<<(parts + 256) / 256, 256, 0, st>>>(cum, size, parts,
                                                  (long long)nnz, bounds);
  n += 2;
  if (launches) *launches += n;
  return cudaGetLastError();
}

}  // namespace bsvd
