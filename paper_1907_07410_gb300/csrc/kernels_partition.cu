// Partition, block means and dense scatter (Section 3, Eq. "datax").
//
// Pass 1 (k_count) maps every training rating to its block and adds its
// count and its value to per-block totals. Values are summed as 64-bit
// fixed point with 32 fraction bits (x * 2^32), so the totals are exact
// integers and do not depend on the order of the atomic adds.
// Pass 2 (k_means) turns the totals into mu_b = fl32(fl64(sum) / count).
// Pass 3 (k_scatter) writes fl32(x - mu_b) into the zeroed dense blocks.
#include "kernels.h"

namespace bsvd {

namespace {

constexpr int kSmemBlocks = 2048;   // per-CTA histogram size limit

__global__ void k_perm_mark(const int32_t *perm, int64_t n, int32_t *seen,
                            int32_t *err) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = perm[t];
    if (v < 0 || (int64_t)v >= n) { atomicOr(err, kErrBadPerm); continue; }
    atomicAdd(&seen[v], 1);
  }
}

__global__ void k_perm_verify(const int32_t *seen, int64_t n, int32_t *err) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    if (seen[t] != 1) atomicOr(err, kErrBadPerm);
}

__device__ __forceinline__ bool rating_ok(float x) {
  return isfinite(x) && fabsf(x) < 2147483648.0f;
}

__device__ __forceinline__ long long fixed32(float x) {
  // x * 2^32 is exact in float64; round to the nearest integer. (An
  // integer-only version with a branch per exponent range measured about
  // 1 ms slower per pass over the large workload's 90 million ratings.)
  return __double2ll_rn(__dmul_rn((double)x, 4294967296.0));
}

__global__ void __launch_bounds__(256)
k_count(GridDesc g, int64_t nnz, const int32_t *__restrict__ u,
        const int32_t *__restrict__ it, const float *__restrict__ x,
        int32_t nblocks, unsigned long long *counts, long long *sums,
        unsigned int *maxabs_bits, int32_t *err) {
  __shared__ unsigned int s_cnt[kSmemBlocks];
  __shared__ unsigned long long s_sum[kSmemBlocks];
  __shared__ unsigned int s_max;
  const bool use_smem = nblocks <= kSmemBlocks;
  if (use_smem) {
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
      s_cnt[b] = 0;
      s_sum[b] = 0;
    }
  }
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  unsigned int local_max = 0;
  int32_t local_err = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t blk, r, c;
    float xv = x[t];
    if (!locate(g, u[t], it[t], &blk, &r, &c)) { local_err |= kErrIndex; continue; }
    if (!rating_ok(xv)) { local_err |= kErrValue; continue; }
    local_max = max(local_max, __float_as_uint(fabsf(xv)));
    long long fx = fixed32(xv);
    if (use_smem) {
      atomicAdd(&s_cnt[blk], 1u);
      atomicAdd(&s_sum[blk], (unsigned long long)fx);
    } else {
      atomicAdd(&counts[blk], 1ull);
      atomicAdd((unsigned long long *)&sums[blk], (unsigned long long)fx);
    }
  }
  // warp-reduce the max and the error bits, one shared atomic per warp
  for (int o = 16; o > 0; o >>= 1) {
    local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    local_err |= __shfl_xor_sync(0xffffffffu, local_err, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&s_max, local_max);
    if (local_err) atomicOr(err, local_err);
  }
  __syncthreads();
  if (use_smem) {
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
      if (s_cnt[b]) {
        atomicAdd(&counts[b], (unsigned long long)s_cnt[b]);
        atomicAdd((unsigned long long *)&sums[b], s_sum[b]);
      }
    }
  }
  if (threadIdx.x == 0 && s_max) atomicMax(maxabs_bits, s_max);
}

__global__ void __launch_bounds__(1024)
k_means(int32_t nblocks, const unsigned long long *counts,
        const long long *sums, const unsigned int *maxabs_bits, float *mu,
        int32_t *err) {
  __shared__ unsigned long long s_c[1024];
  __shared__ long long s_s[1024];
  unsigned long long c = 0;
  long long s = 0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    c += counts[b];
    s += sums[b];
  }
  s_c[threadIdx.x] = c;
  s_s[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_c[threadIdx.x] += s_c[threadIdx.x + w];
      s_s[threadIdx.x] += s_s[threadIdx.x + w];
    }
    __syncthreads();
  }
  const unsigned long long total_c = s_c[0];
  const long long total_s = s_s[0];
  const double xmax = (double)__uint_as_float(*maxabs_bits);
  // |sum| <= count * max|x| * 2^32 must stay inside int64
  if ((double)total_c * xmax >= 2147483648.0) {
    if (threadIdx.x == 0) atomicOr(err, kErrSumRange);
  }
  float gmean = 0.0f;
  if (total_c)
    gmean = __double2float_rn(__ddiv_rn(__dmul_rn((double)total_s, 0x1p-32),
                                        (double)total_c));
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    unsigned long long cb = counts[b];
    mu[b] = cb ? __double2float_rn(__ddiv_rn(
                     __dmul_rn((double)sums[b], 0x1p-32), (double)cb))
               : gmean;
  }
}

__global__ void __launch_bounds__(256)
k_scatter(GridDesc g, const BlockMeta *__restrict__ meta, int64_t nnz,
          const int32_t *__restrict__ u, const int32_t *__restrict__ it,
          const float *__restrict__ x, const float *__restrict__ mu,
          float *__restrict__ W, __nv_bfloat16 *__restrict__ Wh) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t blk, r, c, a, l;
    if (!locate(g, u[t], it[t], &blk, &r, &c)) continue;   // flagged in pass 1
    const BlockMeta &bm = meta[blk];
    if (!bm.owned) continue;                 // another shard's block
    to_w(bm, r, c, &a, &l);
    const float w = __fsub_rn(x[t], mu[blk]);
    if (W) W[bm.w_off + (int64_t)a * bm.L_pad + l] = w;
    // bf16 copy for the bf16 Gram: s128 x L_pad per block at vx_off
    if (Wh) Wh[bm.vx_off + (int64_t)a * bm.L_pad + l] = __float2bfloat16_rn(w);
  }
}

__global__ void __launch_bounds__(256)
k_plane_shift(int32_t nblocks, const unsigned long long *counts,
              const long long *sums, float *shift, float *delta) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblocks;
       b += gridDim.x * blockDim.x) {
    const unsigned long long cb = counts[b];
    double mu = 0.0;
    if (cb) mu = __ddiv_rn(__dmul_rn((double)sums[b], 0x1p-32), (double)cb);
    const double c = rint(mu);
    shift[b] = (float)c;
    delta[b] = __double2float_rn(mu - c);
  }
}

__global__ void __launch_bounds__(256)
k_scatter_planes(GridDesc g, const BlockMeta *__restrict__ meta, int64_t nnz,
                 const int32_t *__restrict__ u, const int32_t *__restrict__ it,
                 const float *__restrict__ x, const float *__restrict__ shift,
                 __nv_bfloat16 *__restrict__ VX, int32_t *flag) {
  int32_t bad = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t blk, r, c, a, l;
    if (!locate(g, u[t], it[t], &blk, &r, &c)) continue;   // flagged in pass 1
    const BlockMeta &bm = meta[blk];
    if (!bm.owned) continue;                 // another shard's block
    to_w(bm, r, c, &a, &l);
    const float y = __fsub_rn(x[t], shift[blk]);
    // exact in bf16, and every Gram partial sum below 2^24 in f32:
    // |y|^2 L_pad < 2^24
    const float lim = sqrtf(16777216.f / (float)bm.L_pad);
    if (!(y == rintf(y) && fabsf(y) <= fminf(lim, 256.f))) bad = 1;
    __nv_bfloat16 *pl = VX + bm.vx_off;
    pl[(int64_t)a * bm.L_pad + l] = __float2bfloat16_rn(y);
    pl[(int64_t)(bm.s128 + a) * bm.L_pad + l] = __float2bfloat16_rn(1.f);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
    atomicOr(flag, kErrNotExact);
}

int grid_for(int64_t n, int per_thread) {
  int64_t want = (n + 256LL * per_thread - 1) / (256LL * per_thread);
  if (want < 1) want = 1;
  if (want > 152 * 8) want = 152 * 8;
  return (int)want;
}

}  // namespace

cudaError_t launch_plane_shift(int32_t nblocks, const unsigned long long *counts,
                               const long long *sums, float *shift,
                               float *delta, cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  k_plane_shift<<<(nblocks + 255) / 256, 256, 0, st>>>(nblocks, counts, sums,
                                                       shift, delta);
  return cudaGetLastError();
}

cudaError_t launch_scatter_planes(const GridDesc &g, const BlockMeta *meta,
                                  int64_t nnz, const int32_t *u,
                                  const int32_t *i, const float *x,
                                  const float *shift, __nv_bfloat16 *VX,
                                  int32_t *flag, cudaStream_t st) {
  if (nnz <= 0) return cudaSuccess;
  k_scatter_planes<<<grid_for(nnz, 4), 256, 0, st>>>(g, meta, nnz, u, i, x,
                                                     shift, VX, flag);
  return cudaGetLastError();
}

cudaError_t launch_perm_check(const int32_t *perm, int64_t n, int32_t *seen,
                              int32_t *err, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(seen, 0, sizeof(int32_t) * n, st);
  if (e != cudaSuccess) return e;
  k_perm_mark<<<grid_for(n, 4), 256, 0, st>>>(perm, n, seen, err);
  k_perm_verify<<<grid_for(n, 4), 256, 0, st>>>(seen, n, err);
  return cudaGetLastError();
}

cudaError_t launch_count(const GridDesc &g, int64_t nnz, const int32_t *u,
                         const int32_t *i, const float *x, int32_t nblocks,
                         unsigned long long *counts, long long *sums,
                         unsigned int *maxabs_bits, int32_t *err,
                         cudaStream_t st) {
  if (nnz <= 0) return cudaSuccess;
  // big grids flush many per-CTA histograms: use fewer, longer CTAs
  int grid = grid_for(nnz, nblocks > 256 ? 16 : 4);
  k_count<<<grid, 256, 0, st>>>(g, nnz, u, i, x, nblocks, counts, sums,
                                maxabs_bits, err);
  return cudaGetLastError();
}

cudaError_t launch_means(int32_t nblocks, const unsigned long long *counts,
                         const long long *sums,
                         const unsigned int *maxabs_bits, float *mu,
                         int32_t *err, cudaStream_t st) {
  k_means<<<1, 1024, 0, st>>>(nblocks, counts, sums, maxabs_bits, mu, err);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const GridDesc &g, const BlockMeta *meta,
                           int64_t nnz, const int32_t *u, const int32_t *i,
                           const float *x, const float *mu, float *W,
                           __nv_bfloat16 *Wh, cudaStream_t st) {
  if (nnz <= 0) return cudaSuccess;
  k_scatter<<<grid_for(nnz, 4), 256, 0, st>>>(g, meta, nnz, u, i, x, mu, W,
                                              Wh);
  return cudaGetLastError();
}

}  // namespace bsvd
