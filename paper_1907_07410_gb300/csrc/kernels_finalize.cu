// Singular values and sign convention of the factors, spread over the GPU.
//
// After the projection, every block holds F_s (s x kp) and F_L = W^T F_s
// (L x kp). The retained singular values are sigma_j = |F_L[:, j]| (the
// Rayleigh-quotient refinement of Section 2's sigma_j, summed in float64),
// and each pair of columns is flipped so that the item-side vector's
// largest-|.| entry is positive (lowest row on ties), which fixes the sign
// that the SVD of Eq. 1 leaves free.
//
// A block's F_L can be 92,840 rows long, so one CTA per block would walk it
// alone. Instead:
//   1. k_colstats, one CTA per 128-row tile of F_L or of F_s: for each
//      column, the tile's float64 sum of squares and its largest |value|
//      with that value's row (first row on ties), reduced in a fixed order;
//   2. k_colcombine, one CTA per block: the tiles' sums in tile order give
//      sigma_j; the item side's tiles give the column's extreme entry and
//      its sign;
//   3. k_colflip, per tile again: negate the flipped columns of F_L and F_s.
// Every reduction has a fixed order, so reruns are bit-identical.
#include <float.h>
#include <limits.h>

#include "kernels.h"

namespace bsvd {

namespace {

constexpr int CT = 128;            // rows per tile
constexpr int kStatThreads = 256;  // at most; a multiple of kp is launched

// Fold (value, row) candidates: larger |value| wins, then the lower row.
__device__ __forceinline__ void pick(float &a, float &v, int &i, float a2,
                                     float v2, int i2) {
  if (a2 > a || (a2 == a && i2 < i)) {
    a = a2;
    v = v2;
    i = i2;
  }
}

// side 0: tiles of F_L (rows l < L); side 1: tiles of F_s (rows a < s).
// Thread t takes column j = t mod kp of the tile's rows g, g + G, ...
// (g = t / kp, G = blockDim / kp), so the CTA reads consecutive floats and
// each thread keeps one column's running sum and extreme entry; the G
// partials of a column are then folded in the order g = 0, 1, ...
__global__ void __launch_bounds__(kStatThreads)
k_colstats(const BlockMeta *__restrict__ meta, const int2 *__restrict__ tiles,
           const float *__restrict__ Fs, const float *__restrict__ FL, int kp,
           int side, ColPartial *__restrict__ out) {
  __shared__ double ssq[kStatThreads];
  __shared__ float sabs[kStatThreads], sval[kStatThreads];
  __shared__ int sidx[kStatThreads];
  pdl_wait();
  pdl_trigger();
  const int2 t = tiles[blockIdx.x];
  const BlockMeta bm = meta[t.x];
  const int G = (int)blockDim.x / kp;
  const int j = (int)threadIdx.x % kp, g = (int)threadIdx.x / kp;
  const int len = side == 0 ? bm.L : bm.s;
  const int rows = bm.owned ? min(CT, len - t.y) : 0;
  const float *src = (side == 0 ? FL + bm.fl_off : Fs + bm.fs_off) +
                     (int64_t)t.y * kp + j;
  double sq = 0.0;
  float a = -1.f, val = 0.f;
  int idx = INT_MAX;
  if (g < G) {
#pragma unroll 4
    for (int r = g; r < rows; r += G) {
      const float v = src[(int64_t)r * kp];
      sq = fma((double)v, (double)v, sq);
      pick(a, val, idx, fabsf(v), v, t.y + r);
    }
    ssq[threadIdx.x] = sq;
    sabs[threadIdx.x] = a;
    sval[threadIdx.x] = val;
    sidx[threadIdx.x] = idx;
  }
  __syncthreads();
  if (threadIdx.x < kp) {
    sq = 0.0;
    a = -1.f;
    val = 0.f;
    idx = INT_MAX;
    for (int q = 0; q < G; ++q) {
      const int o = q * kp + (int)threadIdx.x;
      sq += ssq[o];
      pick(a, val, idx, sabs[o], sval[o], sidx[o]);
    }
    ColPartial &p = out[(int64_t)blockIdx.x * kp + threadIdx.x];
    p.sq = sq;
    p.absmax = a;
    p.val = val;
    p.idx = idx;
  }
}

// One CTA per block, thread j per column.
__global__ void __launch_bounds__(64)
k_colcombine(const BlockMeta *__restrict__ meta,
             const ColPartial *__restrict__ lpart,
             const ColPartial *__restrict__ spart, int kp,
             double *__restrict__ sigma, unsigned char *__restrict__ flip) {
  pdl_wait();
  pdl_trigger();
  const int blk = blockIdx.x;
  const BlockMeta bm = meta[blk];
  const int j = threadIdx.x;
  if (j >= kp) return;
  const bool live = bm.owned && j < bm.keff;
  double sq = 0.0;
  float a = -1.f, val = 0.f;
  int idx = INT_MAX;
  if (live) {
    for (int t = 0; t < bm.npj; ++t)
      sq += lpart[(int64_t)(bm.pj0 + t) * kp + j].sq;
    // the item side: F_s when the Gram side is the items (trans), else F_L
    const ColPartial *ip = bm.trans ? spart : lpart;
    const int t0 = bm.trans ? bm.pt0 : bm.pj0;
    const int nt = bm.trans ? bm.npt : bm.npj;
    for (int t = 0; t < nt; ++t) {
      const ColPartial &p = ip[(int64_t)(t0 + t) * kp + j];
      pick(a, val, idx, p.absmax, p.val, p.idx);
    }
  }
  if (bm.owned) {
    sigma[(int64_t)blk * kp + j] = live ? sqrt(sq) : 0.0;
    flip[(int64_t)blk * kp + j] = (live && val < 0.f) ? 1 : 0;
  }
}

// Negates the flipped columns of one tile, with k_colstats' thread layout.
__global__ void __launch_bounds__(kStatThreads)
k_colflip(const BlockMeta *__restrict__ meta, const int2 *__restrict__ tiles,
          float *__restrict__ M, int kp, int side,
          const unsigned char *__restrict__ flip) {
  pdl_wait();
  pdl_trigger();
  const int2 t = tiles[blockIdx.x];
  const BlockMeta bm = meta[t.x];
  const int G = (int)blockDim.x / kp;
  const int j = (int)threadIdx.x % kp, g = (int)threadIdx.x / kp;
  if (!bm.owned || g >= G || !flip[(int64_t)t.x * kp + j]) return;
  const int len = side == 0 ? bm.L : bm.s;
  const int rows = min(CT, len - t.y);
  float *dst = M + (side == 0 ? bm.fl_off : bm.fs_off) + (int64_t)t.y * kp + j;
#pragma unroll 4
  for (int r = g; r < rows; r += G) dst[(int64_t)r * kp] = -dst[(int64_t)r * kp];
}

}  // namespace

cudaError_t launch_finalize(const BlockMeta *meta, int32_t nblocks,
                            const int2 *ltiles, int32_t nltiles,
                            const int2 *stiles, int32_t nstiles, float *Fs,
                            float *FL, double *sigma, int32_t kp,
                            ColPartial *lpart, ColPartial *spart,
                            unsigned char *flip, int64_t *launches,
                            cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  if (kp > 56 || kp % 4 != 0) return cudaErrorInvalidValue;
  const int threads = (kStatThreads / kp) * kp;
  cudaError_t e = cudaSuccess;
  if (nltiles > 0) {
    e = launch_pdl(k_colstats, dim3(nltiles), dim3(threads), 0, st, meta,
                   ltiles, (const float *)Fs, (const float *)FL, (int)kp, 0,
                   lpart);
    if (e != cudaSuccess) return e;
  }
  if (nstiles > 0) {
    e = launch_pdl(k_colstats, dim3(nstiles), dim3(threads), 0, st, meta,
                   stiles, (const float *)Fs, (const float *)FL, (int)kp, 1,
                   spart);
    if (e != cudaSuccess) return e;
  }
  e = launch_pdl(k_colcombine, dim3(nblocks), dim3(64), 0, st, meta,
                 (const ColPartial *)lpart, (const ColPartial *)spart, (int)kp,
                 sigma, flip);
  if (e != cudaSuccess) return e;
  if (nltiles > 0) {
    e = launch_pdl(k_colflip, dim3(nltiles), dim3(threads), 0, st, meta,
                   ltiles, FL, (int)kp, 0, (const unsigned char *)flip);
    if (e != cudaSuccess) return e;
  }
  if (nstiles > 0)
    e = launch_pdl(k_colflip, dim3(nstiles), dim3(threads), 0, st, meta,
                   stiles, Fs, (int)kp, 1, (const unsigned char *)flip);
  if (launches) *launches += 1 + 2 * ((nltiles > 0) + (nstiles > 0));
  return e;
}

}  // namespace bsvd
