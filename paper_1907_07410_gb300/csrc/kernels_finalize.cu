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

#include <type_traits>

#include "kernels.h"

namespace bsvd {

namespace {

constexpr int CT = 128;            // rows per tile, one per thread

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
template <int KM>
__global__ void __launch_bounds__(CT)
k_colstats(const BlockMeta *__restrict__ meta, const int2 *__restrict__ tiles,
           const float *__restrict__ Fs, const float *__restrict__ FL, int kp,
           int side, ColPartial *__restrict__ out) {
  __shared__ double ssq[CT / 32][KM];
  __shared__ float sabs[CT / 32][KM], sval[CT / 32][KM];
  __shared__ int sidx[CT / 32][KM];
  pdl_wait();
  pdl_trigger();
  const int2 t = tiles[blockIdx.x];
  const BlockMeta bm = meta[t.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = t.y + threadIdx.x;
  const int len = side == 0 ? bm.L : bm.s;
  const float *src = (side == 0 ? FL + bm.fl_off : Fs + bm.fs_off) +
                     (int64_t)row * kp;
  float v[KM];
#pragma unroll
  for (int j = 0; j < KM; ++j) v[j] = 0.f;
  if (bm.owned && row < len) {
#pragma unroll
    for (int j4 = 0; j4 < KM / 4; ++j4) {
      if (4 * j4 < kp) {
        const float4 q = *reinterpret_cast<const float4 *>(src + 4 * j4);
        v[4 * j4] = q.x; v[4 * j4 + 1] = q.y;
        v[4 * j4 + 2] = q.z; v[4 * j4 + 3] = q.w;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < KM; ++j) {
    double sq = (double)v[j] * (double)v[j];
    float a = fabsf(v[j]), val = v[j];
    int idx = row < len ? row : INT_MAX;
    for (int o = 16; o > 0; o >>= 1) {
      sq += __shfl_xor_sync(0xffffffffu, sq, o);
      const float a2 = __shfl_xor_sync(0xffffffffu, a, o);
      const float v2 = __shfl_xor_sync(0xffffffffu, val, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
      pick(a, val, idx, a2, v2, i2);
    }
    if (lane == 0) {
      ssq[warp][j] = sq;
      sabs[warp][j] = a;
      sval[warp][j] = val;
      sidx[warp][j] = idx;
    }
  }
  __syncthreads();
  if (threadIdx.x < kp) {
    const int j = threadIdx.x;
    double sq = 0.0;
    float a = -1.f, val = 0.f;
    int idx = INT_MAX;
    for (int w = 0; w < CT / 32; ++w) {
      sq += ssq[w][j];
      pick(a, val, idx, sabs[w][j], sval[w][j], sidx[w][j]);
    }
    ColPartial &p = out[(int64_t)blockIdx.x * kp + j];
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

template <int KM>
__global__ void __launch_bounds__(CT)
k_colflip(const BlockMeta *__restrict__ meta, const int2 *__restrict__ tiles,
          float *__restrict__ M, int kp, int side,
          const unsigned char *__restrict__ flip) {
  pdl_wait();
  pdl_trigger();
  const int2 t = tiles[blockIdx.x];
  const BlockMeta bm = meta[t.x];
  if (!bm.owned) return;
  const int row = t.y + threadIdx.x;
  const int len = side == 0 ? bm.L : bm.s;
  if (row >= len) return;
  float *dst = M + (side == 0 ? bm.fl_off : bm.fs_off) + (int64_t)row * kp;
  const unsigned char *f = flip + (int64_t)t.x * kp;
#pragma unroll
  for (int j = 0; j < KM; ++j)
    if (j < kp && f[j]) dst[j] = -dst[j];
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
  auto go = [&](auto km) -> cudaError_t {
    constexpr int KM = decltype(km)::value;
    cudaError_t e = cudaSuccess;
    if (nltiles > 0) {
      e = launch_pdl(k_colstats<KM>, dim3(nltiles), dim3(CT), 0, st, meta,
                     ltiles, (const float *)Fs, (const float *)FL, (int)kp, 0,
                     lpart);
      if (e != cudaSuccess) return e;
    }
    if (nstiles > 0) {
      e = launch_pdl(k_colstats<KM>, dim3(nstiles), dim3(CT), 0, st, meta,
                     stiles, (const float *)Fs, (const float *)FL, (int)kp, 1,
                     spart);
      if (e != cudaSuccess) return e;
    }
    e = launch_pdl(k_colcombine, dim3(nblocks), dim3(64), 0, st, meta,
                   (const ColPartial *)lpart, (const ColPartial *)spart,
                   (int)kp, sigma, flip);
    if (e != cudaSuccess) return e;
    if (nltiles > 0) {
      e = launch_pdl(k_colflip<KM>, dim3(nltiles), dim3(CT), 0, st, meta,
                     ltiles, FL, (int)kp, 0, (const unsigned char *)flip);
      if (e != cudaSuccess) return e;
    }
    if (nstiles > 0)
      e = launch_pdl(k_colflip<KM>, dim3(nstiles), dim3(CT), 0, st, meta,
                     stiles, Fs, (int)kp, 1, (const unsigned char *)flip);
    if (launches) *launches += 1 + 2 * ((nltiles > 0) + (nstiles > 0));
    return e;
  };
  switch ((kp + 7) / 8) {
    case 1: return go(std::integral_constant<int, 8>());
    case 2: return go(std::integral_constant<int, 16>());
    case 3: return go(std::integral_constant<int, 24>());
    case 4: return go(std::integral_constant<int, 32>());
    case 5: return go(std::integral_constant<int, 40>());
    case 6: return go(std::integral_constant<int, 48>());
    case 7: return go(std::integral_constant<int, 56>());
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bsvd
