// Gram matrices G_b = W_b W_b^T of every block, float32 on the SIMT pipes.
//
// G_b is the smaller of B^T B and B B^T. Its eigenpairs give the singular
// values and vectors of Section 2, Eq. 1 (sigma_i^2 = lambda_i). G is
// symmetric, so only tiles with tile_i <= tile_j are computed; each
// off-diagonal tile is written twice (as itself and mirrored).
//
// Tile 128 x 128, k-step 8, 256 threads with an 8 x 8 register tile each
// (two 4 x 4 quadrants 64 apart, which keeps shared-memory reads free of
// bank conflicts). The next k-slice is prefetched into registers while the
// current one is multiplied.
#include "kernels.h"

namespace bsvd {

namespace {

constexpr int TM = 128;
constexpr int TK = 8;
constexpr int LDS = TM + 4;

__global__ void __launch_bounds__(256, 2)
k_gram_f32(const BlockMeta *__restrict__ meta, const int4 *__restrict__ tiles,
           const float *__restrict__ W, float *__restrict__ G) {
  __shared__ __align__(16) float As[2][TK][LDS];
  __shared__ __align__(16) float Bs[2][TK][LDS];
  const int4 tl = tiles[blockIdx.x];
  const BlockMeta bm = meta[tl.x];
  const float *Wb = W + bm.w_off;
  float *Gb = G + bm.g_off;
  const int ld = bm.L_pad;
  const int sp = bm.s_pad;
  const int i0 = tl.y * TM, j0 = tl.z * TM;
  const int tid = threadIdx.x;

  // loader: 128 rows x 8 columns per operand, one float4 per thread
  const int lr = tid >> 1, lk = (tid & 1) * 4;
  const bool va = i0 + lr < sp, vb = j0 + lr < sp;
  const float *pa = Wb + (int64_t)(i0 + lr) * ld + lk;
  const float *pb = Wb + (int64_t)(j0 + lr) * ld + lk;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 ra = va ? __ldg(reinterpret_cast<const float4 *>(pa)) : zero;
  float4 rb = vb ? __ldg(reinterpret_cast<const float4 *>(pb)) : zero;
  As[0][lk + 0][lr] = ra.x; As[0][lk + 1][lr] = ra.y;
  As[0][lk + 2][lr] = ra.z; As[0][lk + 3][lr] = ra.w;
  Bs[0][lk + 0][lr] = rb.x; Bs[0][lk + 1][lr] = rb.y;
  Bs[0][lk + 2][lr] = rb.z; Bs[0][lk + 3][lr] = rb.w;
  __syncthreads();

  const int tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;

  int buf = 0;
  for (int k0 = 0; k0 < ld; k0 += TK) {
    const bool more = k0 + TK < ld;
    if (more) {
      ra = va ? __ldg(reinterpret_cast<const float4 *>(pa + k0 + TK)) : zero;
      rb = vb ? __ldg(reinterpret_cast<const float4 *>(pb + k0 + TK)) : zero;
    }
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[8], b[8];
      *reinterpret_cast<float4 *>(&a[0]) =
          *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
      *reinterpret_cast<float4 *>(&a[4]) =
          *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
      *reinterpret_cast<float4 *>(&b[0]) =
          *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
      *reinterpret_cast<float4 *>(&b[4]) =
          *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    if (more) {
      const int nb = buf ^ 1;
      As[nb][lk + 0][lr] = ra.x; As[nb][lk + 1][lr] = ra.y;
      As[nb][lk + 2][lr] = ra.z; As[nb][lk + 3][lr] = ra.w;
      Bs[nb][lk + 0][lr] = rb.x; Bs[nb][lk + 1][lr] = rb.y;
      Bs[nb][lk + 2][lr] = rb.z; Bs[nb][lk + 3][lr] = rb.w;
      __syncthreads();
      buf = nb;
    }
  }

  // rows i0 + {ty*4 + r, 64 + ty*4 + r}, columns j0 + {tx*4 + c, 64 + tx*4 + c}
#pragma unroll
  for (int hr = 0; hr < 2; ++hr) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int gi = i0 + hr * 64 + ty * 4 + r;
      if (gi >= sp) continue;
#pragma unroll
      for (int hc = 0; hc < 2; ++hc) {
        const int gj = j0 + hc * 64 + tx * 4;
        if (gj >= sp) continue;
        float4 v = make_float4(acc[hr * 4 + r][hc * 4 + 0],
                               acc[hr * 4 + r][hc * 4 + 1],
                               acc[hr * 4 + r][hc * 4 + 2],
                               acc[hr * 4 + r][hc * 4 + 3]);
        *reinterpret_cast<float4 *>(Gb + (int64_t)gi * sp + gj) = v;
      }
    }
  }
  if (tl.y != tl.z) {
    // mirrored tile: G[j][i] = G[i][j]
#pragma unroll
    for (int hc = 0; hc < 2; ++hc) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int gj = j0 + hc * 64 + tx * 4 + c;
        if (gj >= sp) continue;
#pragma unroll
        for (int hr = 0; hr < 2; ++hr) {
          const int gi = i0 + hr * 64 + ty * 4;
          if (gi >= sp) continue;
          float4 v = make_float4(acc[hr * 4 + 0][hc * 4 + c],
                                 acc[hr * 4 + 1][hc * 4 + c],
                                 acc[hr * 4 + 2][hc * 4 + c],
                                 acc[hr * 4 + 3][hc * 4 + c]);
          *reinterpret_cast<float4 *>(Gb + (int64_t)gj * sp + gi) = v;
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_gram_f32(const BlockMeta *meta, const int4 *tiles,
                            int32_t ntiles, const float *W, float *G,
                            cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  k_gram_f32<<<ntiles, 256, 0, st>>>(meta, tiles, W, G);
  return cudaGetLastError();
}

}  // namespace bsvd
