// Exact block Gram matrices on the tcgen05 tensor cores.
//
// The Gram G_b = W_b W_b^T of Section 2 (Eq. 1: sigma_i^2 are its top
// eigenvalues) is the only dense contraction of the method. The centred
// block is W = X - mu M, with X the ratings and M the 0/1 observation mask.
// With c = round(mu), Y = X - c M holds small integers (for integer rating
// scales), and with delta = mu - c:
//
//   G = Y Y^T - delta (Y M^T + M Y^T) + delta^2 M M^T.
//
// Y and M are exact in bf16, and every partial sum of the four products is
// an integer below 2^24, so the bf16 MMAs with f32 accumulation are exact.
// The only rounding is the final f32 combination (cancellation is mild,
// since |delta| <= 1/2).
//
// One CTA per 128 x 128 output tile (tile_i <= tile_j) of one block:
//   * the planes of a block are [Y (s128 rows); M (s128 rows)] x L_pad bf16,
//     read by TMA with 128-byte swizzling in 128 x 64 boxes;
//   * a 3-stage shared-memory ring, with full/empty mbarriers;
//   * warp 0 lane 0 issues TMA, warp 1 lane 0 issues tcgen05.mma (M = N =
//     128, K = 16). The four products accumulate in the four 128-column
//     quarters of tensor memory (512 columns);
//   * all four warps then read the accumulators (one row per thread), form
//     G and store the tile and its mirror.
// Every wait is bounded. A timeout sets kErrTimeout, skips the rest of the
// work, and the CTA still waits (bounded) for its copies in flight and frees
// its tensor memory.
#include "kernels.h"
#include "tc_ptx.cuh"

namespace bsvd {

namespace {

constexpr int TT = 128;                      // tile rows = cols
constexpr int KB = 64;                       // bf16 per k-chunk (128 bytes)
constexpr int STAGES = 3;
constexpr int TILE_BYTES = TT * KB * 2;      // 16 KiB
constexpr int STAGE_BYTES = 4 * TILE_BYTES;  // Y_i, M_i, Y_j, M_j
constexpr uint32_t kSpin = 1u << 22;         // mbarrier polls before giving up

struct Ctrl {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t done;
  uint32_t tmem;
  int abort;
  int issued;      // k-chunks whose loads were issued
  int consumed;    // k-chunks whose loads the MMA thread saw complete
};

constexpr size_t kSmemBytes = STAGES * STAGE_BYTES + sizeof(Ctrl) + 1024;

__global__ void __launch_bounds__(128, 1)
k_gram_tc(const BlockMeta *__restrict__ meta, const int4 *__restrict__ tiles,
          const CUtensorMap *__restrict__ maps,
          const float *__restrict__ delta, float *__restrict__ G,
          int32_t *err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Ctrl &ct = *reinterpret_cast<Ctrl *>(base + STAGES * STAGE_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 tl = tiles[blockIdx.x];
  const BlockMeta bm = meta[tl.x];
  const CUtensorMap *map = maps + tl.x;
  const bool diag = tl.y == tl.z;
  const int yi = tl.y * TT, yj = tl.z * TT;
  const int s128 = bm.s128;
  const int nk = (bm.L_pad + KB - 1) / KB;

  if (warp == 0) tc::tmem_alloc(&ct.tmem, 512);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&ct.full[s], 1);
      tc::mbar_init(&ct.empty[s], 1);
    }
    tc::mbar_init(&ct.done, 1);
    ct.abort = 0;
    ct.issued = 0;
    ct.consumed = 0;
    tc::mbar_init_fence();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = ct.tmem;

  if (warp == 0 && lane == 0) {
    // producer: TMA loads into the ring
    const uint32_t bytes = (diag ? 2 : 4) * TILE_BYTES;
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % STAGES;
      const uint32_t ph = (kc / STAGES) & 1;
      if (!tc::mbar_wait(&ct.empty[s], ph ^ 1, kSpin) ||
          *reinterpret_cast<volatile int *>(&ct.abort)) {
        atomicOr(err, kErrTimeout);
        ct.abort = 1;
        break;
      }
      unsigned char *buf = base + s * STAGE_BYTES;
      const int x = kc * KB;
      tc::mbar_expect_tx(&ct.full[s], bytes);
      tc::tma_load_2d(buf, map, x, yi, &ct.full[s]);
      tc::tma_load_2d(buf + TILE_BYTES, map, x, s128 + yi, &ct.full[s]);
      if (!diag) {
        tc::tma_load_2d(buf + 2 * TILE_BYTES, map, x, yj, &ct.full[s]);
        tc::tma_load_2d(buf + 3 * TILE_BYTES, map, x, s128 + yj, &ct.full[s]);
      }
      ct.issued = kc + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = tc::idesc_bf16_f32(TT, TT);
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % STAGES;
      const uint32_t ph = (kc / STAGES) & 1;
      if (!tc::mbar_wait(&ct.full[s], ph, kSpin) ||
          *reinterpret_cast<volatile int *>(&ct.abort)) {
        atomicOr(err, kErrTimeout);
        ct.abort = 1;
        break;
      }
      ct.consumed = kc + 1;
      tc::fence_after_sync();
      unsigned char *buf = base + s * STAGE_BYTES;
      const uint64_t dyi = tc::sdesc_kmajor_sw128(tc::smem_u32(buf));
      const uint64_t dmi = tc::sdesc_kmajor_sw128(tc::smem_u32(buf + TILE_BYTES));
      const uint64_t dyj = diag ? dyi : tc::sdesc_kmajor_sw128(tc::smem_u32(buf + 2 * TILE_BYTES));
      const uint64_t dmj = diag ? dmi : tc::sdesc_kmajor_sw128(tc::smem_u32(buf + 3 * TILE_BYTES));
#pragma unroll
      for (int kk = 0; kk < KB / 16; ++kk) {
        const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
        const uint64_t o = 2 * kk;            // 32 bytes per K=16 slice
        tc::mma_bf16(taddr + 0, dyi + o, dyj + o, idesc, acc);    // Y_i Y_j^T
        tc::mma_bf16(taddr + 128, dyi + o, dmj + o, idesc, acc);  // Y_i M_j^T
        tc::mma_bf16(taddr + 256, dmi + o, dyj + o, idesc, acc);  // M_i Y_j^T
        tc::mma_bf16(taddr + 384, dmi + o, dmj + o, idesc, acc);  // M_i M_j^T
      }
      tc::mma_commit(&ct.empty[s]);           // frees the stage when done
    }
    tc::mma_commit(&ct.done);
  }
  __syncwarp();

  // epilogue: row (warp * 32 + lane) of the tile
  const bool ready = tc::mbar_wait(&ct.done, 0, kSpin);
  if (!ready && lane == 0) atomicOr(err, kErrTimeout);
  __syncwarp();
  if (ready && !*reinterpret_cast<volatile int *>(&ct.abort)) {
    tc::fence_after_sync();
    const int sp = bm.s_pad;
    const int gi = yi + warp * 32 + lane;
    const float dl = delta[tl.x];
    const float dl2 = dl * dl;
    float *Gb = G + bm.g_off;
    const uint32_t lrow = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
    for (int c0 = 0; c0 < TT; c0 += 32) {
      float a[32], c1[32], c2[32], d[32];
      tc::tmem_ld32(taddr + lrow + c0, a);
      tc::tmem_ld32(taddr + lrow + 128 + c0, c1);
      tc::tmem_ld32(taddr + lrow + 256 + c0, c2);
      tc::tmem_ld32(taddr + lrow + 384 + c0, d);
      const int gj0 = yj + c0;
      if (gj0 >= sp) continue;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        a[j] = fmaf(dl2, d[j], fmaf(-dl, c1[j] + c2[j], a[j]));
      if (gi < sp) {
        float4 *dst = reinterpret_cast<float4 *>(Gb + (int64_t)gi * sp + gj0);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          dst[j] = make_float4(a[4 * j], a[4 * j + 1], a[4 * j + 2], a[4 * j + 3]);
        if (!diag) {
#pragma unroll
          for (int j = 0; j < 32; ++j) Gb[(int64_t)(gj0 + j) * sp + gi] = a[j];
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && ct.abort) {
    // drain copies that were issued but never consumed
    for (int kc = ct.consumed; kc < ct.issued; ++kc)
      tc::mbar_wait(&ct.full[kc % STAGES], (kc / STAGES) & 1, kSpin);
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

// Single-product Gram G = W W^T in reduced precision (any rating scale):
//   * k_gram_tf32 reads the float32 blocks, truncated to tf32 by the MMA
//     (10-bit mantissa);
//   * k_gram_bf16 reads a bf16 copy of the centred blocks (8-bit mantissa).
// Both accumulate in f32. Same roles as k_gram_tc (warp 0 TMA, warp 1 MMA,
// all four warps in the epilogue), on the larger tiles below, with boxes of
// 128 rows x 128 bytes (32 floats or 64 bf16). Either way a k-chunk is four
// K slices of 32 bytes each (K = 8 tf32 or K = 16 bf16), so the descriptor
// steps match.
constexpr int KF = 32;                          // floats per k-chunk (128 B)
constexpr int FTILE_BYTES = TT * KF * 4;        // 16 KiB: 128 rows x 128 B

// 256 x 256 output tiles: two 128-row halves of A (rows i0 .. i0+255) and
// the 256 rows j0 .. j0+255 as B (N = 256), one accumulator of 256 columns
// per half (all 512 tensor-memory columns). Per k-chunk the stage holds
// four boxes of 128 rows x 128 bytes, [A0 | A1 | B0 | B1], 64 KiB, and the
// MMA thread issues 8 MMAs (4 K slices x 2 halves): 128 flop per byte
// loaded, twice the 128 x 128 tile's, so the loads no longer set the pace.
// A diagonal tile (i0 = j0) loads A only and reads B from it: [A0 | A1]
// is the same 256 rows, contiguous in shared memory.
constexpr int G2T = 256;
constexpr int G2STAGES = 3;
constexpr int G2STAGE_BYTES = 4 * FTILE_BYTES;       // 64 KiB

struct CtrlG2 {
  uint64_t full[G2STAGES];
  uint64_t empty[G2STAGES];
  uint64_t done;
  uint32_t tmem;
  int abort;
  int issued;
  int consumed;
};

constexpr size_t kSmemBytesG2 =
    G2STAGES * G2STAGE_BYTES + sizeof(CtrlG2) + 1024;

template <bool kBf16>
__device__ __forceinline__ void
gram_single(const BlockMeta *__restrict__ meta, const int4 *__restrict__ tiles,
            const CUtensorMap *__restrict__ maps, float *__restrict__ G,
            int32_t *err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  CtrlG2 &ct = *reinterpret_cast<CtrlG2 *>(base + G2STAGES * G2STAGE_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 tl = tiles[blockIdx.x];
  const BlockMeta bm = meta[tl.x];
  const CUtensorMap *map = maps + tl.x;
  const bool diag = tl.y == tl.z;
  const int yi = tl.y * G2T, yj = tl.z * G2T;
  constexpr int kElems = kBf16 ? 64 : KF;        // elements per k-chunk
  const int nk = (bm.L_pad + kElems - 1) / kElems;

  if (warp == 0) tc::tmem_alloc(&ct.tmem, 512);
  if (threadIdx.x == 0) {
    for (int s = 0; s < G2STAGES; ++s) {
      tc::mbar_init(&ct.full[s], 1);
      tc::mbar_init(&ct.empty[s], 1);
    }
    tc::mbar_init(&ct.done, 1);
    ct.abort = 0;
    ct.issued = 0;
    ct.consumed = 0;
    tc::mbar_init_fence();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = ct.tmem;

  if (warp == 0 && lane == 0) {
    const uint32_t bytes = (diag ? 2 : 4) * FTILE_BYTES;
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % G2STAGES;
      const uint32_t ph = (kc / G2STAGES) & 1;
      if (!tc::mbar_wait(&ct.empty[s], ph ^ 1, kSpin) ||
          *reinterpret_cast<volatile int *>(&ct.abort)) {
        atomicOr(err, kErrTimeout);
        ct.abort = 1;
        break;
      }
      unsigned char *buf = base + s * G2STAGE_BYTES;
      const int x = kc * kElems;
      tc::mbar_expect_tx(&ct.full[s], bytes);
      tc::tma_load_2d(buf, map, x, yi, &ct.full[s]);
      tc::tma_load_2d(buf + FTILE_BYTES, map, x, yi + TT, &ct.full[s]);
      if (!diag) {
        tc::tma_load_2d(buf + 2 * FTILE_BYTES, map, x, yj, &ct.full[s]);
        tc::tma_load_2d(buf + 3 * FTILE_BYTES, map, x, yj + TT, &ct.full[s]);
      }
      ct.issued = kc + 1;
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = kBf16 ? tc::idesc_bf16_f32(TT, G2T)
                                     : tc::idesc_tf32_f32(TT, G2T);
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % G2STAGES;
      const uint32_t ph = (kc / G2STAGES) & 1;
      if (!tc::mbar_wait(&ct.full[s], ph, kSpin) ||
          *reinterpret_cast<volatile int *>(&ct.abort)) {
        atomicOr(err, kErrTimeout);
        ct.abort = 1;
        break;
      }
      ct.consumed = kc + 1;
      tc::fence_after_sync();
      unsigned char *buf = base + s * G2STAGE_BYTES;
      const uint64_t da0 = tc::sdesc_kmajor_sw128(tc::smem_u32(buf));
      const uint64_t da1 =
          tc::sdesc_kmajor_sw128(tc::smem_u32(buf + FTILE_BYTES));
      const uint64_t db =
          diag ? da0 : tc::sdesc_kmajor_sw128(tc::smem_u32(buf + 2 * FTILE_BYTES));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {          // 32 bytes of K per MMA
        const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
        if constexpr (kBf16) {
          tc::mma_bf16(taddr, da0 + 2 * kk, db + 2 * kk, idesc, acc);
          tc::mma_bf16(taddr + G2T, da1 + 2 * kk, db + 2 * kk, idesc, acc);
        } else {
          tc::mma_tf32(taddr, da0 + 2 * kk, db + 2 * kk, idesc, acc);
          tc::mma_tf32(taddr + G2T, da1 + 2 * kk, db + 2 * kk, idesc, acc);
        }
      }
      tc::mma_commit(&ct.empty[s]);
    }
    tc::mma_commit(&ct.done);
  }
  __syncwarp();

  const bool ready = tc::mbar_wait(&ct.done, 0, kSpin);
  if (!ready && lane == 0) atomicOr(err, kErrTimeout);
  __syncwarp();
  if (ready && !*reinterpret_cast<volatile int *>(&ct.abort)) {
    tc::fence_after_sync();
    const int sp = bm.s_pad;
    float *Gb = G + bm.g_off;
    const uint32_t lrow = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int gi = yi + h * TT + warp * 32 + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < G2T; c0 += 32) {
        float a[32];
        tc::tmem_ld32(taddr + lrow + h * G2T + c0, a);
        const int gj0 = yj + c0;
        if (gj0 >= sp) continue;
        if (gi < sp) {
          float4 *dst = reinterpret_cast<float4 *>(Gb + (int64_t)gi * sp + gj0);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            dst[j] = make_float4(a[4 * j], a[4 * j + 1], a[4 * j + 2],
                                 a[4 * j + 3]);
          if (!diag) {
#pragma unroll
            for (int j = 0; j < 32; ++j) Gb[(int64_t)(gj0 + j) * sp + gi] = a[j];
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && ct.abort) {
    for (int kc = ct.consumed; kc < ct.issued; ++kc)
      tc::mbar_wait(&ct.full[kc % G2STAGES], (kc / G2STAGES) & 1, kSpin);
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

__global__ void __launch_bounds__(128, 1)
k_gram_tf32(const BlockMeta *__restrict__ meta, const int4 *__restrict__ tiles,
            const CUtensorMap *__restrict__ maps, float *__restrict__ G,
            int32_t *err) {
  gram_single<false>(meta, tiles, maps, G, err);
}

__global__ void __launch_bounds__(128, 1)
k_gram_bf16(const BlockMeta *__restrict__ meta, const int4 *__restrict__ tiles,
            const CUtensorMap *__restrict__ maps, float *__restrict__ G,
            int32_t *err) {
  gram_single<true>(meta, tiles, maps, G, err);
}

}  // namespace

cudaError_t launch_gram_bf16(const BlockMeta *meta, const int4 *tiles,
                             int32_t ntiles, const CUtensorMap *maps, float *G,
                             int32_t *err, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  static_assert(kSmemBytesG2 <= 227 * 1024, "shared memory");
  cudaError_t e = cudaFuncSetAttribute(
      k_gram_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)kSmemBytesG2);
  if (e != cudaSuccess) return e;
  k_gram_bf16<<<ntiles, 128, kSmemBytesG2, st>>>(meta, tiles, maps, G, err);
  return cudaGetLastError();
}

cudaError_t launch_gram_tf32(const BlockMeta *meta, const int4 *tiles,
                             int32_t ntiles, const CUtensorMap *maps, float *G,
                             int32_t *err, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(
      k_gram_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)kSmemBytesG2);
  if (e != cudaSuccess) return e;
  k_gram_tf32<<<ntiles, 128, kSmemBytesG2, st>>>(meta, tiles, maps, G, err);
  return cudaGetLastError();
}

size_t gram_tc_smem_bytes() { return kSmemBytes; }

cudaError_t launch_gram_tc(const BlockMeta *meta, const int4 *tiles,
                           int32_t ntiles, const CUtensorMap *maps,
                           const float *delta, float *G, int32_t *err,
                           cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(
      k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e != cudaSuccess) return e;
  k_gram_tc<<<ntiles, 128, kSmemBytes, st>>>(meta, tiles, maps, delta, G, err);
  return cudaGetLastError();
}

}  // namespace bsvd
