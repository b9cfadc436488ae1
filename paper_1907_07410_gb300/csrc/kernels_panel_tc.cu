// Panel products of the eigen-solver on the tcgen05 tensor cores:
//   out = alpha G in + beta in + gamma in2
// for one 128-row tile of one block's Gram matrix G (s_pad x s_pad, float32,
// symmetric) and its b-column panel `in` (s_pad x b, row-major).
//
// Precision: three tf32 passes. Every float32 operand x is split into
// hi = x rounded to 10 mantissa bits (exact in tf32) and lo = x - hi
// (exact in float32, |lo| <= 2^-11 |x|), and
//   G in ~= G_hi in_hi + G_hi in_lo + G_lo in_hi.
// The dropped G_lo in_lo term and the tf32 narrowing of the lo parts are
// below 2^-21 relative. Splitting explicitly (rather than leaving the low
// bits to the MMA) makes the result independent of how the hardware narrows
// f32 to tf32.
//
// Accumulation: the tensor core's f32 accumulator does not round to
// nearest at each step (a measured one-signed error growing with the number
// of accumulating MMAs), so long chains drift: one accumulator over the
// whole K range of a 1000-row block gave errors near 1e-5 relative. The
// hi*hi products therefore go round-robin into four accumulators and the
// two small cross terms into a fifth; the epilogue adds the five in a fixed
// order. This brings the product to within about 1e-6 of float64 on such
// blocks, comparable to the FP32 SIMT product, as the 1e-5 residual test of
// the solver needs.
//
// CTA roles (192 threads):
//   * warp 0, one lane: TMA loads into a ring of stages: the G tile, 128 rows
//     x 32 floats with 128-byte swizzling, and the matching 32 rows of `in`
//     (32 x b floats, plain layout);
//   * warps 2-5: split each G tile in place (hi) and into a second buffer
//     (lo) (the swizzle is a permutation of 16-byte chunks, so elementwise
//     work ignores it); split the rows of `in` and store them transposed
//     (one 128-byte row per panel column, the same swizzle), so both MMA
//     operands are K-major;
//   * warp 1, one lane: tcgen05.mma kind::tf32, M = 128, N = b, K = 8,
//     three per K slice, into 5 b TMEM columns; its commit frees the stage.
// Then the epilogue: warp w of warps 2-5 reads TMEM lanes 32 (w mod 4) ..
// +31, i.e. one output row per thread.
//
// Measured on GB300 (clock64 stamps per stage): issuing a stage's 12 MMAs
// takes about 850 cycles, and its conversion about 1000, so the kernel is
// bound by MMA issue and conversion latency, not by memory: per launch it
// is 2.6x faster than the FP32 SIMT product on 4000-row blocks and 1.2-1.5x
// on 1000-row blocks.
//
// Every wait is bounded; a timeout sets kErrTimeout and the CTA drains its
// copies in flight and frees its tensor memory before returning.
#include "kernels.h"
#include "tc_ptx.cuh"

namespace bsvd {

namespace {

constexpr int PT = 128;                  // G rows per CTA (MMA M)
constexpr int PK = 32;                   // floats of K per stage (128 bytes)
constexpr int kMaxStages = 4;
constexpr uint32_t kSpinP = 1u << 22;    // mbarrier polls before giving up
constexpr uint32_t kHiMask = 0xFFFFE000u;
constexpr uint32_t kHiHalf = 0x00001000u;
constexpr int A_BYTES = PT * PK * 4;     // 16 KiB
constexpr int kAcc = 5;                  // 4 hi*hi accumulators + cross terms

template <int B>
struct PanelTc {
  static constexpr int B_BYTES = B * PK * 4;    // B rows of 128 bytes
  static constexpr int X_BYTES = PK * B * 4;    // 32 rows of `in`
  // A hi (TMA destination, split in place), A lo, B hi, B lo, rows of `in`
  static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES + X_BYTES;
  static constexpr int STAGES = B >= 64 ? 3 : 4;
  static constexpr int TMEM_COLS = kAcc * B <= 128 ? 128
                                   : (kAcc * B <= 256 ? 256 : 512);
};

struct PanelCtrl {
  uint64_t full[kMaxStages];    // G tile and rows of `in` landed (TMA bytes)
  uint64_t ready[kMaxStages];   // operands split and stored (4 converter warps)
  uint64_t empty[kMaxStages];   // the stage's MMAs completed
  uint64_t done;                // every MMA completed
  uint32_t tmem;
  int abort;
  int issued;                   // stages whose loads were issued
  int consumed;                 // stages the converters saw land
};

template <int B>
constexpr size_t panel_tc_smem() {
  return PanelTc<B>::STAGES * PanelTc<B>::STAGE + sizeof(PanelCtrl) + 1024;
}

// x rounded to the nearest value with 10 mantissa bits (ties away from 0)
__device__ __forceinline__ float hi1(float x) {
  return __uint_as_float((__float_as_uint(x) + kHiHalf) & kHiMask);
}

__device__ __forceinline__ float4 hi4(float4 v) {
  return make_float4(hi1(v.x), hi1(v.y), hi1(v.z), hi1(v.w));
}

__device__ __forceinline__ float4 sub4(float4 a, float4 b) {
  return make_float4(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y),
                     __fsub_rn(a.z, b.z), __fsub_rn(a.w, b.w));
}

// Byte offset of the 16-byte chunk `c` (0..7) of row `r` in a tile of
// 128-byte rows stored with 128-byte swizzling (tile base 1024-aligned).
__device__ __forceinline__ uint32_t sw128(int r, int c) {
  return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

template <int B>
__global__ void __launch_bounds__(192, 1)
k_gpanel_tc(const BlockMeta *__restrict__ meta, SolverState *state,
            const int2 *__restrict__ tiles, const CUtensorMap *__restrict__ gmaps,
            const CUtensorMap *__restrict__ xmaps, const float *in,
            const float *in2, float *out, int mode, int step, int32_t *err) {
  using L = PanelTc<B>;
  constexpr int PSTAGES = L::STAGES;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  PanelCtrl &ct = *reinterpret_cast<PanelCtrl *>(base + PSTAGES * L::STAGE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int2 t = tiles[blockIdx.x];
  const SolverState st = state[t.x];
  // uniform over the CTA, before any barrier or TMEM is touched
  if (st.status != kRunning) return;
  if (mode >= 1 && step > st.degree) return;
  const BlockMeta bm = meta[t.x];
  const int sp = bm.s_pad, row0 = t.y;
  if (row0 == 0 && threadIdx.x == 0) atomicAdd(&state[t.x].products, 1);
  const int nk = sp / PK;                 // s_pad is a multiple of 32
  const float *inb = in + bm.x_off;
  float alpha, beta, gamma;
  cheb_coeffs(st, mode, step, &alpha, &beta, &gamma);

  auto a_hi = [&](int s) { return base + s * L::STAGE; };
  auto a_lo = [&](int s) { return base + s * L::STAGE + A_BYTES; };
  auto b_hi = [&](int s) { return base + s * L::STAGE + 2 * A_BYTES; };
  auto b_lo = [&](int s) {
    return base + s * L::STAGE + 2 * A_BYTES + L::B_BYTES;
  };
  auto x_raw = [&](int s) {
    return base + s * L::STAGE + 2 * A_BYTES + 2 * L::B_BYTES;
  };

  if (warp == 0) tc::tmem_alloc(&ct.tmem, L::TMEM_COLS);
  if (threadIdx.x == 0) {
    for (int s = 0; s < PSTAGES; ++s) {
      tc::mbar_init(&ct.full[s], 1);
      tc::mbar_init(&ct.ready[s], 4);
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
  volatile int *abort_flag = &ct.abort;

  if (warp == 0) {
    if (lane == 0) {
      const CUtensorMap *map = gmaps + t.x;
      const CUtensorMap *xmap = xmaps + t.x;
      for (int kc = 0; kc < nk; ++kc) {
        const int s = kc % PSTAGES;
        const uint32_t ph = (kc / PSTAGES) & 1;
        if (!tc::mbar_wait(&ct.empty[s], ph ^ 1, kSpinP) || *abort_flag) {
          atomicOr(err, kErrTimeout);
          ct.abort = 1;
          break;
        }
        tc::mbar_expect_tx(&ct.full[s], A_BYTES + L::X_BYTES);
        tc::tma_load_2d(a_hi(s), map, kc * PK, row0, &ct.full[s]);
        tc::tma_load_2d(x_raw(s), xmap, 0, kc * PK, &ct.full[s]);
        ct.issued = kc + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_tf32_f32(PT, B);
      for (int kc = 0; kc < nk; ++kc) {
        const int c = kc % PSTAGES;
        const uint32_t ph = (kc / PSTAGES) & 1;
        if (!tc::mbar_wait(&ct.ready[c], ph, kSpinP) || *abort_flag) {
          atomicOr(err, kErrTimeout);
          ct.abort = 1;
          break;
        }
        tc::fence_after_sync();
        const uint64_t dah = tc::sdesc_kmajor_sw128(tc::smem_u32(a_hi(c)));
        const uint64_t dal = tc::sdesc_kmajor_sw128(tc::smem_u32(a_lo(c)));
        const uint64_t dbh = tc::sdesc_kmajor_sw128(tc::smem_u32(b_hi(c)));
        const uint64_t dbl = tc::sdesc_kmajor_sw128(tc::smem_u32(b_lo(c)));
#pragma unroll
        for (int kk = 0; kk < PK / 8; ++kk) {    // 32 bytes of K per MMA
          const uint64_t o = 2 * kk;
          // hi*hi into accumulator kk (of 4), cross terms into the fifth
          tc::mma_tf32(taddr + kk * B, dah + o, dbh + o, idesc,
                       kc > 0 ? 1u : 0u);
          tc::mma_tf32(taddr + 4 * B, dah + o, dbl + o, idesc,
                       (kc > 0 || kk > 0) ? 1u : 0u);
          tc::mma_tf32(taddr + 4 * B, dal + o, dbh + o, idesc, 1u);
        }
        tc::mma_commit(&ct.empty[c]);
      }
      tc::mma_commit(&ct.done);
    }
  } else {
    // converters: 128 threads
    const int cid = threadIdx.x - 64;
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % PSTAGES;
      const uint32_t ph = (kc / PSTAGES) & 1;
      // warp-uniform: every lane breaks, or none does
      const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&ct.full[s], ph,
                                                            kSpinP) &&
                                                  !*abort_flag);
      if (!ok) {
        if (lane == 0) atomicOr(err, kErrTimeout);
        ct.abort = 1;
        break;
      }
      if (cid == 0) ct.consumed = kc + 1;
      // A: split the 128 x 32 tile in place (hi) and into the lo buffer
      float4 *ah = reinterpret_cast<float4 *>(a_hi(s));
      float4 *al = reinterpret_cast<float4 *>(a_lo(s));
#pragma unroll
      for (int h = 0; h < A_BYTES / 16 / 128; ++h) {
        const int i = cid + 128 * h;
        const float4 g = ah[i];
        const float4 gh = hi4(g);
        ah[i] = gh;
        al[i] = sub4(g, gh);
      }
      // B: rows k0 .. k0+31 of `in` (plain layout), stored transposed.
      // Thread (n, part) takes column n and the 16-byte chunks q = part,
      // part + P, ... of its 128-byte row (4 consecutive k each).
      constexpr int P = 128 / B;              // threads per column (2, 4, 8)
      const int n = cid % B, part = cid / B;
      const float *src = reinterpret_cast<const float *>(x_raw(s)) + n;
#pragma unroll
      for (int q = part; q < PK / 4; q += P) {
        const float4 v = make_float4(src[(4 * q + 0) * B], src[(4 * q + 1) * B],
                                     src[(4 * q + 2) * B], src[(4 * q + 3) * B]);
        const float4 vh = hi4(v);
        const uint32_t off = sw128(n, q);
        *reinterpret_cast<float4 *>(b_hi(s) + off) = vh;
        *reinterpret_cast<float4 *>(b_lo(s) + off) = sub4(v, vh);
      }
      // order these writes before the MMAs' (async proxy) reads
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&ct.ready[s]);
    }
  }
  __syncwarp();

  if (warp >= 2) {
    const bool ready =
        __all_sync(0xffffffffu, tc::mbar_wait(&ct.done, 0, kSpinP));
    if (!ready && lane == 0) atomicOr(err, kErrTimeout);
    // tcgen05.ld is warp-collective: decide for the whole warp
    const bool go = __all_sync(0xffffffffu, ready && !*abort_flag);
    if (go) {
      tc::fence_after_sync();
      const int q = warp & 3;                 // TMEM lane quarter of this warp
      const int r = row0 + q * 32 + lane;     // output row
      const uint32_t lrow = (uint32_t)(q * 32) << 16;
      const float *in2b = in2 ? in2 + bm.x_off : nullptr;
      float *outb = out + bm.x_off;
#pragma unroll 1
      for (int c0 = 0; c0 < B; c0 += 32) {
        // the five accumulators, added in a fixed order (warp-collective
        // loads, before any per-lane branch)
        float a[32], t2[32];
        tc::tmem_ld32(taddr + lrow + c0, a);
        tc::tmem_ld32(taddr + lrow + B + c0, t2);
#pragma unroll
        for (int j = 0; j < 32; ++j) a[j] += t2[j];
        float a23[32];
        tc::tmem_ld32(taddr + lrow + 2 * B + c0, a23);
        tc::tmem_ld32(taddr + lrow + 3 * B + c0, t2);
#pragma unroll
        for (int j = 0; j < 32; ++j) a23[j] += t2[j];
        tc::tmem_ld32(taddr + lrow + 4 * B + c0, t2);
#pragma unroll
        for (int j = 0; j < 32; ++j) a[j] = (a[j] + a23[j]) + t2[j];
        if (r < sp) {
          constexpr int W = B < 32 ? B : 32;
#pragma unroll
          for (int j = 0; j < W; ++j) {
            const int64_t o = (int64_t)r * B + c0 + j;
            float v = alpha * a[j];
            if (beta != 0.f) v = fmaf(beta, inb[o], v);
            if (gamma != 0.f) v = fmaf(gamma, in2b[o], v);
            outb[o] = v;
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && ct.abort) {
    // drain G tiles that were issued but never seen to land
    for (int kc = ct.consumed; kc < ct.issued; ++kc)
      tc::mbar_wait(&ct.full[kc % PSTAGES], (kc / PSTAGES) & 1, kSpinP);
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, L::TMEM_COLS);
}

template <int B>
cudaError_t launch_b(const BlockMeta *meta, SolverState *state,
                     const int2 *tiles, int32_t ntiles,
                     const CUtensorMap *gmaps, const CUtensorMap *xmaps,
                     const float *in, const float *in2, float *out, int mode,
                     int step, int32_t *err, cudaStream_t st) {
  static_assert(panel_tc_smem<B>() <= 227 * 1024, "shared memory");
  static_assert(kAcc * B <= PanelTc<B>::TMEM_COLS, "tensor memory");
  cudaError_t e = cudaFuncSetAttribute(
      k_gpanel_tc<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)panel_tc_smem<B>());
  if (e != cudaSuccess) return e;
  k_gpanel_tc<B><<<ntiles, 192, panel_tc_smem<B>(), st>>>(
      meta, state, tiles, gmaps, xmaps, in, in2, out, mode, step, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gpanel_tc(int32_t bsub, const BlockMeta *meta,
                             SolverState *state, const int2 *tiles,
                             int32_t ntiles, const CUtensorMap *gmaps,
                             const CUtensorMap *xmaps, const float *in,
                             const float *in2, float *out, int mode, int step,
                             int32_t *err, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  switch (bsub) {
    case 16: return launch_b<16>(meta, state, tiles, ntiles, gmaps, xmaps, in,
                                 in2, out, mode, step, err, st);
    case 32: return launch_b<32>(meta, state, tiles, ntiles, gmaps, xmaps, in,
                                 in2, out, mode, step, err, st);
    case 64: return launch_b<64>(meta, state, tiles, ntiles, gmaps, xmaps, in,
                                 in2, out, mode, step, err, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bsvd
