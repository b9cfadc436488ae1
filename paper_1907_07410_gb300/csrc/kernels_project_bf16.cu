// Projection F_L = W^T F_s of the BF16 form on the tcgen05 tensor cores.
//
// Section 2.1 (Eq. 2) predicts with the user and item factors; with the
// Gram side's eigenvectors F_s (s x k) in hand, the other side's factor is
// one product with the centred block, F_L = W^T F_s (L x k). The BF16 form
// factorises the bf16 copy of the centred blocks (its Gram is W_h W_h^T),
// so its projection reads that same copy: 2 bytes per cell instead of the
// float32 arena's 4, which the BF16 form then never writes. F_s is split
// into bf16 hi and lo parts (hi = bf16(F), lo = bf16(F - hi)), so the
// products carry about 16 bits of F_s; W_h's values are used exactly.
//
// A CTA computes 128 consecutive rows l of F_L over the whole K range
// a < s, in stages of 64 rows a:
//   * warp 0: TMA loads of the W_h box (64 rows a x 128 columns l, plain
//     layout) into a ring of W stages, each released as soon as the
//     converters have read it; warp 10: TMA loads of F_s's bf16 B form for
//     those 64 rows (2 kn rows of 64 values, 128-byte swizzle; rows n < kn
//     hold hi, n >= kn hold lo) into the A + B stages, released when their
//     MMAs complete;
//   * warps 2-9 (converters): thread (l, half) reads its column of the box
//     (32 values of a), packs them in pairs and writes one half of row l of
//     the A tile W_h^T (128 rows l x 64 a, K-major, 128-byte swizzle, the
//     layout TMA would write), then fences the writes for the tensor core;
//   * warp 1: four K = 16 MMAs (kind::f16, bf16 x bf16 -> f32) per stage,
//     D[l, n] += A[l, k] B[n, k], round-robin over two accumulators;
//   * epilogue (warps 2-5): F_L[l, j] = sum of the accumulators' hi and lo
//     columns j and kn + j, for j < kp.
// Three W stages of 16 KiB (two when k > 48), two A + B stages and 256
// tensor-memory columns: two CTAs per SM. (With one ring of two 48 KiB
// stages, each held until its MMAs completed, the kernel read W_h at 0.67
// of the measured HBM bandwidth on the mid workload.)
// Every wait is bounded; a timeout sets kErrTimeout and the CTA drains its
// copies in flight and frees its tensor memory before returning.
#include "kernels.h"
#include "tc_ptx.cuh"

namespace bsvd {

namespace {

constexpr int JT = 128;                   // rows l of F_L per CTA (MMA M)
constexpr int JK = 64;                    // rows a of W per stage (K)
constexpr int kJConv = 8;                 // converter warps (2..9)
constexpr int kJBWarp = 10;               // the B-stage producer warp
constexpr int kJThreads = 32 * (kJBWarp + 1);   // 11 warps
constexpr int kJAS = 2;                   // A + B stages
constexpr int kJMaxWS = 3;                // W stages (3 when they fit)
constexpr int kJR = 2;                    // accumulators
constexpr int kJTmemCols = 256;
constexpr uint32_t kJSpin = 1u << 22;     // mbarrier polls before giving up
constexpr int W_BYTES = JK * JT * 2;      // 16 KiB W_h box
constexpr int A_BYTES = JT * JK * 2;      // 16 KiB W_h^T tile
constexpr size_t kJSmemMax = 113 * 1024;  // two CTAs per SM

struct JCtrl {
  uint64_t wfull[kJMaxWS];     // W_h box landed (TMA bytes)
  uint64_t wempty[kJMaxWS];    // the box read by the 8 converter warps
  uint64_t bfull[kJAS];        // B-form rows landed (TMA bytes)
  uint64_t aready[kJAS];       // A tile written (the 8 converter warps)
  uint64_t abempty[kJAS];      // the stage's MMAs completed
  uint64_t done;               // every MMA completed
  uint32_t tmem;
  int abort;
  int wissued, wconsumed;      // W boxes issued / seen to land
  int bissued, bconsumed;      // B stages issued / seen to land
};

// Shared-memory layout for a B form of N = 2 kn rows: the W ring, then the
// A + B ring (each stage an A tile and the B rows, 1024-byte aligned), then
// the control block.
struct JLayout {
  int ws;             // W stages
  int b_bytes;        // one stage's B rows
  int ab_bytes;       // one A + B stage
  size_t ctrl_off;
  size_t smem;        // dynamic shared memory to request
};

__host__ __device__ inline JLayout jlayout(int kn) {
  JLayout L;
  L.b_bytes = ((2 * kn * 128) + 1023) / 1024 * 1024;
  L.ab_bytes = A_BYTES + L.b_bytes;
  L.ws = kJMaxWS;
  for (;;) {
    L.ctrl_off = (size_t)L.ws * W_BYTES + (size_t)kJAS * L.ab_bytes;
    L.smem = L.ctrl_off + sizeof(JCtrl) + 1024;
    if (L.smem <= kJSmemMax || L.ws == 2) break;
    --L.ws;
  }
  return L;
}

__device__ __forceinline__ uint32_t sw128(int r, int c) {
  return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// W boxes and the A + B stages are separate rings: a W box (from HBM) is
// released as soon as the converter warps have read it, an A + B stage when
// its MMAs complete, and the B rows (from L2) have their own producer warp.
__global__ void __launch_bounds__(kJThreads, 2)
k_project_bf16(const BlockMeta *__restrict__ meta,
               const int2 *__restrict__ tiles,
               const CUtensorMap *__restrict__ wmaps,
               const CUtensorMap *__restrict__ fmaps, float *FL, int kp,
               int kn, int32_t *err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const JLayout L = jlayout(kn);
  const int WS = L.ws;
  JCtrl &ct = *reinterpret_cast<JCtrl *>(base + L.ctrl_off);
  auto wbox = [&](int s) { return base + (size_t)s * W_BYTES; };
  auto atile = [&](int s) {
    return base + (size_t)WS * W_BYTES + (size_t)s * L.ab_bytes;
  };
  auto brows = [&](int s) { return atile(s) + A_BYTES; };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int2 t = tiles[blockIdx.x];
  const BlockMeta bm = meta[t.x];
  const int l0 = t.y;
  const int nk = (bm.s_pad + JK - 1) / JK;
  const int N = 2 * kn;

  if (warp == 0) tc::tmem_alloc(&ct.tmem, kJTmemCols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < WS; ++s) {
      tc::mbar_init(&ct.wfull[s], 1);
      tc::mbar_init(&ct.wempty[s], kJConv);
    }
    for (int s = 0; s < kJAS; ++s) {
      tc::mbar_init(&ct.bfull[s], 1);
      tc::mbar_init(&ct.aready[s], kJConv);
      tc::mbar_init(&ct.abempty[s], 1);
    }
    tc::mbar_init(&ct.done, 1);
    ct.abort = 0;
    ct.wissued = ct.wconsumed = 0;
    ct.bissued = ct.bconsumed = 0;
    tc::mbar_init_fence();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  // F_s's B form comes from the previous kernel
  pdl_wait();
  const uint32_t taddr = ct.tmem;
  volatile int *abort_flag = &ct.abort;
  auto give_up = [&]() {
    if (lane == 0) atomicOr(err, kErrTimeout);
    ct.abort = 1;
  };

  if (warp == 0) {
    // W boxes: rows a = 64 kc .. of W_h, columns l0 .. l0 + 127
    const CUtensorMap *wmap = wmaps + t.x;
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % WS;
      const bool ok = __all_sync(
          0xffffffffu,
          tc::mbar_wait(&ct.wempty[s], ((kc / WS) & 1) ^ 1, kJSpin) &&
              !*abort_flag);
      if (!ok) {
        give_up();
        break;
      }
      if (tc::elect_one()) {
        tc::mbar_expect_tx(&ct.wfull[s], W_BYTES);
        tc::tma_load_2d(wbox(s), wmap, l0, kc * JK, &ct.wfull[s]);
        ct.wissued = kc + 1;
      }
      __syncwarp();
    }
  } else if (warp == kJBWarp) {
    // B rows: F_s's bf16 B form for rows a of stage kc
    const CUtensorMap *fmap = fmaps + t.x;
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % kJAS;
      const bool ok = __all_sync(
          0xffffffffu,
          tc::mbar_wait(&ct.abempty[s], ((kc / kJAS) & 1) ^ 1, kJSpin) &&
              !*abort_flag);
      if (!ok) {
        give_up();
        break;
      }
      if (tc::elect_one()) {
        tc::mbar_expect_tx(&ct.bfull[s], (uint32_t)(N * 128));
        tc::tma_load_2d(brows(s), fmap, 0, kc * N, &ct.bfull[s]);
        ct.bissued = kc + 1;
      }
      __syncwarp();
    }
  } else if (warp == 1) {
    const uint32_t idesc = tc::idesc_bf16_f32(JT, (uint32_t)N);
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % kJAS;
      const uint32_t ph = (kc / kJAS) & 1;
      const bool okb = tc::mbar_wait(&ct.bfull[s], ph, kJSpin);
      const bool ok = __all_sync(
          0xffffffffu, okb && tc::mbar_wait(&ct.aready[s], ph, kJSpin) &&
                           !*abort_flag);
      if (!ok) {
        give_up();
        break;
      }
      if (lane == 0) ct.bconsumed = kc + 1;
      tc::fence_after_sync();
      const uint64_t da = tc::sdesc_kmajor_sw128(tc::smem_u32(atile(s)));
      const uint64_t db = tc::sdesc_kmajor_sw128(tc::smem_u32(brows(s)));
      if (tc::elect_one()) {
#pragma unroll
        for (int kk = 0; kk < JK / 16; ++kk) {
          // K slice 16 kk: 32 bytes further along each 128-byte row
          const uint32_t d = taddr + (uint32_t)(N * (kk % kJR));
          const uint32_t acc = (kc > 0 || kk >= kJR) ? 1u : 0u;
          tc::mma_bf16(d, da + 2 * kk, db + 2 * kk, idesc, acc);
        }
        tc::mma_commit(&ct.abempty[s]);
      }
      __syncwarp();
    }
    if (tc::elect_one()) tc::mma_commit(&ct.done);
    __syncwarp();
  } else {
    // converters: thread (r, kh) owns row l0 + r of the A tile, K half kh
    const int cid = threadIdx.x - 64;
    const int r = cid & (JT - 1);
    const int kh = cid >> 7;
    for (int kc = 0; kc < nk; ++kc) {
      const int ws = kc % WS, s = kc % kJAS;
      bool ok = __all_sync(
          0xffffffffu,
          tc::mbar_wait(&ct.wfull[ws], (kc / WS) & 1, kJSpin) && !*abort_flag);
      if (!ok) {
        give_up();
        break;
      }
      if (cid == 0) ct.wconsumed = kc + 1;
      // the box holds rows a of 128 bf16 (l): this thread's column, rows
      // 32 kh .. 32 kh + 31, packed two per 32-bit word (lower a low)
      const unsigned short *wt =
          reinterpret_cast<const unsigned short *>(wbox(ws)) + r;
      uint32_t p[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int a = 32 * kh + 2 * j;
        p[j] = (uint32_t)wt[a * JT] | ((uint32_t)wt[(a + 1) * JT] << 16);
      }
      // the box is in registers: release it to the W loads
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&ct.wempty[ws]);
      // the A tile's previous MMAs have completed
      ok = __all_sync(
          0xffffffffu,
          tc::mbar_wait(&ct.abempty[s], ((kc / kJAS) & 1) ^ 1, kJSpin) &&
              !*abort_flag);
      if (!ok) {
        give_up();
        break;
      }
      unsigned char *arow = atile(s);
#pragma unroll
      for (int c = 0; c < 4; ++c)
        *reinterpret_cast<uint4 *>(arow + sw128(r, 4 * kh + c)) =
            make_uint4(p[4 * c], p[4 * c + 1], p[4 * c + 2], p[4 * c + 3]);
      // generic-proxy writes, read next by the tensor core
      fence_async_shared();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&ct.aready[s]);
    }
  }
  __syncwarp();

  pdl_trigger();
  if (warp >= 2 && warp < 6) {
    const bool ready =
        __all_sync(0xffffffffu, tc::mbar_wait(&ct.done, 0, kJSpin));
    if (!ready && lane == 0) atomicOr(err, kErrTimeout);
    // tcgen05.ld is warp-collective: decide for the whole warp
    const bool go = __all_sync(0xffffffffu, ready && !*abort_flag);
    if (go) {
      tc::fence_after_sync();
      const int q = warp & 3;                 // TMEM lane quarter of this warp
      const int l = l0 + q * 32 + lane;
      const uint32_t lrow = (uint32_t)(q * 32) << 16;
      float *out = FL + bm.fl_off + (int64_t)l * kp;
#pragma unroll 1
      for (int c0 = 0; c0 < kn; c0 += 16) {
        float h0[16], h1[16], o0[16], o1[16];
        tc::tmem_ld16(taddr + lrow + c0, h0);
        tc::tmem_ld16(taddr + lrow + N + c0, h1);
        tc::tmem_ld16(taddr + lrow + kn + c0, o0);
        tc::tmem_ld16(taddr + lrow + N + kn + c0, o1);
        if (l < bm.L) {
          // kp is a multiple of 4: whole float4s up to it
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4) {
            const int j = c0 + 4 * c4;
            if (j < kp) {
              float y[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int e = 4 * c4 + u;
                y[u] = (h0[e] + h1[e]) + (o0[e] + o1[e]);
              }
              *reinterpret_cast<float4 *>(out + j) =
                  make_float4(y[0], y[1], y[2], y[3]);
            }
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && ct.abort) {
    // drain loads that were issued but never seen to land
    for (int kc = ct.wconsumed; kc < ct.wissued; ++kc)
      tc::mbar_wait(&ct.wfull[kc % WS], (kc / WS) & 1, kJSpin);
    for (int kc = ct.bconsumed; kc < ct.bissued; ++kc)
      tc::mbar_wait(&ct.bfull[kc % kJAS], (kc / kJAS) & 1, kJSpin);
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, kJTmemCols);
}

// F_s's bf16 B form for k_project_bf16: per block, for each 64-row chunk c
// of F_s, 2 kn rows of 64 values at row c * 2 kn + n (n < kn: bf16(F[a, n]),
// n >= kn: bf16(F[a, n - kn] - hi)), zero past column kp and row s_pad. One
// CTA per 128-row tile, thread = row a.
__global__ void __launch_bounds__(128)
k_bform_fs16(const BlockMeta *__restrict__ meta, const int2 *__restrict__ tiles,
             const float *__restrict__ Fs, int kp, int kn,
             __nv_bfloat16 *__restrict__ out) {
  pdl_wait();
  pdl_trigger();
  const int2 t = tiles[blockIdx.x];
  const BlockMeta bm = meta[t.x];
  const int a = t.y + threadIdx.x;
  const int nch = (bm.s_pad + JK - 1) / JK;
  const int c = a / JK;
  if (c >= nch) return;
  const int N = 2 * kn;
  __nv_bfloat16 *dst = out + bm.fb_off + (int64_t)c * N * JK + (a % JK);
  const float *src = Fs + bm.fs_off + (int64_t)a * kp;
  for (int j = 0; j < kn; ++j) {
    const float v = (a < bm.s_pad && j < kp) ? src[j] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo =
        __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(h)));
    dst[(int64_t)j * JK] = h;
    dst[(int64_t)(kn + j) * JK] = lo;
  }
}

}  // namespace

int64_t project_bf16_bform_elems(int32_t s_pad, int32_t kn) {
  return (int64_t)((s_pad + JK - 1) / JK) * 2 * kn * JK;
}

cudaError_t launch_project_bf16(const BlockMeta *meta, const int2 *tiles,
                                int32_t ntiles, const CUtensorMap *wmaps,
                                const CUtensorMap *fmaps, float *FL,
                                int32_t kp, int32_t kn, int32_t *err,
                                cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (kn < 16 || kn > 64 || kn % 16 != 0 || kp > kn)
    return cudaErrorInvalidValue;
  const JLayout L = jlayout(kn);
  if (L.smem > kJSmemMax) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(
      k_project_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)L.smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_project_bf16, dim3((unsigned)ntiles), dim3(kJThreads),
                    L.smem, st, meta, tiles, wmaps, fmaps, FL, (int)kp,
                    (int)kn, err);
}

cudaError_t launch_bform_fs16(const BlockMeta *meta, const int2 *tiles,
                              int32_t ntiles, const float *Fs, int32_t kp,
                              int32_t kn, __nv_bfloat16 *out,
                              cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  return launch_pdl(k_bform_fs16, dim3((unsigned)ntiles), dim3(128), 0, st,
                    meta, tiles, Fs, (int)kp, (int)kn, out);
}

}  // namespace bsvd
