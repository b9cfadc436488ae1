// Rank-k reconstruction of one block on the tcgen05 tensor cores.
//
// Section 2 approximates a block by its rank-k truncation U_k S_k V_k^T; the
// library holds it as two factors, the user side P = U_k S_k (mb x k) and
// the item side V (nb x k), so the dense reconstruction is one product with
// a short contraction:
//   out[r, c] = mu + sum_{j < k} P[r, j] V[c, j]     (mb x nb, row-major).
// In the library's storage the Gram side's factor is F_s (s x kp) and the
// other side's F_L (L x kp), both row-major with the k values of a row
// contiguous (K-major, as the MMA wants both operands); P is F_s when the
// Gram side is the users, else F_L.
//
// Persistent: one CTA per SM walks a contiguous run of 128 x 64 output
// tiles (row-major, so consecutive tiles share their 128 rows of P) with
// a group of four loading warps and one of twelve writing warps:
//   * warps 0-3 load: the strip's 128 rows of P when the strip changes and
//     the tile's 64 rows of V (kp floats each), split every value x into
//     hi = x rounded to 10 mantissa bits and lo = x - hi, and write both
//     into shared memory in the 128-byte-swizzled K-major layout (two
//     32-float atoms along K, zeros past kp and past the block's edge);
//     one elected thread then issues, per K = 8 slice, P_hi V_hi, P_hi V_lo
//     and P_lo V_hi (kind::tf32, M = 128, N = 64) into one of two
//     tensor-memory accumulators: the dropped lo x lo term is below 2^-21
//     relative, as in the panel products;
//   * warps 4-7 read: each reads its 32 rows of the finished accumulator
//     (and frees it), adds mu and fills a shared-memory tile; warps 4-15
//     then write the tile's rows to global memory with consecutive threads
//     on consecutive columns. (With the four readers alone writing, the
//     stores in flight limited the kernel to 1.1 TB/s on a 92,840 x 4,619
//     block; twelve writers reach 1.9 TB/s. 16-byte stores along the rows
//     changed nothing.)
// V rows and accumulators are double-buffered, so the next tile's loads
// and MMAs run while the last one's rows are written. Every wait is an
// mbarrier wait with a bound (no named barriers); a timeout sets
// kErrTimeout and both groups stop.
// The contraction is at most 56 long, so the kernel is bound by writing
// out (4 bytes per cell against 2k flops); the tensor cores only keep the
// arithmetic off that path.
#include "kernels.h"
#include "tc_ptx.cuh"

namespace bsvd {

namespace {

constexpr int RT = 128;                       // tile rows (MMA M)
constexpr int CT = 64;                        // tile columns (MMA N)
constexpr int RK = 64;                        // K padded to two swizzle atoms
constexpr int kRThreads = 512;                // 4 loading, 12 writing warps
constexpr int kRWriters = 12;                 // warps 4-15 write out rows
constexpr uint32_t kRSpin = 1u << 22;         // mbarrier polls before giving up
constexpr int A_ATOM = RT * 128;              // 16 KiB: 128 rows x 32 floats
constexpr int B_ATOM = CT * 128;              // 8 KiB: 64 rows x 32 floats
constexpr int A_BYTES = 2 * A_ATOM;           // one part of P, K = 64
constexpr int B_BYTES = 2 * B_ATOM;           // one part of V
constexpr int B_OFF = 2 * A_BYTES;            // V buffers (hi, lo) x 2
constexpr int T_OFF = B_OFF + 4 * B_BYTES;    // the output tile
constexpr int T_BYTES = (RT * (CT + 1) * 4 + 1023) / 1024 * 1024;
constexpr int C_OFF = T_OFF + T_BYTES;        // the control block

struct RCtrl {
  uint64_t mma[2];      // the tile's MMAs completed (buffer b)
  uint64_t tfree[2];    // the writers read accumulator b (4 warps)
  uint64_t loaded[2];   // V (and P) rows of buffer b written (4 warps)
  uint64_t tfull;       // the output tile filled (warps 4-7)
  uint64_t tdone;       // the output tile written out (warps 4-15)
  uint32_t tmem;
  int abort;
};
constexpr int kRSmem = C_OFF + (int)sizeof(RCtrl) + 1024;

__device__ __forceinline__ uint32_t swz(int r, int c) {
  return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Row r (a row past the block's edge when !valid: zeros) of a kp-column
// factor into the hi and lo parts of an operand: 16-byte chunk q of the row
// (4 floats of K) goes to atom q / 8, chunk q mod 8 of the swizzled row.
__device__ __forceinline__ void put_row(unsigned char *hi, unsigned char *lo,
                                        int atom, int r, const float *src,
                                        bool valid, int kp) {
#pragma unroll
  for (int q = 0; q < RK / 4; ++q) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid && 4 * q < kp) v = *reinterpret_cast<const float4 *>(src + 4 * q);
    const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z),
                                 tf32_hi(v.w));
    const float4 l = make_float4(__fsub_rn(v.x, h.x), __fsub_rn(v.y, h.y),
                                 __fsub_rn(v.z, h.z), __fsub_rn(v.w, h.w));
    const uint32_t off = (uint32_t)((q >> 3) * atom) + swz(r, q & 7);
    *reinterpret_cast<float4 *>(hi + off) = h;
    *reinterpret_cast<float4 *>(lo + off) = l;
  }
}

__global__ void __launch_bounds__(kRThreads, 1)
k_reconstruct_tc(const BlockMeta *__restrict__ meta, int32_t b,
                 const float *__restrict__ Fs, const float *__restrict__ FL,
                 int32_t kp, float mu, float *__restrict__ out,
                 int32_t *err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char *a_hi = base, *a_lo = base + A_BYTES;
  auto b_hi = [&](int buf) { return base + B_OFF + buf * 2 * B_BYTES; };
  auto b_lo = [&](int buf) { return b_hi(buf) + B_BYTES; };
  float (*tile)[CT + 1] = reinterpret_cast<float (*)[CT + 1]>(base + T_OFF);
  RCtrl &ct = *reinterpret_cast<RCtrl *>(base + C_OFF);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const BlockMeta bm = meta[b];
  // P (rows r of out) and V (columns c) in the library's storage
  const float *P = bm.trans ? FL + bm.fl_off : Fs + bm.fs_off;
  const float *V = bm.trans ? Fs + bm.fs_off : FL + bm.fl_off;
  const int nct = (bm.nb + CT - 1) / CT;
  const int64_t units = (int64_t)((bm.mb + RT - 1) / RT) * nct;
  const int64_t per = (units + gridDim.x - 1) / gridDim.x;
  const int64_t u0 = (int64_t)blockIdx.x * per;
  const int64_t u1 = u0 + per < units ? u0 + per : units;
  const int ntile = u1 > u0 ? (int)(u1 - u0) : 0;

  if (warp == 0) tc::tmem_alloc(&ct.tmem, 2 * CT);
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&ct.mma[i], 1);
      tc::mbar_init(&ct.tfree[i], 4);
      tc::mbar_init(&ct.loaded[i], 4);
    }
    tc::mbar_init(&ct.tfull, 4);
    tc::mbar_init(&ct.tdone, kRWriters);
    ct.abort = 0;
    tc::mbar_init_fence();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = ct.tmem;
  volatile int *abort_flag = &ct.abort;
  auto give_up = [&]() {
    if (lane == 0) atomicOr(err, kErrTimeout);
    ct.abort = 1;
  };

  if (warp < 4) {
    // loading warps: thread t takes row t of P and, t < 64, row t of V
    const int t = threadIdx.x;
    const int nks = (kp + 7) / 8;                 // K = 8 slices in use
    constexpr uint32_t idesc = tc::idesc_tf32_f32(RT, CT);
    int64_t strip = -1;
    for (int j = 0; j < ntile; ++j) {
      const int64_t u = u0 + j;
      const int64_t su = u / nct;
      const int cu = (int)(u % nct);
      const int buf = j & 1;
      const uint32_t par = (j >> 1) & 1;
      // buffer j mod 2 is free once the MMAs of tile j - 2 completed and
      // the writers read their accumulator
      bool ok = tc::mbar_wait(&ct.mma[buf], par ^ 1, kRSpin) &&
                tc::mbar_wait(&ct.tfree[buf], par ^ 1, kRSpin);
      // P is rewritten for a new strip once the last MMAs that read it
      // (tile j - 1's) completed
      if (ok && su != strip && j > 0)
        ok = tc::mbar_wait(&ct.mma[(j - 1) & 1], ((j - 1) >> 1) & 1, kRSpin);
      ok = __all_sync(0xffffffffu, ok && !*abort_flag);
      if (!ok) {
        give_up();
        break;
      }
      if (su != strip) {
        const int64_t r = su * RT + t;
        put_row(a_hi, a_lo, A_ATOM, t, P + r * kp, r < bm.mb, kp);
        strip = su;
      }
      if (t < CT) {
        const int c = cu * CT + t;
        put_row(b_hi(buf), b_lo(buf), B_ATOM, t, V + (int64_t)c * kp,
                c < bm.nb, kp);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&ct.loaded[buf]);
      if (warp == 0) {
        ok = __all_sync(0xffffffffu,
                        tc::mbar_wait(&ct.loaded[buf], par, kRSpin) &&
                            !*abort_flag);
        if (!ok) {
          give_up();
          break;
        }
        tc::fence_after_sync();
        if (tc::elect_one()) {
          const uint32_t d = taddr + (uint32_t)(buf * CT);
          for (int kk = 0; kk < nks; ++kk) {
            const uint32_t oa = (uint32_t)((kk >> 2) * A_ATOM);
            const uint32_t ob = (uint32_t)((kk >> 2) * B_ATOM);
            const uint32_t k2 = 2 * (kk & 3);
            const uint64_t adh = tc::sdesc_kmajor_sw128(tc::smem_u32(a_hi + oa)) + k2;
            const uint64_t adl = tc::sdesc_kmajor_sw128(tc::smem_u32(a_lo + oa)) + k2;
            const uint64_t bdh = tc::sdesc_kmajor_sw128(tc::smem_u32(b_hi(buf) + ob)) + k2;
            const uint64_t bdl = tc::sdesc_kmajor_sw128(tc::smem_u32(b_lo(buf) + ob)) + k2;
            tc::mma_tf32(d, adh, bdh, idesc, kk > 0 ? 1u : 0u);
            tc::mma_tf32(d, adh, bdl, idesc, 1u);
            tc::mma_tf32(d, adl, bdh, idesc, 1u);
          }
          tc::mma_commit(&ct.mma[buf]);
        }
        __syncwarp();
      }
    }
  } else {
    // writing warps: warps 4-7 read TMEM lanes 32 (w mod 4) .. + 31 into
    // the output tile, then warps 4-15 write its rows out
    const bool reader = warp < 8;
    const int q = warp & 3;
    const int rr = q * 32 + lane;                 // tile row of a reader thread
    const uint32_t lrow = (uint32_t)(q * 32) << 16;
    for (int j = 0; j < ntile; ++j) {
      const int64_t u = u0 + j;
      const int64_t r0 = (u / nct) * RT;
      const int c0 = (int)(u % nct) * CT;
      const int buf = j & 1;
      const uint32_t par = (j >> 1) & 1;
      bool ok = true;
      if (reader) {
        ok = __all_sync(
            0xffffffffu,
            tc::mbar_wait(&ct.mma[buf], par, kRSpin) && !*abort_flag);
        if (!ok) {
          give_up();
          break;
        }
        tc::fence_after_sync();
        float v[CT];
        {
          float w[32];
          tc::tmem_ld32(taddr + lrow + (uint32_t)(buf * CT), w);
#pragma unroll
          for (int c = 0; c < 32; ++c) v[c] = w[c];
          tc::tmem_ld32(taddr + lrow + (uint32_t)(buf * CT + 32), w);
#pragma unroll
          for (int c = 0; c < 32; ++c) v[32 + c] = w[c];
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&ct.tfree[buf]);
        // the output tile is free once the last tile's rows were written
        ok = __all_sync(
            0xffffffffu,
            tc::mbar_wait(&ct.tdone, (j & 1) ^ 1, kRSpin) && !*abort_flag);
        if (!ok) {
          give_up();
          break;
        }
#pragma unroll
        for (int c = 0; c < CT; ++c) tile[rr][c] = mu + v[c];
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&ct.tfull);
      }
      ok = __all_sync(
          0xffffffffu,
          tc::mbar_wait(&ct.tfull, j & 1, kRSpin) && !*abort_flag);
      if (!ok) {
        give_up();
        break;
      }
      const int nr = (int)(bm.mb - r0 < RT ? bm.mb - r0 : RT);
      const int nc = bm.nb - c0 < CT ? bm.nb - c0 : CT;
      for (int r = warp - 4; r < nr; r += kRWriters) {
        float *dst = out + (r0 + r) * (int64_t)bm.nb + c0;
        for (int c = lane; c < nc; c += 32) dst[c] = tile[r][c];
      }
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&ct.tdone);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && ct.abort) {
    // MMAs issued but never seen to finish: wait (bounded) before freeing
    for (int i = 0; i < 2; ++i) {
      tc::mbar_wait(&ct.mma[i], 0, kRSpin);
      tc::mbar_wait(&ct.mma[i], 1, kRSpin);
    }
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, 2 * CT);
}

}  // namespace

cudaError_t launch_reconstruct(const BlockMeta *meta, const BlockMeta &host,
                               int32_t b, const float *Fs, const float *FL,
                               int32_t kp, float mu, float *out, int32_t *err,
                               cudaStream_t st) {
  if (host.mb <= 0 || host.nb <= 0) return cudaSuccess;
  if (kp <= 0 || kp > RK || kp % 4 != 0) return cudaErrorInvalidValue;
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t units = (int64_t)((host.mb + RT - 1) / RT) *
                        ((host.nb + CT - 1) / CT);
  const int grid = (int)(units < nsm ? units : nsm);
  static_assert(kRSmem <= 227 * 1024, "shared memory");
  cudaError_t e = cudaFuncSetAttribute(
      k_reconstruct_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kRSmem);
  if (e != cudaSuccess) return e;
  k_reconstruct_tc<<<grid, kRThreads, kRSmem, st>>>(meta, b, Fs, FL, kp, mu,
                                                   out, err);
  return cudaGetLastError();
}

}  // namespace bsvd
