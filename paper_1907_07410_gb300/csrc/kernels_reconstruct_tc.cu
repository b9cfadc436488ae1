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
// A CTA (4 warps) computes a 128 x 64 tile of out (two CTAs per SM):
//   * the threads load the tile's 128 rows of P and 64 rows of V (kp
//     floats each),
//     split every value x into hi = x rounded to 10 mantissa bits and
//     lo = x - hi, and write hi and lo of both operands into shared memory
//     in the 128-byte-swizzled K-major layout (two 32-float atoms along K,
//     zeros past kp and past the block's edge), then fence them for the
//     tensor core's proxy;
//   * one elected thread issues, per K = 8 slice, P_hi V_hi, P_hi V_lo and
//     P_lo V_hi (kind::tf32, M = 128, N = 64) into one tensor-memory
//     accumulator: the dropped lo x lo term is below 2^-21 relative, as in
//     the panel products;
//   * each warp reads its 32 rows of the accumulator, adds mu and stores the
//     tile into shared memory (over the operands, which the MMAs no longer
//     read); the CTA then writes the tile's rows to global memory with
//     consecutive threads on consecutive columns.
// The contraction is at most 56 long, so the kernel is bound by writing
// out (4 bytes per cell against 2k flops); the tensor cores only keep the
// arithmetic off that path. The one wait (the MMAs' completion) is bounded;
// a timeout sets kErrTimeout, skips the tile's output and frees the tensor
// memory.
#include "kernels.h"
#include "tc_ptx.cuh"

namespace bsvd {

namespace {

constexpr int RT = 128;                       // tile rows (MMA M)
constexpr int CT = 64;                        // tile columns (MMA N)
constexpr int RK = 64;                        // K padded to two swizzle atoms
constexpr int kRThreads = 128;
constexpr uint32_t kRSpin = 1u << 22;         // mbarrier polls before giving up
constexpr int A_ATOM = RT * 128;              // 16 KiB: 128 rows x 32 floats
constexpr int B_ATOM = CT * 128;              // 8 KiB: 64 rows x 32 floats
constexpr int A_BYTES = 2 * A_ATOM;           // one part of P, K = 64
constexpr int B_BYTES = 2 * B_ATOM;           // one part of V
constexpr int OPS = 2 * A_BYTES + 2 * B_BYTES;
// A_hi, A_lo, B_hi, B_lo, then the barrier and the TMEM address
constexpr int kRSmem = OPS + 64 + 1024;
static_assert(RT * (CT + 1) * 4 <= OPS, "the output tile fits");
static_assert(kRSmem <= 113 * 1024, "two CTAs per SM");

__device__ __forceinline__ uint32_t swz(int r, int c) {
  return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Row `row` (< rows, else zeros) of a kp-column factor into the hi and lo
// parts of an operand: 16-byte chunk q of the row (4 floats of K) goes to
// atom q / 8, chunk q mod 8 of the swizzled 128-byte row.
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

__global__ void __launch_bounds__(kRThreads, 2)
k_reconstruct_tc(const BlockMeta *__restrict__ meta, int32_t b,
                 const float *__restrict__ Fs, const float *__restrict__ FL,
                 int32_t kp, float mu, float *__restrict__ out,
                 int32_t *err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char *a_hi = base, *a_lo = base + A_BYTES;
  unsigned char *b_hi = base + 2 * A_BYTES, *b_lo = b_hi + B_BYTES;
  uint64_t *done = reinterpret_cast<uint64_t *>(base + OPS);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(base + OPS + 8);
  float (*tile)[CT + 1] = reinterpret_cast<float (*)[CT + 1]>(base);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const BlockMeta bm = meta[b];
  const int r0 = blockIdx.y * RT, c0 = blockIdx.x * CT;
  // P (rows r of out) and V (columns c) in the library's storage
  const float *P = bm.trans ? FL + bm.fl_off : Fs + bm.fs_off;
  const float *V = bm.trans ? Fs + bm.fs_off : FL + bm.fl_off;

  if (warp == 0) tc::tmem_alloc(tslot, CT);
  if (threadIdx.x == 0) {
    tc::mbar_init(done, 1);
    tc::mbar_init_fence();
  }
  {
    const int t = threadIdx.x;
    const int r = r0 + t, c = c0 + t;
    put_row(a_hi, a_lo, A_ATOM, t, P + (int64_t)r * kp, r < bm.mb, kp);
    if (t < CT)
      put_row(b_hi, b_lo, B_ATOM, t, V + (int64_t)c * kp, c < bm.nb, kp);
  }
  fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *tslot;
  const int nks = (kp + 7) / 8;                   // K = 8 slices in use
  if (warp == 0) {
    constexpr uint32_t idesc = tc::idesc_tf32_f32(RT, CT);
    if (tc::elect_one()) {
      for (int kk = 0; kk < nks; ++kk) {
        const uint32_t oa = (uint32_t)((kk >> 2) * A_ATOM);
        const uint32_t ob = (uint32_t)((kk >> 2) * B_ATOM);
        const uint64_t adh = tc::sdesc_kmajor_sw128(tc::smem_u32(a_hi + oa)) + 2 * (kk & 3);
        const uint64_t adl = tc::sdesc_kmajor_sw128(tc::smem_u32(a_lo + oa)) + 2 * (kk & 3);
        const uint64_t bdh = tc::sdesc_kmajor_sw128(tc::smem_u32(b_hi + ob)) + 2 * (kk & 3);
        const uint64_t bdl = tc::sdesc_kmajor_sw128(tc::smem_u32(b_lo + ob)) + 2 * (kk & 3);
        tc::mma_tf32(taddr, adh, bdh, idesc, kk > 0 ? 1u : 0u);
        tc::mma_tf32(taddr, adh, bdl, idesc, 1u);
        tc::mma_tf32(taddr, adl, bdh, idesc, 1u);
      }
      tc::mma_commit(done);
    }
    __syncwarp();
  }
  const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(done, 0, kRSpin));
  if (!ok && lane == 0) atomicOr(err, kErrTimeout);
  const bool all_ok = __syncthreads_and(ok ? 1 : 0);
  tc::fence_after_sync();
  if (all_ok) {
    // warp w holds rows 32 w .. 32 w + 31 of the accumulator
    const int rr = warp * 32 + lane;
    const uint32_t lrow = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
    for (int cc = 0; cc < CT; cc += 32) {
      float v[32];
      tc::tmem_ld32(taddr + lrow + cc, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) tile[rr][cc + j] = mu + v[j];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (all_ok) {
    const int nr = min(RT, bm.mb - r0), nc = min(CT, bm.nb - c0);
    for (int r = warp; r < nr; r += kRThreads / 32) {
      float *dst = out + (int64_t)(r0 + r) * bm.nb + c0;
      for (int c = lane; c < nc; c += 32) dst[c] = tile[r][c];
    }
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, CT);
}

}  // namespace

cudaError_t launch_reconstruct(const BlockMeta *meta, const BlockMeta &host,
                               int32_t b, const float *Fs, const float *FL,
                               int32_t kp, float mu, float *out, int32_t *err,
                               cudaStream_t st) {
  if (host.mb <= 0 || host.nb <= 0) return cudaSuccess;
  if (kp <= 0 || kp > RK || kp % 4 != 0) return cudaErrorInvalidValue;
  const int64_t gy = (host.mb + RT - 1) / RT, gx = (host.nb + CT - 1) / CT;
  if (gy > 65535 || gx > 0x7fffffff) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(
      k_reconstruct_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kRSmem);
  if (e != cudaSuccess) return e;
  k_reconstruct_tc<<<dim3((unsigned)gx, (unsigned)gy), kRThreads, kRSmem,
                     st>>>(meta, b, Fs, FL, kp, mu, out, err);
  return cudaGetLastError();
}

}  // namespace bsvd
