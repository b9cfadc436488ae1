// Device-side data layout shared by the kernels of libbsvd.
//
// One rating matrix X (m users x n items) is cut into a p x q grid of
// blocks (Section 3, Eq. "datax"). Every block b stores its centred dense
// matrix B_b "Gram-side major":
//
//   W_b = B_b^T (s = n_b items, L = m_b users)  when n_b <= m_b   (trans=1)
//   W_b = B_b   (s = m_b users, L = n_b items)  otherwise         (trans=0)
//
// W_b is s_pad x L_pad row-major in one arena, zero-padded. Its Gram matrix
// G_b = W_b W_b^T (s x s) is the smaller of B^T B and B B^T, and its top-k
// eigenvectors F_s are the singular vectors of the shorter side. The longer
// side's factor is F_L = W_b^T F_s (L x k), i.e. U_k S_k or V_k S_k, so that
// B_b ~ F_s F_L^T in W orientation.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bsvd {

constexpr int kPad = 32;          // s and L are padded to multiples of this

// Programmatic dependent launch. A kernel launched with launch_pdl may be
// scheduled before the previous kernel in the stream has finished:
// pdl_wait() blocks until that kernel has completed and its memory is
// visible (a no-op for a kernel launched normally), so it comes before any
// global access. pdl_trigger() lets the next kernel be scheduled once every
// CTA of this one has called it or exited; single-wave kernels call it at
// entry, so the next launch's scheduling overlaps their work.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The GPU's global nanosecond timer.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// x rounded to the nearest value with 10 mantissa bits, ties away from 0
// (exact in tf32): the "hi" part of the split x = hi + lo that the tensor-
// core kernels use, lo = x - hi exactly.
__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x00001000u) & 0xFFFFE000u);
}

#ifdef __CUDACC__
template <typename... K, typename... A>
cudaError_t launch_pdl(void (*kernel)(K...), dim3 grid, dim3 block,
                       size_t smem, cudaStream_t st, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
#endif

constexpr int kMaxSub = 64;       // widest subspace the small solver handles

struct BlockMeta {
  int32_t mb, nb;       // block shape (users x items)
  int32_t s, L;         // Gram side, reduction side
  int32_t s_pad, L_pad; // padded to kPad
  int32_t trans;        // 1: W = B^T (s indexes items); 0: W = B
  int32_t keff;         // retained rank min(k, s) (set by factor)
  int32_t t0, nt;       // the block's 64-row tiles in the row-tile table
  int32_t s128;         // s rounded up to 128 (rows of each bf16 plane)
  int32_t owned;        // 1: this context holds the block (see set_owned)
  int64_t vx_off;       // bf16 planes offset: [Y; M], 2 s128 x L_pad
  int64_t row0, col0;   // first row / column position of the block
  int64_t w_off;        // W arena offset (floats)
  int64_t g_off;        // Gram offset, s_pad x s_pad
  int64_t x_off;        // subspace panels offset, s_pad x bsub
  int64_t fs_off;       // F_s offset, s_pad x kp
  int64_t fl_off;       // F_L offset, L_pad x kp
  int64_t fb_off;       // bf16 B form of F_s (BF16 form's projection)
  int32_t pt0, npt;     // the block's 128-row tiles of F_s (panel tiles)
  int32_t pj0, npj;     // the block's 128-row tiles of F_L (projection)
  int32_t ch0, nch;     // the block's kChunkRows-row chunks (small Grams)
};

// rows of the panels per chunk of the Rayleigh-Ritz small Grams
constexpr int kChunkRows = 512;

// Per-block state of the subspace iteration.
struct SolverState {
  float cut;            // upper end of the damped interval [0, cut]
  float a0;             // scaling point (largest Ritz value)
  float theta1;         // largest Ritz value
  float resid;          // max residual / theta1 at the last check
  int32_t bsub;         // subspace width used by this block (<= s)
  int32_t iters;        // Rayleigh-Ritz steps taken
  int32_t status;       // kRunning / kConverged / kCapped
  int32_t degree;       // Chebyshev degree of the next filter (even)
  uint64_t refill;      // Ritz columns refilled with random vectors
  int32_t sweeps;       // Jacobi sweeps used so far
  float amp;            // this block's filter amplification cap (0: default)
  int32_t products;     // panel products G X run for this block
  int32_t pad;
  int64_t cycles[3];    // SM clock cycles in the Rayleigh-Ritz kernel:
                        // [0] sums + Cholesky QR + H', [1] Jacobi, [2] rest
};

enum : int32_t { kRunning = 0, kConverged = 1, kCapped = 2 };

// Coefficients of one panel product out = alpha G in + beta in + gamma in2.
// mode 0: the plain product G in. mode 1 and 2: step `step` (1, then 2 ..
// degree) of the scaled three-term Chebyshev recurrence that damps the
// interval [0, cut] and keeps the value at the scaling point a0 at 1
// (Zhou and Saad's filtered subspace iteration).
__device__ __forceinline__ void cheb_coeffs(const SolverState &st, int mode,
                                            int step, float *alpha,
                                            float *beta, float *gamma) {
  *alpha = 1.f;
  *beta = 0.f;
  *gamma = 0.f;
  if (mode < 1) return;
  // damped interval [0, cut]: centre c, half-width e; p(a0) = 1
  const float e = 0.5f * st.cut, c = 0.5f * st.cut;
  const float sig1 = e / (st.a0 - c);
  if (mode == 1) {
    *alpha = sig1 / e;
    *beta = -c * *alpha;
    return;
  }
  const float tau = 2.f / sig1;
  float sig = sig1, sig_prev = sig1;
  for (int j = 2; j <= step; ++j) {
    sig_prev = sig;
    sig = 1.f / (tau - sig);
  }
  *alpha = 2.f * sig / e;
  *beta = -c * *alpha;
  *gamma = -sig_prev * sig;
}

// Error bits raised by kernels (read back by the calling entry point).
enum : int32_t {
  kErrIndex = 1,        // an id outside [0, m) or [0, n)
  kErrValue = 2,        // a non-finite rating or |x| >= 2^31
  kErrSumRange = 4,     // count * max|x| >= 2^31 in some block
  kErrBadPerm = 8,      // a permutation entry out of range or repeated
  kErrTimeout = 16,     // a bounded device-side wait gave up
  kErrNotExact = 32     // a rating is not an exact small integer offset
};

// Grid description used by every kernel that maps (user, item) to a block.
// Every field has a default, so a descriptor filled field by field never
// carries an indeterminate value.
struct GridDesc {
  int64_t m = 0, n = 0;
  int32_t p = 0, q = 0;
  int32_t equal_rows = 0, equal_cols = 0;   // 1: equal ceil-sized blocks
  int32_t diag = 0;                 // 1: only the p diagonal blocks exist
  int32_t pad = 0;
  int64_t br = 0, bc = 0;           // equal block sizes
  const int64_t *row_bounds = nullptr;   // device, p + 1
  const int64_t *col_bounds = nullptr;   // device, q + 1
  const int32_t *row_perm = nullptr;     // device or null
  const int32_t *col_perm = nullptr;     // device or null
};

// Largest j with bounds[j] <= v, for bounds[0] = 0 <= v < bounds[count].
__device__ __forceinline__ int32_t upper_index(const int64_t *bounds,
                                               int32_t count, int64_t v) {
  int32_t lo = 0, hi = count;       // invariant: bounds[lo] <= v < bounds[hi]
  while (hi - lo > 1) {
    int32_t mid = (lo + hi) >> 1;
    if (bounds[mid] <= v) lo = mid; else hi = mid;
  }
  return lo;
}

// Block id and local (row, col) of a rating; false if an id is out of range.
__device__ __forceinline__ bool locate(const GridDesc &g, int32_t u,
                                       int32_t i, int32_t *blk, int32_t *r,
                                       int32_t *c) {
  if (u < 0 || (int64_t)u >= g.m || i < 0 || (int64_t)i >= g.n) return false;
  int64_t ru = g.row_perm ? (int64_t)g.row_perm[u] : (int64_t)u;
  int64_t ci = g.col_perm ? (int64_t)g.col_perm[i] : (int64_t)i;
  int32_t bi, bj;
  if (g.equal_rows) bi = (int32_t)(ru / g.br);
  else bi = upper_index(g.row_bounds, g.p, ru);
  if (g.equal_cols) bj = (int32_t)(ci / g.bc);
  else bj = upper_index(g.col_bounds, g.q, ci);
  if (g.diag) {
    if (bi != bj) return false;     // off the block diagonal
    *blk = bi;
  } else {
    *blk = bi * g.q + bj;
  }
  *r = (int32_t)(ru - g.row_bounds[bi]);
  *c = (int32_t)(ci - g.col_bounds[bj]);
  return true;
}

// (r, c) of B -> (a, l) of W: a on the Gram side, l on the reduction side.
__device__ __forceinline__ void to_w(const BlockMeta &bm, int32_t r,
                                     int32_t c, int32_t *a, int32_t *l) {
  if (bm.trans) { *a = c; *l = r; } else { *a = r; *l = c; }
}

}  // namespace bsvd
