// Truncated eigen-decomposition of the block Gram matrices.
//
// Section 2 defines the truncated SVD: keep the k largest singular values
// and their vectors. For a centred block, sigma_i^2 and v_i are the top
// eigenpairs of G = W W^T. They are found here by Chebyshev-filtered
// subspace iteration (Zhou and Saad, 2007) on a panel X of bsub >= k + 8
// columns per block:
//
//   1. X <- p_d(G) X. p_d is the degree-d Chebyshev polynomial that is small
//      on the unwanted interval [0, cut] and equals 1 at the largest Ritz
//      value a0. It uses the scaled three-term recurrence, so values stay
//      O(1) and float32 cannot overflow.
//   2. Rayleigh-Ritz on span(X) with Cholesky-QR orthonormalisation:
//        S = X^T X, S_n = D^-1 S D^-1 = L L^T (D = diag(S)^1/2),
//        T1 = D^-1 L^-T, so X T1 has orthonormal columns;
//        H' = T1^T (X^T G X) T1 = Y Theta Y^T,
//        X <- X T1 Y, and G X <- (G X) T1 Y without another product.
//      The b x b eigenproblem is solved by cyclic Jacobi with parallel
//      (round-robin) ordering in shared memory. A column whose Cholesky
//      pivot is below kPivotDrop is numerically inside the span of the
//      columns before it; it is dropped from the basis and refilled with a
//      fresh random vector, so the subspace keeps its width.
//   3. Stop a block when |G x_i - theta_i x_i| <= tol * theta_1 for its k
//      wanted pairs; otherwise cut <- smallest Ritz value and go to 1.
//
// The damped interval reaches up to the smallest kept Ritz value (a lower
// bound of the unwanted part of the spectrum), however close it is to
// theta_1. Noise-dominated blocks have flat spectra (sigma_1 / sigma_40
// about 1.1 on the 480,189 x 17,770 workload); capping the cut at
// theta_1 / 2 there left most of the unwanted spectrum undamped and took
// 2.2 times the panel products.
//
// The filter amplifies the top of the spectrum by C_d(t_1), with
// t_1 = 2 theta_1 / cut - 1, relative to the damped interval. In float32
// the columns that should hold the lower Ritz directions drown in rounding
// noise once that ratio nears 1/eps, so each block picks the largest even
// degree d <= max_degree with C_d(t_1) <= kMaxAmplification (at least 2).
// Steep spectra get short filters and more Rayleigh-Ritz steps.
//
// The same ratio is the spread between the filtered columns. Where the
// lower Ritz vectors are still poor (a wanted value near a dense bulk of
// unwanted ones), their errors along the top directions grow by up to
// C_d(t_1), the columns collapse onto those directions, and the Cholesky
// QR drops them. Refilled columns would collapse again in the next filter,
// and a cut taken at the smallest surviving Ritz value lands on a wanted
// one, so the solve stalls. A block that dropped columns therefore divides
// its own cap by kAmpBackoff (down to kMinAmplification) for the rest of
// its solve, and keeps its previous cut for that step.
//
// A block with s <= bsub starts from the identity basis, so the first
// Rayleigh-Ritz step is an exact eigen-decomposition of G.
#include <float.h>

#include <type_traits>

#include "kernels.h"

namespace bsvd {

namespace {

constexpr int TR = 64;       // panel rows per CTA
static_assert(kChunkRows % 32 == 0, "chunks are whole 32-row passes");
constexpr float kMaxAmplification = 3e6f;
constexpr float kMinAmplification = 1e3f;
constexpr float kAmpBackoff = 1e2f;
constexpr float kCutFloor = 1e-3f;   // cut >= kCutFloor * theta_1
// cut <= kCutCeil * theta_1, so that 2 theta_1 / cut - 1 >= 1.105 and the
// filter's degree stays defined when the Ritz values are nearly equal
constexpr float kCutCeil = 0.95f;
constexpr float kPivotDrop = 1e-4f;  // squared sine of the angle to the span
// |a_p . a_q| / (|a_p| |a_q|) to stop. Float32 dot products of 64 terms
// carry rounding near 5e-7 of |a_p| |a_q|, so a bar much below that is
// met only by chance and costs sweeps (3e-7 took about 5 a step at b = 64).
constexpr float kJacobiTol = 1e-6f;
constexpr float kJacobiTolFirst = 1e-3f;  // the same, first step from a random start

// hardware approximations (PTX .approx instructions, flush-to-zero)
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr int KC = 32;       // k-chunk of the panel GEMM

__device__ __forceinline__ float hash_uniform(uint64_t seed, uint64_t a,
                                              uint64_t b) {
  // splitmix64 of (seed, a, b) -> uniform in [-1, 1)
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (a * 0x100000001B3ull + b + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)(z >> 40) * (2.0f / 16777216.0f) - 1.0f;
}

template <int B>
__global__ void __launch_bounds__(256)
k_init_panels(const BlockMeta *__restrict__ meta,
              const SolverState *__restrict__ state,
              const int2 *__restrict__ rowtiles, float *__restrict__ X,
              uint64_t seed) {
  pdl_wait();
  pdl_trigger();
  const int2 t = rowtiles[blockIdx.x];
  const BlockMeta bm = meta[t.x];
  const int s = bm.s;
  const bool direct = s <= B;
  float *Xb = X + bm.x_off;
  for (int e = threadIdx.x; e < TR * B; e += blockDim.x) {
    const int r = t.y + e / B, c = e % B;
    if (r >= bm.s_pad) continue;
    float v = 0.f;
    if (r < s) {
      if (direct) v = (r == c) ? 1.f : 0.f;
      else v = hash_uniform(seed, (uint64_t)t.x, (uint64_t)r * B + c);
    }
    Xb[(int64_t)r * B + c] = v;
  }
}

// out = alpha * G in + beta * in + gamma * in2, on rows [row0, row0 + 64).
// G is symmetric, so the tile G[k0:k0+32, row0:row0+64] is read row-wise.
//
// 512 threads: four groups of 128 split the k range (group g takes chunks
// g, g + 4, ...), each with its own shared buffers, named barrier and a
// register prefetch of its next chunk, so four independent load streams
// are in flight per CTA. Thread (ty, tx) of a group owns rows 4ty..4ty+3 and
// columns tx*CN .. tx*CN+CN-1 (CN = B/8): 2 + CN/4 shared loads feed 4 CN
// FMAs. The four partial tiles are then added in group order (a fixed
// order, so results do not depend on scheduling) and the Chebyshev step is
// applied.
template <int B>
struct PanelSmem {
  float As[4][KC][TR + 4];
  float Bs[4][KC][B + 4];
};

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(128) : "memory");
}

template <int B>
__global__ void __launch_bounds__(512, (B >= 64 ? 1 : 2))
k_gpanel(const BlockMeta *__restrict__ meta, SolverState *state,
         const int2 *__restrict__ rowtiles, const float *__restrict__ G,
         const float *in, const float *in2, float *out, int mode, int step) {
  constexpr int CN = B / 8;                // output columns per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PanelSmem<B> &sm = *reinterpret_cast<PanelSmem<B> *>(smem_raw);
  const int2 t = rowtiles[blockIdx.x];
  const SolverState st = state[t.x];
  if (st.status != kRunning) return;
  if (mode >= 1 && step > st.degree) return;   // this block's filter is done
  if (t.y == 0 && threadIdx.x == 0) atomicAdd(&state[t.x].products, 1);
  const BlockMeta bm = meta[t.x];
  const int sp = bm.s_pad;
  const int row0 = t.y;
  const float *Gb = G + bm.g_off;
  const float *inb = in + bm.x_off;
  float *outb = out + bm.x_off;

  float alpha, beta, gamma;
  cheb_coeffs(st, mode, step, &alpha, &beta, &gamma);

  const int g = threadIdx.x >> 7, tid = threadIdx.x & 127;
  const int ty = tid >> 3, tx = tid & 7;
  float acc[4][CN];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < CN; ++c) acc[r][c] = 0.f;

  constexpr int AV = KC * TR / 4 / 128;            // float4 of G per thread
  constexpr int BV = (KC * B / 4 + 127) / 128;     // float4 of `in` per thread
  float4 ga[AV], gb[BV];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int h = 0; h < AV; ++h) {
      const int idx = tid + 128 * h;
      const int rr = idx >> 4, cc = (idx & 15) * 4;
      ga[h] = (row0 + cc < sp)
                  ? __ldg(reinterpret_cast<const float4 *>(
                        Gb + (int64_t)(k0 + rr) * sp + row0 + cc))
                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int h = 0; h < BV; ++h) {
      const int idx = tid + 128 * h;
      const int rr = idx / (B / 4), cc = (idx % (B / 4)) * 4;
      gb[h] = (idx < KC * B / 4)
                  ? *reinterpret_cast<const float4 *>(inb + (int64_t)(k0 + rr) * B + cc)
                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  const int nchunks = sp / KC;
  if (g < nchunks) fetch(g * KC);
  for (int ch = g; ch < nchunks; ch += 4) {
#pragma unroll
    for (int h = 0; h < AV; ++h) {
      const int idx = tid + 128 * h;
      *reinterpret_cast<float4 *>(&sm.As[g][idx >> 4][(idx & 15) * 4]) = ga[h];
    }
#pragma unroll
    for (int h = 0; h < BV; ++h) {
      const int idx = tid + 128 * h;
      if (idx < KC * B / 4)
        *reinterpret_cast<float4 *>(&sm.Bs[g][idx / (B / 4)][(idx % (B / 4)) * 4]) = gb[h];
    }
    group_sync(g);
    if (ch + 4 < nchunks) fetch((ch + 4) * KC);
#pragma unroll 8
    for (int kk = 0; kk < KC; ++kk) {
      float a[4], b[CN];
      *reinterpret_cast<float4 *>(a) =
          *reinterpret_cast<const float4 *>(&sm.As[g][kk][ty * 4]);
#pragma unroll
      for (int c = 0; c < CN; c += 4) {
        if (CN >= 4) {
          *reinterpret_cast<float4 *>(&b[c]) =
              *reinterpret_cast<const float4 *>(&sm.Bs[g][kk][tx * CN + c]);
        }
      }
      if (CN < 4) {
#pragma unroll
        for (int c = 0; c < CN; ++c) b[c] = sm.Bs[g][kk][tx * CN + c];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < CN; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    group_sync(g);
  }
  // add the four partial tiles in group order, then apply the step
  __syncthreads();
  float (*red)[TR][B + 1] = reinterpret_cast<float (*)[TR][B + 1]>(smem_raw);
  if (g > 0) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < CN; ++c) red[g - 1][ty * 4 + r][tx * CN + c] = acc[r][c];
  }
  __syncthreads();
  if (g != 0) return;
  const float *in2b = in2 ? in2 + bm.x_off : nullptr;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int lr = ty * 4 + r;
    const int row = row0 + lr;
    if (row >= sp) continue;
#pragma unroll
    for (int c = 0; c < CN; ++c) {
      const int col = tx * CN + c;
      const int64_t o = (int64_t)row * B + col;
      const float sum = ((acc[r][c] + red[0][lr][col]) + red[1][lr][col]) + red[2][lr][col];
      float v = alpha * sum;
      if (beta != 0.f) v = fmaf(beta, inb[o], v);
      if (gamma != 0.f) v = fmaf(gamma, in2b[o], v);
      outb[o] = v;
    }
  }
}

template <int B>
size_t panel_smem() {
  const size_t a = sizeof(PanelSmem<B>);
  const size_t r = sizeof(float) * 3 * TR * (B + 1);
  return a > r ? a : r;
}

// N consecutive floats (N = 1, 2 or 4; p aligned to 4 N bytes) in one load
template <int N>
__device__ __forceinline__ void ld_vec(const float *p, float (&v)[N]) {
  if constexpr (N == 4) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else if constexpr (N == 2) {
    const float2 q = *reinterpret_cast<const float2 *>(p);
    v[0] = q.x; v[1] = q.y;
  } else {
    v[0] = p[0];
  }
}

// The same N floats to global memory in one store
template <int N>
__device__ __forceinline__ void st_vec(float *p, const float (&v)[N]) {
  if constexpr (N == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (N == 2) {
    *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
  } else {
    p[0] = v[0];
  }
}

// Partial S = X^T X and H = X^T Z over one chunk of up to kChunkRows rows,
// for every chunk of every running block; k_rr_solve sums a block's chunks
// in a fixed order, so the totals do not depend on scheduling. The 256
// threads form a 16 x 16 grid over the b x b outputs, each thread a TI x TI
// register tile (TI = b / 16): per row, three 16-byte shared loads (its
// slices of the X row for i and j, and of the Z row for j) feed 2 TI^2
// fused multiply-adds. The rows are added in order, 32 at a time staged in
// shared memory.
template <int B>
__global__ void __launch_bounds__(256)
k_small_gram(const BlockMeta *__restrict__ meta,
             const SolverState *__restrict__ state,
             const int2 *__restrict__ chunks, const float *__restrict__ X,
             const float *__restrict__ Z, float *__restrict__ SHp) {
  pdl_wait();
  pdl_trigger();
  constexpr int TI = B / 16;
  constexpr int SR = 32;                   // rows staged per pass
  __shared__ __align__(16) float Xs[SR][B];
  __shared__ __align__(16) float Zs[SR][B];
  const int2 t = chunks[blockIdx.x];
  if (state[t.x].status != kRunning) return;
  const BlockMeta bm = meta[t.x];
  const int rows = min(kChunkRows, bm.s - t.y);
  const float *Xb = X + bm.x_off + (int64_t)t.y * B;
  const float *Zb = Z + bm.x_off + (int64_t)t.y * B;
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
  float sa[TI][TI], ha[TI][TI];
#pragma unroll
  for (int a = 0; a < TI; ++a)
#pragma unroll
    for (int b = 0; b < TI; ++b) sa[a][b] = ha[a][b] = 0.f;
  for (int r0 = 0; r0 < rows; r0 += SR) {
    const int nr = min(SR, rows - r0);
    __syncthreads();                       // the last pass has read Xs, Zs
    for (int e4 = threadIdx.x; e4 < nr * (B / 4); e4 += 256) {
      const int64_t o = (int64_t)r0 * B + 4 * e4;
      reinterpret_cast<float4 *>(&Xs[0][0])[e4] =
          *reinterpret_cast<const float4 *>(Xb + o);
      reinterpret_cast<float4 *>(&Zs[0][0])[e4] =
          *reinterpret_cast<const float4 *>(Zb + o);
    }
    __syncthreads();
    for (int rr = 0; rr < nr; ++rr) {
      float xi[TI], xj[TI], zj[TI];
      ld_vec(&Xs[rr][TI * ti], xi);
      ld_vec(&Xs[rr][TI * tj], xj);
      ld_vec(&Zs[rr][TI * tj], zj);
#pragma unroll
      for (int a = 0; a < TI; ++a)
#pragma unroll
        for (int b = 0; b < TI; ++b) {
          sa[a][b] = fmaf(xi[a], xj[b], sa[a][b]);
          ha[a][b] = fmaf(xi[a], zj[b], ha[a][b]);
        }
    }
  }
  float *S = SHp + (int64_t)blockIdx.x * 2 * B * B;
  float *H = S + B * B;
#pragma unroll
  for (int a = 0; a < TI; ++a)
#pragma unroll
    for (int b = 0; b < TI; ++b) {
      const int idx = (TI * ti + a) * B + TI * tj + b;
      S[idx] = sa[a][b];
      H[idx] = ha[a][b];
    }
}

// Round-robin pairings for cyclic Jacobi on ne (even) indices: round r pairs
// position i with position ne-1-i, where position 0 holds index 0 and
// position j >= 1 holds 1 + (j - 1 + r) mod (ne - 1). Every pair meets once
// per sweep of ne - 1 rounds, and the pairs of a round are disjoint.
__device__ __forceinline__ void build_pairs(int ne, unsigned short *tab) {
  const int np = ne / 2;
  for (int e = threadIdx.x; e < (ne - 1) * np; e += blockDim.x) {
    const int r = e / np, i = e % np;
    const int pa = i, pb = ne - 1 - i;
    const int p = pa == 0 ? 0 : 1 + (pa - 1 + r) % (ne - 1);
    const int q = 1 + (pb - 1 + r) % (ne - 1);
    tab[e] = (unsigned short)(p | (q << 8));
  }
}

// One-sided (Hestenes) Jacobi on a symmetric positive semi-definite n x n
// matrix held by columns: Ac[j][0..n) is column j of A, Vc[j] column j of V
// (V = I on entry). Column pairs are rotated until every pair is
// numerically orthogonal, |a_p.a_q| <= tol |a_p| |a_q|. Then A V = U S with
// orthonormal U, and for a PSD A the columns of V are its eigenvectors and
// the column norms |A v_j| its eigenvalues.
// Round-robin ordering gives np disjoint pairs per round. Each half-warp
// takes one pair (a warp two: pairs 2w + h, 2 (w + nwarps) + h, ...), lane
// l of the half holding rows l, l + 16, ... of the two columns. The three
// dot products are xor-butterfly sums over the half-warp: each step adds
// the same two operands in every lane, so the 16 lanes hold bitwise equal
// sums and apply the same rotation. The loop is issue-bound (one warp per
// pair took about 1600 cycles a round at b = 64: 32 warps' shuffles and
// address arithmetic), so two pairs per warp halve the instructions per
// round. One block-wide barrier per round.
template <int B>
__device__ int onesided_jacobi(float (*Ac)[B + 1], float (*Vc)[B + 1], int n,
                               int max_sweeps, const unsigned short *pairs,
                               int *flag, float tol) {
  constexpr int RPL = (B + 15) / 16;        // rows per lane
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int hl = lane & 15, half = lane >> 4;
  const int nwarps = blockDim.x >> 5;
  const int ne = n + (n & 1), np = ne / 2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int round = 0; round < ne - 1; ++round) {
      const unsigned short *pr = pairs + round * np;
      // warp-uniform trip count: both halves run the shuffles
      for (int w2 = warp; 2 * w2 < np; w2 += nwarps) {
        const int i = 2 * w2 + half;
        const bool has = i < np;
        const int p = has ? (pr[i] & 255) : 0, q = has ? (pr[i] >> 8) : 0;
        const bool valid = has && p < n && q < n;
        float a[RPL], b[RPL];
        float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
        for (int h = 0; h < RPL; ++h) {
          const int r = hl + 16 * h;
          a[h] = (valid && r < n) ? Ac[p][r] : 0.f;
          b[h] = (valid && r < n) ? Ac[q][r] : 0.f;
          al = fmaf(a[h], a[h], al);
          be = fmaf(b[h], b[h], be);
          ga = fmaf(a[h], b[h], ga);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (!valid || !(ga * ga > (tol * tol) * (al * be))) continue;
        // The angle only has to be close to the optimal one (any rotation
        // near it still converges), so t uses the hardware's approximate
        // reciprocal and square root; what must be accurate is c^2 + s^2 = 1,
        // so c = 1/sqrt(1 + t^2) gets one Newton step after the approximate
        // reciprocal square root. |zeta| large enough to overflow zeta^2
        // gives t = 0 and no rotation, as before.
        const float zeta = (be - al) * rcp_approx(2.f * ga);
        const float t = copysignf(
            rcp_approx(fabsf(zeta) + sqrt_approx(fmaf(zeta, zeta, 1.f))), zeta);
        const float x = fmaf(t, t, 1.f);
        float c = rsqrt_approx(x);
        c = c * fmaf(-0.5f * x, c * c, 1.5f);
        const float s = t * c;
        if (s == 0.f) continue;
        if (hl == 0) *flag = 1;
#pragma unroll
        for (int h = 0; h < RPL; ++h) {
          const int r = hl + 16 * h;
          if (r < n) {
            Ac[p][r] = c * a[h] - s * b[h];
            Ac[q][r] = s * a[h] + c * b[h];
            const float va = Vc[p][r], vb = Vc[q][r];
            Vc[p][r] = c * va - s * vb;
            Vc[q][r] = s * va + c * vb;
          }
        }
      }
      __syncthreads();
    }
    const int any = *flag;
    __syncthreads();
    if (!any) break;
  }
  return sweep;
}

template <int B>
struct RRSmem {
  float S[B][B + 1];      // S_n, then its Cholesky factor L (lower)
  float Li[B][B + 1];     // L^-1 (lower)
  float H[B][B + 1];
  float T1[B][B + 1];
  float A[B][B + 1];
  float V[B][B + 1];
  float d[B];
  float key[B];
  int drop[B];
  int rank[B];
  unsigned short pairs[(B - 1) * (B / 2)];
  int flag;
};

// Launched with 1024 threads, or with 512 (enough for the Jacobi's b / 4
// warps at b = 64) when there are more blocks than SMs: two such CTAs share
// an SM (at most 64 registers a thread either way), so 256 blocks run in
// one wave instead of two. Measured on GB300, two CTAs on one SM each take
// about 1.4 times as long as one alone, so with fewer blocks than SMs the
// wider CTA is faster.
template <int B>
__global__ void __launch_bounds__(1024, 1)
k_rr_solve(const BlockMeta *__restrict__ meta, SolverState *__restrict__ state,
           const float *__restrict__ SHp, float *__restrict__ Tout,
           float *__restrict__ theta, int max_sweeps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RRSmem<B> &sm = *reinterpret_cast<RRSmem<B> *>(smem_raw);
  const int blk = blockIdx.x;
  pdl_wait();
  pdl_trigger();
  if (state[blk].status != kRunning) return;
  const BlockMeta bm = meta[blk];
  const int n = state[blk].bsub;
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nw = (int)blockDim.x >> 5;
  const int ne = n + (n & 1), np = ne / 2;
  const long long c0 = clock64();
  build_pairs(ne, sm.pairs);
  // 1. sum the chunk partials in chunk order
  const float *part = SHp + (int64_t)bm.ch0 * 2 * B * B;
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    float s = 0.f, h = 0.f;
    // unrolled so the loads run ahead; the adds stay in chunk order
#pragma unroll 8
    for (int t = 0; t < bm.nch; ++t) {
      s += part[(int64_t)t * 2 * B * B + i * B + j];
      h += part[(int64_t)t * 2 * B * B + B * B + i * B + j];
    }
    sm.S[i][j] = s;
    sm.H[i][j] = h;
  }
  __syncthreads();
  // 2. unit diagonal
  for (int i = tid; i < n; i += blockDim.x) {
    const float sii = sm.S[i][i];
    sm.d[i] = sii > 0.f ? sqrtf(sii) : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    const float di = sm.d[i], dj = sm.d[j];
    sm.S[i][j] = (di > 0.f && dj > 0.f) ? sm.S[i][j] / (di * dj) : (i == j ? 0.f : 0.f);
    sm.Li[i][j] = i == j ? 1.f : 0.f;
  }
  __syncthreads();
  // 3. Cholesky S_n = L L^T, right-looking: for each column j, the pivot
  // S[j][j] already holds S_jj - sum_{l<j} L_jl^2 (subtracted one l at a
  // time, in order), the column below it is scaled, then every thread
  // updates its entries of the trailing triangle, S[i][l] -= L_ij L_lj.
  // This is the same sequence of fused multiply-adds per entry as a
  // left-looking loop over l, but with O(1) work per thread per column.
  // Weak pivots are dropped: the column is treated as zero below its unit
  // diagonal, so it also changes nothing in the trailing update.
  // 4. L^-1 in the same sweep: Li starts as I; at step j row j is divided by
  // L_jj (it has received all its updates) and then the rows below get
  // Li[i][c] -= L_ij Li[j][c] for c <= j. Per entry these are the fused
  // multiply-adds of forward substitution in the same order (l ascending,
  // then the division), so the result is bitwise the same, but every step
  // is parallel over the entries instead of one dependent chain per column.
  for (int j = 0; j < n; ++j) {
    const float piv = sm.S[j][j];
    const bool drop = !(piv > kPivotDrop);
    const float ljj = drop ? 1.f : __fsqrt_rn(piv);
    const float inv = __frcp_rn(ljj);
    for (int i = j + 1 + tid; i < n; i += blockDim.x)
      sm.S[i][j] = drop ? 0.f : sm.S[i][j] * inv;
    for (int c = tid; c <= j; c += blockDim.x) sm.Li[j][c] = sm.Li[j][c] / ljj;
    if (tid == 0) {
      sm.drop[j] = drop;
      sm.key[j] = ljj;          // L's diagonal; S[j][j] stays readable
    }
    __syncthreads();
    // trailing triangle j < l <= i < n: a warp per row, lanes over l
    for (int i = j + 1 + wid; i < n; i += nw) {
      const float sij = sm.S[i][j];
      for (int l = j + 1 + lane; l <= i; l += 32)
        sm.S[i][l] = fmaf(-sij, sm.S[l][j], sm.S[i][l]);
      // the row of L^-1, columns 0 .. j
      for (int c = lane; c <= j; c += 32)
        sm.Li[i][c] = fmaf(-sij, sm.Li[j][c], sm.Li[i][c]);
    }
    __syncthreads();
  }
  // 5. T1 = D^-1 L^-T, dropped basis columns are zero
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    float v = 0.f;
    if (!sm.drop[j] && sm.d[i] > 0.f) v = sm.Li[j][i] / sm.d[i];
    sm.T1[i][j] = v;
  }
  __syncthreads();
  // 6. H' = T1^T H T1 (Li reused as scratch for H T1); A holds H' by
  // columns (A[j][i] = H'_ij, symmetrised), V = I
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    float acc = 0.f;
    for (int l = 0; l < n; ++l) acc = fmaf(sm.H[i][l], sm.T1[l][j], acc);
    sm.Li[i][j] = acc;
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    float acc = 0.f;
    for (int l = 0; l < n; ++l) acc = fmaf(sm.T1[l][i], sm.Li[l][j], acc);
    sm.V[i][j] = acc;
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    sm.A[j][i] = 0.5f * (sm.V[i][j] + sm.V[j][i]);
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x)
    sm.V[e / n][e % n] = (e / n == e % n) ? 1.f : 0.f;
  __syncthreads();
  // 7. eigen-decomposition of H' (V by columns: V[j] is eigenvector j)
  const long long c1 = clock64();
  // The first step works on a random start: unless the block is no wider
  // than the subspace (then this one step is exact), it cannot converge,
  // and what the next filter needs is the Ritz values (accurate to second
  // order in the off-diagonal) and the subspace, not an accurate basis of
  // it. So its columns only need to be orthogonal to 1e-3; every later
  // step goes to kJacobiTol. Convergence is still decided by the residual
  // test.
  const float tol =
      (state[blk].iters == 0 && n < bm.s) ? kJacobiTolFirst : kJacobiTol;
  const int sweeps = onesided_jacobi<B>(sm.A, sm.V, n, max_sweeps, sm.pairs,
                                        &sm.flag, tol);
  const long long c2 = clock64();
  // 8. eigenvalues = column norms; descending order, dropped directions last
  for (int j = tid; j < n; j += blockDim.x) {
    float nn = 0.f;
    for (int r = 0; r < n; ++r) nn = fmaf(sm.A[j][r], sm.A[j][r], nn);
    sm.d[j] = sqrtf(nn);                  // d is free after step 5
    sm.key[j] = sm.drop[j] ? -INFINITY : sm.d[j];
  }
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) {
    const float ki = sm.key[i];
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const float kj = sm.key[j];
      r += (kj > ki) || (kj == ki && j < i);
    }
    sm.rank[i] = r;
  }
  __syncthreads();
  float *Tb = Tout + (int64_t)blk * B * B;
  for (int e = tid; e < B * B; e += blockDim.x) {
    const int i = e / B, j = e % B;
    if (i < n && j < n) {
      float acc = 0.f;
      for (int l = 0; l < n; ++l) acc = fmaf(sm.T1[i][l], sm.V[j][l], acc);
      Tb[i * B + sm.rank[j]] = acc;
    } else {
      Tb[i * B + j] = 0.f;
    }
  }
  for (int i = tid; i < B; i += blockDim.x) {
    if (i < n) theta[(int64_t)blk * B + sm.rank[i]] = sm.drop[i] ? 0.f : sm.d[i];
    else theta[(int64_t)blk * B + i] = 0.f;
  }
  if (tid == 0) {
    unsigned long long mask = 0ull;
    for (int i = 0; i < n; ++i)
      if (sm.drop[i]) mask |= 1ull << sm.rank[i];
    state[blk].refill = mask;
    state[blk].sweeps += sweeps;
    state[blk].cycles[0] += c1 - c0;
    state[blk].cycles[1] += c2 - c1;
    state[blk].cycles[2] += clock64() - c2;
  }
}

// X <- X T and Z <- Z T on one 64-row tile, in place; refilled columns get
// fresh random values (and Z = 0 until the next product). Writes the tile's
// partial |Z_j - theta_j X_j|^2 and |X_j|^2 for every column j: each
// thread's four rows in float32 (one rounding for the residual entry, one
// per square and add), then float64 over the threads in a fixed order.
// The 256 threads form a 16 x 16 grid over the tile's 64 rows x b columns,
// each thread 4 rows x TJ = b / 16 columns in registers. X and Z are staged
// transposed (column l of the tile is row l of XT, ZT), so for each l one
// 16-byte load of XT, of ZT and of T's row l feed 8 TJ fused multiply-adds;
// every output is still the sum over l in ascending order.
template <int B>
__global__ void __launch_bounds__(256)
k_rotate(const BlockMeta *__restrict__ meta,
         const SolverState *__restrict__ state,
         const int2 *__restrict__ rowtiles, const float *__restrict__ T,
         const float *__restrict__ theta, float *X, float *Z,
         double *__restrict__ RP, uint64_t seed, int32_t *running,
         float *__restrict__ XB) {
  constexpr int TJ = B / 16;
  constexpr int LD = TR + 4;                 // XT, ZT rows: 16-byte multiples
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float (*Ts)[B] = reinterpret_cast<float (*)[B]>(smem_raw);
  float (*XT)[LD] = reinterpret_cast<float (*)[LD]>(smem_raw +
                                                     sizeof(float) * B * B);
  float (*ZT)[LD] = XT + B;
  // the new X rows for the B form, over XT and ZT once they are read
  float (*Os)[B + 1] = reinterpret_cast<float (*)[B + 1]>(&XT[0][0]);
  __shared__ double r2s[16][B], x2s[16][B];
  pdl_wait();
  pdl_trigger();
  // k_check, next in the stream, counts the blocks still running here
  if (blockIdx.x == 0 && threadIdx.x < 2) running[threadIdx.x] = 0;
  const int2 t = rowtiles[blockIdx.x];
  const SolverState st = state[t.x];
  if (st.status != kRunning) return;
  const BlockMeta bm = meta[t.x];
  const int rows = min(TR, bm.s - t.y);
  const float *Tb = T + (int64_t)t.x * B * B;
  const float *th = theta + (int64_t)t.x * B;
  float *Xb = X + bm.x_off + (int64_t)t.y * B;
  float *Zb = Z + bm.x_off + (int64_t)t.y * B;
  for (int e4 = threadIdx.x; e4 < B * B / 4; e4 += blockDim.x)
    reinterpret_cast<float4 *>(&Ts[0][0])[e4] =
        reinterpret_cast<const float4 *>(Tb)[e4];
  for (int e = threadIdx.x; e < TR * B; e += blockDim.x) {
    const int r = e / B, l = e % B;
    const bool ok = r < rows;
    XT[l][r] = ok ? Xb[e] : 0.f;
    ZT[l][r] = ok ? Zb[e] : 0.f;
  }
  __syncthreads();
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
  float ax[4][TJ], az[4][TJ];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < TJ; ++b) ax[a][b] = az[a][b] = 0.f;
#pragma unroll 4
  for (int l = 0; l < B; ++l) {
    float xv[4], zv[4], tv[TJ];
    ld_vec(&XT[l][4 * tr], xv);
    ld_vec(&ZT[l][4 * tr], zv);
    ld_vec(&Ts[l][TJ * tc], tv);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < TJ; ++b) {
        ax[a][b] = fmaf(xv[a], tv[b], ax[a][b]);
        az[a][b] = fmaf(zv[a], tv[b], az[a][b]);
      }
  }
  __syncthreads();                           // XT, ZT read: Os may reuse them
#pragma unroll
  for (int b = 0; b < TJ; ++b) {
    const int j = TJ * tc + b;
    const bool refill = (st.refill >> j) & 1ull;
    const float tj = th[j];
    float pr2 = 0.f, px2 = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = 4 * tr + a;
      if (refill) {
        ax[a][b] = hash_uniform(
            seed ^ (0x51ED270Bull * (uint64_t)(st.iters + 1)), (uint64_t)t.x,
            (uint64_t)(t.y + r) * B + j);
        az[a][b] = 0.f;
      }
      if (r < rows) {
        const float d = fmaf(-tj, ax[a][b], az[a][b]);
        pr2 = fmaf(d, d, pr2);
        px2 = fmaf(ax[a][b], ax[a][b], px2);
        Os[r][j] = ax[a][b];
      }
    }
    r2s[tr][j] = (double)pr2;
    x2s[tr][j] = (double)px2;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = 4 * tr + a;
    if (r < rows) {
      st_vec(Xb + (int64_t)r * B + TJ * tc, ax[a]);
      st_vec(Zb + (int64_t)r * B + TJ * tc, az[a]);
    }
  }
  __syncthreads();
  if (XB) {
    // the B form of X for the tensor-core products that follow: for each
    // column, consecutive threads take consecutive rows of a 32-row chunk,
    // so a warp stores 128 contiguous bytes (rows past s keep the zeros an
    // earlier conversion wrote)
    for (int e = threadIdx.x; e < TR * B; e += blockDim.x) {
      const int c = e / TR, rr = e % TR;
      if (rr >= rows) continue;
      const int gr = t.y + rr;
      float *bf = XB + 2 * bm.x_off + (int64_t)(gr >> 5) * 2 * B * 32 + (gr & 31);
      const float v = Os[rr][c];
      const float h = tf32_hi(v);
      bf[c * 32] = h;
      bf[(B + c) * 32] = __fsub_rn(v, h);
    }
  }
  if (threadIdx.x < B) {
    double a = 0.0, b = 0.0;
    for (int g = 0; g < 16; ++g) { a += r2s[g][threadIdx.x]; b += x2s[g][threadIdx.x]; }
    double *rp = RP + (int64_t)blockIdx.x * 2 * B;
    rp[threadIdx.x] = a;
    rp[B + threadIdx.x] = b;
  }
}

// Residuals, convergence, next filter. When a block is done, its columns'
// float32 reciprocal norms go to Finv (k_publish_fs normalises X into F_s
// after the loop, spread over row tiles).
template <int B>
__global__ void __launch_bounds__(256)
k_check(const BlockMeta *__restrict__ meta, SolverState *__restrict__ state,
        const double *__restrict__ RP, const float *__restrict__ theta,
        float *__restrict__ Finv, int max_iters, int max_degree, float tol,
        int32_t *running) {
  __shared__ double r2[B], x2[B];
  __shared__ int s_done;
  const int blk = blockIdx.x;
  pdl_wait();
  pdl_trigger();
  SolverState st = state[blk];
  if (st.status != kRunning) return;
  const BlockMeta bm = meta[blk];
  const int n = st.bsub, s = bm.s, keff = bm.keff;
  const float *th = theta + (int64_t)blk * B;
  if (threadIdx.x < B) {
    double a = 0.0, b = 0.0;
#pragma unroll 8
    for (int t = 0; t < bm.nt; ++t) {
      const double *rp = RP + (int64_t)(bm.t0 + t) * 2 * B;
      a += rp[threadIdx.x];
      b += rp[B + threadIdx.x];
    }
    r2[threadIdx.x] = a;
    x2[threadIdx.x] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // The convergence test, in float64: |G x_j - theta_j x_j| / |x_j| <=
    // tol theta_1 for the wanted pairs. For orthonormal Ritz vectors it
    // also bounds the off-diagonal entries |x_i^T G x_j| = |x_i^T r_j| of
    // the Rayleigh quotient matrix by the same amount.
    const float t1 = th[0];
    double worst = 0.0;
    for (int j = 0; j < keff && j < n; ++j)
      worst = fmax(worst, x2[j] > 0.0 ? sqrt(r2[j] / x2[j]) : sqrt(r2[j]));
    const unsigned long long wanted =
        keff >= 64 ? ~0ull : ((1ull << keff) - 1ull);
    st.iters += 1;
    st.theta1 = t1;
    st.resid = t1 > 0.f ? (float)(worst / (double)t1) : 0.f;
    const bool refilled_wanted = (st.refill & wanted) != 0ull;
    const bool conv = !refilled_wanted &&
                      ((s <= B) || !(t1 > 1e-30f) ||
                       (worst <= (double)tol * (double)t1));
    if (conv || st.iters >= max_iters) {
      st.status = conv ? kConverged : kCapped;
      s_done = 1;
    } else {
      const int ndrop = __popcll(st.refill);
      float amp = st.amp > 0.f ? st.amp : kMaxAmplification;
      float cut = th[max(0, n - 1 - ndrop)];
      if (ndrop > 0) {
        amp = fmaxf(amp / kAmpBackoff, kMinAmplification);
        if (st.cut > 0.f) cut = fminf(cut, st.cut);
      }
      st.amp = amp;
      cut = fmaxf(cut, kCutFloor * t1);
      if (cut >= kCutCeil * t1) cut = kCutCeil * t1;
      st.cut = cut;
      st.a0 = t1;
      const float tt = 2.f * t1 / cut - 1.f;   // >= 1.105
      const float at = acoshf(tt);
      int d = 2;
      while (d + 2 <= max_degree && coshf((float)(d + 2) * at) <= amp)
        d += 2;
      st.degree = d;
      atomicAdd(running, 1);
      atomicMax(running + 1, d);
      s_done = 0;
    }
    state[blk] = st;
  }
  __syncthreads();
  if (!s_done) return;
  // unit columns: one float64 reciprocal norm per column
  if (threadIdx.x < B) {
    const double nn = x2[threadIdx.x];
    Finv[(int64_t)blk * B + threadIdx.x] =
        nn > 0.0 ? (float)(1.0 / sqrt(nn)) : 0.f;
  }
}

// F_s = the first keff columns of X, each scaled by its reciprocal norm
// (zero elsewhere), for one 128-row tile of a finished block. Thread t takes
// column t mod kp of the rows t / kp, t / kp + G, ... (G = blockDim / kp),
// so a CTA writes consecutive floats of F_s. A block that never reached a
// Rayleigh-Ritz step (keff = 0) gets zeros.
template <int B>
__global__ void __launch_bounds__(256)
k_publish_fs(const BlockMeta *__restrict__ meta,
             const SolverState *__restrict__ state,
             const int2 *__restrict__ tiles, const float *__restrict__ X,
             const float *__restrict__ Finv, float *__restrict__ Fs, int kp) {
  pdl_wait();
  pdl_trigger();
  const int2 t = tiles[blockIdx.x];
  const BlockMeta bm = meta[t.x];
  const SolverState st = state[t.x];
  const int G = (int)blockDim.x / kp;
  const int j = (int)threadIdx.x % kp, g = (int)threadIdx.x / kp;
  if (g >= G) return;
  const int rows = min(128, bm.s - t.y);
  const bool live = st.iters > 0 && st.status != kRunning && j < bm.keff &&
                    j < st.bsub;
  const float inv = live ? Finv[(int64_t)t.x * B + j] : 0.f;
  const float *Xb = X + bm.x_off + (int64_t)t.y * B;
  float *Fb = Fs + bm.fs_off + (int64_t)t.y * kp;
  for (int r = g; r < rows; r += G)
    Fb[(int64_t)r * kp + j] = live ? Xb[(int64_t)r * B + j] * inv : 0.f;
}

// Asynchronous 4-byte global -> shared copy (no register staging); with
// `valid` false the destination is zero-filled and nothing is read.
__device__ __forceinline__ void cp_async4(float *dst, const float *src,
                                          bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d),
               "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// F_L[l, :] = sum_a W[a, l] F_s[a, :] for kProjCols = 64 consecutive l: lane
// t owns l = l0 + 2t, l0 + 2t + 1 (one float2 of each W row), warp w takes
// the rows a = w, w + 8, ... and a row of F_s is read from shared memory as
// float4s, so each shared load feeds 8 FMAs. The 8 warps' partial sums are
// added in warp order. The next 64-row chunk is in flight while the current
// one's products run: the warp's W rows in registers, F_s as asynchronous
// copies into the other half of a double-buffered shared array. KM: kp
// rounded up to 8.
template <int KM>
__global__ void __launch_bounds__(256)
k_project(const BlockMeta *__restrict__ meta, const int2 *__restrict__ ltiles,
          const float *__restrict__ W, const float *__restrict__ Fs,
          float *__restrict__ FL, int kp) {
  constexpr int CH = 64;
  __shared__ __align__(16) float Fsh[2][CH][KM];
  __shared__ float red[8][64][9];
  pdl_wait();
  const int2 t = ltiles[blockIdx.x];
  const BlockMeta bm = meta[t.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = t.y + 2 * lane;
  const bool lv = l < bm.L_pad;          // padded columns of W are zero
  const float *Wb = W + bm.w_off;
  const float *Fb = Fs + bm.fs_off;
  float acc[2][KM];
#pragma unroll
  for (int j = 0; j < KM; ++j) { acc[0][j] = 0.f; acc[1][j] = 0.f; }
  // W rows of the chunk at a0 that this warp handles: warp + 8 h
  auto load_w = [&](int a0, float2 (&w)[CH / 8]) {
    const int lim = min(CH, bm.s - a0);
#pragma unroll
    for (int h = 0; h < CH / 8; ++h) {
      const int rr = warp + 8 * h;
      w[h] = (lv && rr < lim) ? *reinterpret_cast<const float2 *>(
                                    Wb + (int64_t)(a0 + rr) * bm.L_pad + l)
                              : make_float2(0.f, 0.f);
    }
  };
  // F_s rows a0 .. a0+63 into Fsh[buf] (zeros past s and past kp)
  auto load_f = [&](int a0, int buf) {
    for (int e = threadIdx.x; e < CH * KM; e += blockDim.x) {
      const int rr = e / KM, j = e % KM;
      const bool ok = a0 + rr < bm.s && j < kp;
      cp_async4(&Fsh[buf][rr][j], ok ? Fb + (int64_t)(a0 + rr) * kp + j : Fb,
                ok);
    }
    cp_async_commit();
  };
  float2 w[CH / 8], wn[CH / 8];
  load_w(0, w);
  load_f(0, 0);
  int buf = 0;
  for (int a0 = 0; a0 < bm.s; a0 += CH, buf ^= 1) {
    const bool more = a0 + CH < bm.s;
    if (more) {
      load_f(a0 + CH, buf ^ 1);
      cp_async_wait<1>();      // this chunk's copies have landed
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    if (more) load_w(a0 + CH, wn);
    const int lim = min(CH, bm.s - a0);
    if (lv) {
#pragma unroll
      for (int h = 0; h < CH / 8; ++h) {
        const int rr = warp + 8 * h;
        if (rr >= lim) break;
#pragma unroll
        for (int j = 0; j < KM; j += 4) {
          const float4 f = *reinterpret_cast<const float4 *>(&Fsh[buf][rr][j]);
          acc[0][j] = fmaf(w[h].x, f.x, acc[0][j]);
          acc[0][j + 1] = fmaf(w[h].x, f.y, acc[0][j + 1]);
          acc[0][j + 2] = fmaf(w[h].x, f.z, acc[0][j + 2]);
          acc[0][j + 3] = fmaf(w[h].x, f.w, acc[0][j + 3]);
          acc[1][j] = fmaf(w[h].y, f.x, acc[1][j]);
          acc[1][j + 1] = fmaf(w[h].y, f.y, acc[1][j + 1]);
          acc[1][j + 2] = fmaf(w[h].y, f.z, acc[1][j + 2]);
          acc[1][j + 3] = fmaf(w[h].y, f.w, acc[1][j + 3]);
        }
      }
    }
#pragma unroll
    for (int h = 0; h < CH / 8; ++h) w[h] = wn[h];
    // every warp is done with Fsh[buf] before the next chunk refills it
    __syncthreads();
  }
#pragma unroll
  for (int jc = 0; jc < KM; jc += 8) {
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      red[warp][2 * lane][jj] = acc[0][jc + jj];
      red[warp][2 * lane + 1][jj] = acc[1][jc + jj];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * 8; e += blockDim.x) {
      const int ln = e >> 3, jj = e & 7, j = jc + jj;
      const int ll = t.y + ln;
      if (ll < bm.L && j < kp) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += red[w][ln][jj];
        FL[bm.fl_off + (int64_t)ll * kp + j] = s;
      }
    }
    __syncthreads();
  }
}

template <int B>
size_t rr_smem() { return sizeof(RRSmem<B>); }

template <int B>
size_t rot_smem() { return sizeof(float) * (B * B + 2 * B * (TR + 4)); }
static_assert(TR * (16 + 1) <= 2 * 16 * (TR + 4), "Os fits over XT and ZT");

template <int B>
cudaError_t set_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_rr_solve<B>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)rr_smem<B>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_rotate<B>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)rot_smem<B>());
}

template <typename F>
cudaError_t by_width(int b, F &&f) {
  switch (b) {
    case 16: return f(std::integral_constant<int, 16>());
    case 32: return f(std::integral_constant<int, 32>());
    case 64: return f(std::integral_constant<int, 64>());
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_init_panels(const EigBuffers &e, const int2 *rowtiles,
                               int32_t ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  return by_width(e.bsub, [&](auto w) {
    constexpr int B = decltype(w)::value;
    return launch_pdl(k_init_panels<B>, dim3(ntiles), dim3(256), 0, st, e.meta,
                      e.state, rowtiles, e.X, e.seed);
  });
}

cudaError_t launch_gpanel(const EigBuffers &e, const int2 *rowtiles,
                          int32_t ntiles, int32_t mode, int32_t step,
                          int32_t degree, const float *in, const float *in2,
                          float *out, cudaStream_t st) {
  (void)degree;
  if (ntiles <= 0) return cudaSuccess;
  return by_width(e.bsub, [&](auto w) {
    constexpr int B = decltype(w)::value;
    cudaError_t err = cudaFuncSetAttribute(
        k_gpanel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)panel_smem<B>());
    if (err != cudaSuccess) return err;
    k_gpanel<B><<<ntiles, 512, panel_smem<B>(), st>>>(e.meta, e.state, rowtiles,
                                                      e.G, in, in2, out, mode,
                                                      step);
    return cudaGetLastError();
  });
}

cudaError_t launch_small_gram(const EigBuffers &e, const int2 *chunks,
                              int32_t nchunks, cudaStream_t st) {
  if (nchunks <= 0) return cudaSuccess;
  return by_width(e.bsub, [&](auto w) {
    constexpr int B = decltype(w)::value;
    return launch_pdl(k_small_gram<B>, dim3(nchunks), dim3(256), 0, st, e.meta,
                      e.state, chunks, (const float *)e.X,
                      (const float *)e.Z, e.SH);
  });
}

cudaError_t launch_rr_solve(const EigBuffers &e, cudaStream_t st) {
  return by_width(e.bsub, [&](auto w) {
    constexpr int B = decltype(w)::value;
    cudaError_t err = set_attrs<B>();
    if (err != cudaSuccess) return err;
    const int threads = B < 32 ? 256 : (e.nblocks > e.nsm ? 512 : 1024);
    return launch_pdl(k_rr_solve<B>, dim3(e.nblocks), dim3(threads),
                      rr_smem<B>(), st, e.meta, e.state, (const float *)e.SH,
                      e.T, e.theta, e.max_sweeps);
  });
}

cudaError_t launch_rotate(const EigBuffers &e, const int2 *rowtiles,
                          int32_t ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  return by_width(e.bsub, [&](auto w) {
    constexpr int B = decltype(w)::value;
    cudaError_t err = set_attrs<B>();
    if (err != cudaSuccess) return err;
    return launch_pdl(k_rotate<B>, dim3(ntiles), dim3(256), rot_smem<B>(), st,
                      e.meta, (const SolverState *)e.state, rowtiles,
                      (const float *)e.T, (const float *)e.theta, e.X, e.Z,
                      e.RP, e.seed, e.running, e.XB);
  });
}

cudaError_t launch_check(const EigBuffers &e, cudaStream_t st) {
  return by_width(e.bsub, [&](auto w) {
    constexpr int B = decltype(w)::value;
    return launch_pdl(k_check<B>, dim3(e.nblocks), dim3(256), 0, st, e.meta,
                      e.state, (const double *)e.RP, (const float *)e.theta,
                      e.Finv, e.max_iters, e.max_degree, e.tol, e.running);
  });
}

cudaError_t launch_publish_fs(const EigBuffers &e, const int2 *tiles,
                              int32_t ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (e.kp <= 0 || e.kp > 256) return cudaErrorInvalidValue;
  const int threads = (256 / e.kp) * e.kp;
  return by_width(e.bsub, [&](auto w) {
    constexpr int B = decltype(w)::value;
    return launch_pdl(k_publish_fs<B>, dim3(ntiles), dim3(threads), 0, st,
                      e.meta, (const SolverState *)e.state, tiles,
                      (const float *)e.X, (const float *)e.Finv, e.Fs,
                      (int)e.kp);
  });
}

// One thread: the step's running counters to the host, then the sequence
// number (after a system-scope fence, so the host never sees the new
// sequence number with old counters).
__global__ void k_publish(const int32_t *__restrict__ running,
                          volatile int32_t *host, int32_t seq) {
  pdl_wait();
  host[0] = running[0];
  host[1] = running[1];
  __threadfence_system();
  host[2] = seq;
}

__global__ void k_loopctl(const int32_t *__restrict__ running,
                          int32_t *count, int32_t max,
                          cudaGraphConditionalHandle handle, LoopHandles steps) {
  pdl_wait();
  if (threadIdx.x == 0) {
    const int32_t it = ++count[0];
    const bool any = running[0] > 0;
    cudaGraphSetConditional(handle, (any && it < max) ? 1u : 0u);
    int32_t opened = 0;
    for (int j = 0; j < steps.n; ++j) {
      const bool go = any && running[1] >= steps.first + j;
      cudaGraphSetConditional(steps.h[j], go ? 1u : 0u);
      opened += go;
    }
    count[1] += opened;
  }
}

cudaError_t launch_loopctl(const int32_t *running, int32_t *count,
                           int32_t max, cudaGraphConditionalHandle handle,
                           const LoopHandles &steps, cudaStream_t st) {
  k_loopctl<<<1, 32, 0, st>>>(running, count, max, handle, steps);
  return cudaGetLastError();
}

cudaError_t launch_publish(const int32_t *running, int32_t *host, int32_t seq,
                           cudaStream_t st) {
  return launch_pdl(k_publish, dim3(1), dim3(1), 0, st, running,
                    (volatile int32_t *)host, seq);
}

template <typename F>
cudaError_t by_kmax(int kp, F &&f) {
  switch ((kp + 7) / 8) {
    case 1: return f(std::integral_constant<int, 8>());
    case 2: return f(std::integral_constant<int, 16>());
    case 3: return f(std::integral_constant<int, 24>());
    case 4: return f(std::integral_constant<int, 32>());
    case 5: return f(std::integral_constant<int, 40>());
    case 6: return f(std::integral_constant<int, 48>());
    case 7: return f(std::integral_constant<int, 56>());
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_project(const BlockMeta *meta, const int2 *ltiles,
                           int32_t ntiles, const float *W, const float *Fs,
                           float *FL, int32_t kp, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  return by_kmax(kp, [&](auto km) {
    constexpr int KM = decltype(km)::value;
    return launch_pdl(k_project<KM>, dim3(ntiles), dim3(256), 0, st, meta,
                      ltiles, W, Fs, FL, kp);
  });
}


}  // namespace bsvd
