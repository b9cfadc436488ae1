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
//   2. Rayleigh-Ritz with SVQB orthonormalisation (Stathopoulos and Wu,
//      2002):
//        S = X^T X, S_n = D^-1 S D^-1 = Q L Q^T,
//        T1 = D^-1 Q L^-1/2,
//        H' = T1^T (X^T G X) T1 = Y Theta Y^T,
//        X <- X T1 Y.
//      Both small symmetric eigenproblems are solved by cyclic Jacobi with
//      parallel (round-robin) ordering in shared memory.
//   3. Stop a block when |G x_i - theta_i x_i| <= tol * theta_1 for its k
//      wanted pairs; otherwise cut <- smallest Ritz value and go to 1.
//
// The filter amplifies the top of the spectrum by C_d(t_1), with
// t_1 = 2 theta_1 / cut - 1, relative to the damped interval. In float32
// the columns that should hold the lower Ritz directions drown in rounding
// noise once that ratio nears 1/eps, so each block picks the largest even
// degree d <= max_degree with C_d(t_1) <= kMaxAmplification (at least 2).
// Steep spectra get short filters and more Rayleigh-Ritz steps.
//
// A block with s <= bsub starts from the identity basis, so the first
// Rayleigh-Ritz step is an exact eigen-decomposition of G.
#include <float.h>

#include <type_traits>

#include "kernels.h"

namespace bsvd {

namespace {

constexpr int TR = 64;       // panel rows per CTA
constexpr float kMaxAmplification = 3e6f;
constexpr float kCutFloor = 1e-3f;   // cut >= kCutFloor * theta_1
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
template <int B>
__global__ void __launch_bounds__(256)
k_gpanel(const BlockMeta *__restrict__ meta,
         const SolverState *__restrict__ state,
         const int2 *__restrict__ rowtiles, const float *__restrict__ G,
         const float *in, const float *in2, float *out, int mode, int step) {
  constexpr int CN = B / 16;               // output columns per thread
  __shared__ __align__(16) float As[KC][TR + 4];
  __shared__ __align__(16) float Bs[KC][B + 4];
  const int2 t = rowtiles[blockIdx.x];
  const SolverState st = state[t.x];
  if (st.status != kRunning) return;
  if (mode >= 1 && step > st.degree) return;   // this block's filter is done
  const BlockMeta bm = meta[t.x];
  const int sp = bm.s_pad;
  const int row0 = t.y;
  const float *Gb = G + bm.g_off;
  const float *inb = in + bm.x_off;
  float *outb = out + bm.x_off;

  float alpha = 1.f, beta = 0.f, gamma = 0.f;
  if (mode >= 1) {
    // damped interval [0, cut]: centre c, half-width e; p(a0) = 1
    const float e = 0.5f * st.cut, c = 0.5f * st.cut;
    const float sig1 = e / (st.a0 - c);
    if (mode == 1) {
      alpha = sig1 / e;
      beta = -c * alpha;
    } else {
      const float tau = 2.f / sig1;
      float sig = sig1, sig_prev = sig1;
      for (int j = 2; j <= step; ++j) {
        sig_prev = sig;
        sig = 1.f / (tau - sig);
      }
      alpha = 2.f * sig / e;
      beta = -c * alpha;
      gamma = -sig_prev * sig;
    }
  }

  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  float acc[4][CN];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < CN; ++c) acc[r][c] = 0.f;

  for (int k0 = 0; k0 < sp; k0 += KC) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int idx = tid + 256 * h;
      const int rr = idx >> 4, cc = (idx & 15) * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k0 + rr < sp && row0 + cc < sp)
        v = __ldg(reinterpret_cast<const float4 *>(
            Gb + (int64_t)(k0 + rr) * sp + row0 + cc));
      *reinterpret_cast<float4 *>(&As[rr][cc]) = v;
    }
    for (int idx = tid; idx < KC * B / 4; idx += 256) {
      const int rr = idx / (B / 4), cc = (idx % (B / 4)) * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k0 + rr < sp)
        v = *reinterpret_cast<const float4 *>(inb + (int64_t)(k0 + rr) * B + cc);
      *reinterpret_cast<float4 *>(&Bs[rr][cc]) = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < KC; ++kk) {
      float a[4], b[CN];
      *reinterpret_cast<float4 *>(a) =
          *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
#pragma unroll
      for (int c = 0; c < CN; ++c) b[c] = Bs[kk][tx * CN + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < CN; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
  const float *in2b = in2 ? in2 + bm.x_off : nullptr;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int row = row0 + ty * 4 + r;
    if (row >= sp) continue;
#pragma unroll
    for (int c = 0; c < CN; ++c) {
      const int col = tx * CN + c;
      const int64_t o = (int64_t)row * B + col;
      float v = alpha * acc[r][c];
      if (beta != 0.f) v = fmaf(beta, inb[o], v);
      if (gamma != 0.f) v = fmaf(gamma, in2b[o], v);
      outb[o] = v;
    }
  }
}

// S = X^T X and H = X^T Z over the block's s rows (float32 sums).
template <int B>
__global__ void __launch_bounds__(256)
k_small_gram(const BlockMeta *__restrict__ meta,
             const SolverState *__restrict__ state,
             const float *__restrict__ X, const float *__restrict__ Z,
             float *__restrict__ SH) {
  constexpr int CH = 32;
  constexpr int PER = (B * B + 255) / 256;
  __shared__ float Xs[CH][B + 1];
  __shared__ float Zs[CH][B + 1];
  const int blk = blockIdx.x;
  if (state[blk].status != kRunning) return;
  const BlockMeta bm = meta[blk];
  const float *Xb = X + bm.x_off;
  const float *Zb = Z + bm.x_off;
  float s_acc[PER], h_acc[PER];
#pragma unroll
  for (int e = 0; e < PER; ++e) { s_acc[e] = 0.f; h_acc[e] = 0.f; }
  for (int r0 = 0; r0 < bm.s; r0 += CH) {
    for (int e = threadIdx.x; e < CH * B; e += 256) {
      const int rr = e / B, c = e % B;
      const bool ok = r0 + rr < bm.s;
      Xs[rr][c] = ok ? Xb[(int64_t)(r0 + rr) * B + c] : 0.f;
      Zs[rr][c] = ok ? Zb[(int64_t)(r0 + rr) * B + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const int idx = threadIdx.x + 256 * e;
      if (idx < B * B) {
        const int i = idx / B, j = idx % B;
        float sa = s_acc[e], ha = h_acc[e];
#pragma unroll 8
        for (int rr = 0; rr < CH; ++rr) {
          const float xi = Xs[rr][i];
          sa = fmaf(xi, Xs[rr][j], sa);
          ha = fmaf(xi, Zs[rr][j], ha);
        }
        s_acc[e] = sa;
        h_acc[e] = ha;
      }
    }
    __syncthreads();
  }
  float *S = SH + (int64_t)blk * 2 * B * B;
  float *H = S + B * B;
#pragma unroll
  for (int e = 0; e < PER; ++e) {
    const int idx = threadIdx.x + 256 * e;
    if (idx < B * B) { S[idx] = s_acc[e]; H[idx] = h_acc[e]; }
  }
}

// Cyclic Jacobi for a symmetric n x n matrix A (n <= B) in shared memory.
// On return A is diagonal (to the tolerance) and A_in = V diag(A) V^T.
// Round-robin ordering: n_even - 1 rounds per sweep, n_even / 2 disjoint
// pairs per round, so all rotations of a round commute.
template <int B>
__device__ void jacobi_eig(float (*A)[B + 1], float (*V)[B + 1], int n,
                           int max_sweeps, float *rc, float *rs, int *rp,
                           int *rq, int *flag) {
  const int tid = threadIdx.x;
  const int ne = n + (n & 1);
  const int np = ne / 2;
  for (int e = tid; e < n * n; e += blockDim.x)
    V[e / n][e % n] = (e / n == e % n) ? 1.f : 0.f;
  // absolute floor: rotations below it cannot change float32 results
  float dmax = 0.f;
  for (int i = 0; i < n; ++i) dmax = fmaxf(dmax, fabsf(A[i][i]));
  __syncthreads();
  const float floor_abs = dmax * 1e-9f;
  const float tol = 3e-7f;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int round = 0; round < ne - 1; ++round) {
      if (tid < np) {
        const int pa = tid, pb = ne - 1 - tid;
        const int p = pa == 0 ? 0 : 1 + (pa - 1 + round) % (ne - 1);
        const int q = 1 + (pb - 1 + round) % (ne - 1);
        float c = 1.f, s = 0.f;
        if (p < n && q < n) {
          const float app = A[p][p], aqq = A[q][q], apq = A[p][q];
          const float thr = fmaxf(tol * sqrtf(fabsf(app) * fabsf(aqq)), floor_abs);
          if (fabsf(apq) > thr) {
            const float theta = (aqq - app) / (2.f * apq);
            const float t = copysignf(1.f, theta) /
                            (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f)));
            c = 1.f / sqrtf(fmaf(t, t, 1.f));
            s = t * c;
            *flag = 1;
          }
        }
        rc[tid] = c; rs[tid] = s; rp[tid] = p; rq[tid] = q;
      }
      __syncthreads();
      // A <- J^T A J on the 2 x 2 sub-blocks (pair i, pair j), i <= j; the
      // (j, i) sub-block is written as the transpose so A stays symmetric.
      for (int e = tid; e < np * np; e += blockDim.x) {
        const int i = e / np, j = e % np;
        if (i > j) continue;
        const float si = rs[i], sj = rs[j];
        if (si == 0.f && sj == 0.f) continue;
        const float ci = rc[i], cj = rc[j];
        const int pi = rp[i], qi = rq[i], pj = rp[j], qj = rq[j];
        const bool vpi = pi < n, vqi = qi < n, vpj = pj < n, vqj = qj < n;
        const float x00 = (vpi && vpj) ? A[pi][pj] : 0.f;
        const float x01 = (vpi && vqj) ? A[pi][qj] : 0.f;
        const float x10 = (vqi && vpj) ? A[qi][pj] : 0.f;
        const float x11 = (vqi && vqj) ? A[qi][qj] : 0.f;
        // rows: J^T from the left
        const float y00 = ci * x00 - si * x10, y01 = ci * x01 - si * x11;
        const float y10 = si * x00 + ci * x10, y11 = si * x01 + ci * x11;
        // columns: J from the right
        float z00 = cj * y00 - sj * y01, z01 = sj * y00 + cj * y01;
        float z10 = cj * y10 - sj * y11, z11 = sj * y10 + cj * y11;
        if (i == j) { z01 = 0.f; z10 = 0.f; }
        if (vpi && vpj) A[pi][pj] = z00;
        if (vpi && vqj) A[pi][qj] = z01;
        if (vqi && vpj) A[qi][pj] = z10;
        if (vqi && vqj) A[qi][qj] = z11;
        if (i != j) {
          if (vpi && vpj) A[pj][pi] = z00;
          if (vpi && vqj) A[qj][pi] = z01;
          if (vqi && vpj) A[pj][qi] = z10;
          if (vqi && vqj) A[qj][qi] = z11;
        }
      }
      for (int e = tid; e < n * np; e += blockDim.x) {
        const int x = e / np, j = e % np;
        const float sj = rs[j];
        if (sj == 0.f) continue;
        const float cj = rc[j];
        const int pj = rp[j], qj = rq[j];
        const float v0 = V[x][pj], v1 = V[x][qj];
        V[x][pj] = cj * v0 - sj * v1;
        V[x][qj] = sj * v0 + cj * v1;
      }
      __syncthreads();
    }
    const int any = *flag;
    __syncthreads();
    if (!any) break;
  }
}

template <int B>
struct RRSmem {
  float A[B][B + 1];
  float V[B][B + 1];
  float T1[B][B + 1];
  float Tm[B][B + 1];
  float d[B];
  float lam[B];
  float rc[B / 2 + 1], rs[B / 2 + 1];
  int rp[B / 2 + 1], rq[B / 2 + 1];
  int rank[B];
  int flag;
};

template <int B>
__global__ void __launch_bounds__(256)
k_rr_solve(const BlockMeta *__restrict__ meta,
           const SolverState *__restrict__ state,
           const float *__restrict__ SH, float *__restrict__ Tout,
           float *__restrict__ theta, int max_sweeps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RRSmem<B> &sm = *reinterpret_cast<RRSmem<B> *>(smem_raw);
  const int blk = blockIdx.x;
  const SolverState st = state[blk];
  if (st.status != kRunning) return;
  const int n = st.bsub;
  const int tid = threadIdx.x;
  const float *S = SH + (int64_t)blk * 2 * B * B;
  const float *H = S + B * B;

  // SVQB: normalise S to unit diagonal, eigen-decompose
  for (int i = tid; i < n; i += blockDim.x) {
    const float sii = S[i * B + i];
    sm.d[i] = sii > 0.f ? sqrtf(sii) : 1.f;
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    sm.A[i][j] = S[i * B + j] / (sm.d[i] * sm.d[j]);
  }
  __syncthreads();
  jacobi_eig<B>(sm.A, sm.V, n, max_sweeps, sm.rc, sm.rs, sm.rp, sm.rq,
                &sm.flag);
  if (tid == 0) {
    float lmax = 0.f;
    for (int i = 0; i < n; ++i) lmax = fmaxf(lmax, sm.A[i][i]);
    const float lfloor = fmaxf(lmax * 1e-6f, FLT_MIN);
    for (int i = 0; i < n; ++i) sm.lam[i] = 1.f / sqrtf(fmaxf(sm.A[i][i], lfloor));
  }
  __syncthreads();
  // T1 = D^-1 Q L^-1/2
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    sm.T1[i][j] = sm.V[i][j] * sm.lam[j] / sm.d[i];
  }
  __syncthreads();
  // Tm = H T1, then A = T1^T Tm (symmetrised)
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    float acc = 0.f;
    for (int l = 0; l < n; ++l) acc = fmaf(H[i * B + l], sm.T1[l][j], acc);
    sm.Tm[i][j] = acc;
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    float acc = 0.f;
    for (int l = 0; l < n; ++l) acc = fmaf(sm.T1[l][i], sm.Tm[l][j], acc);
    sm.V[i][j] = acc;          // V is free until the next Jacobi call
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    sm.A[i][j] = 0.5f * (sm.V[i][j] + sm.V[j][i]);
  }
  __syncthreads();
  jacobi_eig<B>(sm.A, sm.V, n, max_sweeps, sm.rc, sm.rs, sm.rp, sm.rq,
                &sm.flag);
  // descending order, ties by index
  for (int i = tid; i < n; i += blockDim.x) {
    const float ti = sm.A[i][i];
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const float tj = sm.A[j][j];
      r += (tj > ti) || (tj == ti && j < i);
    }
    sm.rank[i] = r;
  }
  __syncthreads();
  float *Tb = Tout + (int64_t)blk * B * B;
  for (int e = tid; e < B * B; e += blockDim.x) {
    const int i = e / B, j = e % B;
    float acc = 0.f;
    if (i < n && j < n) {
      for (int l = 0; l < n; ++l) acc = fmaf(sm.T1[i][l], sm.V[l][j], acc);
      Tb[i * B + sm.rank[j]] = acc;
    } else {
      Tb[i * B + j] = 0.f;
    }
  }
  for (int i = tid; i < B; i += blockDim.x)
    if (i < n) theta[(int64_t)blk * B + sm.rank[i]] = sm.A[i][i];
    else theta[(int64_t)blk * B + i] = 0.f;
}

// X <- X T and Z <- Z T on rows [row0, row0 + 64), in place.
template <int B>
__global__ void __launch_bounds__(256)
k_rotate(const BlockMeta *__restrict__ meta,
         const SolverState *__restrict__ state,
         const int2 *__restrict__ rowtiles, const float *__restrict__ T,
         float *X, float *Z) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float (*Ts)[B + 1] = reinterpret_cast<float (*)[B + 1]>(smem_raw);
  float (*Xs)[B + 1] = Ts + B;
  float (*Zs)[B + 1] = Xs + TR;
  const int2 t = rowtiles[blockIdx.x];
  if (state[t.x].status != kRunning) return;
  const BlockMeta bm = meta[t.x];
  const int rows = min(TR, bm.s - t.y);
  if (rows <= 0) return;
  const float *Tb = T + (int64_t)t.x * B * B;
  float *Xb = X + bm.x_off + (int64_t)t.y * B;
  float *Zb = Z + bm.x_off + (int64_t)t.y * B;
  for (int e = threadIdx.x; e < B * B; e += blockDim.x)
    Ts[e / B][e % B] = Tb[e];
  for (int e = threadIdx.x; e < rows * B; e += blockDim.x) {
    Xs[e / B][e % B] = Xb[e];
    Zs[e / B][e % B] = Zb[e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rows * B; e += blockDim.x) {
    const int r = e / B, j = e % B;
    float ax = 0.f, az = 0.f;
#pragma unroll 8
    for (int l = 0; l < B; ++l) {
      const float tl = Ts[l][j];
      ax = fmaf(Xs[r][l], tl, ax);
      az = fmaf(Zs[r][l], tl, az);
    }
    Xb[e] = ax;
    Zb[e] = az;
  }
}

// Residuals, convergence, next filter interval; copies F_s when done.
template <int B>
__global__ void __launch_bounds__(256)
k_check(const BlockMeta *__restrict__ meta, SolverState *__restrict__ state,
        const float *__restrict__ X, const float *__restrict__ Z,
        const float *__restrict__ theta, float *__restrict__ Fs, int kp,
        int max_iters, int max_degree, float tol, int32_t *running) {
  constexpr int G = 256 / B;          // row groups
  __shared__ float rs[G][B], xs[G][B];
  __shared__ int s_done;
  const int blk = blockIdx.x;
  SolverState st = state[blk];
  if (st.status != kRunning) return;
  const BlockMeta bm = meta[blk];
  const int n = st.bsub, s = bm.s, keff = bm.keff;
  const float *Xb = X + bm.x_off;
  const float *Zb = Z + bm.x_off;
  const float *th = theta + (int64_t)blk * B;
  const int col = threadIdx.x % B, grp = threadIdx.x / B;
  float r2 = 0.f, x2 = 0.f;
  const float tc = th[col];
  for (int r = grp; r < s; r += G) {
    const float xv = Xb[(int64_t)r * B + col];
    const float d = Zb[(int64_t)r * B + col] - tc * xv;
    r2 = fmaf(d, d, r2);
    x2 = fmaf(xv, xv, x2);
  }
  rs[grp][col] = r2;
  xs[grp][col] = x2;
  __syncthreads();
  if (threadIdx.x == 0) {
    const float t1 = th[0];
    float worst = 0.f;
    for (int j = 0; j < keff && j < n; ++j) {
      float a = 0.f;
      for (int g = 0; g < G; ++g) a += rs[g][j];
      worst = fmaxf(worst, sqrtf(a));
    }
    st.iters += 1;
    st.theta1 = t1;
    st.resid = t1 > 0.f ? worst / t1 : 0.f;
    const bool conv = (s <= B) || !(t1 > 1e-30f) || (worst <= tol * t1);
    if (conv || st.iters >= max_iters) {
      st.status = conv ? kConverged : kCapped;
      s_done = 1;
    } else {
      float cut = th[n - 1];
      cut = fmaxf(cut, kCutFloor * t1);
      if (cut >= 0.5f * t1) cut = 0.5f * t1;
      st.cut = cut;
      st.a0 = t1;
      const float tt = 2.f * t1 / cut - 1.f;   // >= 3
      const float at = acoshf(tt);
      int d = 2;
      while (d + 2 <= max_degree && coshf((float)(d + 2) * at) <= kMaxAmplification)
        d += 2;
      st.degree = d;
      atomicAdd(running, 1);
      s_done = 0;
    }
    state[blk] = st;
  }
  __syncthreads();
  if (!s_done) return;
  // F_s = normalised first keff Ritz vectors
  for (int e = threadIdx.x; e < s * kp; e += blockDim.x) {
    const int r = e / kp, j = e % kp;
    float v = 0.f;
    if (j < keff && j < n) {
      float nn = 0.f;
      for (int g = 0; g < G; ++g) nn += xs[g][j];
      v = nn > 0.f ? Xb[(int64_t)r * B + j] / sqrtf(nn) : 0.f;
    }
    Fs[bm.fs_off + (int64_t)r * kp + j] = v;
  }
}

// F_L[l, :] = sum_a W[a, l] F_s[a, :] for 128 consecutive l.
template <int KM>
__global__ void __launch_bounds__(128)
k_project(const BlockMeta *__restrict__ meta, const int2 *__restrict__ ltiles,
          const float *__restrict__ W, const float *__restrict__ Fs,
          float *__restrict__ FL, int kp) {
  constexpr int CH = 32;
  __shared__ float Fsh[CH][KM];
  const int2 t = ltiles[blockIdx.x];
  const BlockMeta bm = meta[t.x];
  const int l = t.y + threadIdx.x;
  const float *Wb = W + bm.w_off;
  const float *Fb = Fs + bm.fs_off;
  float acc[KM];
#pragma unroll
  for (int j = 0; j < KM; ++j) acc[j] = 0.f;
  for (int a0 = 0; a0 < bm.s; a0 += CH) {
    for (int e = threadIdx.x; e < CH * KM; e += blockDim.x) {
      const int rr = e / KM, j = e % KM;
      Fsh[rr][j] = (a0 + rr < bm.s && j < kp) ? Fb[(int64_t)(a0 + rr) * kp + j] : 0.f;
    }
    __syncthreads();
    const int lim = min(CH, bm.s - a0);
    if (l < bm.L) {
      for (int rr = 0; rr < lim; ++rr) {
        const float w = Wb[(int64_t)(a0 + rr) * bm.L_pad + l];
#pragma unroll
        for (int j = 0; j < KM; ++j) acc[j] = fmaf(w, Fsh[rr][j], acc[j]);
      }
    }
    __syncthreads();
  }
  if (l < bm.L) {
    float *out = FL + bm.fl_off + (int64_t)l * kp;
#pragma unroll
    for (int j = 0; j < KM; ++j)
      if (j < kp) out[j] = acc[j];
  }
}

// sigma_j = |F_L[:, j]| in float64; flip (F_s_j, F_L_j) so the item-side
// vector's largest-|.| entry (lowest index on ties) is positive.
__global__ void __launch_bounds__(256)
k_finalize(const BlockMeta *__restrict__ meta, float *Fs, float *FL,
           double *sigma, int kp, int k) {
  const int blk = blockIdx.x;
  const BlockMeta bm = meta[blk];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float *Fsb = Fs + bm.fs_off;
  float *FLb = FL + bm.fl_off;
  for (int j = warp; j < kp; j += 8) {
    if (j >= bm.keff) {
      if (lane == 0) sigma[(int64_t)blk * kp + j] = 0.0;
      continue;
    }
    double acc = 0.0;
    for (int l = lane; l < bm.L; l += 32) {
      const double v = FLb[(int64_t)l * kp + j];
      acc = fma(v, v, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    // item-side vector: F_s when trans (s indexes items), else F_L
    const float *vec = bm.trans ? Fsb : FLb;
    const int len = bm.trans ? bm.s : bm.L;
    float best = -1.f;
    int bidx = 0x7fffffff;
    for (int a = lane; a < len; a += 32) {
      const float v = fabsf(vec[(int64_t)a * kp + j]);
      if (v > best) { best = v; bidx = a; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    const bool flip = bidx < len && vec[(int64_t)bidx * kp + j] < 0.f;
    __syncwarp();
    if (flip) {
      for (int a = lane; a < bm.s; a += 32) Fsb[(int64_t)a * kp + j] *= -1.f;
      for (int l = lane; l < bm.L; l += 32) FLb[(int64_t)l * kp + j] *= -1.f;
    }
    if (lane == 0) sigma[(int64_t)blk * kp + j] = sqrt(acc);
  }
}

template <int B>
size_t rr_smem() { return sizeof(RRSmem<B>); }

template <int B>
size_t rot_smem() { return sizeof(float) * (B + 2 * TR) * (B + 1); }

template <int B>
cudaError_t set_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_rr_solve<B>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)rr_smem<B>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_rotate<B>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)rot_smem<B>());
  return e;
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
    k_init_panels<B><<<ntiles, 256, 0, st>>>(e.meta, e.state, rowtiles, e.X,
                                             e.seed);
    return cudaGetLastError();
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
    k_gpanel<B><<<ntiles, 256, 0, st>>>(e.meta, e.state, rowtiles, e.G, in,
                                        in2, out, mode, step);
    return cudaGetLastError();
  });
}

cudaError_t launch_small_gram(const EigBuffers &e, cudaStream_t st) {
  return by_width(e.bsub, [&](auto w) {
    constexpr int B = decltype(w)::value;
    k_small_gram<B><<<e.nblocks, 256, 0, st>>>(e.meta, e.state, e.X, e.Z,
                                               e.SH);
    return cudaGetLastError();
  });
}

cudaError_t launch_rr_solve(const EigBuffers &e, cudaStream_t st) {
  return by_width(e.bsub, [&](auto w) {
    constexpr int B = decltype(w)::value;
    cudaError_t err = set_attrs<B>();
    if (err != cudaSuccess) return err;
    k_rr_solve<B><<<e.nblocks, 256, rr_smem<B>(), st>>>(
        e.meta, e.state, e.SH, e.T, e.theta, e.max_sweeps);
    return cudaGetLastError();
  });
}

cudaError_t launch_rotate(const EigBuffers &e, const int2 *rowtiles,
                          int32_t ntiles, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  return by_width(e.bsub, [&](auto w) {
    constexpr int B = decltype(w)::value;
    cudaError_t err = set_attrs<B>();
    if (err != cudaSuccess) return err;
    k_rotate<B><<<ntiles, 256, rot_smem<B>(), st>>>(e.meta, e.state,
                                                    rowtiles, e.T, e.X, e.Z);
    return cudaGetLastError();
  });
}

cudaError_t launch_check(const EigBuffers &e, cudaStream_t st) {
  return by_width(e.bsub, [&](auto w) {
    constexpr int B = decltype(w)::value;
    k_check<B><<<e.nblocks, 256, 0, st>>>(e.meta, e.state, e.X, e.Z,
                                          e.theta, e.Fs, e.kp, e.max_iters,
                                          e.max_degree, e.tol, e.running);
    return cudaGetLastError();
  });
}

cudaError_t launch_project(const BlockMeta *meta, const int2 *ltiles,
                           int32_t ntiles, const float *W, const float *Fs,
                           float *FL, int32_t kp, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (kp <= 16) k_project<16><<<ntiles, 128, 0, st>>>(meta, ltiles, W, Fs, FL, kp);
  else if (kp <= 32) k_project<32><<<ntiles, 128, 0, st>>>(meta, ltiles, W, Fs, FL, kp);
  else k_project<56><<<ntiles, 128, 0, st>>>(meta, ltiles, W, Fs, FL, kp);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const BlockMeta *meta, int32_t nblocks,
                            float *Fs, float *FL, double *sigma, int32_t kp,
                            int32_t k, cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  k_finalize<<<nblocks, 256, 0, st>>>(meta, Fs, FL, sigma, kp, k);
  return cudaGetLastError();
}

}  // namespace bsvd
