// Held-out prediction and scoring.
//
// A rating is predicted from its block's factors (Section 2.1, Eq. 2, with
// the singular values merged into one side): yhat = mu_b + P[r,:] . V[c,:].
// In W orientation that is mu_b + F_s[a,:] . F_L[l,:]. The score is the RMSE
// of Section 5 (Table 1, "Test RMSE").
//
// The squared errors are summed in float64 with a fixed grid, a fixed
// per-thread stride and a fixed reduction tree. The sum therefore does not
// depend on scheduling, and reruns are bit-identical.
#include "kernels.h"

namespace bsvd {

namespace {

__device__ __forceinline__ bool predict_one(const PredictArgs &a, int32_t u,
                                            int32_t i, float *out) {
  int32_t blk, r, c, wa, wl;
  if (!locate(a.g, u, i, &blk, &r, &c)) return false;
  const BlockMeta &bm = a.meta[blk];
  float y = a.mu[blk];
  if (bm.keff > 0) {
    to_w(bm, r, c, &wa, &wl);
    const float4 *fs = reinterpret_cast<const float4 *>(
        a.Fs + bm.fs_off + (int64_t)wa * a.kp);
    const float4 *fl = reinterpret_cast<const float4 *>(
        a.FL + bm.fl_off + (int64_t)wl * a.kp);
    // both rows' loads in chunks of 5 float4s, each chunk's loads issued
    // before its products (in column order)
    constexpr int kChunk = 5;
    const int n4 = a.kp / 4;
    float dot = 0.f;
    for (int j0 = 0; j0 < n4; j0 += kChunk) {
      float4 p[kChunk], q[kChunk];
#pragma unroll
      for (int j = 0; j < kChunk; ++j) {
        if (j0 + j < n4) {
          p[j] = __ldg(fs + j0 + j);
          q[j] = __ldg(fl + j0 + j);
        }
      }
#pragma unroll
      for (int j = 0; j < kChunk; ++j) {
        if (j0 + j < n4) {
          dot = fmaf(p[j].x, q[j].x, dot);
          dot = fmaf(p[j].y, q[j].y, dot);
          dot = fmaf(p[j].z, q[j].z, dot);
          dot = fmaf(p[j].w, q[j].w, dot);
        }
      }
    }
    y += dot;
  }
  if (a.clamp) y = fminf(fmaxf(y, a.lo), a.hi);
  *out = y;
  return true;
}

__global__ void __launch_bounds__(256)
k_predict(PredictArgs a, int64_t nq, const int32_t *__restrict__ u,
          const int32_t *__restrict__ it, float *__restrict__ yhat,
          int32_t *err) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nq;
       t += (int64_t)gridDim.x * blockDim.x) {
    float y = 0.f;
    if (!predict_one(a, u[t], it[t], &y)) atomicOr(err, kErrIndex);
    yhat[t] = y;
  }
}

// With a.owned_only, queries in blocks this context does not hold are
// skipped; the CTA's count of summed queries goes to counts.
__global__ void __launch_bounds__(256)
k_sqerr(PredictArgs a, int64_t nq, const int32_t *__restrict__ u,
        const int32_t *__restrict__ it, const float *__restrict__ y,
        double *__restrict__ partials, long long *__restrict__ counts,
        int32_t *err) {
  __shared__ double red[256];
  __shared__ long long cnt[256];
  double acc = 0.0;
  long long n = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nq;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (a.owned_only) {
      int32_t blk, r, c;
      if (locate(a.g, u[t], it[t], &blk, &r, &c) && !a.meta[blk].owned)
        continue;
    }
    float yh;
    if (!predict_one(a, u[t], it[t], &yh)) { atomicOr(err, kErrIndex); continue; }
    const double d = (double)yh - (double)y[t];
    acc = fma(d, d, acc);
    ++n;
  }
  red[threadIdx.x] = acc;
  cnt[threadIdx.x] = n;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[threadIdx.x] += red[threadIdx.x + w];
      cnt[threadIdx.x] += cnt[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = red[0];
    counts[blockIdx.x] = cnt[0];
  }
}

// out[0] = sum of the partial sums (fixed tree); out[1] = their count, as
// a float64 holding an exact integer below 2^53.
__global__ void __launch_bounds__(512)
k_sum_partials(const double *__restrict__ partials,
               const long long *__restrict__ counts, int n, double *out) {
  __shared__ double red[512];
  __shared__ long long cnt[512];
  red[threadIdx.x] = threadIdx.x < n ? partials[threadIdx.x] : 0.0;
  cnt[threadIdx.x] = threadIdx.x < n ? counts[threadIdx.x] : 0;
  __syncthreads();
  for (int w = 256; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[threadIdx.x] += red[threadIdx.x + w];
      cnt[threadIdx.x] += cnt[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = red[0];
    out[1] = (double)cnt[0];
  }
}

int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > 152 * 8) g = 152 * 8;
  return (int)g;
}

}  // namespace

cudaError_t launch_predict(const PredictArgs &a, int64_t nq, const int32_t *u,
                           const int32_t *i, float *yhat, int32_t *err,
                           cudaStream_t st) {
  if (nq <= 0) return cudaSuccess;
  k_predict<<<grid_for(nq), 256, 0, st>>>(a, nq, u, i, yhat, err);
  return cudaGetLastError();
}

cudaError_t launch_sqerr(const PredictArgs &a, int64_t nq, const int32_t *u,
                         const int32_t *i, const float *y, double *partials,
                         double *out, int32_t *err, cudaStream_t st) {
  static_assert(kSqerrBlocks <= 512, "final sum is one CTA of 512");
  long long *counts = reinterpret_cast<long long *>(partials + kSqerrBlocks);
  k_sqerr<<<kSqerrBlocks, 256, 0, st>>>(a, nq, u, i, y, partials, counts, err);
  k_sum_partials<<<1, 512, 0, st>>>(partials, counts, kSqerrBlocks, out);
  return cudaGetLastError();
}

}  // namespace bsvd
