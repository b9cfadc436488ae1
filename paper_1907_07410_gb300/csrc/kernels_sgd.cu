// The paper's own method: blocked stochastic gradient descent on the biased
// latent-factor model (Section 2.2, Eq. 3 and 10-13; Algorithms 1-2), with
// the blocks of one schedule step (Figure 2) processed at once.
//
// Epoch order. Algorithm 2 walks a block row by row, then column by column,
// so each block's ratings are laid out row-major once, on the device:
//   * bucket = (block column bj, the user's row position in the grid), so a
//     block (bi, bj) is the consecutive buckets bj * m + [rb[bi], rb[bi+1]);
//   * count, exclusive scan (one CTA, fixed order), scatter, then sort each
//     bucket by (local column, input index): the order is deterministic
//     even though the scatter is not.
//
// Step kernel. One warp per block of the step (the blocks of a step share
// no user and no item, so they are independent). The warp walks its block's
// ratings in order; lane f holds factor f of the current user and item.
// The dot product is summed over f = 0 .. k-1 in order (every lane runs the
// same chain of shuffles and adds, so all hold the same value) and every
// operation is an explicitly rounded float64 add/sub/mul, so the result is
// bit-identical to a sequential float64 loop without contraction.
#include "kernels.h"

namespace bsvd {

namespace {

__device__ __forceinline__ int64_t sgd_bucket(const GridDesc &g, int32_t blk,
                                              int32_t r, int64_t m) {
  const int32_t bi = g.diag ? blk : blk / g.q;
  const int32_t bj = g.diag ? blk : blk % g.q;
  int64_t row0 = g.equal_rows ? (int64_t)bi * g.br : g.row_bounds[bi];
  if (row0 > m) row0 = m;
  return (int64_t)bj * m + row0 + r;
}

__global__ void __launch_bounds__(256)
k_sgd_count(GridDesc g, int64_t nnz, const int32_t *__restrict__ u,
            const int32_t *__restrict__ it, unsigned long long *__restrict__ cnt,
            int32_t *err) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t blk, r, c;
    if (!locate(g, u[t], it[t], &blk, &r, &c)) {
      atomicOr(err, kErrIndex);
      continue;
    }
    atomicAdd(&cnt[sgd_bucket(g, blk, r, g.m)], 1ull);
  }
}

// Exclusive prefix sum of n counts into off[0 .. n] (off[n] = total), by one
// CTA of 1024 threads: each thread sums a contiguous segment, the segment
// sums are scanned in shared memory, then each thread writes its segment.
__global__ void __launch_bounds__(1024)
k_scan_exclusive(int64_t n, const unsigned long long *__restrict__ cnt,
                 int64_t *__restrict__ off) {
  __shared__ long long part[1024];
  const int64_t seg = (n + 1023) / 1024;
  const int64_t a = (int64_t)threadIdx.x * seg;
  const int64_t b = a + seg < n ? a + seg : n;
  long long s = 0;
  for (int64_t e = a; e < b; ++e) s += (long long)cnt[e];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 1; w < 1024; w <<= 1) {
    const long long v = threadIdx.x >= w ? part[threadIdx.x - w] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  long long run = part[threadIdx.x] - s;    // exclusive prefix of the segment
  for (int64_t e = a; e < b; ++e) {
    off[e] = run;
    run += (long long)cnt[e];
  }
  if (threadIdx.x == 1023) off[n] = part[1023];
}

__global__ void __launch_bounds__(256)
k_sgd_fill(GridDesc g, int64_t nnz, const int32_t *__restrict__ u,
           const int32_t *__restrict__ it, const int64_t *__restrict__ off,
           unsigned long long *__restrict__ cursor,
           int64_t *__restrict__ key, int64_t *__restrict__ src) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t blk, r, c;
    if (!locate(g, u[t], it[t], &blk, &r, &c)) continue;   // flagged before
    const int64_t bkt = sgd_bucket(g, blk, r, g.m);
    const int64_t slot = off[bkt] + (int64_t)atomicAdd(&cursor[bkt], 1ull);
    key[slot] = ((int64_t)c << 40) | t;     // nnz < 2^40 is checked by the host
    src[slot] = t;
  }
}

// Buckets are sorted by key (local column, then input index; the keys are
// distinct). One thread per bucket sorts a small bucket by insertion; a
// bucket of more than kSortSmall ratings is appended to a list (big[1..],
// count in big[0]) for k_sgd_sort_big. The list's order depends on
// scheduling, the sorted buckets do not.
constexpr int64_t kSortSmall = 64;
constexpr int kSortTile = 16384;       // keys of a shared-memory bitonic sort

__global__ void __launch_bounds__(256)
k_sgd_sort(int64_t nbuckets, const int64_t *__restrict__ off,
           int64_t *__restrict__ key, int64_t *__restrict__ src,
           unsigned long long *__restrict__ big) {
  for (int64_t bk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       bk < nbuckets; bk += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = off[bk], b = off[bk + 1];
    if (b - a > kSortSmall) {
      big[1 + atomicAdd(&big[0], 1ull)] = (unsigned long long)bk;
      continue;
    }
    for (int64_t e = a + 1; e < b; ++e) {
      const int64_t kv = key[e], sv = src[e];
      int64_t d = e - 1;
      while (d >= a && key[d] > kv) {
        key[d + 1] = key[d];
        src[d + 1] = src[d];
        --d;
      }
      key[d + 1] = kv;
      src[d + 1] = sv;
    }
  }
}

// One CTA per listed bucket (grid-stride over the list): a bitonic sort of
// its keys in shared memory, padded with all-ones keys to a power of two;
// the input index is the key's low 40 bits, so src is rewritten from the
// sorted keys. A bucket of more than kSortTile ratings (more than that many
// of one user's items in one block column) is sorted by insertion in
// global memory by one thread: correct, slow, and not met by the workloads
// here.
__global__ void __launch_bounds__(1024)
k_sgd_sort_big(const int64_t *__restrict__ off,
               const unsigned long long *__restrict__ big,
               int64_t *__restrict__ key, int64_t *__restrict__ src) {
  extern __shared__ unsigned long long sk[];
  const unsigned long long nbig = big[0];
  for (unsigned long long li = blockIdx.x; li < nbig; li += gridDim.x) {
    const int64_t bk = (int64_t)big[1 + li];
    const int64_t a = off[bk], n = off[bk + 1] - a;
    if (n > kSortTile) {
      if (threadIdx.x == 0) {
        for (int64_t e = a + 1; e < a + n; ++e) {
          const int64_t kv = key[e];
          int64_t d = e - 1;
          while (d >= a && key[d] > kv) { key[d + 1] = key[d]; --d; }
          key[d + 1] = kv;
        }
        for (int64_t e = a; e < a + n; ++e) src[e] = key[e] & ((1ll << 40) - 1);
      }
      __syncthreads();
      continue;
    }
    int p2 = 1;
    while (p2 < n) p2 <<= 1;
    for (int t = threadIdx.x; t < p2; t += blockDim.x)
      sk[t] = t < n ? (unsigned long long)key[a + t] : ~0ull;
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < p2; t += blockDim.x) {
          const int o = t ^ j;
          if (o > t) {
            const unsigned long long x = sk[t], y = sk[o];
            const bool up = (t & k) == 0;
            if ((x > y) == up) { sk[t] = y; sk[o] = x; }
          }
        }
        __syncthreads();
      }
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      key[a + t] = (int64_t)sk[t];
      src[a + t] = (int64_t)(sk[t] & ((1ull << 40) - 1));
    }
    __syncthreads();
  }
}

// Gathers the ratings into epoch order. Only the first *placed entries of
// src were written (a rating with an id out of range was counted nowhere and
// is reported by k_sgd_count), so only those are read.
__global__ void __launch_bounds__(256)
k_sgd_gather(GridDesc g, const int64_t *__restrict__ placed,
             const int64_t *__restrict__ src,
             const int32_t *__restrict__ u, const int32_t *__restrict__ it,
             const float *__restrict__ x, int32_t *__restrict__ su,
             int32_t *__restrict__ si, float *__restrict__ sx,
             int32_t *__restrict__ sr, int32_t *__restrict__ sc) {
  const int64_t nnz = *placed;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = src[t];
    const int32_t uu = u[s], ii = it[s];
    int32_t blk = 0, r = 0, c = 0;
    locate(g, uu, ii, &blk, &r, &c);      // in range: checked by k_sgd_count
    su[t] = uu;
    si[t] = ii;
    sx[t] = x[s];
    sr[t] = r;
    sc[t] = c;
  }
}

// [start, end) of every block's ratings in the epoch order
__global__ void __launch_bounds__(256)
k_sgd_ranges(GridDesc g, int32_t nblocks, const int64_t *__restrict__ off,
             int64_t *__restrict__ range) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblocks;
       b += gridDim.x * blockDim.x) {
    const int32_t bi = g.diag ? b : b / g.q;
    const int32_t bj = g.diag ? b : b % g.q;
    // with equal blocks, trailing block rows can lie wholly past m (e.g.
    // 256 rows of ceil(6040 / 256) = 24): clamp both ends, so such a block
    // has an empty range and every index stays inside off[0 .. buckets]
    int64_t r0 = g.equal_rows ? (int64_t)bi * g.br : g.row_bounds[bi];
    int64_t r1 = g.equal_rows ? (int64_t)(bi + 1) * g.br : g.row_bounds[bi + 1];
    if (r0 > g.m) r0 = g.m;
    if (r1 > g.m) r1 = g.m;
    range[2 * b] = off[(int64_t)bj * g.m + r0];
    range[2 * b + 1] = off[(int64_t)bj * g.m + r1];
  }
}

// One schedule step: warp w takes block blocks[w] and runs Algorithm 2 on it.
//
// Software pipelined: while rating t is updated, the ids, rating, factor
// rows and biases of rating t+1 are loaded. A user (item) shared by t and
// t+1 is not reloaded: the values just computed for t are carried in
// registers instead (every lane computes the new biases the same way, lane
// 0 stores them). Anything else t+1 reads was last written by an earlier
// rating, in program order in the same lane (factors) or before the
// __syncwarp that ends that rating (biases). The arithmetic is unchanged,
// so the results stay bit-identical to the sequential order.
__global__ void __launch_bounds__(32)
k_sgd_step(const int32_t *__restrict__ blocks, const int64_t *__restrict__ range,
           const int32_t *__restrict__ su, const int32_t *__restrict__ si,
           const float *__restrict__ sx, int64_t nnz, int32_t k, double *P,
           double *Q, double *bu, double *bi, SgdRates r, int32_t *err) {
  const int lane = threadIdx.x;
  const int32_t b = blocks[blockIdx.x];
  const int64_t t0 = range[2 * b], t1 = range[2 * b + 1];
  if (t0 < 0 || t1 > nnz || t0 > t1) {     // never expected: refuse to run
    if (lane == 0) atomicOr(err, kErrIndex);
    return;
  }
  if (t0 == t1) return;
  const bool mine = lane < k;
  int32_t uu = su[t0], ii = si[t0];
  float xx = sx[t0];
  double pf = mine ? P[(int64_t)uu * k + lane] : 0.0;
  double qf = mine ? Q[(int64_t)ii * k + lane] : 0.0;
  double bu0 = bu[uu], bi0 = bi[ii];
  for (int64_t t = t0; t < t1; ++t) {
    // loads for rating t+1, except rows and biases it shares with t
    const bool more = t + 1 < t1;
    const int32_t un = more ? su[t + 1] : uu;
    const int32_t in = more ? si[t + 1] : ii;
    const float xn = more ? sx[t + 1] : 0.f;
    const bool new_u = un != uu, new_i = in != ii;
    const double pn = (mine && new_u) ? P[(int64_t)un * k + lane] : 0.0;
    const double qn = (mine && new_i) ? Q[(int64_t)in * k + lane] : 0.0;
    const double bun = new_u ? bu[un] : 0.0;
    const double bin = new_i ? bi[in] : 0.0;
    // rating t
    const double prod = __dmul_rn(pf, qf);
    double dot = 0.0;
    for (int f = 0; f < k; ++f)
      dot = __dadd_rn(dot, __shfl_sync(0xffffffffu, prod, f));
    const double e = __dsub_rn(__dsub_rn(__dsub_rn((double)xx, bu0), bi0), dot);
    const double bu1 = __dadd_rn(bu0, __dmul_rn(r.a_ubias, __dsub_rn(
                                          e, __dmul_rn(r.b_ubias, bu0))));
    const double bi1 = __dadd_rn(bi0, __dmul_rn(r.a_ibias, __dsub_rn(
                                          e, __dmul_rn(r.b_ibias, bi0))));
    const double p1 = __dadd_rn(pf, __dmul_rn(r.a_user, __dsub_rn(
                                        __dmul_rn(e, qf), __dmul_rn(r.b_user, pf))));
    const double q1 = __dadd_rn(qf, __dmul_rn(r.a_item, __dsub_rn(
                                        __dmul_rn(e, pf), __dmul_rn(r.b_item, qf))));
    if (lane == 0) {
      bu[uu] = bu1;
      bi[ii] = bi1;
    }
    if (mine) {
      P[(int64_t)uu * k + lane] = p1;
      Q[(int64_t)ii * k + lane] = q1;
    }
    // the next rating's loads (issued above or in the next iteration) may
    // read what this one wrote, in another lane
    __syncwarp();
    pf = new_u ? pn : p1;
    qf = new_i ? qn : q1;
    bu0 = new_u ? bun : bu1;
    bi0 = new_i ? bin : bi1;
    uu = un;
    ii = in;
    xx = xn;
  }
}

// ---- the float32 form -----------------------------------------------------
//
// A block's walk is a chain of dependent operations, each rating's update
// feeding the next rating's dot product. In float64 on GB300 one link of
// that chain costs about as much as a whole float32 rating, so the float32
// form runs the same operations, in the same order and with the same
// single rounding each, in float32.
//
// Parameters live as rows of k + 1 floats: factors 0 .. k-1, then the bias.
// One CTA per block of the step. When the step's blocks fit in shared
// memory, the CTA first stages its block's rows (the users of its block row
// and the items of its block column that have ratings in the block), the
// first warp walks the ratings against shared memory (lane f owns factor f;
// lane 0 stores the biases), and the CTA writes the rows back. The next
// rating's rows are loaded one rating ahead and its ids two ahead; a row it
// shares with the current rating is carried in registers. Otherwise the
// warp works on the rows in global memory the same way.

__global__ void __launch_bounds__(256)
k_sgd_narrow(int64_t m, int64_t n, int32_t k, const double *__restrict__ P,
             const double *__restrict__ Q, const double *__restrict__ bu,
             const double *__restrict__ bi, float *__restrict__ P32,
             float *__restrict__ Q32) {
  const int64_t kk = k + 1, np = m * kk, total = np + n * kk;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const bool user = e < np;
    const int64_t a = user ? e : e - np;
    const int64_t row = a / kk, f = a - row * kk;
    double v;
    if (user) v = f < k ? P[row * k + f] : bu[row];
    else v = f < k ? Q[row * k + f] : bi[row];
    if (user) P32[a] = __double2float_rn(v);
    else Q32[a] = __double2float_rn(v);
  }
}

__global__ void __launch_bounds__(256)
k_sgd_widen(int64_t m, int64_t n, int32_t k, const float *__restrict__ P32,
            const float *__restrict__ Q32, double *__restrict__ P,
            double *__restrict__ Q, double *__restrict__ bu,
            double *__restrict__ bi) {
  const int64_t kk = k + 1, np = m * kk, total = np + n * kk;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const bool user = e < np;
    const int64_t a = user ? e : e - np;
    const int64_t row = a / kk, f = a - row * kk;
    const double v = (double)(user ? P32[a] : Q32[a]);
    if (user) {
      if (f < k) P[row * k + f] = v;
      else bu[row] = v;
    } else {
      if (f < k) Q[row * k + f] = v;
      else bi[row] = v;
    }
  }
}

// The walk of one block's ratings [t0, t1) by one warp. Rows are
// Pr + ru[t] * (k + 1) and Qr + ci[t] * (k + 1): shared memory with local
// indices, or global memory with ids.
__device__ __forceinline__ void sgd_walk_f32(
    int64_t t0, int64_t t1, const int32_t *__restrict__ ru,
    const int32_t *__restrict__ ci, const float *__restrict__ sx, int32_t k,
    float *Pr, float *Qr, const SgdRates32 &r) {
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x;
  const bool mine = lane < k;
  const int64_t kk = k + 1;
  int32_t uu = ru[t0], ii = ci[t0];
  float xx = sx[t0];
  const bool two = t0 + 1 < t1;
  int32_t un = two ? ru[t0 + 1] : uu, in = two ? ci[t0 + 1] : ii;
  float xn = two ? sx[t0 + 1] : 0.f;
  float pf = mine ? Pr[uu * kk + lane] : 0.f;
  float qf = mine ? Qr[ii * kk + lane] : 0.f;
  float bu0 = Pr[uu * kk + k], bi0 = Qr[ii * kk + k];
  for (int64_t t = t0; t < t1; ++t) {
    // ids of rating t + 2; the rows of t + 1 unless shared with t
    const bool more = t + 1 < t1, more2 = t + 2 < t1;
    const int32_t u2 = more2 ? ru[t + 2] : un;
    const int32_t i2 = more2 ? ci[t + 2] : in;
    const float x2 = more2 ? sx[t + 2] : 0.f;
    const bool new_u = more && un != uu, new_i = more && in != ii;
    float pn = 0.f, qn = 0.f, bun = 0.f, bin = 0.f;
    if (new_u) {
      pn = mine ? Pr[un * kk + lane] : 0.f;
      bun = Pr[un * kk + k];
    }
    if (new_i) {
      qn = mine ? Qr[in * kk + lane] : 0.f;
      bin = Qr[in * kk + k];
    }
    // rating t: the dot product in f order, in chunks of eight shuffles
    const float prod = __fmul_rn(pf, qf);
    float dot = 0.f;
#pragma unroll
    for (int j0 = 0; j0 < 32; j0 += 8) {
      if (j0 < k) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __shfl_sync(kAll, prod, j0 + j);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (j0 + j < k) dot = __fadd_rn(dot, v[j]);
      }
    }
    const float e = __fsub_rn(__fsub_rn(__fsub_rn(xx, bu0), bi0), dot);
    const float bu1 = __fadd_rn(bu0, __fmul_rn(r.a_ubias, __fsub_rn(
                                         e, __fmul_rn(r.b_ubias, bu0))));
    const float bi1 = __fadd_rn(bi0, __fmul_rn(r.a_ibias, __fsub_rn(
                                         e, __fmul_rn(r.b_ibias, bi0))));
    const float p1 = __fadd_rn(pf, __fmul_rn(r.a_user, __fsub_rn(
                                       __fmul_rn(e, qf), __fmul_rn(r.b_user, pf))));
    const float q1 = __fadd_rn(qf, __fmul_rn(r.a_item, __fsub_rn(
                                       __fmul_rn(e, pf), __fmul_rn(r.b_item, qf))));
    if (mine) {
      Pr[uu * kk + lane] = p1;
      Qr[ii * kk + lane] = q1;
    }
    if (lane == 0) {
      Pr[uu * kk + k] = bu1;
      Qr[ii * kk + k] = bi1;
    }
    // every lane reads the biases lane 0 stored, at a later rating
    __syncwarp();
    pf = new_u ? pn : p1;
    qf = new_i ? qn : q1;
    bu0 = new_u ? bun : bu1;
    bi0 = new_i ? bin : bi1;
    uu = un;
    ii = in;
    xx = xn;
    un = u2;
    in = i2;
    xn = x2;
  }
}

__global__ void __launch_bounds__(256)
k_sgd_step_f32(GridDesc g, const int32_t *__restrict__ blocks,
               const int64_t *__restrict__ range,
               const int32_t *__restrict__ sr, const int32_t *__restrict__ sc,
               const int32_t *__restrict__ su, const int32_t *__restrict__ si,
               const float *__restrict__ sx, int64_t nnz, int32_t k,
               float *P32, float *Q32, SgdRates32 r, int staged, int32_t *err) {
  extern __shared__ float stage[];
  const int32_t b = blocks[blockIdx.x];
  const int64_t t0 = range[2 * b], t1 = range[2 * b + 1];
  if (t0 < 0 || t1 > nnz || t0 > t1) {     // never expected: refuse to run
    if (threadIdx.x == 0) atomicOr(err, kErrIndex);
    return;
  }
  if (t0 == t1) return;
  if (!staged) {
    if (threadIdx.x < 32) sgd_walk_f32(t0, t1, su, si, sx, k, P32, Q32, r);
    return;
  }
  const int32_t bi = g.diag ? b : b / g.q, bj = g.diag ? b : b % g.q;
  const int64_t rows = g.row_bounds[bi + 1] - g.row_bounds[bi];
  const int64_t cols = g.col_bounds[bj + 1] - g.col_bounds[bj];
  const int64_t kk = k + 1;
  float *Ps = stage;
  float *Qs = Ps + rows * kk;
  int32_t *ids = reinterpret_cast<int32_t *>(Qs + cols * kk);  // rows, cols
  const int tid = threadIdx.x, nt = blockDim.x;
  // slot -> id of the users and items the block's ratings touch (-1: none)
  for (int64_t s = tid; s < rows + cols; s += nt) ids[s] = -1;
  __syncthreads();
  for (int64_t t = t0 + tid; t < t1; t += nt) {
    ids[sr[t]] = su[t];
    ids[rows + sc[t]] = si[t];
  }
  __syncthreads();
  for (int64_t e = tid; e < (rows + cols) * kk; e += nt) {
    const int64_t s = e / kk;
    const int32_t id = ids[s];
    if (id >= 0)
      stage[e] = s < rows ? P32[(int64_t)id * kk + (e - s * kk)]
                          : Q32[(int64_t)id * kk + (e - s * kk)];
  }
  __syncthreads();
  if (tid < 32) sgd_walk_f32(t0, t1, sr, sc, sx, k, Ps, Qs, r);
  __syncthreads();
  for (int64_t e = tid; e < (rows + cols) * kk; e += nt) {
    const int64_t s = e / kk;
    const int32_t id = ids[s];
    if (id >= 0) {
      float *dst = s < rows ? P32 : Q32;
      dst[(int64_t)id * kk + (e - s * kk)] = stage[e];
    }
  }
}

// Eq. 3 in the oracle's order: (sum_f p_f q_f, in f order) + bu + bi
__device__ __forceinline__ double sgd_eval(int32_t k, const double *P,
                                           const double *Q, const double *bu,
                                           const double *bi, int32_t uu,
                                           int32_t ii) {
  const double *p = P + (int64_t)uu * k;
  const double *q = Q + (int64_t)ii * k;
  double dot = 0.0;
  for (int f = 0; f < k; ++f) dot = __dadd_rn(dot, __dmul_rn(p[f], q[f]));
  return __dadd_rn(__dadd_rn(dot, bu[uu]), bi[ii]);
}

__global__ void __launch_bounds__(256)
k_sgd_predict(int64_t nq, const int32_t *__restrict__ u,
              const int32_t *__restrict__ it, int32_t k, int64_t m, int64_t n,
              const double *__restrict__ P, const double *__restrict__ Q,
              const double *__restrict__ bu, const double *__restrict__ bi,
              double *__restrict__ yhat, int32_t *err) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nq;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t uu = u[t], ii = it[t];
    if (uu < 0 || uu >= m || ii < 0 || ii >= n) {
      atomicOr(err, kErrIndex);
      yhat[t] = 0.0;
      continue;
    }
    yhat[t] = sgd_eval(k, P, Q, bu, bi, uu, ii);
  }
}

// Squared training errors: per-CTA partial sums in a fixed tree, then one
// CTA adds the partials in index order.
__global__ void __launch_bounds__(256)
k_sgd_sqerr(int64_t nnz, const int32_t *__restrict__ u,
            const int32_t *__restrict__ it, const float *__restrict__ x,
            int32_t k, const double *__restrict__ P,
            const double *__restrict__ Q, const double *__restrict__ bu,
            const double *__restrict__ bi, double *__restrict__ partials) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double d = __dsub_rn((double)x[t], sgd_eval(k, P, Q, bu, bi, u[t],
                                                      it[t]));
    acc = __dadd_rn(acc, __dmul_rn(d, d));
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(512)
k_sgd_sum(const double *__restrict__ partials, int n, double *out) {
  __shared__ double red[512];
  red[threadIdx.x] = threadIdx.x < n ? partials[threadIdx.x] : 0.0;
  __syncthreads();
  for (int w = 256; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

int sgd_grid(int64_t n) {
  int64_t want = (n + 255) / 256;
  if (want < 1) want = 1;
  if (want > 152 * 8) want = 152 * 8;
  return (int)want;
}

}  // namespace

cudaError_t launch_sgd_order(const GridDesc &g, int32_t nblocks, int64_t nnz,
                             const int32_t *u, const int32_t *i, const float *x,
                             unsigned long long *cnt, int64_t *off,
                             int64_t *key, int64_t *src, int32_t *su,
                             int32_t *si, float *sx, int32_t *sr, int32_t *sc,
                             int64_t *range, int32_t *err, cudaStream_t st) {
  const int64_t nbuckets = (int64_t)(g.diag ? g.p : g.q) * g.m;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * nbuckets,
                                  st);
  if (e != cudaSuccess) return e;
  if (nnz > 0)
    k_sgd_count<<<sgd_grid(nnz), 256, 0, st>>>(g, nnz, u, i, cnt, err);
  k_scan_exclusive<<<1, 1024, 0, st>>>(nbuckets, cnt, off);
  e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * nbuckets, st);
  if (e != cudaSuccess) return e;
  if (nnz > 0) {
    k_sgd_fill<<<sgd_grid(nnz), 256, 0, st>>>(g, nnz, u, i, off, cnt, key, src);
    // the bucket counts are no longer needed: cnt holds the big-bucket list
    e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_sgd_sort<<<sgd_grid(nbuckets), 256, 0, st>>>(nbuckets, off, key, src,
                                                   cnt);
    e = cudaFuncSetAttribute(k_sgd_sort_big,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(unsigned long long) * kSortTile));
    if (e != cudaSuccess) return e;
    k_sgd_sort_big<<<152 * 2, 1024, sizeof(unsigned long long) * kSortTile,
                     st>>>(off, cnt, key, src);
    k_sgd_gather<<<sgd_grid(nnz), 256, 0, st>>>(g, off + nbuckets, src, u, i,
                                                x, su, si, sx, sr, sc);
  }
  k_sgd_ranges<<<(nblocks + 255) / 256, 256, 0, st>>>(g, nblocks, off, range);
  return cudaGetLastError();
}

cudaError_t launch_sgd_step(int32_t nb, const int32_t *blocks,
                            const int64_t *range, const int32_t *su,
                            const int32_t *si, const float *sx, int64_t nnz,
                            int32_t k, double *P, double *Q, double *bu,
                            double *bi, const SgdRates &r, int32_t *err,
                            cudaStream_t st) {
  if (nb <= 0) return cudaSuccess;
  k_sgd_step<<<nb, 32, 0, st>>>(blocks, range, su, si, sx, nnz, k, P, Q, bu,
                                bi, r, err);
  return cudaGetLastError();
}

cudaError_t launch_sgd_narrow(int64_t m, int64_t n, int32_t k, const double *P,
                              const double *Q, const double *bu,
                              const double *bi, float *P32, float *Q32,
                              cudaStream_t st) {
  k_sgd_narrow<<<sgd_grid((m + n) * (k + 1)), 256, 0, st>>>(m, n, k, P, Q, bu,
                                                            bi, P32, Q32);
  return cudaGetLastError();
}

cudaError_t launch_sgd_widen(int64_t m, int64_t n, int32_t k, const float *P32,
                             const float *Q32, double *P, double *Q,
                             double *bu, double *bi, cudaStream_t st) {
  k_sgd_widen<<<sgd_grid((m + n) * (k + 1)), 256, 0, st>>>(m, n, k, P32, Q32,
                                                           P, Q, bu, bi);
  return cudaGetLastError();
}

cudaError_t launch_sgd_step_f32(const GridDesc &g, int32_t nb,
                                const int32_t *blocks, const int64_t *range,
                                const int32_t *sr, const int32_t *sc,
                                const int32_t *su, const int32_t *si,
                                const float *sx, int64_t nnz, int32_t k,
                                float *P32, float *Q32, const SgdRates32 &r,
                                size_t stage_bytes, int32_t *err,
                                cudaStream_t st) {
  if (nb <= 0) return cudaSuccess;
  if (stage_bytes > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_sgd_step_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)stage_bytes);
    if (e != cudaSuccess) return e;
  }
  k_sgd_step_f32<<<nb, 256, stage_bytes, st>>>(g, blocks, range, sr, sc, su,
                                                si, sx, nnz, k, P32, Q32, r,
                                                stage_bytes > 0 ? 1 : 0, err);
  return cudaGetLastError();
}

cudaError_t launch_sgd_sqerr(int64_t nnz, const int32_t *u, const int32_t *i,
                             const float *x, int32_t k, const double *P,
                             const double *Q, const double *bu,
                             const double *bi, double *partials, double *out,
                             cudaStream_t st) {
  static_assert(kSqerrBlocks <= 512, "final sum is one CTA of 512");
  k_sgd_sqerr<<<kSqerrBlocks, 256, 0, st>>>(nnz, u, i, x, k, P, Q, bu, bi,
                                            partials);
  k_sgd_sum<<<1, 512, 0, st>>>(partials, kSqerrBlocks, out);
  return cudaGetLastError();
}

cudaError_t launch_sgd_predict(int64_t nq, const int32_t *u, const int32_t *i,
                               int32_t k, int64_t m, int64_t n,
                               const double *P, const double *Q,
                               const double *bu, const double *bi,
                               double *yhat, int32_t *err, cudaStream_t st) {
  if (nq <= 0) return cudaSuccess;
  k_sgd_predict<<<sgd_grid(nq), 256, 0, st>>>(nq, u, i, k, m, n, P, Q, bu, bi,
                                              yhat, err);
  return cudaGetLastError();
}

}  // namespace bsvd
