// Launchers of the libbsvd kernels (host side). Every launcher queues work
// on the given stream and returns the launch status.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace bsvd {

// ---- partition (kernels_partition.cu) ----------------------------------
cudaError_t launch_perm_check(const int32_t *perm, int64_t n, int32_t *seen,
                              int32_t *err, cudaStream_t st);
cudaError_t launch_count(const GridDesc &g, int64_t nnz, const int32_t *u,
                         const int32_t *i, const float *x, int32_t nblocks,
                         unsigned long long *counts, long long *sums,
                         unsigned int *maxabs_bits, int32_t *err,
                         cudaStream_t st);
cudaError_t launch_means(int32_t nblocks, const unsigned long long *counts,
                         const long long *sums,
                         const unsigned int *maxabs_bits, float *mu,
                         int32_t *err, cudaStream_t st);
// W (float32 arena) and Wh (bf16 copy) are each written when not null.
cudaError_t launch_scatter(const GridDesc &g, const BlockMeta *meta,
                           int64_t nnz, const int32_t *u, const int32_t *i,
                           const float *x, const float *mu, float *W,
                           __nv_bfloat16 *Wh, cudaStream_t st);

// ---- activity-quantile cut of one side (kernels_grid.cu) ----------------
// Keys are padded to quantile_cut_padded(size) entries. counts: size,
// keys: padded, cum: size + 1, perm: size, bounds: parts + 1 (device).
// *launches is increased by the number of kernels queued.
int64_t quantile_cut_padded(int64_t size);
cudaError_t launch_quantile_cut(const int32_t *ids, int64_t nnz, int64_t size,
                                int32_t parts, unsigned int *counts,
                                unsigned long long *keys, long long *cum,
                                int32_t *perm, int64_t *bounds, int32_t *err,
                                int64_t *launches, cudaStream_t st);

// ---- Gram (kernels_gram.cu) ---------------------------------------------
// tiles: (block, tile_i, tile_j, 0) with tile_i <= tile_j, 128 x 128 tiles.
cudaError_t launch_gram_f32(const BlockMeta *meta, const int4 *tiles,
                            int32_t ntiles, const float *W, float *G,
                            cudaStream_t st);

// ---- exact tensor-core Gram (kernels_gram_tc.cu) ------------------------
// maps: one TMA map per block over its [Y; M] bf16 planes (2 s128 x L_pad,
// 128 x 64 boxes, 128-byte swizzle); delta: mu - round(mu) per block.
cudaError_t launch_gram_tc(const BlockMeta *meta, const int4 *tiles,
                           int32_t ntiles, const CUtensorMap *maps,
                           const float *delta, float *G, int32_t *err,
                           cudaStream_t st);

// Single-pass tf32 Gram of the float32 blocks; maps: one TMA map per block
// over W (s_pad x L_pad f32, 128 x 32 boxes, 128-byte swizzle). This and
// launch_gram_bf16 take tiles (block, tile_i, tile_j, 0), tile_i <= tile_j,
// of 256 x 256.
cudaError_t launch_gram_tf32(const BlockMeta *meta, const int4 *tiles,
                             int32_t ntiles, const CUtensorMap *maps, float *G,
                             int32_t *err, cudaStream_t st);

// single-product bf16 Gram over the bf16 copy of the centred blocks
cudaError_t launch_gram_bf16(const BlockMeta *meta, const int4 *tiles,
                             int32_t ntiles, const CUtensorMap *maps, float *G,
                             int32_t *err, cudaStream_t st);

// ---- bf16 planes for the tensor-core Gram (kernels_partition.cu) ----------
// shift[b] = round(mu_b) (exact mean from the sums), delta[b] = mu_b - shift.
cudaError_t launch_plane_shift(int32_t nblocks, const unsigned long long *counts,
                               const long long *sums, float *shift,
                               float *delta, cudaStream_t st);
// Y = x - shift, M = 1 at every rating, into the zeroed planes; sets
// kErrNotExact in *flag when some x - shift is not an integer small enough
// (|y|^2 L_pad < 2^24, |y| <= 256) for the tensor-core Gram to be exact.
cudaError_t launch_scatter_planes(const GridDesc &g, const BlockMeta *meta,
                                  int64_t nnz, const int32_t *u,
                                  const int32_t *i, const float *x,
                                  const float *shift, __nv_bfloat16 *VX,
                                  int32_t *flag, cudaStream_t st);

// ---- subspace iteration (kernels_eig.cu) --------------------------------
struct EigBuffers {
  const BlockMeta *meta;
  SolverState *state;
  float *G;          // s_pad x s_pad Gram per block
  float *X;          // panels, s_pad x bsub per block
  float *Z;          // G X panels
  float *SH;         // per chunk: partial S (bsub^2) then H (bsub^2)
  double *RP;        // per row tile: partial residual^2 and norm^2 (2 bsub)
  float *T;          // per block: bsub^2 transform
  float *theta;      // per block: bsub Ritz values, descending
  float *Fs;         // s_pad x kp per block
  float *Finv;       // per block: bsub reciprocal column norms of X (done)
  int32_t *running;  // [0] blocks still iterating, [1] their largest degree
  float *XB = nullptr;  // the B form of X for the tensor-core products, or null
  int32_t bsub, kp, k;
  int32_t nblocks;
  int32_t nsm = 152;   // SMs of the device
  int32_t max_iters, max_sweeps;
  int32_t max_degree;  // cap on the per-block Chebyshev degree (even)
  float tol;
  uint64_t seed;
};

// Panel product on the tensor cores (three tf32 passes): tiles are
// (block, first row) pairs of 128 rows, gmaps one TMA map per block over G,
// xmaps one per block over the B form of `in` (32-float rows, 2 bsub-row
// boxes, 128-byte swizzle). The B form of a panel P (s_pad x bsub) sits at
// 2 x_off: for each 32-row chunk, bsub rows of hi(P) then bsub rows of
// lo(P), 32 floats each (hi = P rounded to 10 mantissa bits, lo = P - hi).
// out_bf (optional) receives the B form of `out`.
// Persistent: nctas CTAs (one per SM) take the tiles of the running blocks
// from the counter ctl[0] (ctl: 2 ints, zero before the first launch; the
// kernel leaves them zero). ptime[0] gains the launch's span in ns (first
// CTA start to last CTA end), ptime[2] counts launches; ptime[1] must hold
// ~0 before the first launch (the kernel leaves it so).
cudaError_t launch_gpanel_tc(int32_t bsub, const BlockMeta *meta,
                             SolverState *state, const int2 *tiles,
                             int32_t ntiles, int32_t nctas, int32_t *ctl,
                             unsigned long long *ptime,
                             const CUtensorMap *gmaps,
                             const CUtensorMap *xmaps, const float *in,
                             const float *in2, float *out, float *out_bf,
                             int mode, int step, int32_t *err,
                             cudaStream_t st);
// F_L = W^T F_s on the tensor cores (three tf32 passes): tiles are (block,
// first column l) pairs of 128 columns of W; wmaps one TMA map per block
// over W (32-row x 128-column boxes, plain layout), fmaps one per block over
// the B form of F_s (as xmaps), written by launch_bform_fs.
cudaError_t launch_project_tc(int32_t bsub, const BlockMeta *meta,
                              const int2 *tiles, int32_t ntiles,
                              const CUtensorMap *wmaps,
                              const CUtensorMap *fmaps, float *FL, int32_t kp,
                              int32_t *err, cudaStream_t st);
// B form of F_s (s_pad x kp per block, at fs_off) at 2 x_off of out_bf, in
// the panel layout with bsub columns (zero past kp); tiles as for the
// panel products.
cudaError_t launch_bform_fs(int32_t bsub, const BlockMeta *meta,
                            const int2 *tiles, int32_t ntiles, const float *Fs,
                            int32_t kp, float *out_bf, cudaStream_t st);
// BF16 form: F_L = W_h^T F_s from the bf16 copy of the centred blocks (the
// BF16 Gram's operand) with F_s split into bf16 hi and lo: tiles are (block,
// first column l) pairs of 128 columns; wmaps one TMA map per block over
// W_h (s128 rows x L_pad bf16, 128 x 64 boxes, plain layout); fmaps one per
// block over F_s's bf16 B form (64-value rows, 2 kn-row boxes, 128-byte
// swizzle), written by launch_bform_fs16 at fb_off. kn = kp rounded up to
// 16 (16 .. 64).
int64_t project_bf16_bform_elems(int32_t s_pad, int32_t kn);
cudaError_t launch_project_bf16(const BlockMeta *meta, const int2 *tiles,
                                int32_t ntiles, const CUtensorMap *wmaps,
                                const CUtensorMap *fmaps, float *FL,
                                int32_t kp, int32_t kn, int32_t *err,
                                cudaStream_t st);
// tiles: (block, first row) pairs of 128 rows of F_s.
cudaError_t launch_bform_fs16(const BlockMeta *meta, const int2 *tiles,
                              int32_t ntiles, const float *Fs, int32_t kp,
                              int32_t kn, __nv_bfloat16 *out, cudaStream_t st);
// B form of `in` for the blocks still running (tiles as above).
cudaError_t launch_bform(int32_t bsub, const BlockMeta *meta,
                         const SolverState *state, const int2 *tiles,
                         int32_t ntiles, const float *in, float *in_bf,
                         cudaStream_t st);

// row tiles: (block, first row) pairs, 64 rows each.
cudaError_t launch_init_panels(const EigBuffers &e, const int2 *rowtiles,
                               int32_t ntiles, cudaStream_t st);
// mode 0: Z = G X. mode 1: first Chebyshev step X -> Z. mode 2: step j >= 2.
cudaError_t launch_gpanel(const EigBuffers &e, const int2 *rowtiles,
                          int32_t ntiles, int32_t mode, int32_t step,
                          int32_t degree, const float *in, const float *in2,
                          float *out, cudaStream_t st);
cudaError_t launch_small_gram(const EigBuffers &e, const int2 *chunks,
                              int32_t nchunks, cudaStream_t st);
cudaError_t launch_rr_solve(const EigBuffers &e, cudaStream_t st);
cudaError_t launch_rotate(const EigBuffers &e, const int2 *rowtiles,
                          int32_t ntiles, cudaStream_t st);
cudaError_t launch_check(const EigBuffers &e, cudaStream_t st);
// F_s of every finished block from X and Finv, over 128-row tiles
// (block, first row) of F_s.
cudaError_t launch_publish_fs(const EigBuffers &e, const int2 *tiles,
                              int32_t ntiles, cudaStream_t st);
// The IF nodes of filter steps first .. first + n - 1.
struct LoopHandles {
  cudaGraphConditionalHandle h[62];
  int32_t first, n;
};
// The device-driven loop's decisions, after a Rayleigh-Ritz step: one more
// step while blocks are still iterating and ++count[0] < max; filter step
// first + j runs when some running block's degree (running[1]) reaches it.
// count[1] sums the steps opened.
cudaError_t launch_loopctl(const int32_t *running, int32_t *count,
                           int32_t max, cudaGraphConditionalHandle handle,
                           const LoopHandles &steps, cudaStream_t st);
// Copies running[0..1] to host-mapped memory `host` (device pointer), then
// writes `seq` to host[2], so a host thread that sees seq in host[2] reads
// the counters of this step.
cudaError_t launch_publish(const int32_t *running, int32_t *host, int32_t seq,
                           cudaStream_t st);

// F_L = W^T F_s on the FP32 SIMT pipes.
// ltiles: (block, first column l) pairs, kProjCols columns each.
constexpr int kProjCols = 64;
cudaError_t launch_project(const BlockMeta *meta, const int2 *ltiles,
                           int32_t ntiles, const float *W, const float *Fs,
                           float *FL, int32_t kp, cudaStream_t st);

// One tile's statistics of one factor column (kernels_finalize.cu).
struct ColPartial {
  double sq;        // float64 sum of squares over the tile's rows
  float absmax;     // largest |value| (first row on ties)
  float val;        // that value
  int32_t idx;      // its row
  int32_t pad;
};
// sigma_j = |F_L[:, j]| in float64 and the sign convention (the item-side
// vector's largest-|.| entry positive), then the flips applied to F_s and
// F_L. ltiles / stiles: (block, first row) pairs of 128 rows of F_L / F_s
// (BlockMeta pj0, npj / pt0, npt index them); lpart, spart: nltiles * kp
// and nstiles * kp partials; flip: nblocks * kp bytes.
cudaError_t launch_finalize(const BlockMeta *meta, int32_t nblocks,
                            const int2 *ltiles, int32_t nltiles,
                            const int2 *stiles, int32_t nstiles, float *Fs,
                            float *FL, double *sigma, int32_t kp,
                            ColPartial *lpart, ColPartial *spart,
                            unsigned char *flip, int64_t *launches,
                            cudaStream_t st);

// ---- blocked SGD, the paper's Algorithms 1-2 (kernels_sgd.cu) -------------
struct SgdRates {
  double a_user, b_user, a_item, b_item, a_ubias, b_ubias, a_ibias, b_ibias;
};
struct SgdRates32 {
  float a_user, b_user, a_item, b_item, a_ubias, b_ubias, a_ibias, b_ibias;
};

// Epoch order of the ratings: cnt and off hold (diag ? p : q) * m (+1)
// buckets; key, src, su, si, sx, and the local row and column sr, sc, hold
// nnz entries; range 2 per block.
cudaError_t launch_sgd_order(const GridDesc &g, int32_t nblocks, int64_t nnz,
                             const int32_t *u, const int32_t *i, const float *x,
                             unsigned long long *cnt, int64_t *off,
                             int64_t *key, int64_t *src, int32_t *su,
                             int32_t *si, float *sx, int32_t *sr, int32_t *sc,
                             int64_t *range, int32_t *err, cudaStream_t st);
// One schedule step: nb blocks (ids in `blocks`), one warp each.
cudaError_t launch_sgd_step(int32_t nb, const int32_t *blocks,
                            const int64_t *range, const int32_t *su,
                            const int32_t *si, const float *sx, int64_t nnz,
                            int32_t k, double *P, double *Q, double *bu,
                            double *bi, const SgdRates &r, int32_t *err,
                            cudaStream_t st);
// The float32 form: parameters as rows of k + 1 floats (k factors, then
// the bias), P32 m rows, Q32 n rows. narrow: float64 P, Q, bu, bi -> P32,
// Q32 (rounded to nearest); widen: back (exact).
cudaError_t launch_sgd_narrow(int64_t m, int64_t n, int32_t k, const double *P,
                              const double *Q, const double *bu,
                              const double *bi, float *P32, float *Q32,
                              cudaStream_t st);
cudaError_t launch_sgd_widen(int64_t m, int64_t n, int32_t k, const float *P32,
                             const float *Q32, double *P, double *Q,
                             double *bu, double *bi, cudaStream_t st);
// Shared memory a block of `rows` users and `cols` items stages.
inline size_t sgd_stage_bytes(int64_t rows, int64_t cols, int32_t k) {
  return (size_t)(rows + cols) * sizeof(float) * (size_t)(k + 2);
}
// One schedule step of the float32 form: nb blocks, one CTA each (its
// first warp walks the ratings). stage_bytes > 0: every block stages its
// rows and columns in that much shared memory (the largest block's
// sgd_stage_bytes); 0: the blocks work in global memory.
cudaError_t launch_sgd_step_f32(const GridDesc &g, int32_t nb,
                                const int32_t *blocks, const int64_t *range,
                                const int32_t *sr, const int32_t *sc,
                                const int32_t *su, const int32_t *si,
                                const float *sx, int64_t nnz, int32_t k,
                                float *P32, float *Q32, const SgdRates32 &r,
                                size_t stage_bytes, int32_t *err,
                                cudaStream_t st);
// Sum of squared training errors into *out (fixed order); partials holds
// kSqerrBlocks doubles.
cudaError_t launch_sgd_sqerr(int64_t nnz, const int32_t *u, const int32_t *i,
                             const float *x, int32_t k, const double *P,
                             const double *Q, const double *bu,
                             const double *bi, double *partials, double *out,
                             cudaStream_t st);
cudaError_t launch_sgd_predict(int64_t nq, const int32_t *u, const int32_t *i,
                               int32_t k, int64_t m, int64_t n,
                               const double *P, const double *Q,
                               const double *bu, const double *bi,
                               double *yhat, int32_t *err, cudaStream_t st);

// ---- prediction (kernels_predict.cu) ------------------------------------
struct PredictArgs {
  GridDesc g;
  const BlockMeta *meta;
  const float *mu;
  const float *Fs;
  const float *FL;
  int32_t kp;
  int32_t clamp;
  float lo, hi;
  int32_t owned_only = 0;   // squared errors: only blocks this context holds
};
cudaError_t launch_predict(const PredictArgs &a, int64_t nq, const int32_t *u,
                           const int32_t *i, float *yhat, int32_t *err,
                           cudaStream_t st);
// Squared-error partial sums: one float64 per CTA of a fixed grid, then a
// fixed-order final sum into out[0] and the number of queries summed into
// out[1]. partials must hold 2 kSqerrBlocks doubles (sums, then counts).
constexpr int kSqerrBlocks = 304;
cudaError_t launch_sqerr(const PredictArgs &a, int64_t nq, const int32_t *u,
                         const int32_t *i, const float *y, double *partials,
                         double *out, int32_t *err, cudaStream_t st);
// Rank-k reconstruction of block b on the tensor cores
// (kernels_reconstruct_tc.cu): out (mb x nb, row-major, device) = mu +
// P V^T from the block's factors; `host` is the block's metadata on the host
// (for the grid). A timed-out wait sets kErrTimeout in *err.
cudaError_t launch_reconstruct(const BlockMeta *meta, const BlockMeta &host,
                               int32_t b, const float *Fs, const float *FL,
                               int32_t kp, float mu, float *out, int32_t *err,
                               cudaStream_t st);

}  // namespace bsvd
