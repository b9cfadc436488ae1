/*
 * bsvd.h: C ABI of the block-SVD recommender library (libbsvd.so).
 *
 * The library runs one method on one GPU: the block-based truncated SVD
 * recommender of Bhavana, Kumar and Padmanabhan, "Block based Singular
 * Value Decomposition approach to matrix factorization for recommender
 * systems" (arXiv 1907.07410).
 *
 *   1. bsvd_partition: scatter the training ratings into a p x q grid of
 *      dense blocks (Section 3, Eq. "datax"), centre each block on its
 *      mean rating and fill missing cells with that mean (so they become 0).
 *   2. bsvd_factor: truncated rank-k SVD of every block (Section 2, Eq. 1
 *      and the rank-k truncation after it).
 *   3. bsvd_predict / bsvd_rmse: predict held-out ratings as
 *      mu_b + p_u . q_i (Section 2.1, Eq. 2) and score them by RMSE
 *      (Section 5, Table 1 "Test RMSE").
 *
 * Conventions shared by every call:
 *   - Ids are 0-based. A rating is observed when it is listed in the COO
 *     input. Ratings must be finite, |x| < 2^31, and the number of
 *     ratings times the largest |x| must stay below 2^31: the block sums,
 *     and their total (which gives an empty block's mean), are 64-bit
 *     fixed point with 32 fraction bits (otherwise BSVD_EINVAL). Block sums
 *     are then exact for every rating that is a multiple of 2^-32; in
 *     float32 that is every value with |x| >= 2^-9. Smaller non-zero
 *     ratings are rounded to a multiple of 2^-32 before they are summed.
 *   - Pointers named "host or device" may point to either kind of memory.
 *     The library asks the CUDA runtime which kind it is. Host data is
 *     copied to device buffers that the context owns; device data is used
 *     in place. The caller keeps ownership of every pointer it passes. The
 *     library never frees or keeps caller memory after a call returns.
 *   - Work is queued on the stream in the config (NULL: the legacy default
 *     stream). Every call below synchronises that stream before it
 *     returns, so its status also covers the GPU work it launched.
 *   - Errors come back as status codes; no exception crosses the ABI and the
 *     library never exits, aborts or traps on the device. After an error,
 *     bsvd_last_error() describes it. A device-side check that fails (an id
 *     out of range, a non-finite rating) sets a flag that the call reads
 *     back as BSVD_EINVAL.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef BSVD_H
#define BSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bsvd_ctx bsvd_ctx;

typedef enum {
    BSVD_OK = 0,
    BSVD_EINVAL = 1,    /* bad argument or bad input data */
    BSVD_ENOMEM = 2,    /* device or host allocation failed */
    BSVD_ECUDA = 3,     /* a CUDA runtime call failed */
    BSVD_ENOTCONV = 4,  /* an eigen-solver hit its iteration cap */
    BSVD_ETIMEOUT = 5,  /* a bounded device-side wait gave up; copies of
                           the kernel that gave up may still have been in
                           flight, so discard the context (and the CUDA
                           context's results) instead of retrying in place */
    BSVD_ESTATE = 6     /* call out of order (e.g. factor before partition) */
} bsvd_status;

typedef enum {
    BSVD_FP32 = 0,      /* float32 result: exact tensor-core Gram when the
                           ratings allow it, else FP32 SIMT Gram */
    BSVD_TF32 = 1,      /* single-pass TF32 tensor-core Gram (inputs
                           truncated to 10-bit mantissas); float32 solver,
                           float64 norms for sigma */
    BSVD_BF16 = 2       /* single-pass BF16 tensor-core Gram over a bf16
                           copy of the centred blocks (8-bit mantissas),
                           f32 accumulation; float32 solver and projection,
                           float64 norms for sigma */
} bsvd_precision;

typedef struct {
    int32_t precision;    /* bsvd_precision */
    int32_t clamp;        /* 1: clip predictions to [clamp_lo, clamp_hi] */
    float clamp_lo;
    float clamp_hi;
    int32_t oversample;   /* subspace columns beyond k; <= 0: default */
    int32_t cheb_degree;  /* largest Chebyshev filter degree, even;
                             <= 0: default (8) */
    int32_t max_iters;    /* subspace iterations cap; <= 0: default (30) */
    int32_t max_sweeps;   /* Jacobi sweeps cap per small solve; <= 0: 30 */
    int32_t profile;      /* 1: time each phase with CUDA events */
    int32_t gram_path;    /* BSVD_FP32 only (the others always use their
                             tensor-core Gram). 0: tensor cores when exact,
                             else FP32 SIMT; 1: FP32 SIMT always; 2: tensor
                             cores or BSVD_EINVAL from bsvd_factor */
    double tol;           /* residual |G v - theta v| <= tol * theta_1;
                             <= 0: default, 1e-5 for BSVD_FP32, 1e-4 for
                             BSVD_TF32 and 5e-4 for BSVD_BF16 (their Gram
                             products already carry errors near 1e-3
                             relative, and the bf16 copy of the data
                             limits the BF16 form's agreement with the
                             float32 problem to about 2e-3, so a tighter
                             residual buys no accuracy) */
    uint64_t seed;        /* seed of the start basis */
    void *stream;         /* cudaStream_t, or NULL for the default stream */
    int32_t panel_path;   /* panel products G X of the eigen-solver and
                             the projection F_L = W^T F_s:
                             0: tensor cores (three tf32 passes, float32
                             accuracy); 1: FP32 SIMT */
    int32_t loop;         /* eigen loop: 0 (default) device-driven from
                             the second bsvd_factor of a block layout on
                             (one CUDA graph whose loop a kernel ends; the
                             first factorisation of a layout runs the
                             host-driven loop, since a layout seen once
                             may never repeat); 1 always host-driven
                             (per-step phase times); 2 always the graph */
} bsvd_config;

/* Fill *cfg with the defaults listed above. */
void bsvd_config_default(bsvd_config *cfg);

/*
 * Create a context on the current CUDA device. cfg may be NULL (defaults).
 * Errors: BSVD_EINVAL (bad config), BSVD_ECUDA (no usable device),
 * BSVD_ENOMEM.
 */
bsvd_status bsvd_create(const bsvd_config *cfg, bsvd_ctx **out);

/* Free the context and every device buffer it owns. NULL is ignored. */
void bsvd_destroy(bsvd_ctx *ctx);

/* Description of the last error on this context ("" if none). */
const char *bsvd_last_error(const bsvd_ctx *ctx);

/*
 * Partition (Section 3, Eq. "datax") plus block means and the dense,
 * centred blocks.
 *
 * m, n       users and items of the rating matrix X (m x n); m, n >= 1.
 * nnz        number of training ratings (>= 0).
 * u, i, x    host or device arrays of nnz entries: user id, item id and
 *            rating. A (u, i) pair must not repeat (not checked).
 * p, q       block rows and block columns, 1 <= p <= m, 1 <= q <= n.
 * row_bounds host array of p + 1 increasing positions with row_bounds[0]
 *            = 0 and row_bounds[p] = m; block row bi holds row positions
 *            [row_bounds[bi], row_bounds[bi+1]). NULL selects the paper's
 *            equal blocks: ceil(m/p) rows each, the last holding the rest.
 * col_bounds the same for the q block columns over n items.
 * row_perm   host or device array of m entries, a permutation mapping user
 *            id -> row position; NULL means position = id.
 * col_perm   the same for items (n entries).
 *
 * Block b = bi * q + bj. Its mean mu_b is the exact sum of its training
 * ratings divided by their count in float64, then rounded to float32. An
 * empty block takes the global training mean (0 if nnz = 0). The dense
 * block holds float32(x - mu_b) at observed cells and 0 elsewhere.
 * A new partition discards any previous partition and factors.
 * Errors: BSVD_EINVAL (bad sizes, bounds or permutation; an id out of
 * range; a non-finite or too large rating), BSVD_ENOMEM, BSVD_ECUDA.
 */
bsvd_status bsvd_partition(bsvd_ctx *ctx, int64_t m, int64_t n, int64_t nnz,
                           const int32_t *u, const int32_t *i,
                           const float *x, int32_t p, int32_t q,
                           const int64_t *row_bounds,
                           const int64_t *col_bounds,
                           const int32_t *row_perm, const int32_t *col_perm);

/*
 * Partition a batch of independent rating matrices (Section 3's blocks
 * used one by one; each is factorised as its own block). The nb matrices
 * are stacked block-diagonally: matrix b owns rows [row_bounds[b],
 * row_bounds[b+1]) and columns [col_bounds[b], col_bounds[b+1]) of one
 * row_bounds[nb] x col_bounds[nb] matrix, and only these nb diagonal blocks
 * exist (block b is matrix b). u, i, x as in bsvd_partition, in the
 * stacked coordinates; a rating outside the diagonal blocks is an error.
 * row_bounds, col_bounds: host arrays of nb + 1 non-decreasing positions
 * starting at 0. Predictions take ids in the same stacked coordinates.
 * Errors as bsvd_partition.
 */
bsvd_status bsvd_partition_diag(bsvd_ctx *ctx, int32_t nb,
                                const int64_t *row_bounds,
                                const int64_t *col_bounds, int64_t nnz,
                                const int32_t *u, const int32_t *i,
                                const float *x);

/*
 * Uneven grid cut at rating-activity quantiles, for bsvd_partition (the
 * batched form; the paper's own grid, Section 3 Eq. "datax", has equal
 * blocks, which on long-tailed data leaves a few blocks holding most
 * ratings). Users are ordered by their number of training ratings, busiest
 * first, lower id first on ties; row_perm[u] is user u's position. Block
 * row bound g (0 < g < p) is the smallest position j whose preceding users
 * hold at least g / p of the nnz ratings, parts * C_j >= g * nnz in exact
 * integers; row_bounds[0] = 0 and row_bounds[p] = m. Items and the q block
 * columns likewise. The results plug into bsvd_partition unchanged.
 * m, n, nnz, u, i, p, q  as in bsvd_partition (x is not needed); nnz must
 *            be below 2^32 and 1 <= p <= m, 1 <= q <= n.
 * row_perm, col_perm     host or device arrays of m and n entries, written.
 * row_bounds, col_bounds host arrays of p + 1 and q + 1 entries, written.
 * Errors: BSVD_EINVAL (bad sizes, an id out of range), BSVD_ENOMEM,
 * BSVD_ECUDA.
 */
bsvd_status bsvd_quantile_grid(bsvd_ctx *ctx, int64_t m, int64_t n,
                               int64_t nnz, const int32_t *u,
                               const int32_t *i, int32_t p, int32_t q,
                               int32_t *row_perm, int32_t *col_perm,
                               int64_t *row_bounds, int64_t *col_bounds);

/*
 * bsvd_quantile_grid followed by bsvd_partition in one call, for the
 * batched form: the activity-quantile grid of (u, i) (same rule as
 * bsvd_quantile_grid) and the partition of (u, i, x) on it. Host ratings
 * are uploaded once (x while the grid is being cut), and the permutations
 * stay on the device.
 * m, n, nnz, u, i, x, p, q  as in bsvd_partition (u, i, x host or device);
 *            nnz must be below 2^32 and 1 <= p <= m, 1 <= q <= n.
 * row_bounds, col_bounds    host arrays of p + 1 and q + 1 entries that
 *            receive the grid's bounds, or NULL.
 * Errors: as bsvd_quantile_grid and bsvd_partition.
 */
bsvd_status bsvd_partition_quantile(bsvd_ctx *ctx, int64_t m, int64_t n,
                                    int64_t nnz, const int32_t *u,
                                    const int32_t *i, const float *x,
                                    int32_t p, int32_t q, int64_t *row_bounds,
                                    int64_t *col_bounds);

/*
 * Truncated SVD of every block (Section 2, Eq. 1 and the rank-k truncation
 * after it): keep the k_eff = min(k, min(m_b, n_b)) largest singular values
 * of each centred block B_b and their singular vectors.
 *
 * The library forms the Gram matrix of the block's shorter side and finds
 * its top eigenpairs by Chebyshev-filtered subspace iteration with
 * Rayleigh-Ritz steps solved by Jacobi. Factors stay on the device.
 * With BSVD_FP32 the Gram runs on the tensor cores, exactly, when every
 * rating minus its block's rounded mean is a small integer (integer rating
 * scales), else on the FP32 SIMT pipes; gram_path in the config can force
 * either. BSVD_TF32 and BSVD_BF16 run a single reduced-precision product
 * on the tensor cores.
 * k >= 0; k = 0 keeps no factor (predictions are then the block means).
 * The limit is k <= 56.
 * Errors: BSVD_ESTATE (no partition), BSVD_EINVAL (k out of range),
 * BSVD_ENOTCONV (some block hit the iteration cap; its factors are still
 * stored and usable), BSVD_ENOMEM, BSVD_ECUDA.
 */
bsvd_status bsvd_factor(bsvd_ctx *ctx, int32_t k);

/*
 * bsvd_factor with a rank per block: ks is a host array of one k per block
 * (p*q entries, or nb after bsvd_partition_diag), each in [0, 56].
 */
bsvd_status bsvd_factor_ks(bsvd_ctx *ctx, const int32_t *ks);

/*
 * Predict nq ratings (Section 2.1, Eq. 2): yhat = mu_b + P_b[r,:] . V_b[c,:]
 * with P_b = U_k S_k, clipped to [clamp_lo, clamp_hi] when clamp = 1.
 * u, i: host or device arrays of nq ids. yhat: host or device array of nq
 * floats, written by the call. nq >= 0.
 * Errors: BSVD_ESTATE (no factors), BSVD_EINVAL (id out of range).
 */
bsvd_status bsvd_predict(bsvd_ctx *ctx, int64_t nq, const int32_t *u,
                         const int32_t *i, float *yhat);

/*
 * Root mean squared error of the predictions for nq held-out ratings y
 * (Section 5, Table 1 "Test RMSE"): sqrt(sum (yhat - y)^2 / nq). The
 * squared errors are summed in float64 in a fixed order, so the result is
 * the same on every run. Every query counts, including those of blocks a
 * shard does not hold (bsvd_set_owned), which predict the block mean; a
 * shard reports its part with bsvd_sqerr instead. u, i, y: host or device
 * arrays of nq entries; nq >= 1. *out_rmse: host double.
 * Errors: BSVD_ESTATE, BSVD_EINVAL.
 */
bsvd_status bsvd_rmse(bsvd_ctx *ctx, int64_t nq, const int32_t *u,
                      const int32_t *i, const float *y, double *out_rmse);

/*
 * Restrict the context to a subset of the blocks, for sharding one matrix
 * over several GPUs (Section 3's blocks are independent: a block's factors
 * need only its own ratings, so each GPU can hold and factorise its own
 * blocks). owned: host array of nblocks flags (nonzero: held), one per
 * block of the next partition (p * q, or nb after bsvd_partition_diag);
 * nblocks = 0 (owned may be NULL) holds every block again. The next
 * partition still counts every block and computes every block mean, but
 * stores dense blocks only for the held ones; bsvd_factor factorises only
 * those (the others keep k_eff = 0, so their predictions are the block
 * means). bsvd_sqerr then sums the squared errors of the held blocks'
 * queries. Takes effect at the next partition (a mask of the wrong length
 * is rejected there with BSVD_EINVAL); discards any partition and factors.
 * Errors: BSVD_EINVAL.
 */
bsvd_status bsvd_set_owned(bsvd_ctx *ctx, int32_t nblocks,
                           const uint8_t *owned);

/*
 * The held-out error of the blocks this context holds (see bsvd_set_owned;
 * every block when no mask is set): *out_sum = sum of (yhat - y)^2 over the
 * queries whose block is held, in float64 in a fixed order, and
 * *out_count = the number of those queries. Summed over the shards, these
 * give the RMSE of Section 5, sqrt(sum / count). u, i, y: host or device
 * arrays of nq entries, nq >= 0. out_sum, out_count: host.
 * Errors: BSVD_ESTATE (no factors), BSVD_EINVAL (an id out of range).
 */
bsvd_status bsvd_sqerr(bsvd_ctx *ctx, int64_t nq, const int32_t *u,
                       const int32_t *i, const float *y, double *out_sum,
                       int64_t *out_count);

/*
 * Grid information after a partition: number of blocks and the count and
 * mean of each. counts (int64) and mu (float): host arrays of p*q entries,
 * either may be NULL.
 */
bsvd_status bsvd_block_stats(bsvd_ctx *ctx, int32_t *nblocks,
                             int64_t *counts, float *mu);

/*
 * Copy one block's results to host memory. Any output pointer may be NULL.
 *   mb, nb    block shape; keff retained rank; mu the block mean.
 *   sigma     keff singular values, descending (float64 norms |B v_i|).
 *   P         mb x keff, row-major: U_k S_k (user side).
 *   V         nb x keff, row-major: V_k (item side, unit columns). Each
 *             pair (P_i, V_i) has the sign that makes the largest-|.|
 *             entry of V_i positive.
 *   dense     mb x nb, row-major float32: the centred dense block as
 *             stored on the device (needs only a partition). The BF16 form
 *             (with the tensor-core panel path) stores only the bf16
 *             rounding of each cell, so that is what it returns.
 * A block another shard holds (bsvd_set_owned) reports keff = 0 and has
 * no dense block (BSVD_EINVAL when dense is asked for).
 * Errors: BSVD_ESTATE, BSVD_EINVAL (b out of range).
 */
bsvd_status bsvd_get_block(bsvd_ctx *ctx, int32_t b, int32_t *mb,
                           int32_t *nb, int32_t *keff, float *mu,
                           double *sigma, float *P, float *V, float *dense);

/*
 * Rank-k reconstruction of block b (the low-rank matrix of Section 2):
 * out[r * nb + c] = (add_mean ? mu_b : 0) + P[r,:] . V[c,:], for the
 * mb x nb block, computed on the tensor cores in 128 x 128 tiles (three
 * tf32 products of the factors' hi and lo parts: float32-level accuracy).
 * out: host or device array of mb * nb floats, owned by the caller.
 * Errors: BSVD_ESTATE (no factors), BSVD_EINVAL (b out of range, a block
 * another shard holds), BSVD_ETIMEOUT (a device-side wait gave up: discard
 * the context).
 */
bsvd_status bsvd_reconstruct(bsvd_ctx *ctx, int32_t b, int32_t add_mean,
                             float *out);

/*
 * Per-block solver report after bsvd_factor (host arrays of p*q entries,
 * any may be NULL): Rayleigh-Ritz steps used, 1 where the block converged,
 * Jacobi sweeps summed over the steps, SM clock cycles spent in the
 * Rayleigh-Ritz kernel (3 per block: partial sums + Cholesky QR + H',
 * Jacobi, ordering + output) summed over the steps, the last
 * relative residual max_i |G v_i - theta_i v_i| / theta_1 over the k_eff
 * wanted pairs (converged means <= tol), and the number of panel products
 * G X run for the block (each 2 s_pad^2 b multiply-adds' worth of work).
 */
bsvd_status bsvd_factor_report(bsvd_ctx *ctx, int32_t *iters,
                               int32_t *converged, int32_t *sweeps,
                               int64_t *cycles, float *resid,
                               int32_t *products);

/*
 * Phase timings of the last calls, in milliseconds of device time between
 * CUDA events on the context's stream (needs profile = 1 in the config):
 *   ms[0] partition (count, means, scatter)   ms[1] Gram products
 *   ms[2] subspace iteration (eigen-solve)    ms[3] projection and norms
 *   ms[4] prediction / squared-error sum
 *   ms[5] inside ms[2]: the tensor-core panel products' own device time
 *         (each launch's span, first CTA start to last CTA end, summed on
 *         the device; 0 on the FP32 SIMT panel path)
 *   ms[6] inside ms[2]: Rayleigh-Ritz kernels (Grams, solve, rotate,
 *         check); with the loop in a graph, the rest of ms[2]
 *   ms[7] the rest of ms[2] (start basis, host round trips between steps)
 * Phases the last calls did not run read as 0. ms: host array of 8.
 */
bsvd_status bsvd_phase_times(bsvd_ctx *ctx, double *ms);

/*
 * Number of kernels this context has launched since it was created (every
 * launch of the library's own kernels; memory copies and sets excluded).
 * Returns -1 for a NULL context.
 */
int64_t bsvd_kernel_launches(const bsvd_ctx *ctx);

/*
 * Which Gram kernel the last bsvd_factor ran: 1 FP32 SIMT, 2 tensor cores
 * (exact), 3 tensor cores (single-pass tf32), 4 tensor cores (single-pass
 * bf16), 0 none yet (or k = 0), -1 for a NULL context.
 */
int32_t bsvd_gram_path(const bsvd_ctx *ctx);

/*
 * How the last bsvd_factor ran its eigen loop: 1 host-driven, 2 one CUDA
 * graph with the loop decided on the device (see bsvd_config.loop), 0 no
 * factorisation yet, -1 for a NULL context.
 */
int32_t bsvd_loop_form(const bsvd_ctx *ctx);

/*
 * Launches of the tensor-core panel products G X in the last bsvd_factor
 * (counted on the device, so also inside a graph), -1 for a NULL context.
 * Their summed device time is bsvd_phase_times' ms[5].
 */
int64_t bsvd_panel_launches(const bsvd_ctx *ctx);

/*
 * ---- The paper's own method: blocked SGD (Algorithms 1-2) ----------------
 *
 * The biased latent-factor model of Section 2.2 (Eq. 3):
 *   x_ui ~ p_u . q_i + bu_u + bi_i,
 * fitted by stochastic gradient descent (Eq. 10-13) block by block.
 *   * Schedule (Section 3, Figure 2): the blocks of the last bsvd_partition
 *     grid are visited in steps of blocks that share no block row and no
 *     block column: step s holds blocks ((j + s) mod p, j), j < q, when
 *     p >= q, else (i, (i + s) mod q), i < p. The blocks of a step run at
 *     once, one warp each.
 *   * Within a block (Algorithm 2): its ratings row by row, then column by
 *     column. For each rating, with err = x - bu - bi - p . q:
 *       bu += a_ubias (err - b_ubias bu),  bi += a_ibias (err - b_ibias bi),
 *       p_f += a_user (err q_f - b_user p_f),
 *       q_f += a_item (err p_f - b_item q_f)   (p_f before this rating).
 *     Where Algorithm 2 and Eq. 10-13 differ, this follows the equations:
 *     each bias is regularised by itself.
 *   * Epochs (Algorithm 1): up to max_steps passes over all blocks; after
 *     each, the training RMSE is measured and training stops once it
 *     improved by less than delta.
 * Arithmetic (the precision field):
 *   * BSVD_SGD_FP64 (the default): float64 with one rounding per operation
 *     (no fused multiply-add) and the dot product summed over f = 0 .. k-1
 *     in order, so results equal a sequential float64 implementation bit
 *     for bit. A block's walk is a chain of dependent float64 operations.
 *   * BSVD_SGD_FP32: the same operations in the same order in float32 (no
 *     fused multiply-add), on float32 copies of P0, Q0 (rounded to nearest)
 *     and rates rounded to float32; each block stages its users' and items'
 *     parameters in shared memory when they fit (else it works in global
 *     memory). Results equal a sequential float32 implementation bit for
 *     bit. The RMSE, bsvd_sgd_predict and bsvd_sgd_get see the float32
 *     values widened to float64.
 */
typedef enum {
    BSVD_SGD_FP64 = 0,
    BSVD_SGD_FP32 = 1
} bsvd_sgd_precision;

typedef struct {
    double a_user, b_user;     /* user factors p_u (Eq. 10) */
    double a_item, b_item;     /* item factors q_i (Eq. 11) */
    double a_ubias, b_ubias;   /* user biases (Eq. 12) */
    double a_ibias, b_ibias;   /* item biases (Eq. 13) */
    double delta;              /* minimum RMSE improvement per epoch */
    int32_t k;                 /* latent factors, 1 .. 32 */
    int32_t max_steps;         /* STEPS of Algorithm 1, >= 0 */
    int32_t precision;         /* bsvd_sgd_precision */
} bsvd_sgd_params;

/*
 * The experiments' values (Section 5, "Hyper-parameters", SVD model):
 * user factors a = 0.019, b = 0.019; item factors a = 0.004, b = 0.019;
 * user biases a = 0.004, b = 0.019; item biases a = 0.013, b = 0.007;
 * delta = 1e-4; k = 13; max_steps = 100; precision BSVD_SGD_FP64.
 */
void bsvd_sgd_params_default(bsvd_sgd_params *prm);

/*
 * Lay out the training ratings in epoch order on the device, for the grid
 * of the last bsvd_partition or bsvd_partition_diag call (same ids; the
 * ratings themselves need not be the ones partitioned).
 * u, i, x: host or device arrays of nnz entries; nnz < 2^40, and no block
 * wider than 2^23 columns. Repeated (u, i) cells are kept, in input order.
 * Errors: BSVD_ESTATE (no partition), BSVD_EINVAL (sizes, an id out of
 * range or off the block diagonal), BSVD_ENOMEM, BSVD_ECUDA.
 */
bsvd_status bsvd_sgd_prepare(bsvd_ctx *ctx, int64_t nnz, const int32_t *u,
                             const int32_t *i, const float *x);

/*
 * Algorithm 1 from factors P0 (m x k) and Q0 (n x k), row-major float64,
 * host or device (the starting values are the caller's: the paper draws
 * them at random), and zero biases. The model stays on the device.
 * rmse: host array of max_steps + 1 doubles, or NULL: the training RMSE
 * before the first epoch, then after each epoch run. *steps_run (may be
 * NULL): epochs run.
 * Errors: BSVD_ESTATE (no bsvd_sgd_prepare), BSVD_EINVAL (parameters),
 * BSVD_ENOMEM, BSVD_ECUDA.
 */
bsvd_status bsvd_sgd_train(bsvd_ctx *ctx, const bsvd_sgd_params *prm,
                           const double *P0, const double *Q0, double *rmse,
                           int32_t *steps_run);

/*
 * Eq. 3 for nq (user, item) pairs of the trained model:
 * yhat = (sum_f p_uf q_if, in f order) + bu_u + bi_i. u, i: host or device
 * arrays; yhat: host or device array of nq doubles.
 * Errors: BSVD_ESTATE (not trained), BSVD_EINVAL (an id out of range).
 */
bsvd_status bsvd_sgd_predict(bsvd_ctx *ctx, int64_t nq, const int32_t *u,
                             const int32_t *i, double *yhat);

/*
 * Copy the trained model to host arrays (any may be NULL): P (m x k), Q
 * (n x k), row-major, bu (m), bi (n).
 * Errors: BSVD_ESTATE (not trained), BSVD_ECUDA.
 */
bsvd_status bsvd_sgd_get(bsvd_ctx *ctx, double *P, double *Q, double *bu,
                         double *bi);

/*
 * Block counts and block means of a rating matrix, for callers that cannot
 * allocate device memory during the call (the paper has no counterpart:
 * this serves deployment, not the method). A serving process that has
 * handed all of its device memory to its own pool, or a real-time loop
 * whose memory is fixed before it starts, cannot call cudaMalloc; the
 * context-based bsvd_partition does (it owns its buffers). This entry
 * point allocates nothing: its scratch (per-block rating sums, block
 * bounds, the largest |rating|, an error word; about 96 KiB) is one
 * file-scope __device__ array that every GPU that loads the library holds
 * until the process exits.
 *
 * Same grid and means as bsvd_partition with equal blocks (NULL bounds and
 * permutations): counts[b] and mu[b] for b = bi * q + bj equal what
 * bsvd_block_stats returns after bsvd_partition on the same input.
 * m, n, nnz, p, q  as in bsvd_partition; p * q <= 4096, p, q <= 4096.
 * u, i, x          device arrays of nnz entries (host memory is rejected,
 *                  since staging it would need an allocation).
 * counts, mu       device arrays of p * q entries, written by the call.
 * stream           cudaStream_t (NULL: the legacy default stream); the call
 *                  reads an error word back and synchronises the stream
 *                  before returning, so it must never be made on a stream
 *                  that is being captured.
 * The first call on each device looks up the scratch array's device
 * address (once per device, with that device current); make that first
 * call before another thread starts a global-mode stream capture. The
 * address is kept for the life of the process: after cudaDeviceReset this
 * entry point must not be called again. Every call shares the array and
 * clears the parts it accumulates into; calls that overlap on the GPU
 * (other threads or streams, or work queued before this call finishes)
 * race on it and must not be made. Device pointers must belong to the
 * current device (or be managed memory).
 * Errors (status only, there is no context): BSVD_EINVAL (bad sizes, a
 * grid over the limit, a host pointer, an id out of range, a non-finite or
 * too large rating), BSVD_ECUDA.
 */
bsvd_status bsvd_block_means_noalloc(int64_t m, int64_t n, int64_t nnz,
                                     const int32_t *u, const int32_t *i,
                                     const float *x, int32_t p, int32_t q,
                                     int64_t *counts, float *mu,
                                     void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BSVD_H */
