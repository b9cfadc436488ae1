/*
 * FP64 one-sided Jacobi SVD: the test oracle's factorisation step.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links or calls this
 * file. It shares no code with the CUDA library.
 *
 * Computes the singular value decomposition X = U S V^T of Section 2, Eq. 1:
 * U and V have orthonormal columns, S is diagonal, and s_1 >= s_2 >= ... >= 0.
 * (The text says "incremental order" but then writes s_1 >= s_2, so the
 * order is read as descending.) Truncating to the k largest values, as
 * Section 2 describes, is left to the caller.
 *
 * Method: one-sided (Hestenes) Jacobi. Column pairs (a_p, a_q) are
 * rotated until every pair is numerically orthogonal. The rotation angle
 * uses Rutishauser's formulas:
 *     zeta = (|a_q|^2 - |a_p|^2) / (2 a_p.a_q),
 *     t    = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
 *     c    = 1 / sqrt(1 + t^2),  s = c t,
 *     a_p <- c a_p - s a_q,  a_q <- s a_p + c a_q.
 * A pair is rotated only when |a_p.a_q| > tol |a_p| |a_q| with
 * tol = 1e-15 sqrt(m). This is the relative test of Demmel and Veselic
 * (1992). A column whose norm has fallen below tol |A|_F is zero to
 * working precision and is not rotated. Pairs are visited cyclically by
 * rows. The loop stops after a sweep with no rotation, or after max_sweeps
 * sweeps.
 *
 * Then sigma_i = |a_i|, u_i = a_i / sigma_i (zero when sigma_i == 0), and the
 * accumulated rotations form V. Columns are sorted by descending sigma. Ties
 * are kept in original column order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static double dot(const double *a, const double *b, int64_t m) {
    /* four partial sums; any order is a valid FP64 sum */
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    int64_t i = 0;
    for (; i + 4 <= m; i += 4) {
        s0 += a[i] * b[i];
        s1 += a[i + 1] * b[i + 1];
        s2 += a[i + 2] * b[i + 2];
        s3 += a[i + 3] * b[i + 3];
    }
    for (; i < m; ++i) s0 += a[i] * b[i];
    return (s0 + s1) + (s2 + s3);
}

static void rotate(double *a, double *b, int64_t m, double c, double s) {
    for (int64_t i = 0; i < m; ++i) {
        double x = a[i], y = b[i];
        a[i] = c * x - s * y;
        b[i] = s * x + c * y;
    }
}

typedef struct { double key; int idx; } sort_item;

static int cmp_desc(const void *pa, const void *pb) {
    const sort_item *a = pa, *b = pb;
    if (a->key > b->key) return -1;
    if (a->key < b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);   /* stable tie-break */
}

/*
 * A: m x n, column-major (column j at A + j*m), m >= n >= 0. Overwritten.
 * U: m x n column-major, out. S: n, out. V: n x n column-major, out.
 * Returns the number of sweeps used, or -1 if max_sweeps was reached
 * with rotations still happening, or -2 on bad arguments / no memory.
 */
int oracle_jacobi_svd(double *A, int64_t m, int64_t n, double *U, double *S,
                      double *V, int max_sweeps) {
    if (m < n || n < 0 || m < 0) return -2;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) V[j * n + i] = (i == j) ? 1.0 : 0.0;
    const double tol = 1e-15 * sqrt((double)(m > 0 ? m : 1));
    double fro2 = 0.0;
    for (int64_t j = 0; j < n; ++j) fro2 += dot(A + j * m, A + j * m, m);
    const double tiny2 = tol * tol * fro2;
    int sweeps = 0, converged = (n < 2);
    while (!converged && sweeps < max_sweeps) {
        int64_t rotations = 0;
        for (int64_t p = 0; p + 1 < n; ++p) {
            for (int64_t q = p + 1; q < n; ++q) {
                double *ap = A + p * m, *aq = A + q * m;
                double alpha = dot(ap, ap, m);
                double beta = dot(aq, aq, m);
                double gamma = dot(ap, aq, m);
                if (alpha <= tiny2 || beta <= tiny2 || gamma == 0.0 ||
                    fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta))
                    continue;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0 ? 1.0 : -1.0) /
                           (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = c * t;
                rotate(ap, aq, m, c, s);
                rotate(V + p * n, V + q * n, n, c, s);
                ++rotations;
            }
        }
        ++sweeps;
        if (rotations == 0) converged = 1;
    }
    sort_item *items = malloc(sizeof(sort_item) * (size_t)(n > 0 ? n : 1));
    double *Vs = malloc(sizeof(double) * (size_t)(n > 0 ? n * n : 1));
    if (!items || !Vs) { free(items); free(Vs); return -2; }
    for (int64_t j = 0; j < n; ++j) {
        items[j].key = sqrt(dot(A + j * m, A + j * m, m));
        items[j].idx = (int)j;
    }
    qsort(items, (size_t)n, sizeof(sort_item), cmp_desc);
    for (int64_t r = 0; r < n; ++r) {
        int64_t j = items[r].idx;
        double sg = items[r].key;
        S[r] = sg;
        for (int64_t i = 0; i < m; ++i)
            U[r * m + i] = sg > 0 ? A[j * m + i] / sg : 0.0;
        memcpy(Vs + r * n, V + j * n, sizeof(double) * (size_t)n);
    }
    memcpy(V, Vs, sizeof(double) * (size_t)(n * n));
    free(items);
    free(Vs);
    return converged ? sweeps : -1;
}
