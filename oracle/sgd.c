/*
 * One pass of the paper's blocked stochastic gradient descent over a
 * sequence of ratings: the test oracle for Algorithms 1 and 2.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links or calls this
 * file. It shares no code with the CUDA library.
 *
 * Model (Section 2.2, Eq. 3): x_ui ~ p_u . q_i + bu_u + bi_i. For each
 * rating, in the order given (the caller lays the blocks out in schedule
 * order and each block row by row, as Algorithm 2 loops over rows, then
 * columns):
 *
 *   err = x - bu[u] - bi[i] - p_u . q_i          (dot product over f = 0..k-1)
 *   bu[u] <- bu[u] + a_ubias (err - b_ubias bu[u])       (Eq. 12)
 *   bi[i] <- bi[i] + a_ibias (err - b_ibias bi[i])       (Eq. 13)
 *   for each factor f, with the value of p_u[f] before this rating:
 *     p_u[f] <- p_u[f] + a_user (err q_i[f] - b_user p_u[f])   (Eq. 10)
 *     q_i[f] <- q_i[f] + a_item (err p_u[f] - b_item q_i[f])   (Eq. 11)
 *
 * Readings (Algorithm 2 and Eq. 10-13 disagree): each bias is
 * regularised by itself, as Eq. 12-13 write; the item-factor update uses the
 * user factor from before this rating, as Eq. 10-11 imply; the learning and
 * regularisation rates are named by the parameter they update.
 *
 * Arithmetic is float64, evaluated left to right as written, one rounding
 * per operation (compile without floating-point contraction).
 * oracle_sgd_pass_f32 is the same pass in float32, for the library's
 * float32 form.
 */
#include <float.h>
#include <stdint.h>

#if FLT_EVAL_METHOD != 0
#error "float expressions must be evaluated in float"
#endif

typedef struct {
  double a_user, b_user;    /* user factors */
  double a_item, b_item;    /* item factors */
  double a_ubias, b_ubias;  /* user biases */
  double a_ibias, b_ibias;  /* item biases */
} oracle_sgd_rates;

void oracle_sgd_pass(int64_t n, const int32_t *u, const int32_t *i,
                     const float *x, int32_t k, double *P, double *Q,
                     double *bu, double *bi, const oracle_sgd_rates *r) {
  for (int64_t t = 0; t < n; ++t) {
    double *p = P + (int64_t)u[t] * k;
    double *q = Q + (int64_t)i[t] * k;
    double dot = 0.0;
    for (int32_t f = 0; f < k; ++f) dot = dot + p[f] * q[f];
    const double err = (double)x[t] - bu[u[t]] - bi[i[t]] - dot;
    bu[u[t]] = bu[u[t]] + r->a_ubias * (err - r->b_ubias * bu[u[t]]);
    bi[i[t]] = bi[i[t]] + r->a_ibias * (err - r->b_ibias * bi[i[t]]);
    for (int32_t f = 0; f < k; ++f) {
      const double pf = p[f];
      p[f] = pf + r->a_user * (err * q[f] - r->b_user * pf);
      q[f] = q[f] + r->a_item * (err * pf - r->b_item * q[f]);
    }
  }
}

/*
 * The same pass in float32: the parameters are float arrays, the rates are
 * the float64 rates rounded to float32, and every operation rounds once to
 * float32, in the order of oracle_sgd_pass (C evaluates float expressions
 * in float on the targets this builds for: FLT_EVAL_METHOD 0).
 */
void oracle_sgd_pass_f32(int64_t n, const int32_t *u, const int32_t *i,
                         const float *x, int32_t k, float *P, float *Q,
                         float *bu, float *bi, const oracle_sgd_rates *r) {
  const float a_user = (float)r->a_user, b_user = (float)r->b_user;
  const float a_item = (float)r->a_item, b_item = (float)r->b_item;
  const float a_ubias = (float)r->a_ubias, b_ubias = (float)r->b_ubias;
  const float a_ibias = (float)r->a_ibias, b_ibias = (float)r->b_ibias;
  for (int64_t t = 0; t < n; ++t) {
    float *p = P + (int64_t)u[t] * k;
    float *q = Q + (int64_t)i[t] * k;
    float dot = 0.0f;
    for (int32_t f = 0; f < k; ++f) dot = dot + p[f] * q[f];
    const float err = x[t] - bu[u[t]] - bi[i[t]] - dot;
    bu[u[t]] = bu[u[t]] + a_ubias * (err - b_ubias * bu[u[t]]);
    bi[i[t]] = bi[i[t]] + a_ibias * (err - b_ibias * bi[i[t]]);
    for (int32_t f = 0; f < k; ++f) {
      const float pf = p[f];
      p[f] = pf + a_user * (err * q[f] - b_user * pf);
      q[f] = q[f] + a_item * (err * pf - b_item * q[f]);
    }
  }
}
