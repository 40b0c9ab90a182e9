/*
 * Oracle for tall-skinny QR — TEST INFRASTRUCTURE, NOT PRODUCT CODE.
 *
 * A plain, slow, obviously correct FP64 CPU restatement of what the TSQR hot path
 * computes. Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * this file; the CUDA library shares no code, header, table or helper with it.
 *
 * What it computes and where that is defined:
 *   - The QR factorization A = QR of an m-by-n real matrix, built from successive
 *     Householder reflections H = I - tau v v^T (paper §2.2). TSQR (paper §2.3)
 *     reaches the same factorization by another operation order: the reduce
 *     operator "QR of [R1; R2], keep R" is associative, so the R of the whole
 *     matrix equals the R of its row blocks' R factors. The oracle is therefore the
 *     plain definition: one unblocked Householder QR of the whole matrix.
 *   - The factorization is essentially unique: unique once the diagonal of R is
 *     made positive (paper §2.2, and the commutativity remark of §2.3). The oracle
 *     normalises signs with D = diag(sign(r_jj)), sign(0) = +1: R <- D R, Q <- Q D.
 *   - Implicit application of Q^T and Q, and explicit formation of the thin Q
 *     (paper §4, Table 2 counts Q as "R again"; Property 1).
 *   - Least squares min ||A x - b||: c = (Q^T b)[0:n], back substitution R x = c.
 *   - Mixed-precision least squares: an FP32 Householder QR used inside Bjorck's
 *     augmented-system iterative refinement with FP64 residuals and corrections
 *     (Bjorck 1967; Higham, "Accuracy and Stability of Numerical Algorithms",
 *     §20.5), and Bjorck's corrected semi-normal equations (Bjorck 1987), the
 *     refinement the library runs, iterated around the R of the mixed-precision TSQR
 *     (FP32 Householder QR of each leaf, FP64 QR of the stacked leaf triangles: the
 *     paper's TSQR of §2.3 with the library's precision pattern). The paper has no
 *     mixed-precision algorithm; these are the readings the library documents.
 *   - Error measures ||A - QR||_F / ||A||_F and ||Q^T Q - I||_F, accumulated with
 *     Neumaier's compensated summation (Neumaier 1974).
 *
 * Householder convention (Golub & Van Loan, "Matrix Computations", §5.1.2-5.1.3):
 * for x = A[j:m, j], alpha = x_0, sigma = ||x_{1:}||_2 (overflow-safe: scaled by
 * max |x_i|). If sigma == 0: tau = 0, H = I. Otherwise
 * beta = -sign(alpha) sqrt(alpha^2 + sigma^2) with sign(0) = +1, tau = (beta-alpha)/beta,
 * v = [1; x_{1:} / (alpha - beta)], and A[j,j] becomes beta. v_0 = 1 is implicit; the
 * rest of v is stored below the diagonal of A (unit lower trapezoidal V).
 *
 * Parallelism: the loops over the trailing columns may run on several OpenMP
 * threads. Each column's dot product and update stays a sequential loop in one
 * thread, so the arithmetic and its order are identical for any thread count.
 *
 * Layout: every matrix is column-major with a leading dimension (element (i,j)
 * at p[i + j*ld]). Every function here owns nothing and allocates only the
 * scratch it frees before returning.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define AT(p, i, j, ld) ((p)[(int64_t)(i) + (int64_t)(j) * (int64_t)(ld)])

/* ------------------------------------------------------------------ utilities */

/* Neumaier's compensated sum: add x to the running pair (s, c). */
static void kahan_add(double *s, double *c, double x) {
  double t = *s + x;
  if (fabs(*s) >= fabs(x))
    *c += (*s - t) + x;
  else
    *c += (x - t) + *s;
  *s = t;
}

/* Overflow-safe Euclidean norm: scale by the largest magnitude, then sum squares. */
static double nrm2_safe(int64_t len, const double *x) {
  double amax = 0.0;
  for (int64_t i = 0; i < len; i++) amax = fmax(amax, fabs(x[i]));
  if (amax == 0.0) return 0.0;
  double s = 0.0;
  for (int64_t i = 0; i < len; i++) {
    double t = x[i] / amax;
    s += t * t;
  }
  return amax * sqrt(s);
}

static float nrm2_safe_f32(int64_t len, const float *x) {
  float amax = 0.0f;
  for (int64_t i = 0; i < len; i++) amax = fmaxf(amax, fabsf(x[i]));
  if (amax == 0.0f) return 0.0f;
  float s = 0.0f;
  for (int64_t i = 0; i < len; i++) {
    float t = x[i] / amax;
    s += t * t;
  }
  return amax * sqrtf(s);
}

/* sign with sign(0) = +1 */
static double sgn(double a) { return a < 0.0 ? -1.0 : 1.0; }

/* ------------------------------------------------------------ Householder QR */

/* Apply H_j = I - tau v v^T (v_0 = 1 at row j, v_i = V[i,j] for i > j) to column c
 * of B (rows j..m-1). */
static void reflect_column(int64_t m, int64_t j, const double *V, int64_t ldv, double tau,
                           double *Bc) {
  if (tau == 0.0) return;
  double w = Bc[j];
  for (int64_t i = j + 1; i < m; i++) w += AT(V, i, j, ldv) * Bc[i];
  w *= tau;
  Bc[j] -= w;
  for (int64_t i = j + 1; i < m; i++) Bc[i] -= AT(V, i, j, ldv) * w;
}

/* Unblocked Householder QR in place (paper §2.2). On return R is in the upper
 * triangle of A, the reflector tails below the diagonal, tau[j] the scalars. */
void oracle_geqr2(int64_t m, int64_t n, double *A, int64_t lda, double *tau) {
  for (int64_t j = 0; j < n; j++) {
    double *x = &AT(A, j, j, lda);
    double alpha = x[0];
    double sigma = nrm2_safe(m - j - 1, x + 1);
    if (sigma == 0.0) {
      tau[j] = 0.0;
    } else {
      double beta = -sgn(alpha) * hypot(alpha, sigma);
      tau[j] = (beta - alpha) / beta;
      double denom = alpha - beta;
      for (int64_t i = 1; i < m - j; i++) x[i] = x[i] / denom;
      x[0] = beta;
    }
    double tj = tau[j];
#pragma omp parallel for schedule(static)
    for (int64_t k = j + 1; k < n; k++) reflect_column(m, j, A, lda, tj, &AT(A, 0, k, lda));
  }
}

/* B <- Q^T B with Q = H_0 H_1 ... H_{n-1}: H_0 is applied first. */
void oracle_apply_qt(int64_t m, int64_t n, const double *V, int64_t ldv, const double *tau,
                     int64_t k, double *B, int64_t ldb) {
  for (int64_t j = 0; j < n; j++) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < k; c++) reflect_column(m, j, V, ldv, tau[j], &AT(B, 0, c, ldb));
  }
}

/* B <- Q B: H_{n-1} is applied first. */
void oracle_apply_q(int64_t m, int64_t n, const double *V, int64_t ldv, const double *tau,
                    int64_t k, double *B, int64_t ldb) {
  for (int64_t j = n - 1; j >= 0; j--) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < k; c++) reflect_column(m, j, V, ldv, tau[j], &AT(B, 0, c, ldb));
  }
}

/* Thin Q = Q [I_n; 0] (m-by-n). */
void oracle_form_q(int64_t m, int64_t n, const double *V, int64_t ldv, const double *tau,
                   double *Q, int64_t ldq) {
  for (int64_t j = 0; j < n; j++)
    for (int64_t i = 0; i < m; i++) AT(Q, i, j, ldq) = (i == j) ? 1.0 : 0.0;
  oracle_apply_q(m, n, V, ldv, tau, n, Q, ldq);
}

/* R (n-by-n, zero below the diagonal) from the factored A. */
void oracle_extract_r(int64_t n, const double *A, int64_t lda, double *R, int64_t ldr) {
  for (int64_t j = 0; j < n; j++)
    for (int64_t i = 0; i < n; i++) AT(R, i, j, ldr) = (i <= j) ? AT(A, i, j, lda) : 0.0;
}

/* d[j] = sign(R_jj) (sign(0) = +1); R <- D R. */
void oracle_sign_normalise_r(int64_t n, double *R, int64_t ldr, double *d) {
  for (int64_t j = 0; j < n; j++) d[j] = sgn(AT(R, j, j, ldr));
  for (int64_t j = 0; j < n; j++)
    for (int64_t i = 0; i <= j; i++) AT(R, i, j, ldr) *= d[i];
}

/* rows 0..n-1 of B <- D B (for Q^T b) */
void oracle_scale_rows(int64_t n, const double *d, int64_t k, double *B, int64_t ldb) {
  for (int64_t c = 0; c < k; c++)
    for (int64_t i = 0; i < n; i++) AT(B, i, c, ldb) *= d[i];
}

/* columns of Q <- Q D */
void oracle_scale_cols(int64_t m, int64_t n, const double *d, double *Q, int64_t ldq) {
  for (int64_t j = 0; j < n; j++)
    for (int64_t i = 0; i < m; i++) AT(Q, i, j, ldq) *= d[j];
}

/* Back substitution R x = c, R upper triangular, x overwrites c. Returns 1 when some
 * R_ii == 0 (x is then left unfinished). */
int oracle_trsv_upper(int64_t n, const double *R, int64_t ldr, double *x) {
  for (int64_t i = n - 1; i >= 0; i--) {
    double s = x[i];
    for (int64_t l = i + 1; l < n; l++) s -= AT(R, i, l, ldr) * x[l];
    if (AT(R, i, i, ldr) == 0.0) return 1;
    x[i] = s / AT(R, i, i, ldr);
  }
  return 0;
}

/* Forward substitution R^T x = g (R^T lower triangular), x overwrites g. */
int oracle_trsv_upper_t(int64_t n, const double *R, int64_t ldr, double *x) {
  for (int64_t i = 0; i < n; i++) {
    double s = x[i];
    for (int64_t l = 0; l < i; l++) s -= AT(R, l, i, ldr) * x[l];
    if (AT(R, i, i, ldr) == 0.0) return 1;
    x[i] = s / AT(R, i, i, ldr);
  }
  return 0;
}

/* Least squares min ||A x - B||, one column of B at a time. A (m-by-n, m >= n) is
 * overwritten by its factorization and B by Q^T B. X is n-by-k. Returns 0, or 4
 * when R has an exactly zero diagonal entry. */
int oracle_lstsq(int64_t m, int64_t n, double *A, int64_t lda, int64_t k, double *B,
                 int64_t ldb, double *X, int64_t ldx) {
  double *tau = (double *)malloc(sizeof(double) * (size_t)n);
  oracle_geqr2(m, n, A, lda, tau);
  oracle_apply_qt(m, n, A, lda, tau, k, B, ldb);
  int rc = 0;
  for (int64_t c = 0; c < k; c++) {
    double *x = &AT(X, 0, c, ldx);
    for (int64_t i = 0; i < n; i++) x[i] = AT(B, i, c, ldb);
    if (oracle_trsv_upper(n, A, lda, x)) rc = 4;
  }
  free(tau);
  return rc;
}

/* --------------------------------------------------------------- error measures */

/* ||A - Q R||_F / ||A||_F with compensated sums; Q m-by-n, R n-by-n upper. */
double oracle_backward_error(int64_t m, int64_t n, const double *A, int64_t lda,
                             const double *Q, int64_t ldq, const double *R, int64_t ldr) {
  double s_num = 0.0, c_num = 0.0, s_den = 0.0, c_den = 0.0;
  for (int64_t j = 0; j < n; j++) {
    for (int64_t i = 0; i < m; i++) {
      double qr = 0.0, cq = 0.0;
      for (int64_t l = 0; l <= j; l++) kahan_add(&qr, &cq, AT(Q, i, l, ldq) * AT(R, l, j, ldr));
      double diff = AT(A, i, j, lda) - (qr + cq);
      kahan_add(&s_num, &c_num, diff * diff);
      kahan_add(&s_den, &c_den, AT(A, i, j, lda) * AT(A, i, j, lda));
    }
  }
  double den = s_den + c_den;
  return den > 0.0 ? sqrt(s_num + c_num) / sqrt(den) : sqrt(s_num + c_num);
}

/* ||Q^T Q - I||_F with compensated sums. */
double oracle_orth_error(int64_t m, int64_t n, const double *Q, int64_t ldq) {
  double s = 0.0, c = 0.0;
  for (int64_t a = 0; a < n; a++) {
    for (int64_t b = a; b < n; b++) {
      double g = 0.0, cg = 0.0;
      for (int64_t i = 0; i < m; i++) kahan_add(&g, &cg, AT(Q, i, a, ldq) * AT(Q, i, b, ldq));
      double e = (g + cg) - (a == b ? 1.0 : 0.0);
      kahan_add(&s, &c, (a == b ? 1.0 : 2.0) * e * e);
    }
  }
  return sqrt(s + c);
}

/* ------------------------------------------------- FP32 Householder (mixed) */

static void reflect_column_f32(int64_t m, int64_t j, const float *V, int64_t ldv, float tau,
                               float *Bc) {
  if (tau == 0.0f) return;
  float w = Bc[j];
  for (int64_t i = j + 1; i < m; i++) w += AT(V, i, j, ldv) * Bc[i];
  w *= tau;
  Bc[j] -= w;
  for (int64_t i = j + 1; i < m; i++) Bc[i] -= AT(V, i, j, ldv) * w;
}

/* The same Householder QR as oracle_geqr2, every operation in FP32. */
void oracle_geqr2_f32(int64_t m, int64_t n, float *A, int64_t lda, float *tau) {
  for (int64_t j = 0; j < n; j++) {
    float *x = &AT(A, j, j, lda);
    float alpha = x[0];
    float sigma = nrm2_safe_f32(m - j - 1, x + 1);
    if (sigma == 0.0f) {
      tau[j] = 0.0f;
    } else {
      float beta = -(alpha < 0.0f ? -1.0f : 1.0f) * hypotf(alpha, sigma);
      tau[j] = (beta - alpha) / beta;
      float denom = alpha - beta;
      for (int64_t i = 1; i < m - j; i++) x[i] = x[i] / denom;
      x[0] = beta;
    }
    float tj = tau[j];
#pragma omp parallel for schedule(static)
    for (int64_t k = j + 1; k < n; k++)
      reflect_column_f32(m, j, A, lda, tj, &AT(A, 0, k, lda));
  }
}

void oracle_apply_qt_f32(int64_t m, int64_t n, const float *V, int64_t ldv, const float *tau,
                         float *b) {
  for (int64_t j = 0; j < n; j++) reflect_column_f32(m, j, V, ldv, tau[j], b);
}

void oracle_apply_q_f32(int64_t m, int64_t n, const float *V, int64_t ldv, const float *tau,
                        float *b) {
  for (int64_t j = n - 1; j >= 0; j--) reflect_column_f32(m, j, V, ldv, tau[j], b);
}

/*
 * Mixed-precision least squares by augmented-system iterative refinement
 * (Bjorck 1967; Higham §20.5). The system [I A; A^T 0][r; x] = [b; 0] is refined
 * with FP64 residuals; each correction is solved through an FP32 QR A ~ Q [R; 0]:
 *   f = b - r - A x,  g = -A^T r                       (FP64)
 *   [d1; d2] = Q^T f                                   (FP32 reflectors)
 *   h = R^{-T} g,  dx = R^{-1} (d1 - h)                (FP64, R promoted)
 *   dr = Q [h; d2]                                     (FP32 reflectors)
 *   x += dx, r += dr                                   (FP64)
 * Start: x0 = R^{-1} (Q^T b)[0:n], r0 = b - A x0. Stops when ||dx|| <= tol ||x|| or
 * after max_steps corrections. One right-hand side b (length m); x (n) and r (m)
 * are outputs. hist[s] receives ||dx||/||x|| of step s (length max_steps, may be
 * NULL). Returns the number of corrections taken, or -4 if R is singular.
 */
int oracle_lstsq_refine_mixed(int64_t m, int64_t n, const double *A, int64_t lda,
                              const double *b, int32_t max_steps, double tol, double *x,
                              double *r, double *hist) {
  float *A32 = (float *)malloc(sizeof(float) * (size_t)(m * n));
  float *tau = (float *)malloc(sizeof(float) * (size_t)n);
  float *w32 = (float *)malloc(sizeof(float) * (size_t)m);
  double *R = (double *)malloc(sizeof(double) * (size_t)(n * n));
  double *f = (double *)malloc(sizeof(double) * (size_t)m);
  double *g = (double *)malloc(sizeof(double) * (size_t)n);
  double *dx = (double *)malloc(sizeof(double) * (size_t)n);
  int steps = 0;
  for (int64_t j = 0; j < n; j++)
    for (int64_t i = 0; i < m; i++) A32[i + j * m] = (float)AT(A, i, j, lda);
  oracle_geqr2_f32(m, n, A32, m, tau);
  for (int64_t j = 0; j < n; j++)
    for (int64_t i = 0; i < n; i++) R[i + j * n] = (i <= j) ? (double)A32[i + j * m] : 0.0;

  /* x0 = R^{-1} (Q^T b)[0:n] */
  for (int64_t i = 0; i < m; i++) w32[i] = (float)b[i];
  oracle_apply_qt_f32(m, n, A32, m, tau, w32);
  for (int64_t i = 0; i < n; i++) x[i] = (double)w32[i];
  if (oracle_trsv_upper(n, R, n, x)) { steps = -4; goto done; }
  /* r0 = b - A x0 */
  for (int64_t i = 0; i < m; i++) {
    double s = b[i];
    for (int64_t j = 0; j < n; j++) s -= AT(A, i, j, lda) * x[j];
    r[i] = s;
  }
  for (int32_t s = 0; s < max_steps; s++) {
    for (int64_t i = 0; i < m; i++) {
      double t = b[i] - r[i];
      for (int64_t j = 0; j < n; j++) t -= AT(A, i, j, lda) * x[j];
      f[i] = t;
    }
    for (int64_t j = 0; j < n; j++) {
      double t = 0.0;
      for (int64_t i = 0; i < m; i++) t -= AT(A, i, j, lda) * r[i];
      g[j] = t;
    }
    for (int64_t i = 0; i < m; i++) w32[i] = (float)f[i];
    oracle_apply_qt_f32(m, n, A32, m, tau, w32);            /* [d1; d2] */
    if (oracle_trsv_upper_t(n, R, n, g)) { steps = -4; goto done; } /* g <- h */
    for (int64_t i = 0; i < n; i++) dx[i] = (double)w32[i] - g[i];
    oracle_trsv_upper(n, R, n, dx);
    for (int64_t i = 0; i < n; i++) w32[i] = (float)g[i];     /* [h; d2] */
    oracle_apply_q_f32(m, n, A32, m, tau, w32);
    double nx = 0.0, ndx = 0.0;
    for (int64_t i = 0; i < n; i++) {
      x[i] += dx[i];
      nx += x[i] * x[i];
      ndx += dx[i] * dx[i];
    }
    for (int64_t i = 0; i < m; i++) r[i] += (double)w32[i];
    double rel = nx > 0.0 ? sqrt(ndx / nx) : sqrt(ndx);
    if (hist) hist[s] = rel;
    steps = s + 1;
    if (rel <= tol) break;
  }
done:
  free(A32); free(tau); free(w32); free(R); free(f); free(g); free(dx);
  return steps;
}

/*
 * Negative control: "x-only" refinement x += R^{-1} (Q^T (b - A x))[0:n] with the
 * same FP32 QR. Its fixed point carries the FP32 perturbation of the pseudo-inverse,
 * so for an inconsistent system with kappa(A) ~ 1e4 it stalls far above FP64
 * accuracy. Same arguments as oracle_lstsq_refine_mixed (no r).
 */
int oracle_lstsq_refine_x_only(int64_t m, int64_t n, const double *A, int64_t lda,
                               const double *b, int32_t max_steps, double *x, double *hist) {
  float *A32 = (float *)malloc(sizeof(float) * (size_t)(m * n));
  float *tau = (float *)malloc(sizeof(float) * (size_t)n);
  float *w32 = (float *)malloc(sizeof(float) * (size_t)m);
  double *R = (double *)malloc(sizeof(double) * (size_t)(n * n));
  double *dx = (double *)malloc(sizeof(double) * (size_t)n);
  int steps = 0;
  for (int64_t j = 0; j < n; j++)
    for (int64_t i = 0; i < m; i++) A32[i + j * m] = (float)AT(A, i, j, lda);
  oracle_geqr2_f32(m, n, A32, m, tau);
  for (int64_t j = 0; j < n; j++)
    for (int64_t i = 0; i < n; i++) R[i + j * n] = (i <= j) ? (double)A32[i + j * m] : 0.0;
  for (int64_t i = 0; i < n; i++) x[i] = 0.0;
  for (int32_t s = 0; s < max_steps; s++) {
    for (int64_t i = 0; i < m; i++) {
      double t = b[i];
      for (int64_t j = 0; j < n; j++) t -= AT(A, i, j, lda) * x[j];
      w32[i] = (float)t;
    }
    oracle_apply_qt_f32(m, n, A32, m, tau, w32);
    for (int64_t i = 0; i < n; i++) dx[i] = (double)w32[i];
    if (oracle_trsv_upper(n, R, n, dx)) { steps = -4; break; }
    double nx = 0.0, ndx = 0.0;
    for (int64_t i = 0; i < n; i++) {
      x[i] += dx[i];
      nx += x[i] * x[i];
      ndx += dx[i] * dx[i];
    }
    if (hist) hist[s] = nx > 0.0 ? sqrt(ndx / nx) : sqrt(ndx);
    steps = s + 1;
  }
  free(A32); free(tau); free(w32); free(R); free(dx);
  return steps;
}

/*
 * R of the mixed-precision TSQR (the library's precision pattern for the mixed path on
 * the paper's TSQR, §2.3): the rows are split into leaves of h rows (the last leaf takes the
 * remainder; one leaf when m < 2h), each leaf is rounded to FP32 and factored by the FP32
 * Householder QR, and the stacked leaf triangles (promoted to FP64) are factored by the
 * FP64 Householder QR, whose R is returned (n-by-n, any diagonal signs, zeros below).
 * Every tree shape gives the same R up to rounding (the reduce operator is associative),
 * so one combine of all leaves stands for any tree. Requires h >= n.
 */
void oracle_r_mixed(int64_t m, int64_t n, const double *A, int64_t lda, int64_t h, double *R, int64_t ldr) {
  const int64_t P = m / h > 0 ? m / h : 1;
  double *S = (double *)malloc(sizeof(double) * (size_t)(P * n * n));
  double *tau = (double *)malloc(sizeof(double) * (size_t)n);
  float *L = (float *)malloc(sizeof(float) * (size_t)((m - (P - 1) * h) * n));
  float *tau32 = (float *)malloc(sizeof(float) * (size_t)n);
  const int64_t lds = P * n;
  for (int64_t l = 0; l < P; l++) {
    const int64_t r0 = l * h, rows = (l == P - 1) ? m - r0 : h;
    for (int64_t j = 0; j < n; j++)
      for (int64_t i = 0; i < rows; i++) L[i + j * rows] = (float)AT(A, r0 + i, j, lda);
    oracle_geqr2_f32(rows, n, L, rows, tau32);
    for (int64_t j = 0; j < n; j++)
      for (int64_t i = 0; i < n; i++) AT(S, l * n + i, j, lds) = (i <= j) ? (double)L[i + j * rows] : 0.0;
  }
  oracle_geqr2(lds, n, S, lds, tau);
  oracle_extract_r(n, S, lds, R, ldr);
  free(S); free(tau); free(L); free(tau32);
}

/*
 * Mixed-precision least squares by corrected semi-normal equations, iterated
 * (Bjorck, "Stability analysis of the method of seminormal equations for linear least
 * squares problems", 1987; Higham, "Accuracy and Stability", §20.6). This is the
 * refinement the library runs; the paper has no mixed-precision algorithm. R is the R
 * of the mixed-precision TSQR with 128-row FP32 leaves (oracle_r_mixed); every other
 * operation is FP64. From x = 0:
 *   r = b - A x,  g = A^T r,  R^T y = g,  R d = y,  x <- x + d.
 * Stopping rule (the library's reading): stop after the step whose ||d|| / ||x|| is
 * <= 1e-15; or, from the second step on, once ||d|| / ||x|| times rho / (1 - rho) is
 * <= tol with rho < 1/2, rho the largest ratio of successive corrections seen so far;
 * or, from the third step on, once a correction exceeds half the previous one; or after
 * max_steps steps. One right-hand side b (length m); x (n) is the output and hist[s]
 * (length max_steps, may be NULL) receives ||d|| / ||x|| of step s. Returns the number
 * of steps taken, or -4 if R is singular.
 */
int oracle_lstsq_refine_csne(int64_t m, int64_t n, const double *A, int64_t lda, const double *b,
                             int32_t max_steps, double tol, double *x, double *hist) {
  double *R = (double *)malloc(sizeof(double) * (size_t)(n * n));
  double *r = (double *)malloc(sizeof(double) * (size_t)m);
  double *y = (double *)malloc(sizeof(double) * (size_t)n);
  double *h = (double *)malloc(sizeof(double) * (size_t)(max_steps > 0 ? max_steps : 1));
  int steps = 0;
  oracle_r_mixed(m, n, A, lda, n > 128 ? n : 128, R, n);
  for (int64_t i = 0; i < n; i++) x[i] = 0.0;
  for (int32_t s = 0; s < max_steps; s++) {
    for (int64_t i = 0; i < m; i++) {          /* r = b - A x */
      double t = b[i];
      for (int64_t j = 0; j < n; j++) t -= AT(A, i, j, lda) * x[j];
      r[i] = t;
    }
    for (int64_t j = 0; j < n; j++) {          /* g = A^T r */
      double t = 0.0;
      for (int64_t i = 0; i < m; i++) t += AT(A, i, j, lda) * r[i];
      y[j] = t;
    }
    if (oracle_trsv_upper_t(n, R, n, y) || oracle_trsv_upper(n, R, n, y)) { steps = -4; break; }
    double nx = 0.0, nd = 0.0;
    for (int64_t i = 0; i < n; i++) {
      x[i] += y[i];
      nx += x[i] * x[i];
      nd += y[i] * y[i];
    }
    const double ratio = nx > 0.0 ? sqrt(nd / nx) : (nd > 0.0 ? 1.0 : 0.0);
    h[s] = ratio;
    if (hist) hist[s] = ratio;
    steps = s + 1;
    if (ratio <= 1e-15) break;
    if (s >= 1) {
      double rho = 0.0;
      for (int32_t q = 1; q <= s; q++)
        if (h[q - 1] > 0.0) rho = fmax(rho, h[q] / h[q - 1]);
      if (s >= 2 && ratio > 0.5 * h[s - 1]) break;
      if (rho < 0.5 && ratio * rho / (1.0 - rho) <= tol) break;
    }
  }
  free(R); free(r); free(y); free(h);
  return steps;
}
