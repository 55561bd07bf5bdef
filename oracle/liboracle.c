/*
 * Oracle: plain CPU FP64 kernels for the least-squares reference.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg use it.  It shares no code, header or table with the CUDA
 * library.
 *
 * Contents (all row-major, all FP64, no blocking):
 *   or_householder_qr : unblocked Householder QR, one reflector per column,
 *                       v = x + sign(x_1)||x|| e_1 normalised to unit length and
 *                       A <- A - 2 v (v^T A).  Householder QR is the
 *                       factorisation the paper's analysis assumes for the
 *                       sketch (Sec. 2.1; Lemma 6.3).
 *   or_apply_qt       : b <- Q^T b with the stored reflectors.
 *   or_backsub        : R x = y by back substitution (Sec. 6: "All triangular
 *                       solves ... are computed by back substitution").
 *   or_backsub_t      : R^T x = y by forward substitution.
 *   or_resid_dot2     : r = b - A x and g = A^T r, both evaluated with the
 *                       compensated dot product Dot2 (Ogita, Rump, Oishi,
 *                       SISC 2005), r returned as an unevaluated sum r_hi+r_lo
 *                       (used by the Karlson-Walden backward-error estimate).
 *
 * Parallelism: OpenMP splits only over independent outputs (columns of the
 * trailing matrix, rows of the residual), never inside one sum, so every
 * sum is accumulated in the textbook order whatever the thread count.
 * Build with -ffp-contract=off so no a*b+c is silently fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Error-free transformations (Knuth TwoSum; TwoProd via the exact fma). */
static inline void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}
static inline void two_prod(double a, double b, double *p, double *e) {
  double x = a * b;
  *e = fma(a, b, -x);
  *p = x;
}

/*
 * Householder QR of the m x n row-major matrix A (leading dimension lda),
 * m >= n.  On return the upper triangle of A holds R (below-diagonal entries
 * set to zero) and V (m x n row-major, leading dimension n) holds the unit
 * reflector vectors, V[i, k] = 0 for i < k.  A zero column gives v = 0 and
 * R_kk = 0.  Returns 0.
 */
int or_householder_qr(int64_t m, int64_t n, double *A, int64_t lda, double *V) {
  double *w = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  memset(V, 0, sizeof(double) * (size_t)m * (size_t)n);
  for (int64_t k = 0; k < n; k++) {
    double s = 0.0;
    for (int64_t i = k; i < m; i++) s += A[i * lda + k] * A[i * lda + k];
    double nx = sqrt(s);
    double x0 = A[k * lda + k];
    double sg = (x0 >= 0.0) ? 1.0 : -1.0;
    for (int64_t i = k; i < m; i++) V[i * n + k] = A[i * lda + k];
    V[k * n + k] += sg * nx;
    double sv = 0.0;
    for (int64_t i = k; i < m; i++) sv += V[i * n + k] * V[i * n + k];
    double nv = sqrt(sv);
    if (nv > 0.0) {
      for (int64_t i = k; i < m; i++) V[i * n + k] /= nv;
    } else {
      for (int64_t i = k; i < m; i++) V[i * n + k] = 0.0;
    }
    /* trailing columns j > k:  w_j = v^T A[k:, j],  A[k:, j] -= 2 v w_j */
    int64_t nt = n - k - 1;
    if (nt > 0 && nv > 0.0) {
#pragma omp parallel
      {
#ifdef _OPENMP
        extern int omp_get_thread_num(void);
        extern int omp_get_num_threads(void);
        int tid = omp_get_thread_num(), nth = omp_get_num_threads();
#else
        int tid = 0, nth = 1;
#endif
        int64_t chunk = (nt + nth - 1) / nth;
        int64_t j0 = k + 1 + (int64_t)tid * chunk;
        int64_t j1 = j0 + chunk;
        if (j1 > n) j1 = n;
        if (j0 < j1) {
          for (int64_t j = j0; j < j1; j++) w[j] = 0.0;
          for (int64_t i = k; i < m; i++) {
            double vi = V[i * n + k];
            const double *ai = A + i * lda;
            for (int64_t j = j0; j < j1; j++) w[j] += vi * ai[j];
          }
          for (int64_t i = k; i < m; i++) {
            double tv = 2.0 * V[i * n + k];
            double *ai = A + i * lda;
            for (int64_t j = j0; j < j1; j++) ai[j] -= tv * w[j];
          }
        }
      }
    }
    A[k * lda + k] = -sg * nx;
    for (int64_t i = k + 1; i < m; i++) A[i * lda + k] = 0.0;
  }
  free(w);
  return 0;
}

/* b <- Q^T b, applying the reflectors stored in V (m x n) in order k = 0..n-1. */
int or_apply_qt(int64_t m, int64_t n, const double *V, double *b) {
  for (int64_t k = 0; k < n; k++) {
    double w = 0.0;
    for (int64_t i = k; i < m; i++) w += V[i * n + k] * b[i];
    for (int64_t i = k; i < m; i++) b[i] -= 2.0 * V[i * n + k] * w;
  }
  return 0;
}

/* Solve R x = y (R upper triangular n x n, leading dimension ldr). x may alias y. */
int or_backsub(int64_t n, const double *R, int64_t ldr, const double *y, double *x) {
  for (int64_t i = n - 1; i >= 0; i--) {
    double s = y[i];
    for (int64_t j = i + 1; j < n; j++) s -= R[i * ldr + j] * x[j];
    x[i] = s / R[i * ldr + i];
  }
  return 0;
}

/* Solve R^T x = y (R upper triangular, so R^T lower). x may alias y. */
int or_backsub_t(int64_t n, const double *R, int64_t ldr, const double *y, double *x) {
  for (int64_t i = 0; i < n; i++) {
    double s = y[i];
    for (int64_t j = 0; j < i; j++) s -= R[j * ldr + i] * x[j];
    x[i] = s / R[i * ldr + i];
  }
  return 0;
}

/*
 * r = b - A x and g = A^T r with the compensated dot product Dot2.
 * r is returned as r_hi + r_lo (r_hi = fl(r), r_lo = the rounding remainder),
 * g_j = sum_i A_ij (r_hi,i + r_lo,i) evaluated with Dot2 and rounded once.
 * A is m x n row-major with leading dimension lda.
 */
int or_resid_dot2(int64_t m, int64_t n, const double *A, int64_t lda, const double *b,
                  const double *x, double *r_hi, double *r_lo, double *g) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; i++) {
    const double *ai = A + i * lda;
    double s = b[i], c = 0.0;
    for (int64_t j = 0; j < n; j++) {
      double p, ep, t, es;
      two_prod(ai[j], -x[j], &p, &ep);
      two_sum(s, p, &t, &es);
      s = t;
      c += ep + es;
    }
    double hi, lo;
    two_sum(s, c, &hi, &lo);
    r_hi[i] = hi;
    r_lo[i] = lo;
  }
#pragma omp parallel
  {
#ifdef _OPENMP
    extern int omp_get_thread_num(void);
    extern int omp_get_num_threads(void);
    int tid = omp_get_thread_num(), nth = omp_get_num_threads();
#else
    int tid = 0, nth = 1;
#endif
    int64_t chunk = (n + nth - 1) / nth;
    int64_t j0 = (int64_t)tid * chunk, j1 = j0 + chunk;
    if (j1 > n) j1 = n;
    if (j0 < j1) {
      int64_t w = j1 - j0;
      double *s = (double *)calloc((size_t)w * 2, sizeof(double));
      double *c = s + w;
      for (int64_t i = 0; i < m; i++) {
        const double *ai = A + i * lda;
        double rh = r_hi[i], rl = r_lo[i];
        for (int64_t j = j0; j < j1; j++) {
          double p, ep, t, es;
          two_prod(ai[j], rh, &p, &ep);
          two_sum(s[j - j0], p, &t, &es);
          s[j - j0] = t;
          c[j - j0] += ep + es + ai[j] * rl;
        }
      }
      for (int64_t j = j0; j < j1; j++) g[j] = s[j - j0] + c[j - j0];
      free(s);
    }
  }
  return 0;
}
