/*
 * Oracle for the left / lower / no-transpose triangular solve  L X = alpha B.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file; only the test-suite, the smoke check and the CPU
 * baseline arm of the benchmark do.  It shares no code, header, table or helper
 * with the CUDA path.
 *
 * What it computes (Section 2.1, the forward-substitution formula, repeated in
 * Section 4.2.1):
 *
 *     x_ij = ( alpha * b_ij  -  sum_{k < i} a_ik * x_kj ) / a_ii
 *
 * for every column j independently (Section 4.2.1: columns of one row are
 * independent).  L is the lower triangle of A; with diag = unit the diagonal is
 * taken as 1 and never read, and the strict upper triangle is never read.
 *
 * Evaluation order.  Each column is swept in the column-oriented ("axpy")
 * order: x := alpha*b; for k = 0..m-1 { x_k := x_k / a_kk; x_i -= a_ik x_k
 * for i > k }.  For every i this performs exactly the operations of the
 * formula above, in the same ascending-k order, with the same roundings:
 * s_i = (((alpha b_i - a_i0 x_0) - a_i1 x_1) - ...) and then s_i / a_ii.
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 *
 * Complex arithmetic is written out: a*b = (ar br - ai bi, ar bi + ai br);
 * a/b by Smith's algorithm (R. L. Smith, "Algorithm 116: Complex division",
 * CACM 5(8), 1962).
 *
 * The backward-error checker forms residuals with compensated dot products
 * (the Dot2 algorithm of Ogita, Rump and Oishi, "Accurate sum and dot
 * product", SIAM J. Sci. Comput. 26(6), 2005), using Dekker's TwoProduct
 * (T. J. Dekker, 1971) so that no fused multiply-add is needed.
 *
 * OpenMP parallelises over columns (or batch instances) only; results do not
 * depend on the thread count.
 *
 * Matrices are column-major with leading dimensions lda, ldb (in elements).
 * Complex values are stored as interleaved (re, im) doubles.
 */
#include <stdint.h>
#include <stddef.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double re, im; } zv;

static zv z_mul(zv a, zv b) {
  zv r;
  r.re = a.re * b.re - a.im * b.im;
  r.im = a.re * b.im + a.im * b.re;
  return r;
}

static zv z_sub(zv a, zv b) {
  zv r;
  r.re = a.re - b.re;
  r.im = a.im - b.im;
  return r;
}

/* Smith (1962): scale by the larger component of the divisor. */
static zv z_div(zv a, zv b) {
  zv r;
  if (fabs(b.re) >= fabs(b.im)) {
    double t = b.im / b.re;
    double d = b.re + b.im * t;
    r.re = (a.re + a.im * t) / d;
    r.im = (a.im - a.re * t) / d;
  } else {
    double t = b.re / b.im;
    double d = b.re * t + b.im;
    r.re = (a.re * t + a.im) / d;
    r.im = (a.im * t - a.re) / d;
  }
  return r;
}

static int bad_args(int64_t m, int64_t n, int64_t lda, int64_t ldb) {
  if (m < 0 || n < 0) return 1;
  if (lda < (m > 1 ? m : 1) || ldb < (m > 1 ? m : 1)) return 1;
  return 0;
}

/* Real solve, one column j.  x is column j of B, overwritten in place. */
static void solve_col_d(int unit, int64_t m, double alpha, const double *A, int64_t lda, double *x) {
  for (int64_t i = 0; i < m; i++) x[i] = alpha * x[i];
  for (int64_t k = 0; k < m; k++) {
    if (!unit) x[k] = x[k] / A[k + k * lda];
    const double xk = x[k];
    const double *ak = A + k * lda;
    for (int64_t i = k + 1; i < m; i++) x[i] = x[i] - ak[i] * xk;
  }
}

static void solve_col_z(int unit, int64_t m, zv alpha, const zv *A, int64_t lda, zv *x) {
  for (int64_t i = 0; i < m; i++) x[i] = z_mul(alpha, x[i]);
  for (int64_t k = 0; k < m; k++) {
    if (!unit) x[k] = z_div(x[k], A[k + k * lda]);
    const zv xk = x[k];
    const zv *ak = A + k * lda;
    for (int64_t i = k + 1; i < m; i++) x[i] = z_sub(x[i], z_mul(ak[i], xk));
  }
}

/* alpha == 0: B := 0 and A is not referenced (the usual BLAS convention). */
int oracle_trsm_llnn_d(int unit, int64_t m, int64_t n, double alpha,
                       const double *A, int64_t lda, double *B, int64_t ldb) {
  if (bad_args(m, n, lda, ldb)) return 1;
  if (m == 0 || n == 0) return 0;
  if (alpha == 0.0) {
    for (int64_t j = 0; j < n; j++)
      for (int64_t i = 0; i < m; i++) B[i + j * ldb] = 0.0;
    return 0;
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < n; j++) solve_col_d(unit, m, alpha, A, lda, B + j * ldb);
  return 0;
}

int oracle_trsm_llnn_z(int unit, int64_t m, int64_t n, const double *alpha,
                       const double *A, int64_t lda, double *B, int64_t ldb) {
  if (bad_args(m, n, lda, ldb)) return 1;
  if (m == 0 || n == 0) return 0;
  zv al = {alpha[0], alpha[1]};
  zv *Bz = (zv *)B;
  if (al.re == 0.0 && al.im == 0.0) {
    for (int64_t j = 0; j < n; j++)
      for (int64_t i = 0; i < m; i++) { Bz[i + j * ldb].re = 0.0; Bz[i + j * ldb].im = 0.0; }
    return 0;
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < n; j++) solve_col_z(unit, m, al, (const zv *)A, lda, Bz + j * ldb);
  return 0;
}

/* ---------------------------------------------------------------------------
 * The other BLAS triangular-solve variants, by their definition (the paper
 * studies the left / lower / no-transpose case only; these extend it):
 *
 *   side 0 (left):   op(A) X = alpha B,  A is m x m
 *   side 1 (right):  X op(A) = alpha B,  A is n x n
 *   uplo 0 / 1:      the lower / upper triangle of A is referenced
 *   trans 0 / 1 / 2: op(A) = A, A^T, or A^H (conjugate transpose)
 *   unit:            the diagonal of A is taken as 1 and never read
 *
 * T(p, q) denotes op(A)'s entry.  Left: each column x of X solves T x = alpha b
 * by forward substitution when T is lower triangular and backward when it is
 * upper, x_i = (alpha b_i - sum_k T(i,k) x_k) / T(i,i) over the already solved
 * k, summed in ascending k.  Right: each row y of X solves y T = alpha b, i.e.
 * y_k = (alpha b_k - sum_l y_l T(l,k)) / T(k,k) over the solved l (ascending),
 * forward in k when T is upper, backward when lower.  Real data runs through
 * the same complex operations with zero imaginary parts, which round exactly
 * as the real ones.
 * ------------------------------------------------------------------------- */
static zv g_get(int cx, const double *A, int64_t lda, int64_t i, int64_t k) {
  zv v;
  if (cx) {
    v.re = A[2 * (i + k * lda)];
    v.im = A[2 * (i + k * lda) + 1];
  } else {
    v.re = A[i + k * lda];
    v.im = 0.0;
  }
  return v;
}

static zv g_op(int cx, int trans, const double *A, int64_t lda, int64_t p, int64_t q) {
  if (trans == 0) return g_get(cx, A, lda, p, q);
  zv v = g_get(cx, A, lda, q, p);
  if (trans == 2) v.im = -v.im;
  return v;
}

static void g_put(int cx, double *B, int64_t ldb, int64_t i, int64_t j, zv v) {
  if (cx) {
    B[2 * (i + j * ldb)] = v.re;
    B[2 * (i + j * ldb) + 1] = v.im;
  } else {
    B[i + j * ldb] = v.re;
  }
}

int oracle_trsm_general(int cx, int side, int uplo, int trans, int unit, int64_t m, int64_t n,
                        const double *alpha, const double *A, int64_t lda, double *B, int64_t ldb) {
  const int64_t na = side == 0 ? m : n; /* order of A */
  if (m < 0 || n < 0 || side < 0 || side > 1 || uplo < 0 || uplo > 1 || trans < 0 || trans > 2) return 1;
  if (lda < (na > 1 ? na : 1) || ldb < (m > 1 ? m : 1)) return 1;
  if (!cx && trans == 2) trans = 1; /* A^H = A^T for real A */
  if (m == 0 || n == 0) return 0;
  const zv al = {alpha[0], cx ? alpha[1] : 0.0};
  const int t_lower = (uplo == 0) != (trans != 0);
  if (al.re == 0.0 && al.im == 0.0) {
    const zv z = {0.0, 0.0};
    for (int64_t j = 0; j < n; j++)
      for (int64_t i = 0; i < m; i++) g_put(cx, B, ldb, i, j, z);
    return 0;
  }
  if (side == 0) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; j++) {
      for (int64_t t = 0; t < m; t++) {
        const int64_t i = t_lower ? t : m - 1 - t;
        zv s = z_mul(al, g_get(cx, B, ldb, i, j));
        const int64_t k0 = t_lower ? 0 : i + 1, k1 = t_lower ? i : m;
        for (int64_t k = k0; k < k1; k++) s = z_sub(s, z_mul(g_op(cx, trans, A, lda, i, k), g_get(cx, B, ldb, k, j)));
        if (!unit) s = z_div(s, g_op(cx, trans, A, lda, i, i));
        g_put(cx, B, ldb, i, j, s);
      }
    }
  } else {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < m; i++) {
      for (int64_t t = 0; t < n; t++) {
        const int64_t k = t_lower ? n - 1 - t : t;
        zv s = z_mul(al, g_get(cx, B, ldb, i, k));
        const int64_t l0 = t_lower ? k + 1 : 0, l1 = t_lower ? n : k;
        for (int64_t l = l0; l < l1; l++) s = z_sub(s, z_mul(g_get(cx, B, ldb, i, l), g_op(cx, trans, A, lda, l, k)));
        if (!unit) s = z_div(s, g_op(cx, trans, A, lda, k, k));
        g_put(cx, B, ldb, i, k, s);
      }
    }
  }
  return 0;
}

/* Only the listed columns of B (column indices cols[0..ncols-1]) are solved;
 * the others are left untouched.  Columns are independent, so each listed
 * column equals the corresponding column of a full solve. */
int oracle_trsm_llnn_cols_d(int unit, int64_t m, double alpha, const double *A, int64_t lda,
                            double *B, int64_t ldb, const int64_t *cols, int64_t ncols) {
  if (bad_args(m, ncols, lda, ldb)) return 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < ncols; c++) {
    double *x = B + cols[c] * ldb;
    if (alpha == 0.0) { for (int64_t i = 0; i < m; i++) x[i] = 0.0; continue; }
    solve_col_d(unit, m, alpha, A, lda, x);
  }
  return 0;
}

int oracle_trsm_llnn_cols_z(int unit, int64_t m, const double *alpha, const double *A, int64_t lda,
                            double *B, int64_t ldb, const int64_t *cols, int64_t ncols) {
  if (bad_args(m, ncols, lda, ldb)) return 1;
  zv al = {alpha[0], alpha[1]};
  zv *Bz = (zv *)B;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < ncols; c++) {
    zv *x = Bz + cols[c] * ldb;
    if (al.re == 0.0 && al.im == 0.0) {
      for (int64_t i = 0; i < m; i++) { x[i].re = 0.0; x[i].im = 0.0; }
      continue;
    }
    solve_col_z(unit, m, al, (const zv *)A, lda, x);
  }
  return 0;
}

/* Batch of independent solves (instance b: m[b] x m[b] A, m[b] x n[b] B,
 * packed back to back in A and B at element offsets offA[b], offB[b], with
 * lda = ldb = m[b]).  Complex data interleaved when is_complex. */
int oracle_trsm_llnn_batch(int is_complex, int unit, int64_t batch, const int64_t *m, const int64_t *n,
                           const double *alpha, const double *A, const int64_t *offA,
                           double *B, const int64_t *offB) {
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int64_t b = 0; b < batch; b++) {
    int64_t mb = m[b], nb = n[b], ld = mb > 1 ? mb : 1;
    if (mb < 0 || nb < 0) { err |= 1; continue; }
    if (mb == 0 || nb == 0) continue;
    if (!is_complex) {
      if (alpha[0] == 0.0) {
        for (int64_t e = 0; e < mb * nb; e++) B[offB[b] + e] = 0.0;
        continue;
      }
      for (int64_t j = 0; j < nb; j++)
        solve_col_d(unit, mb, alpha[0], A + offA[b], ld, B + offB[b] + j * ld);
    } else {
      zv al = {alpha[0], alpha[1]};
      zv *Bz = (zv *)(B + 2 * offB[b]);
      if (al.re == 0.0 && al.im == 0.0) {
        for (int64_t e = 0; e < mb * nb; e++) { Bz[e].re = 0.0; Bz[e].im = 0.0; }
        continue;
      }
      for (int64_t j = 0; j < nb; j++)
        solve_col_z(unit, mb, al, (const zv *)(A + 2 * offA[b]), ld, Bz + j * ld);
    }
  }
  return err;
}

/* ---------------------------------------------------------------------------
 * Error-free transformations (Knuth TwoSum, Dekker TwoProduct with Veltkamp's
 * split) and Dot2 accumulation, for the backward-error checker.
 * ------------------------------------------------------------------------- */
static void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}

static void split(double a, double *hi, double *lo) {
  const double factor = 134217729.0; /* 2^27 + 1 */
  double c = factor * a;
  double h = c - (c - a);
  *hi = h;
  *lo = a - h;
}

static void two_prod(double a, double b, double *p, double *e) {
  double ah, al, bh, bl;
  double x = a * b;
  split(a, &ah, &al);
  split(b, &bh, &bl);
  *e = al * bl - (((x - ah * bh) - al * bh) - ah * bl);
  *p = x;
}

typedef struct { double s, c; } acc2; /* Dot2 running sum and compensation */

static void acc_add(acc2 *a, double v) {
  double s, e;
  two_sum(a->s, v, &s, &e);
  a->s = s;
  a->c += e;
}

static void acc_fma(acc2 *a, double x, double y) { /* a += x*y */
  double p, ep, s, es;
  two_prod(x, y, &p, &ep);
  two_sum(a->s, p, &s, &es);
  a->s = s;
  a->c += ep + es;
}

static double acc_val(const acc2 *a) { return a->s + a->c; }

/* Normwise backward error
 *     eta = ||L X - alpha B||_F / ( ||L||_F ||X||_F + |alpha| ||B||_F )
 * L = lower triangle of A (unit diagonal when unit != 0).  Residual entries
 * are formed with Dot2; the norms in plain double (they only scale eta). */
double oracle_backward_error_d(int unit, int64_t m, int64_t n, double alpha,
                               const double *A, int64_t lda, const double *B, int64_t ldb,
                               const double *X, int64_t ldx) {
  double rr = 0.0, nl = 0.0, nx = 0.0, nb = 0.0;
  for (int64_t k = 0; k < m; k++)
    for (int64_t i = k; i < m; i++) {
      double v = (i == k && unit) ? 1.0 : A[i + k * lda];
      nl += v * v;
    }
#pragma omp parallel for reduction(+ : rr, nx, nb) schedule(dynamic, 1)
  for (int64_t j = 0; j < n; j++) {
    for (int64_t i = 0; i < m; i++) {
      acc2 a = {0.0, 0.0};
      for (int64_t k = 0; k < i; k++) acc_fma(&a, A[i + k * lda], X[k + j * ldx]);
      if (unit) acc_add(&a, X[i + j * ldx]);
      else acc_fma(&a, A[i + i * lda], X[i + j * ldx]);
      acc_fma(&a, -alpha, B[i + j * ldb]);
      double r = acc_val(&a);
      rr += r * r;
      nx += X[i + j * ldx] * X[i + j * ldx];
      nb += B[i + j * ldb] * B[i + j * ldb];
    }
  }
  double den = sqrt(nl) * sqrt(nx) + fabs(alpha) * sqrt(nb);
  return den > 0.0 ? sqrt(rr) / den : sqrt(rr);
}

double oracle_backward_error_z(int unit, int64_t m, int64_t n, const double *alpha,
                               const double *A, int64_t lda, const double *B, int64_t ldb,
                               const double *X, int64_t ldx) {
  const zv *Az = (const zv *)A, *Bz = (const zv *)B, *Xz = (const zv *)X;
  zv al = {alpha[0], alpha[1]};
  double rr = 0.0, nl = 0.0, nx = 0.0, nb = 0.0;
  for (int64_t k = 0; k < m; k++)
    for (int64_t i = k; i < m; i++) {
      if (i == k && unit) { nl += 1.0; continue; }
      zv v = Az[i + k * lda];
      nl += v.re * v.re + v.im * v.im;
    }
#pragma omp parallel for reduction(+ : rr, nx, nb) schedule(dynamic, 1)
  for (int64_t j = 0; j < n; j++) {
    for (int64_t i = 0; i < m; i++) {
      acc2 re = {0.0, 0.0}, im = {0.0, 0.0};
      for (int64_t k = 0; k <= i; k++) {
        zv a = (k == i && unit) ? (zv){1.0, 0.0} : Az[i + k * lda];
        zv x = Xz[k + j * ldx];
        acc_fma(&re, a.re, x.re);
        acc_fma(&re, -a.im, x.im);
        acc_fma(&im, a.re, x.im);
        acc_fma(&im, a.im, x.re);
      }
      zv b = Bz[i + j * ldb];
      acc_fma(&re, -al.re, b.re);
      acc_fma(&re, al.im, b.im);
      acc_fma(&im, -al.re, b.im);
      acc_fma(&im, -al.im, b.re);
      double r0 = acc_val(&re), r1 = acc_val(&im);
      rr += r0 * r0 + r1 * r1;
      zv xv = Xz[i + j * ldx];
      nx += xv.re * xv.re + xv.im * xv.im;
      nb += b.re * b.re + b.im * b.im;
    }
  }
  double den = sqrt(nl) * sqrt(nx) + hypot(al.re, al.im) * sqrt(nb);
  return den > 0.0 ? sqrt(rr) / den : sqrt(rr);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_num_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}
