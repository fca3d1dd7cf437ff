/*
 * CPU FP64 oracle for the LOBPCG eigensolver of arXiv 2305.06668.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test-suite, the smoke check and the CPU
 * baseline of the benchmark; never by the GPU library.  It is written for reading,
 * not for speed: every step follows the paper's Algorithms 1-3 in their order and
 * notation, with plain loops (OpenMP only spreads independent rows / matrix entries
 * over threads, which does not change any result).
 *
 * Readings of points the paper leaves open (each is also listed in the design notes):
 *  R1  Algorithm 1, initialisation: the initial Rayleigh-Ritz step solves a^[0] and
 *      forms R = AX - X lambda from the rotated X; the lock/exit test of the main loop
 *      is applied to this initial residual as well.
 *  R2  The initial block is orthonormalised with Algorithm 2 first (the initial
 *      Rayleigh-Ritz is a standard eigenproblem only for orthonormal X0).
 *  R3  ||X^T X - I|| and ||Y^T X|| are max-abs entry norms; Algorithm 2 stops after
 *      `ortho_cap` Cholesky-QR passes and Algorithm 3 after `ortho2_cap` projection
 *      passes (a cap hit is counted, not an error).
 *  R4  Shift of Sec. 3.2 / Algorithm 2: sigma_0 = 100 * eps * trace(M)
 *      (= 100 eps ||X||_F^2, which bounds ||M||_2), multiplied by 10 after every
 *      further failure, at most 8 shifted attempts; then an SVQB step (Stathopoulos &
 *      Wu) with eigenvalues floored at eps * max.
 *  R5  Algorithm 2 tests ||X^T X - I|| before each factorisation (so a successful call
 *      costs passes + 1 Gram matrices).  Algorithm 3 runs its body at least once
 *      (project, then ortho) and repeats while ||Y^T X|| > tau: the printed loop would
 *      otherwise return a non-orthonormal X whenever X~ happens to be orthogonal to Y.
 *  R6  Diagonal preconditioner (Sec. 2): w_ij = r_ij / delta with delta = d_i - lambda_j,
 *      replaced by sign(delta) * 1e-8 * max(1, |lambda_j|) when smaller than that in
 *      magnitude (sign(0) = +1).  Each column uses its own Ritz value.
 *  R7  Locking (Sec. 3.1): after each Rayleigh-Ritz step the longest prefix of converged
 *      pairs (in the new ascending order) is locked; locked vectors stay in X and in the
 *      Rayleigh-Ritz problem but get no new W or P.  The prefix is recomputed every
 *      step: the Rayleigh-Ritz step can move a lower, unconverged Ritz vector in front of
 *      a converged one, and that column must become active again.  Exit once the first
 *      k pairs are converged.
 *  R8  P coefficients (Sec. 3.1, Eq. (a_block)/(neweigv)): u~_p = u_x[:, act] minus the
 *      identity columns of the active indices in the X-block rows; then
 *      u_p = ortho(u~_p; u_x) in R^s with Algorithm 3.
 *  R9  The Rayleigh-Ritz matrix is symmetrised as (a + a^T) / 2 before the eigensolve.
 *  R10 Reported residual norms are recomputed with a fresh product A X at exit.
 *  R15 Algorithm 2 factors the diagonally scaled overlap D M D, D = diag(M)^{-1/2}, and
 *      sets X <- X D L^{-T} (scaled Cholesky-QR).  In exact arithmetic this is the same Q
 *      (the QR factor of X D equals that of X); in floating point it makes the shift of
 *      R4 (now 100 eps trace(D M D) = 100 eps p) relative to unit columns, so a column
 *      whose norm is at the rounding level of the others is still normalised.  Without
 *      it such a column (a P direction of a Ritz vector that did not move) stays
 *      unnormalised through every pass and breaks the orthonormality of V.
 *  R16 Algorithm 3 (and the Algorithm 2 inside it) may stop at a pass cap without having
 *      produced orthonormal columns orthogonal to Y.  Only then (a cap was hit during
 *      the call) are the columns whose largest overlap with Y is above sqrt(tau), or
 *      whose norm differs from 1 by more than sqrt(tau), dropped; the kept columns are
 *      packed to the front in their order.  When no cap is hit every column passed the
 *      tau tests and the rule cannot fire, so it never changes a run in which the
 *      paper's loops succeed.  It differs from dropping ill-conditioned directions
 *      during the orthogonalisation (Sec. 1, Duersch et al.): nothing is dropped while
 *      the shifted Cholesky-QR still works, only directions the loops could not make
 *      part of an orthonormal basis.  The cases that reach it are degenerate: a W~
 *      column that is exactly zero (an active pair whose residual is exactly zero; its
 *      direction is already in X), more columns than the complement of Y holds (u_p in
 *      R^s after a column was unlocked: s - m directions for a_act columns), both
 *      applied to W (n rows) and to u_p (s rows).  Kept, such a column would make V
 *      rank-deficient and give a spurious Ritz value with a vanishing vector.
 *  R14 A P direction exists only where x_j moved: the coefficient vector u~_p of column j,
 *      after projecting out u_x, is (I - u_x u_x^T) e_j; when it vanishes exactly (norm
 *      <= 1e-200, e.g. when the Rayleigh-Ritz coupling of a localised vector is exactly
 *      zero and its Jacobi column stays e_j) the column is dropped from P (P then has fewer
 *      than m_act columns).  A zero vector cannot be normalised by Algorithm 2, and in V it
 *      would produce a spurious Ritz value 0 with a zero "residual".  Columns that are
 *      merely small (rounding noise) are kept, as the printed algorithm does.
 *  R24 Tridiagonal preconditioner (Sec. 4.4): w_j = (T - lambda_j I)^{-1} r_j with T the
 *      diagonal and the first sub- and super-diagonals of A, solved by Gaussian
 *      elimination with partial pivoting between neighbouring rows (the scheme of
 *      LAPACK's tridiagonal solver).  A pivot smaller in magnitude than
 *      1e-8 * max(1, |lambda_j|) is replaced by that value with its sign (sign(0) = +1),
 *      the guard of R6.  With zero off-diagonals it is exactly the diagonal
 *      preconditioner of R6.
 */
#include "lobpcg_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EPS DBL_EPSILON

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ basic blocks */

/* Pairwise (recursive halving) summation of x_i * y_i: error grows like log2(n) eps. */
static double pairwise_dot(const double* x, const double* y, int64_t len) {
  if (len <= 32) {
    double s = 0.0;
    for (int64_t i = 0; i < len; ++i) s += x[i] * y[i];
    return s;
  }
  int64_t h = len / 2;
  return pairwise_dot(x, y, h) + pairwise_dot(x + h, y + h, len - h);
}

void oracle_gram(int64_t n, int p, const double* X, int q, const double* Y, double* C) {
  int64_t total = (int64_t)p * q;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t e = 0; e < total; ++e) {
    int i = (int)(e % p), j = (int)(e / p);
    C[i + (int64_t)j * p] = pairwise_dot(X + (int64_t)i * n, Y + (int64_t)j * n, n);
  }
}

/* Z = X U  (X: n x p, U: p x q, Z: n x q).  Z must not alias X. */
static void block_times_small(int64_t n, int p, const double* X, int q, const double* U,
                              double* Z) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < q; ++j) {
      double s = 0.0;
      for (int l = 0; l < p; ++l) s += X[i + (int64_t)l * n] * U[l + (int64_t)j * p];
      Z[i + (int64_t)j * n] = s;
    }
}

/* X <- X - Y C  (X: n x p, Y: n x q, C: q x p). */
static void block_minus_times(int64_t n, int p, double* X, int q, const double* Y,
                              const double* C) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < p; ++j) {
      double s = 0.0;
      for (int l = 0; l < q; ++l) s += Y[i + (int64_t)l * n] * C[l + (int64_t)j * q];
      X[i + (int64_t)j * n] -= s;
    }
}

void oracle_apply(const oracle_matrix* A, int p, const double* X, double* Y) {
  const int64_t n = A->n;
  if (A->dense) {
    /* y_i = sum_c a_ic x_c, with a_ic = dense[i + c*ld]; column-oriented sweep. */
    for (int j = 0; j < p; ++j) {
      const double* x = X + (int64_t)j * n;
      double* y = Y + (int64_t)j * n;
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t c = 0; c < n; ++c) s += A->dense[c + i * A->ld] * x[c]; /* a_ci = a_ic */
        y[i] = s;
      }
    }
    return;
  }
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < p; ++j) {
      double s = 0.0;
      for (int64_t e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e)
        s += A->val[e] * X[(int64_t)A->col_idx[e] + (int64_t)j * n];
      Y[i + (int64_t)j * n] = s;
    }
}

static double max_abs_minus_identity(int p, const double* M) {
  double worst = 0.0;
  for (int j = 0; j < p; ++j)
    for (int i = 0; i < p; ++i) {
      double v = fabs(M[i + j * p] - (i == j ? 1.0 : 0.0));
      if (!(v <= worst)) worst = v; /* NaN propagates as "large" */
    }
  return worst;
}

static double max_abs(int64_t len, const double* v) {
  double worst = 0.0;
  for (int64_t i = 0; i < len; ++i) {
    double a = fabs(v[i]);
    if (!(a <= worst)) worst = a;
  }
  return worst;
}

/* ----------------------------------------------------------- dense small kernels */

int oracle_cholesky(int p, double* M) {
  for (int j = 0; j < p; ++j) {
    double d = M[j + j * p];
    for (int l = 0; l < j; ++l) d -= M[j + l * p] * M[j + l * p];
    if (!(d > 0.0)) return j + 1;
    double ljj = sqrt(d);
    M[j + j * p] = ljj;
    for (int i = j + 1; i < p; ++i) {
      double s = M[i + j * p];
      for (int l = 0; l < j; ++l) s -= M[i + l * p] * M[j + l * p];
      M[i + j * p] = s / ljj;
    }
  }
  return 0;
}

/* X <- X L^{-T}: each row x solves z L^T = x, i.e. L z^T = x^T (forward substitution). */
static void right_solve_lower_transpose(int64_t n, int p, double* X, const double* L) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < p; ++j) {
      double s = X[i + (int64_t)j * n];
      for (int l = 0; l < j; ++l) s -= L[j + l * p] * X[i + (int64_t)l * n];
      X[i + (int64_t)j * n] = s / L[j + j * p];
    }
}

/* Cyclic-by-row Jacobi with the classical (smaller-angle) rotation, as in Golub & Van
 * Loan, Matrix Computations, Sec. 8.5 (sym.schur2 + cyclic sweep). */
int oracle_jacobi_eig(int s, const double* a_in, double* lam, double* U) {
  double* a = (double*)malloc(sizeof(double) * (size_t)s * s);
  double* vec = (double*)malloc(sizeof(double) * (size_t)s * s);
  int* order = (int*)malloc(sizeof(int) * (size_t)(s > 0 ? s : 1));
  memcpy(a, a_in, sizeof(double) * (size_t)s * s);
  for (int j = 0; j < s; ++j)
    for (int i = 0; i < s; ++i) vec[i + j * s] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int e = 0; e < s * s; ++e) fro += a[e] * a[e];
  fro = sqrt(fro);
  int sweeps = 0, converged = 0;
  for (; sweeps <= 100; ++sweeps) {
    double off = 0.0;
    for (int j = 0; j < s; ++j)
      for (int i = 0; i < s; ++i)
        if (i != j) off += a[i + j * s] * a[i + j * s];
    if (sqrt(off) <= 1e-15 * fro) {
      converged = 1;
      break;
    }
    for (int p = 0; p < s - 1; ++p)
      for (int q = p + 1; q < s; ++q) {
        double apq = a[p + q * s];
        if (apq == 0.0) continue;
        double tau = (a[q + q * s] - a[p + p * s]) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
        /* A <- A J: columns p and q */
        for (int i = 0; i < s; ++i) {
          double aip = a[i + p * s], aiq = a[i + q * s];
          a[i + p * s] = c * aip - sn * aiq;
          a[i + q * s] = sn * aip + c * aiq;
        }
        /* A <- J^T A: rows p and q */
        for (int j = 0; j < s; ++j) {
          double apj = a[p + j * s], aqj = a[q + j * s];
          a[p + j * s] = c * apj - sn * aqj;
          a[q + j * s] = sn * apj + c * aqj;
        }
        a[p + q * s] = 0.0;
        a[q + p * s] = 0.0;
        /* U <- U J */
        for (int i = 0; i < s; ++i) {
          double vip = vec[i + p * s], viq = vec[i + q * s];
          vec[i + p * s] = c * vip - sn * viq;
          vec[i + q * s] = sn * vip + c * viq;
        }
      }
  }
  /* ascending order, ties keep index order (stable insertion sort) */
  for (int i = 0; i < s; ++i) order[i] = i;
  for (int i = 1; i < s; ++i) {
    int key = order[i];
    int j = i - 1;
    while (j >= 0 && a[order[j] + order[j] * s] > a[key + key * s]) {
      order[j + 1] = order[j];
      --j;
    }
    order[j + 1] = key;
  }
  for (int j = 0; j < s; ++j) {
    lam[j] = a[order[j] + order[j] * s];
    memcpy(U + (size_t)j * s, vec + (size_t)order[j] * s, sizeof(double) * (size_t)s);
  }
  free(a);
  free(vec);
  free(order);
  return converged ? sweeps : -1;
}

/* ------------------------------------------------------ Algorithms 2 and 3 (Sec. 3.2) */

/* SVQB step (Stathopoulos & Wu), the fallback when even shifted Cholesky fails:
 * D = diag(M)^{-1/2}, D M D = Z Theta Z^T, X <- X D Z Theta^{-1/2}. */
void oracle_svqb(int64_t n, int p, double* X, const double* M) {
  if (p <= 0) return;
  double* dmd = (double*)malloc(sizeof(double) * (size_t)p * p);
  double* Z = (double*)malloc(sizeof(double) * (size_t)p * p);
  double* th = (double*)malloc(sizeof(double) * (size_t)p);
  double* Dv = (double*)malloc(sizeof(double) * (size_t)p);
  double* T = (double*)malloc(sizeof(double) * (size_t)p * p);
  double* Xc = (double*)malloc(sizeof(double) * (size_t)n * p);
  for (int i = 0; i < p; ++i) Dv[i] = M[i + i * p] > 0.0 ? 1.0 / sqrt(M[i + i * p]) : 0.0;
  for (int j = 0; j < p; ++j)
    for (int i = 0; i < p; ++i) dmd[i + j * p] = Dv[i] * M[i + j * p] * Dv[j];
  oracle_jacobi_eig(p, dmd, th, Z);
  double tmax = 0.0;
  for (int i = 0; i < p; ++i) tmax = fmax(tmax, th[i]);
  for (int j = 0; j < p; ++j) {
    double t = fmax(th[j], EPS * tmax);
    for (int i = 0; i < p; ++i) T[i + j * p] = Dv[i] * Z[i + j * p] / sqrt(t);
  }
  memcpy(Xc, X, sizeof(double) * (size_t)n * p);
  block_times_small(n, p, Xc, p, T, X);
  free(dmd), free(Z), free(th), free(Dv), free(T), free(Xc);
}

/* Algorithm 2.  With trim (Sec. 3.2, the estimate of ||L^{-T}|| that makes the final
 * re-check unnecessary, reading R17): after an unshifted pass whose scaled overlap
 * S = D M D = I + F has ||F||_F <= 1/2, ||L^{-T}||_2^2 = 1 / lambda_min(S) <= 1 / (1 - ||F||_F)
 * <= 2, so the new vectors are orthonormal to about twice the Gram's rounding and the
 * loop ends without forming X^T X again.  d2_first (nullable, p) receives diag of the
 * first X^T X (the squared input column norms) and *l2_first the bound on
 * ||L^{-T}||_2^2 of the first pass (1 when no pass was needed, HUGE_VAL after a shift or
 * an SVQB step): the error amplification Algorithm 3's growth factor needs. */
static int ortho_impl(int64_t n, int p, double* X, double tau, int cap, int trim, oracle_ortho_stats* st,
                      double* d2_first, double* l2_first) {
  if (l2_first) *l2_first = 1.0;
  if (p <= 0) return 0;
  double* M = (double*)malloc(sizeof(double) * (size_t)p * p);
  double* L = (double*)malloc(sizeof(double) * (size_t)p * p);
  int passes = 0;
  oracle_gram(n, p, X, p, X, M); /* M = X^T X */
  st->grams++;
  if (d2_first)
    for (int j = 0; j < p; ++j) d2_first[j] = M[j + j * p];
  for (;;) {
    if (max_abs_minus_identity(p, M) <= tau) break;
    if (passes >= cap) {
      st->cap_hits++;
      break;
    }
    ++passes;
    /* scaled overlap D M D, D = diag(M)^{-1/2}  (R15) */
    double* Dv = (double*)malloc(sizeof(double) * (size_t)p);
    double* Ms = (double*)malloc(sizeof(double) * (size_t)p * p);
    for (int i = 0; i < p; ++i) Dv[i] = M[i + i * p] > 0.0 ? 1.0 / sqrt(M[i + i * p]) : 1.0;
    for (int j = 0; j < p; ++j)
      for (int i = 0; i < p; ++i) Ms[i + j * p] = Dv[i] * M[i + j * p] * Dv[j];
    double fro_off = 0.0; /* ||F||_F, F = S - I */
    for (int j = 0; j < p; ++j)
      for (int i = 0; i < p; ++i) {
        const double f = Ms[i + j * p] - (i == j ? 1.0 : 0.0);
        fro_off += f * f;
      }
    fro_off = sqrt(fro_off);
    memcpy(L, Ms, sizeof(double) * (size_t)p * p);
    int fail = oracle_cholesky(p, L);
    const int shifted = fail != 0;
    if (fail) {
      /* level shift (Sec. 3.2), grown by 10x until the factorisation succeeds */
      double tr = 0.0;
      for (int i = 0; i < p; ++i) tr += Ms[i + i * p];
      double sigma = 100.0 * EPS * tr;
      for (int t = 0; t < 8 && fail; ++t, sigma *= 10.0) {
        memcpy(L, Ms, sizeof(double) * (size_t)p * p);
        for (int i = 0; i < p; ++i) L[i + i * p] += sigma;
        st->shifts++;
        fail = oracle_cholesky(p, L);
      }
    }
    free(Ms);
    if (passes == 1 && l2_first) *l2_first = (!shifted && fro_off < 1.0) ? 1.0 / (1.0 - fro_off) : HUGE_VAL;
    if (fail) {
      free(Dv);
      st->svqb++;
      oracle_svqb(n, p, X, M);
    } else {
      for (int j = 0; j < p; ++j)
        for (int64_t i = 0; i < n; ++i) X[i + (int64_t)j * n] *= Dv[j];
      free(Dv);
      right_solve_lower_transpose(n, p, X, L); /* X <- X D L^{-T} */
      if (trim && !shifted && fro_off <= 0.5) { /* R17: ||L^{-T}||^2 <= 2, no re-check */
        st->skipped_recheck++;
        break;
      }
    }
    oracle_gram(n, p, X, p, X, M); /* M = X^T X */
    st->grams++;
  }
  if (passes > st->cholqr_passes_max) st->cholqr_passes_max = passes;
  st->passes = passes;
  free(M);
  free(L);
  return passes;
}

/* Algorithm 3.  With trim (Sec. 3.2, the growth factor of ortho(X), reading R18): the
 * projection X - Y C leaves a Y-component of about eps sqrt(q) ||x~_j|| per column, and
 * ortho(X) amplifies it by g_j = (||x~_j|| / ||x_proj,j||) ||L^{-T}||, with ||x~_j||^2 =
 * ||C_j||^2 + ||x_proj,j||^2 (Y orthonormal).  When eps sqrt(q) max_j g_j <= tau the
 * overlap after the pass is below tau and the loop ends without forming Y^T X again. */
static int ortho_against_impl(int64_t n, int p, double* X, int q, const double* Y, double tau, int cap,
                              int cap2, int trim, oracle_ortho_stats* st) {
  if (p <= 0) return 0;
  double* C = (double*)malloc(sizeof(double) * (size_t)(q > 0 ? q : 1) * p);
  double* d2 = (double*)malloc(sizeof(double) * (size_t)p);
  int passes = 0, have_c = 0;
  for (;;) {
    if (q > 0) {
      if (!have_c) {
        oracle_gram(n, q, Y, p, X, C); /* C = Y^T X */
        st->grams++;
      }
      block_minus_times(n, p, X, q, Y, C); /* X <- X - Y Y^T X */
    }
    oracle_ortho_stats in;
    memset(&in, 0, sizeof in);
    double l2 = 1.0;
    ortho_impl(n, p, X, tau, cap, trim, &in, d2, &l2);
    st->grams += in.grams, st->shifts += in.shifts, st->svqb += in.svqb, st->cap_hits += in.cap_hits;
    st->skipped_recheck += in.skipped_recheck;
    if (in.cholqr_passes_max > st->cholqr_passes_max) st->cholqr_passes_max = in.cholqr_passes_max;
    ++passes;
    if (q == 0) break;
    if (trim && l2 < HUGE_VAL) {
      double g2 = 0.0;
      for (int j = 0; j < p; ++j) {
        double c2 = 0.0;
        for (int i = 0; i < q; ++i) c2 += C[i + (size_t)j * q] * C[i + (size_t)j * q];
        const double gj = d2[j] > 0.0 ? (c2 + d2[j]) / d2[j] * l2 : HUGE_VAL;
        if (!(gj <= g2)) g2 = gj;
      }
      if (EPS * sqrt((double)q) * sqrt(g2) <= tau) { /* R18: moderate growth, no test */
        st->skipped_test++;
        break;
      }
    }
    oracle_gram(n, q, Y, p, X, C);
    st->grams++;
    have_c = 1;
    if (max_abs((int64_t)q * p, C) <= tau) break;
    if (passes >= cap2) {
      st->cap_hits++;
      break;
    }
  }
  st->passes = passes;
  free(C);
  free(d2);
  return passes;
}

int oracle_ortho(int64_t n, int p, double* X, double tau, int cap, int* shifts, int* svqb,
                 int* cap_hit, int* passes_max) {
  oracle_ortho_stats st;
  memset(&st, 0, sizeof st);
  const int passes = ortho_impl(n, p, X, tau, cap, 0, &st, NULL, NULL);
  if (shifts) *shifts += st.shifts;
  if (svqb) *svqb += st.svqb;
  if (cap_hit) *cap_hit += st.cap_hits;
  if (passes_max && passes > *passes_max) *passes_max = passes;
  return passes;
}

int oracle_ortho_against(int64_t n, int p, double* X, int q, const double* Y, double tau,
                         int cap, int cap2, int* shifts, int* svqb, int* cap_hit,
                         int* cholqr_passes_max) {
  oracle_ortho_stats st;
  memset(&st, 0, sizeof st);
  const int passes = ortho_against_impl(n, p, X, q, Y, tau, cap, cap2, 0, &st);
  if (shifts) *shifts += st.shifts;
  if (svqb) *svqb += st.svqb;
  if (cap_hit) *cap_hit += st.cap_hits;
  if (cholqr_passes_max && st.cholqr_passes_max > *cholqr_passes_max) *cholqr_passes_max = st.cholqr_passes_max;
  return passes;
}

int oracle_ortho_ex(int64_t n, int p, double* X, double tau, int cap, int trim, oracle_ortho_stats* st) {
  memset(st, 0, sizeof *st);
  return ortho_impl(n, p, X, tau, cap, trim, st, NULL, NULL);
}

int oracle_ortho_against_ex(int64_t n, int p, double* X, int q, const double* Y, double tau, int cap, int cap2,
                            int trim, oracle_ortho_stats* st) {
  memset(st, 0, sizeof *st);
  return ortho_against_impl(n, p, X, q, Y, tau, cap, cap2, trim, st);
}

/* R16: drop the columns of W whose overlap with Y is above sqrt(tau) (and, with
 * check_norm, whose norm is not 1 to sqrt(tau)); the kept columns are packed to the
 * front in their order.  Returns their number.  Algorithm 1 calls it only after an
 * Algorithm 2/3 pass cap was hit. */
int oracle_drop_unorthogonal_columns(int64_t n, int p, double* W, int q, const double* Y, double tau,
                                     int check_norm) {
  if (p <= 0) return 0;
  double* Cm = (double*)malloc(sizeof(double) * (size_t)(q > 0 ? q : 1) * p);
  if (q > 0) oracle_gram(n, q, Y, p, W, Cm);
  int kept = 0;
  for (int j = 0; j < p; ++j) {
    const double worst = q > 0 ? max_abs(q, Cm + (size_t)j * q) : 0.0;
    const double nrm = sqrt(pairwise_dot(W + (size_t)j * n, W + (size_t)j * n, n));
    if (worst <= sqrt(tau) && (!check_norm || fabs(nrm - 1.0) <= sqrt(tau))) {
      if (kept != j) memcpy(W + (size_t)kept * n, W + (size_t)j * n, sizeof(double) * n);
      ++kept;
    }
  }
  free(Cm);
  return kept;
}

/* ------------------------------------------------------------- Algorithm 1 (Sec. 3.1) */

static int column_converged(int64_t n, const double* r, double tol, int tol_kind,
                            double* norm_out) {
  double nrm = sqrt(pairwise_dot(r, r, n));
  *norm_out = nrm;
  if (tol_kind == 1) {
    double rms = nrm / sqrt((double)n);
    return rms <= 0.1 * tol && max_abs(n, r) <= tol;
  }
  return nrm <= tol;
}

/* R = AX - X diag(lambda), norms and convergence flags for every column. */
static void residuals(int64_t n, int m, const double* X, const double* AX, const double* lam,
                      double* R, double* nrm, int* conv, double tol, int tol_kind) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j)
      R[i + (int64_t)j * n] = AX[i + (int64_t)j * n] - lam[j] * X[i + (int64_t)j * n];
  for (int j = 0; j < m; ++j)
    conv[j] = column_converged(n, R + (int64_t)j * n, tol, tol_kind, &nrm[j]);
}

/* Row t of the history: Ritz values and residual norms after Rayleigh-Ritz step t, the
 * active count that follows, and the widths of W and P in the basis of that step. */
static void record(oracle_history* h, int m, const double* lam, const double* nrm, int m_act, int w_cols,
                   int p_cols) {
  if (!h || h->rows >= h->cap) return;
  if (h->w_cols) h->w_cols[h->rows] = w_cols;
  if (h->p_cols) h->p_cols[h->rows] = p_cols;
  if (h->lambda) memcpy(h->lambda + (size_t)h->rows * m, lam, sizeof(double) * (size_t)m);
  if (h->resnorm) memcpy(h->resnorm + (size_t)h->rows * m, nrm, sizeof(double) * (size_t)m);
  if (h->m_act) h->m_act[h->rows] = m_act;
  h->rows++;
}

/* Precondition the active residual columns (R6): W~ = T R[:, act]. */
void oracle_precondition(int64_t n, int m_conv, int m_act, const double* R, const double* lam,
                         const double* diag, int precond, double* W) {
  for (int c = 0; c < m_act; ++c) {
    int j = m_conv + c;
    const double* r = R + (int64_t)j * n;
    double* w = W + (int64_t)c * n;
    double floor_ = 1e-8 * fmax(1.0, fabs(lam[j]));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      if (precond == 1) {
        double delta = diag[i] - lam[j];
        if (fabs(delta) < floor_) delta = (delta >= 0.0 ? 1.0 : -1.0) * floor_;
        w[i] = r[i] / delta;
      } else {
        w[i] = r[i];
      }
    }
  }
}

/* R24: x = (T - shift I)^{-1} b, T tridiagonal with sub-diagonal dl (T[i+1][i], n-1
 * entries), diagonal d and super-diagonal du (T[i][i+1], n-1 entries).  Gaussian
 * elimination with partial pivoting: at step i the pivot is the larger in magnitude of
 * the two candidates in column i (rows i and i+1), and an interchange of the two rows
 * puts a second super-diagonal entry (fill-in) into row i.  Then back substitution. */
void oracle_tridiag_solve(int64_t n, const double* dl, const double* d, const double* du, double shift,
                          const double* b, double* x) {
  if (n <= 0) return;
  const double fl = 1e-8 * fmax(1.0, fabs(shift));
  double* p = malloc(sizeof(double) * (size_t)n);  /* pivots (diagonal of U) */
  double* u1 = malloc(sizeof(double) * (size_t)n); /* first super-diagonal of U */
  double* u2 = malloc(sizeof(double) * (size_t)n); /* second super-diagonal of U (fill-in) */
  double* y = malloc(sizeof(double) * (size_t)n);  /* right-hand side, eliminated */
  for (int64_t i = 0; i < n; ++i) {
    p[i] = d[i] - shift;
    u1[i] = i + 1 < n ? du[i] : 0.0;
    u2[i] = 0.0;
    y[i] = b[i];
  }
  for (int64_t i = 0; i + 1 < n; ++i) {
    /* rows i and i+1 hold column i: p[i] (row i) and dl[i] (row i+1) */
    const double sub = dl[i];
    if (fabs(p[i]) >= fabs(sub)) {
      if (fabs(p[i]) < fl) p[i] = (p[i] >= 0.0 ? 1.0 : -1.0) * fl;
      const double f = sub / p[i];
      p[i + 1] -= f * u1[i];
      y[i + 1] -= f * y[i];
    } else {
      /* interchange rows i and i+1: row i becomes (sub, p[i+1], u1[i+1]) */
      const double piv = fabs(sub) < fl ? (sub >= 0.0 ? 1.0 : -1.0) * fl : sub;
      const double f = p[i] / piv;
      const double a1 = p[i + 1], a2 = u1[i + 1]; /* old row i+1: columns i+1, i+2 */
      const double b1 = u1[i];                    /* old row i: column i+1 */
      p[i] = piv;
      u1[i] = a1;
      u2[i] = a2;
      p[i + 1] = b1 - f * a1;
      u1[i + 1] = -f * a2;
      const double yi = y[i];
      y[i] = y[i + 1];
      y[i + 1] = yi - f * y[i];
    }
  }
  if (fabs(p[n - 1]) < fl) p[n - 1] = (p[n - 1] >= 0.0 ? 1.0 : -1.0) * fl;
  for (int64_t i = n - 1; i >= 0; --i) {
    double t = y[i];
    if (i + 1 < n) t -= u1[i] * x[i + 1];
    if (i + 2 < n) t -= u2[i] * x[i + 2];
    x[i] = t / p[i];
  }
  free(p), free(u1), free(u2), free(y);
}

/* The first sub- and super-diagonals of A: dl[i] = A[i+1][i], du[i] = A[i][i+1]
 * (duplicate CSR entries summed, as the product sums them). */
void oracle_tridiag_of(const oracle_matrix* A, double* dl, double* du) {
  const int64_t n = A->n;
  for (int64_t i = 0; i + 1 < n; ++i) {
    double lo = 0.0, up = 0.0;
    if (A->dense) {
      lo = A->dense[i * A->ld + (i + 1)]; /* column i, row i+1 (column-major) */
      up = A->dense[(i + 1) * A->ld + i]; /* column i+1, row i */
    } else {
      for (int64_t e = A->row_ptr[i + 1]; e < A->row_ptr[i + 2]; ++e)
        if (A->col_idx[e] == i) lo += A->val[e];
      for (int64_t e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e)
        if (A->col_idx[e] == i + 1) up += A->val[e];
    }
    dl[i] = lo;
    du[i] = up;
  }
}

/* R24 on the active residual columns: W[:, c] = (T - lam_j I)^{-1} R[:, j], j = m_conv + c. */
void oracle_precondition_tridiag(int64_t n, int m_conv, int m_act, const double* R, const double* lam,
                                 const double* dl, const double* diag, const double* du, double* W) {
#pragma omp parallel for schedule(static)
  for (int c = 0; c < m_act; ++c) {
    const int j = m_conv + c;
    oracle_tridiag_solve(n, dl, diag, du, lam[j], R + (int64_t)j * n, W + (int64_t)c * n);
  }
}

static void finish_outputs(const oracle_matrix* A, int64_t n, int k, const double* X,
                           const double* lam, double* evals, double* evecs, double* resnorms) {
  double* AXk = (double*)malloc(sizeof(double) * (size_t)n * k);
  for (int j = 0; j < k; ++j) {
    const double* x = X + (int64_t)j * n;
    double* e = evecs + (int64_t)j * n;
    double big = 0.0;
    int64_t at = 0;
    for (int64_t i = 0; i < n; ++i)
      if (fabs(x[i]) > big) big = fabs(x[i]), at = i;
    double sgn = x[at] < 0.0 ? -1.0 : 1.0;
    double nrm = sqrt(pairwise_dot(x, x, n));
    for (int64_t i = 0; i < n; ++i) e[i] = sgn * x[i] / nrm;
    evals[j] = lam[j];
  }
  oracle_apply(A, k, evecs, AXk);
  for (int j = 0; j < k; ++j) {
    double* r = AXk + (int64_t)j * n;
    for (int64_t i = 0; i < n; ++i) r[i] -= evals[j] * evecs[i + (int64_t)j * n];
    resnorms[j] = sqrt(pairwise_dot(r, r, n));
  }
  free(AXk);
}

/* Algorithm 2 / 3 on an n-row block with the run's options; statistics go to *loc.  The
 * cost trims (R17, R18) apply to these n-row orthogonalisations only: the u_p one in
 * R^s costs nothing worth saving. */
static void add_stats(oracle_info* loc, const oracle_ortho_stats* st) {
  loc->shifts += st->shifts;
  loc->svqb += st->svqb;
  loc->cap_hits += st->cap_hits;
  loc->ortho_grams += st->grams;
  loc->skipped_recheck += st->skipped_recheck;
  loc->skipped_test += st->skipped_test;
  if (st->cholqr_passes_max > loc->cholqr_passes_max) loc->cholqr_passes_max = st->cholqr_passes_max;
}

static void run_ortho(int64_t n, int p, double* X, double tau, int cap, int trim, oracle_info* loc) {
  oracle_ortho_stats st;
  oracle_ortho_ex(n, p, X, tau, cap, trim, &st);
  add_stats(loc, &st);
}

static int run_ortho_against(int64_t n, int p, double* X, int q, const double* Y, double tau, int cap, int cap2,
                             int trim, oracle_info* loc) {
  oracle_ortho_stats st;
  const int passes = oracle_ortho_against_ex(n, p, X, q, Y, tau, cap, cap2, trim, &st);
  add_stats(loc, &st);
  if (passes > loc->ortho_passes_max) loc->ortho_passes_max = passes;
  return passes;
}

int oracle_lobpcg(const oracle_matrix* A, const double* diag, const oracle_opts* opt,
                  const double* X0, double* evals, double* evecs, double* resnorms,
                  oracle_info* info, oracle_history* hist) {
  const int64_t n = A->n;
  const int k = opt->k, m = opt->k + opt->extra;
  const double tau = opt->tau > 0 ? opt->tau : 1e-14;
  const int cap = opt->ortho_cap > 0 ? opt->ortho_cap : 6;
  const int cap2 = opt->ortho2_cap > 0 ? opt->ortho2_cap : 4;
  oracle_info loc;
  memset(&loc, 0, sizeof loc);
  if (k < 1 || opt->extra < 0 || 3 * (int64_t)m > n || !X0 || !evals || !evecs || !resnorms)
    return ORACLE_EINVAL;
  if ((opt->precond == 1 || opt->precond == 3) && !diag) return ORACLE_EINVAL;
  if (opt->precond < 0 || opt->precond > 3 || opt->precond == 2) return ORACLE_EINVAL;
  if (hist) hist->rows = 0;

  const int smax = 3 * m;
  double *X = malloc(sizeof(double) * n * m), *AX = malloc(sizeof(double) * n * m);
  double *W = malloc(sizeof(double) * n * m), *AW = malloc(sizeof(double) * n * m);
  double *P = malloc(sizeof(double) * n * m), *AP = malloc(sizeof(double) * n * m);
  double *R = malloc(sizeof(double) * n * m), *Y = malloc(sizeof(double) * n * 2 * m);
  double *V = malloc(sizeof(double) * n * smax), *AV = malloc(sizeof(double) * n * smax);
  double *a = malloc(sizeof(double) * smax * smax), *U = malloc(sizeof(double) * smax * smax);
  double *lam_all = malloc(sizeof(double) * smax), *lam = malloc(sizeof(double) * m);
  double *up = malloc(sizeof(double) * smax * m), *nrm = malloc(sizeof(double) * m);
  int* conv = malloc(sizeof(int) * m);
  if (!X || !AX || !W || !AW || !P || !AP || !R || !Y || !V || !AV || !a || !U || !lam_all ||
      !lam || !up || !nrm || !conv) {
    free(X), free(AX), free(W), free(AW), free(P), free(AP), free(R), free(Y), free(V);
    free(AV), free(a), free(U), free(lam_all), free(lam), free(up), free(nrm), free(conv);
    return ORACLE_ENOMEM;
  }
  int status = ORACLE_ENOCONV;
  double *tdl = NULL, *tdu = NULL; /* tridiagonal part of A (R24) */
  if (opt->precond == 3) {
    tdl = calloc((size_t)(n > 1 ? n - 1 : 1), sizeof(double));
    tdu = calloc((size_t)(n > 1 ? n - 1 : 1), sizeof(double));
    oracle_tridiag_of(A, tdl, tdu);
  }

  /* ---- Algorithm 1, initialisation ---- */
  memcpy(X, X0, sizeof(double) * n * m);
  run_ortho(n, m, X, tau, cap, opt->trim, &loc);                          /* R2 */
  oracle_apply(A, m, X, AX);                                              /* AX = A X */
  loc.spmm_columns += m;
  oracle_gram(n, m, X, m, AX, a);                                         /* a = X^T AX */
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < j; ++i) a[i + j * m] = a[j + i * m] = 0.5 * (a[i + j * m] + a[j + i * m]);
  oracle_jacobi_eig(m, a, lam, U);                                        /* a u = u lambda */
  memcpy(V, X, sizeof(double) * n * m);
  memcpy(AV, AX, sizeof(double) * n * m);
  block_times_small(n, m, V, m, U, X);                                    /* X = X u, AX = AX u */
  block_times_small(n, m, AV, m, U, AX);
  residuals(n, m, X, AX, lam, R, nrm, conv, opt->tol, opt->tol_kind);     /* R = AX - X lambda */
  int m_conv = 0;
  while (m_conv < m && conv[m_conv]) ++m_conv;                            /* R1, R7 */
  int m_act = m - m_conv;
  record(hist, m, lam, nrm, m_act, 0, 0);
  int have_p = 0, it = 0;
  if (m_conv >= k) {
    status = ORACLE_OK;
    goto done;
  }
  if (opt->precond == 3)
    oracle_precondition_tridiag(n, m_conv, m_act, R, lam, tdl, diag, tdu, W);   /* W~ = T R (R24) */
  else
    oracle_precondition(n, m_conv, m_act, R, lam, diag, opt->precond, W);        /* W~ = T R */
  int w_cols = m_act; /* columns of W (R16) */
  {
    const int hits0 = loc.cap_hits;
    run_ortho_against(n, m_act, W, m, X, tau, cap, cap2, opt->trim, &loc); /* W = ortho(W~; X) */
    if (loc.cap_hits > hits0) w_cols = oracle_drop_unorthogonal_columns(n, m_act, W, m, X, tau, 1); /* R16 */
    loc.w_dropped += m_act - w_cols;
  }
  oracle_apply(A, w_cols, W, AW);                                         /* AW = A W */
  loc.spmm_columns += w_cols;

  /* ---- Algorithm 1, main loop ---- */
  for (it = 1; it <= opt->maxiter; ++it) {
    /* expansion subspace: V = (X, W) on the first pass, (X, W, P) afterwards */
    const int s = m + w_cols + have_p;
    memcpy(V, X, sizeof(double) * n * m);
    memcpy(V + n * m, W, sizeof(double) * n * w_cols);
    memcpy(AV, AX, sizeof(double) * n * m);
    memcpy(AV + n * m, AW, sizeof(double) * n * w_cols);
    if (have_p) {
      memcpy(V + n * (m + w_cols), P, sizeof(double) * n * have_p);
      memcpy(AV + n * (m + w_cols), AP, sizeof(double) * n * have_p);
    }
    oracle_gram(n, s, V, s, AV, a);                                       /* a = V^T AV */
    for (int j = 0; j < s; ++j)
      for (int i = 0; i < j; ++i)
        a[i + j * s] = a[j + i * s] = 0.5 * (a[i + j * s] + a[j + i * s]); /* R9 */
    oracle_jacobi_eig(s, a, lam_all, U);                                  /* Rayleigh-Ritz */
    memcpy(lam, lam_all, sizeof(double) * m);                             /* u_x = U[:, :m] */
    block_times_small(n, s, V, m, U, X);                                  /* X = V u_x, AX = AV u_x */
    block_times_small(n, s, AV, m, U, AX);
    residuals(n, m, X, AX, lam, R, nrm, conv, opt->tol, opt->tol_kind);   /* R = AX - X lambda */
    m_conv = 0;
    while (m_conv < m && conv[m_conv]) ++m_conv;                          /* lock, R7 */
    m_act = m - m_conv;
    record(hist, m, lam, nrm, m_act, w_cols, have_p);
    if (m_conv >= k) {
      status = ORACLE_OK;
      break;
    }
    /* P coefficients: u~_p = u_x[:, act] - E_act, u_p = ortho(u~_p; u_x)  (R8, R14) */
    int p_cols = 0;
    for (int c = 0; c < m_act; ++c) {
      int j = m_conv + c;
      double* col = up + (size_t)p_cols * s;
      memcpy(col, U + (size_t)j * s, sizeof(double) * s);
      col[j] -= 1.0;
      /* norm of (I - u_x u_x^T) u~_p_j: keep the column only if x_j moved */
      double* proj = (double*)malloc(sizeof(double) * s);
      memcpy(proj, col, sizeof(double) * s);
      for (int q = 0; q < m; ++q) {
        double d = 0.0;
        for (int i = 0; i < s; ++i) d += U[i + (size_t)q * s] * col[i];
        for (int i = 0; i < s; ++i) proj[i] -= d * U[i + (size_t)q * s];
      }
      double nrm = 0.0;
      for (int i = 0; i < s; ++i) nrm += proj[i] * proj[i];
      free(proj);
      if (sqrt(nrm) > 1e-200) ++p_cols;
    }
    loc.p_dropped += m_act - p_cols; /* R14 */
    if (p_cols > 0) {
      const int hits0 = loc.cap_hits, asked = p_cols;
      int p2 = oracle_ortho_against(s, p_cols, up, m, U, tau, cap, cap2, &loc.shifts,
                                    &loc.svqb, &loc.cap_hits, &loc.cholqr_passes_max);
      (void)p2;
      if (loc.cap_hits > hits0) p_cols = oracle_drop_unorthogonal_columns(s, p_cols, up, m, U, tau, 1); /* R16 in R^s */
      loc.p_dropped += asked - p_cols;
    }
    block_times_small(n, s, V, p_cols, up, P);                            /* P = V u_p, AP = AV u_p */
    block_times_small(n, s, AV, p_cols, up, AP);
    have_p = p_cols;
    if (opt->precond == 3)
      oracle_precondition_tridiag(n, m_conv, m_act, R, lam, tdl, diag, tdu, W); /* W~ = T R (R24) */
    else
      oracle_precondition(n, m_conv, m_act, R, lam, diag, opt->precond, W);      /* W~ = T R */
    memcpy(Y, X, sizeof(double) * n * m);                                 /* Y = (X, P) */
    memcpy(Y + n * m, P, sizeof(double) * n * have_p);
    {
      const int hits0 = loc.cap_hits;
      run_ortho_against(n, m_act, W, m + have_p, Y, tau, cap, cap2, opt->trim, &loc); /* W = ortho(W~; (X, P)) */
      w_cols = m_act;
      if (loc.cap_hits > hits0)
        w_cols = oracle_drop_unorthogonal_columns(n, m_act, W, m + have_p, Y, tau, 1); /* R16 */
      loc.w_dropped += m_act - w_cols;
    }
    oracle_apply(A, w_cols, W, AW);                                       /* AW = A W */
    loc.spmm_columns += w_cols;
  }
  if (it > opt->maxiter) it = opt->maxiter;

done:
  loc.iterations = it;
  loc.converged = m_conv;
  finish_outputs(A, n, k, X, lam, evals, evecs, resnorms);                /* R10 */
  if (info) *info = loc;
  free(X), free(AX), free(W), free(AW), free(P), free(AP), free(R), free(Y), free(V);
  free(AV), free(a), free(U), free(lam_all), free(lam), free(up), free(nrm), free(conv);
  free(tdl), free(tdu);
  return status;
}

/* ================================================ generalised problem A x = lambda B x (Sec. 3.3)
 *
 * B symmetric positive definite.  The basis V = (X, W, P) is kept B-orthonormal, so the
 * Rayleigh-Ritz problem stays the standard one a = V^T A V; B V is carried along like A V
 * and updated by the same coefficients.  Following Sec. 3.3:
 *   - W^ = ortho(W~, (B X, B P)): Algorithm 3 against an orthonormal basis Q of
 *     span(B X, B P) (reading R19: the printed ortho(X, Y) needs orthonormal Y, so Q is
 *     formed from (B X, B P) with Algorithm 2).  W^ is then B-orthogonal to X and P and
 *     orthonormal in the Euclidean product, hence well conditioned in the B product.
 *   - W = W^ L^{-T} with L L^T = W^T B W^ (Cholesky-QR in the B product, repeated while
 *     ||W^T B W - I|| > tau as in Algorithm 2), and B W = (B W^) L^{-T} re-using the one
 *     application of B to W^.
 * Residuals are A x - lambda B x, the diagonal preconditioner is
 * (diag(A) - theta diag(B))^{-1} (guarded as in R6), and x_j is returned with x^T B x = 1.
 * X0 is B-orthonormalised the same way (reading R20).  Without B (B = I) every step reduces
 * to Algorithm 1 exactly. */

/* T (p x p) of one Cholesky-QR pass on the overlap M (R15 scaling, R4 shift, SVQB when
 * the shift fails): X <- X T.  Counts go to loc. */
static void cholqr_transform(int p, const double* M, double* T, oracle_info* loc) {
  double* Dv = (double*)malloc(sizeof(double) * (size_t)p);
  double* Ms = (double*)malloc(sizeof(double) * (size_t)p * p);
  double* L = (double*)malloc(sizeof(double) * (size_t)p * p);
  for (int i = 0; i < p; ++i) Dv[i] = M[i + i * p] > 0.0 ? 1.0 / sqrt(M[i + i * p]) : 1.0;
  for (int j = 0; j < p; ++j)
    for (int i = 0; i < p; ++i) Ms[i + j * p] = Dv[i] * M[i + j * p] * Dv[j];
  memcpy(L, Ms, sizeof(double) * (size_t)p * p);
  int fail = oracle_cholesky(p, L);
  if (fail) {
    double tr = 0.0;
    for (int i = 0; i < p; ++i) tr += Ms[i + i * p];
    double sigma = 100.0 * EPS * tr;
    for (int t = 0; t < 8 && fail; ++t, sigma *= 10.0) {
      memcpy(L, Ms, sizeof(double) * (size_t)p * p);
      for (int i = 0; i < p; ++i) L[i + i * p] += sigma;
      loc->shifts++;
      fail = oracle_cholesky(p, L);
    }
  }
  if (!fail) {
    /* T = D L^{-T}: column j of L^{-T} is row j of L^{-1} (forward substitution) */
    for (int j = 0; j < p; ++j)
      for (int i = 0; i < p; ++i) T[i + j * p] = 0.0;
    for (int c = 0; c < p; ++c) { /* column c of L^{-1} */
      for (int i = 0; i < p; ++i) {
        double s = i == c ? 1.0 : 0.0;
        for (int l = 0; l < i; ++l) s -= L[i + l * p] * T[c + l * p];
        T[c + i * p] = i < c ? 0.0 : s / L[i + i * p]; /* T(c, i) = (L^{-1})(i, c) */
      }
    }
    for (int j = 0; j < p; ++j)
      for (int i = 0; i < p; ++i) T[i + j * p] *= Dv[i];
  } else {
    /* SVQB: D M D = Z Theta Z^T, T = D Z Theta^{-1/2} (Theta floored at eps max) */
    double* Z = (double*)malloc(sizeof(double) * (size_t)p * p);
    double* th = (double*)malloc(sizeof(double) * (size_t)p);
    loc->svqb++;
    oracle_jacobi_eig(p, Ms, th, Z);
    double tmax = 0.0;
    for (int i = 0; i < p; ++i) tmax = fmax(tmax, th[i]);
    for (int j = 0; j < p; ++j) {
      const double t = fmax(th[j], EPS * tmax);
      for (int i = 0; i < p; ++i) T[i + j * p] = Dv[i] * Z[i + j * p] / sqrt(t);
    }
    free(Z), free(th);
  }
  free(Dv), free(Ms), free(L);
}

/* X <- X T and, when Y != NULL, Y <- Y T (same T): the re-use of B applications. */
static void apply_transform(int64_t n, int p, double* X, double* Y, const double* T) {
  double* tmp = (double*)malloc(sizeof(double) * (size_t)n * p);
  memcpy(tmp, X, sizeof(double) * (size_t)n * p);
  block_times_small(n, p, tmp, p, T, X);
  if (Y) {
    memcpy(tmp, Y, sizeof(double) * (size_t)n * p);
    block_times_small(n, p, tmp, p, T, Y);
  }
  free(tmp);
}

/* Algorithm 2 in the B product with re-use: M = X^T (B X), stop when ||M - I|| <= tau,
 * else X <- X T and B X <- (B X) T.  Returns the passes; a cap hit is counted. */
static int b_ortho(int64_t n, int p, double* X, double* BX, double tau, int cap, oracle_info* loc) {
  if (p <= 0) return 0;
  double* M = (double*)malloc(sizeof(double) * (size_t)p * p);
  double* T = (double*)malloc(sizeof(double) * (size_t)p * p);
  int passes = 0;
  for (;;) {
    oracle_gram(n, p, X, p, BX, M);
    for (int j = 0; j < p; ++j)
      for (int i = 0; i < j; ++i) M[i + j * p] = M[j + i * p] = 0.5 * (M[i + j * p] + M[j + i * p]);
    if (max_abs_minus_identity(p, M) <= tau) break;
    if (passes >= cap) {
      loc->cap_hits++;
      break;
    }
    ++passes;
    cholqr_transform(p, M, T, loc);
    apply_transform(n, p, X, BX, T);
  }
  if (passes > loc->cholqr_passes_max) loc->cholqr_passes_max = passes;
  free(M), free(T);
  return passes;
}

/* R16 in the generalised form: keep the columns of W (and B W) whose overlap with the
 * orthonormal Q is <= sqrt(tau) and whose B-norm is 1 to sqrt(tau); pack to the front. */
static int drop_gen(int64_t n, int p, double* W, double* BW, int q, const double* Q, double tau) {
  double* Cm = (double*)malloc(sizeof(double) * (size_t)(q > 0 ? q : 1) * p);
  if (q > 0) oracle_gram(n, q, Q, p, W, Cm);
  int kept = 0;
  for (int j = 0; j < p; ++j) {
    const double worst = q > 0 ? max_abs(q, Cm + (size_t)j * q) : 0.0;
    const double bn = sqrt(fabs(pairwise_dot(W + (size_t)j * n, BW + (size_t)j * n, n)));
    if (worst <= sqrt(tau) && fabs(bn - 1.0) <= sqrt(tau)) {
      if (kept != j) {
        memcpy(W + (size_t)kept * n, W + (size_t)j * n, sizeof(double) * n);
        memcpy(BW + (size_t)kept * n, BW + (size_t)j * n, sizeof(double) * n);
      }
      ++kept;
    }
  }
  free(Cm);
  return kept;
}

/* R = AX - BX diag(lambda), norms and convergence flags. */
static void residuals_gen(int64_t n, int m, const double* AX, const double* BX, const double* lam, double* R,
                          double* nrm, int* conv, double tol, int tol_kind) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j)
      R[i + (int64_t)j * n] = AX[i + (int64_t)j * n] - lam[j] * BX[i + (int64_t)j * n];
  for (int j = 0; j < m; ++j) conv[j] = column_converged(n, R + (int64_t)j * n, tol, tol_kind, &nrm[j]);
}

/* W~ = T R over the active columns with T = (diag(A) - theta diag(B))^{-1}, guarded (R6). */
static void precondition_gen(int64_t n, int m_conv, int m_act, const double* R, const double* lam,
                             const double* dA, const double* dB, int precond, double* W) {
  for (int c = 0; c < m_act; ++c) {
    const int j = m_conv + c;
    const double* r = R + (int64_t)j * n;
    double* w = W + (int64_t)c * n;
    const double floor_ = 1e-8 * fmax(1.0, fabs(lam[j]));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      if (precond == 1) {
        double delta = dA[i] - lam[j] * dB[i];
        if (fabs(delta) < floor_) delta = (delta >= 0.0 ? 1.0 : -1.0) * floor_;
        w[i] = r[i] / delta;
      } else {
        w[i] = r[i];
      }
    }
  }
}

int oracle_lobpcg_gen(const oracle_matrix* A, const oracle_matrix* B, const double* dA, const double* dB,
                      const oracle_opts* opt, const double* X0, double* evals, double* evecs, double* resnorms,
                      oracle_info* info, oracle_history* hist) {
  const int64_t n = A->n;
  const int k = opt->k, m = opt->k + opt->extra;
  const double tau = opt->tau > 0 ? opt->tau : 1e-14;
  const int cap = opt->ortho_cap > 0 ? opt->ortho_cap : 6;
  const int cap2 = opt->ortho2_cap > 0 ? opt->ortho2_cap : 4;
  oracle_info loc;
  memset(&loc, 0, sizeof loc);
  if (!B || B->n != n || k < 1 || opt->extra < 0 || 3 * (int64_t)m > n || !X0 || !evals || !evecs || !resnorms)
    return ORACLE_EINVAL;
  if (opt->precond == 1 && (!dA || !dB)) return ORACLE_EINVAL;
  if (hist) hist->rows = 0;
  const int smax = 3 * m;
  const size_t blk = sizeof(double) * (size_t)n * m;
  double *X = malloc(blk), *AX = malloc(blk), *BX = malloc(blk), *W = malloc(blk), *AW = malloc(blk);
  double *BW = malloc(blk), *P = malloc(blk), *AP = malloc(blk), *BP = malloc(blk), *R = malloc(blk);
  double* Q = malloc(2 * blk);
  double *V = malloc(sizeof(double) * n * smax), *AV = malloc(sizeof(double) * n * smax);
  double* BV = malloc(sizeof(double) * n * smax);
  double *a = malloc(sizeof(double) * smax * smax), *U = malloc(sizeof(double) * smax * smax);
  double *lam_all = malloc(sizeof(double) * smax), *lam = malloc(sizeof(double) * m);
  double *up = malloc(sizeof(double) * smax * m), *nrm = malloc(sizeof(double) * m);
  int* conv = malloc(sizeof(int) * m);
  int status = ORACLE_ENOCONV;
  int m_conv = 0, m_act = m, have_p = 0, it = 0, w_cols = 0;

  /* ---- initialisation: B-orthonormal X0 (R20), Rayleigh-Ritz, residual ---- */
  memcpy(X, X0, blk);
  oracle_apply(B, m, X, BX);
  b_ortho(n, m, X, BX, tau, cap, &loc);
  oracle_apply(A, m, X, AX);
  loc.spmm_columns += m;
  oracle_gram(n, m, X, m, AX, a);
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < j; ++i) a[i + j * m] = a[j + i * m] = 0.5 * (a[i + j * m] + a[j + i * m]);
  oracle_jacobi_eig(m, a, lam, U);
  memcpy(V, X, blk), memcpy(AV, AX, blk), memcpy(BV, BX, blk);
  block_times_small(n, m, V, m, U, X);
  block_times_small(n, m, AV, m, U, AX);
  block_times_small(n, m, BV, m, U, BX);
  residuals_gen(n, m, AX, BX, lam, R, nrm, conv, opt->tol, opt->tol_kind);
  while (m_conv < m && conv[m_conv]) ++m_conv;
  m_act = m - m_conv;
  record(hist, m, lam, nrm, m_act, 0, 0);
  if (m_conv >= k) {
    status = ORACLE_OK;
    goto done;
  }
  for (it = 1;; ++it) {
    /* W = B-ortho(ortho(T R, orth(B X, B P))), B W re-used (Sec. 3.3) */
    precondition_gen(n, m_conv, m_act, R, lam, dA, dB, opt->precond, W);
    const int q = m + have_p;
    memcpy(Q, BX, blk);
    memcpy(Q + (size_t)n * m, BP, sizeof(double) * (size_t)n * have_p);
    const int hits0 = loc.cap_hits;
    run_ortho(n, q, Q, tau, cap, opt->trim, &loc);                        /* Q = orth(BX, BP) (R19) */
    run_ortho_against(n, m_act, W, q, Q, tau, cap, cap2, opt->trim, &loc); /* W^ = ortho(W~, Q) */
    oracle_apply(B, m_act, W, BW);                                         /* B W^ */
    b_ortho(n, m_act, W, BW, tau, cap, &loc);                              /* W = W^ L^{-T}, BW re-used */
    w_cols = m_act;
    if (loc.cap_hits > hits0) w_cols = drop_gen(n, m_act, W, BW, q, Q, tau); /* R16 */
    loc.w_dropped += m_act - w_cols;
    oracle_apply(A, w_cols, W, AW);
    loc.spmm_columns += w_cols;
    if (it > opt->maxiter) break;
    /* ---- Rayleigh-Ritz on V = (X, W, P) ---- */
    const int s = m + w_cols + have_p;
    memcpy(V, X, blk), memcpy(AV, AX, blk), memcpy(BV, BX, blk);
    memcpy(V + n * m, W, sizeof(double) * n * w_cols);
    memcpy(AV + n * m, AW, sizeof(double) * n * w_cols);
    memcpy(BV + n * m, BW, sizeof(double) * n * w_cols);
    memcpy(V + n * (m + w_cols), P, sizeof(double) * n * have_p);
    memcpy(AV + n * (m + w_cols), AP, sizeof(double) * n * have_p);
    memcpy(BV + n * (m + w_cols), BP, sizeof(double) * n * have_p);
    oracle_gram(n, s, V, s, AV, a);
    for (int j = 0; j < s; ++j)
      for (int i = 0; i < j; ++i) a[i + j * s] = a[j + i * s] = 0.5 * (a[i + j * s] + a[j + i * s]);
    oracle_jacobi_eig(s, a, lam_all, U);
    memcpy(lam, lam_all, sizeof(double) * m);
    block_times_small(n, s, V, m, U, X);
    block_times_small(n, s, AV, m, U, AX);
    block_times_small(n, s, BV, m, U, BX);
    residuals_gen(n, m, AX, BX, lam, R, nrm, conv, opt->tol, opt->tol_kind);
    m_conv = 0;
    while (m_conv < m && conv[m_conv]) ++m_conv;
    m_act = m - m_conv;
    record(hist, m, lam, nrm, m_act, w_cols, have_p);
    if (m_conv >= k) {
      status = ORACLE_OK;
      break;
    }
    if (it >= opt->maxiter) break;
    /* P coefficients in R^s, as in Algorithm 1 (R8, R14, R16) */
    int p_cols = 0;
    for (int c = 0; c < m_act; ++c) {
      const int j = m_conv + c;
      double* col = up + (size_t)p_cols * s;
      memcpy(col, U + (size_t)j * s, sizeof(double) * s);
      col[j] -= 1.0;
      double* proj = (double*)malloc(sizeof(double) * s);
      memcpy(proj, col, sizeof(double) * s);
      for (int qq = 0; qq < m; ++qq) {
        double d = 0.0;
        for (int i = 0; i < s; ++i) d += U[i + (size_t)qq * s] * col[i];
        for (int i = 0; i < s; ++i) proj[i] -= d * U[i + (size_t)qq * s];
      }
      double pn = 0.0;
      for (int i = 0; i < s; ++i) pn += proj[i] * proj[i];
      free(proj);
      if (sqrt(pn) > 1e-200) ++p_cols;
    }
    loc.p_dropped += m_act - p_cols;
    if (p_cols > 0) {
      const int hp = loc.cap_hits, asked = p_cols;
      oracle_ortho_against(s, p_cols, up, m, U, tau, cap, cap2, &loc.shifts, &loc.svqb, &loc.cap_hits,
                           &loc.cholqr_passes_max);
      if (loc.cap_hits > hp) p_cols = oracle_drop_unorthogonal_columns(s, p_cols, up, m, U, tau, 1);
      loc.p_dropped += asked - p_cols;
    }
    block_times_small(n, s, V, p_cols, up, P);
    block_times_small(n, s, AV, p_cols, up, AP);
    block_times_small(n, s, BV, p_cols, up, BP);
    have_p = p_cols;
  }
  if (it > opt->maxiter) it = opt->maxiter;

done:
  loc.iterations = it;
  loc.converged = m_conv;
  {
    /* outputs: x^T B x = 1, largest |entry| positive, fresh residual A x - lambda B x */
    double* Bx = (double*)malloc(blk);
    double* Ax = (double*)malloc(blk);
    oracle_apply(B, k, X, Bx);
    for (int j = 0; j < k; ++j) {
      const double* x = X + (int64_t)j * n;
      double big = 0.0;
      int64_t at = 0;
      for (int64_t i = 0; i < n; ++i)
        if (fabs(x[i]) > big) big = fabs(x[i]), at = i;
      const double sgn = x[at] < 0.0 ? -1.0 : 1.0;
      const double bn = sqrt(pairwise_dot(x, Bx + (int64_t)j * n, n));
      for (int64_t i = 0; i < n; ++i) evecs[i + (int64_t)j * n] = sgn * x[i] / bn;
      evals[j] = lam[j];
    }
    oracle_apply(A, k, evecs, Ax);
    oracle_apply(B, k, evecs, Bx);
    for (int j = 0; j < k; ++j) {
      double* r = Ax + (int64_t)j * n;
      for (int64_t i = 0; i < n; ++i) r[i] -= evals[j] * Bx[i + (int64_t)j * n];
      resnorms[j] = sqrt(pairwise_dot(r, r, n));
    }
    free(Bx), free(Ax);
  }
  if (info) *info = loc;
  free(X), free(AX), free(BX), free(W), free(AW), free(BW), free(P), free(AP), free(BP), free(R), free(Q);
  free(V), free(AV), free(BV), free(a), free(U), free(lam_all), free(lam), free(up), free(nrm), free(conv);
  return status;
}
