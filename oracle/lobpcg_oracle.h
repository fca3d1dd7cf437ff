/*
 * CPU FP64 oracle for the LOBPCG eigensolver of "Robust and efficient LOBPCG for
 * quantum chemistry" (arXiv 2305.06668).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that the GPU
 * path is checked against.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it; the GPU library never includes, links or calls it.
 *
 * Conventions: every n x p block is column-major (column j starts at X + j*n), FP64.
 * Small p x q matrices are column-major too.
 */
#ifndef LOBPCG_ORACLE_H
#define LOBPCG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Symmetric operator: CSR (row_ptr/col_idx/val) or dense column-major (dense, ld). */
typedef struct {
  int64_t n;
  const int64_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
  const double* dense; /* non-NULL selects the dense form */
  int64_t ld;
} oracle_matrix;

typedef struct {
  int k;          /* eigenpairs sought */
  int extra;      /* block size m = k + extra (Sec. 2, larger block than sought) */
  int maxiter;    /* iteration cap of the main loop */
  int tol_kind;   /* 0: ||r_j||_2 <= tol;  1: rms(r_j) <= tol/10 and max|r_ij| <= tol */
  int precond;    /* 0: none, 1: diagonal (diag(A) - theta)^-1, 3: tridiagonal (R24) */
  int ortho_cap;  /* cap on Cholesky-QR passes in ortho(X)        (default 6) */
  int ortho2_cap; /* cap on projection passes in ortho(X, Y)      (default 4) */
  double tol;     /* residual tolerance */
  double tau;     /* orthogonality threshold tau_ortho (Sec. 4: 1e-14) */
  int trim;       /* 1: the cost trims of Sec. 3.2 in the n-row orthogonalisations (R17, R18) */
} oracle_opts;

typedef struct {
  int iterations;        /* main-loop iterations executed */
  int converged;         /* number of leading converged (locked) pairs at exit */
  int cholqr_passes_max; /* most Cholesky-QR passes in one ortho(X) call */
  int ortho_passes_max;  /* most projection passes in one ortho(X, Y) call */
  int shifts;            /* shifted Cholesky attempts, summed over the run */
  int svqb;              /* SVQB fallbacks, summed over the run */
  int cap_hits;          /* ortho loops that stopped at their pass cap */
  int spmm_columns;      /* columns multiplied by A, summed over the run */
  int w_dropped;         /* W columns dropped by R16, summed over the run */
  int p_dropped;         /* P columns dropped by R14 (x_j did not move) or R16, summed */
  int ortho_grams;       /* n-row Gram matrices formed by the orthogonalisations of W and X0 */
  int skipped_recheck;   /* Algorithm 2 re-check Grams skipped by the ||L^-T|| estimate (R17) */
  int skipped_test;      /* Algorithm 3 test Grams skipped by the growth factor (R18) */
} oracle_info;

/* Statistics of one Algorithm 2 / 3 call. */
typedef struct {
  int passes;            /* Cholesky-QR passes (Algorithm 2) or projection passes (Algorithm 3) */
  int grams;             /* n-row Gram matrices formed (X^T X and Y^T X) */
  int shifts, svqb, cap_hits, cholqr_passes_max;
  int skipped_recheck;   /* Algorithm 2 re-check Grams skipped (R17) */
  int skipped_test;      /* Algorithm 3 test Grams skipped (R18) */
} oracle_ortho_stats;

/* Per-iteration history (optional; any pointer may be NULL).  Row t (t = 0 is the
 * initial Rayleigh-Ritz) holds the m Ritz values / residual norms and the active count. */
typedef struct {
  int cap;          /* rows available */
  double* lambda;   /* cap x m, row-major */
  double* resnorm;  /* cap x m, row-major */
  int* m_act;       /* cap */
  int rows;         /* rows written */
  int* w_cols;      /* cap: columns of W in the basis of step t (0 for the initial step) */
  int* p_cols;      /* cap: columns of P in the basis of step t */
} oracle_history;

enum { ORACLE_OK = 0, ORACLE_EINVAL = 1, ORACLE_ENOMEM = 2, ORACLE_ENOCONV = 4, ORACLE_EBREAKDOWN = 5 };

/* Y = A X for an n x p block X. */
void oracle_apply(const oracle_matrix* A, int p, const double* X, double* Y);

/* Eigen-decomposition of a symmetric s x s matrix by cyclic Jacobi rotations.
 * lam ascending (ties keep Jacobi's index order), U column-major s x s eigenvectors.
 * Returns the number of sweeps, or -1 if it did not converge within 100 sweeps. */
int oracle_jacobi_eig(int s, const double* a, double* lam, double* U);

/* In-place lower Cholesky factor of p x p M (upper part untouched).
 * Returns 0 on success, else j+1 for the first non-positive pivot j. */
int oracle_cholesky(int p, double* M);

/* C = X^T Y (p x q) with pairwise summation over the n rows. */
void oracle_gram(int64_t n, int p, const double* X, int q, const double* Y, double* C);

/* SVQB step (Stathopoulos & Wu) on X given M = X^T X: X <- X D Z Theta^{-1/2}, where
 * D = diag(M)^{-1/2} and D M D = Z Theta Z^T (Theta floored at eps * max Theta). */
void oracle_svqb(int64_t n, int p, double* X, const double* M);

/* Algorithm 2 in place on the n x p block X.  Returns the number of Cholesky-QR
 * passes; *shifts / *svqb / *cap_hit accumulate (may be NULL). */
int oracle_ortho(int64_t n, int p, double* X, double tau, int cap, int* shifts, int* svqb,
                 int* cap_hit, int* passes_max);

/* Algorithm 2 with the optional cost trim of Sec. 3.2 (trim = 1, reading R17): the final
 * re-check X^T X is skipped after an unshifted pass whose scaled overlap I + F has
 * ||F||_F <= 1/2.  *st receives the call's statistics. */
int oracle_ortho_ex(int64_t n, int p, double* X, double tau, int cap, int trim, oracle_ortho_stats* st);

/* Algorithm 3 with the optional cost trim of Sec. 3.2 (trim = 1, reading R18): the test
 * Y^T X is skipped when eps sqrt(q) times the growth factor of the pass is <= tau (and the
 * Algorithm 2 calls inside use R17). */
int oracle_ortho_against_ex(int64_t n, int p, double* X, int q, const double* Y, double tau, int cap, int cap2,
                            int trim, oracle_ortho_stats* st);

/* Algorithm 3 in place: orthonormalise X (n x p) against orthonormal Y (n x q).
 * Returns the number of projection passes. */
int oracle_ortho_against(int64_t n, int p, double* X, int q, const double* Y, double tau,
                         int cap, int cap2, int* shifts, int* svqb, int* cap_hit,
                         int* cholqr_passes_max);

/* Diagonal preconditioner of Sec. 2 on the active residual columns (reading R6):
 * W[:, c] = R[:, m_conv + c] / delta, delta = diag - lam[m_conv + c] guarded away from zero;
 * precond == 0 copies R.  R: n x m, W: n x m_act, column-major. */
void oracle_precondition(int64_t n, int m_conv, int m_act, const double* R, const double* lam,
                         const double* diag, int precond, double* W);

/* Tridiagonal preconditioner (Sec. 4.4, reading R24).  oracle_tridiag_solve: x = (T -
 * shift I)^{-1} b by Gaussian elimination with partial pivoting, T given by its
 * sub-diagonal dl (T[i+1][i]), diagonal d and super-diagonal du (T[i][i+1]); pivots below
 * 1e-8 max(1, |shift|) are replaced by that value with their sign.  oracle_tridiag_of: dl
 * and du (n - 1 entries each) of A.  oracle_precondition_tridiag: W[:, c] = (T -
 * lam[m_conv + c] I)^{-1} R[:, m_conv + c] (column-major, R n x m, W n x m_act). */
void oracle_tridiag_solve(int64_t n, const double* dl, const double* d, const double* du, double shift,
                          const double* b, double* x);
void oracle_tridiag_of(const oracle_matrix* A, double* dl, double* du);
void oracle_precondition_tridiag(int64_t n, int m_conv, int m_act, const double* R, const double* lam,
                                 const double* dl, const double* diag, const double* du, double* W);

/* Reading R16: drop the columns of W (n x p) whose largest |overlap| with Y (n x q) is
 * above sqrt(tau), and with check_norm those whose 2-norm differs from 1 by more than
 * sqrt(tau); kept columns are packed to the front in order.  Returns their number. */
int oracle_drop_unorthogonal_columns(int64_t n, int p, double* W, int q, const double* Y, double tau,
                                     int check_norm);

/* Algorithm 1.  diag = diag(A) (length n).  X0 = n x m initial block (m = k + extra),
 * required.  Outputs: evals (k), evecs (n x k column-major), resnorms (k) = ||A x_j -
 * lambda_j x_j||_2 recomputed with a fresh product.  info, hist may be NULL. */
int oracle_lobpcg(const oracle_matrix* A, const double* diag, const oracle_opts* opt,
                  const double* X0, double* evals, double* evecs, double* resnorms,
                  oracle_info* info, oracle_history* hist);

/* Algorithm 1 for the generalised problem A x = lambda B x (Sec. 3.3), B symmetric
 * positive definite: B-orthonormal basis, B V carried along, W^ = ortho(W~, (B X, B P))
 * then Cholesky-QR in the B product with re-use of B W^.  dA, dB: diagonals of A and B
 * (preconditioner (dA - theta dB)^{-1}).  Outputs as oracle_lobpcg with x^T B x = 1 and
 * resnorms = ||A x - lambda B x||_2. */
int oracle_lobpcg_gen(const oracle_matrix* A, const oracle_matrix* B, const double* dA, const double* dB,
                      const oracle_opts* opt, const double* X0, double* evals, double* evecs, double* resnorms,
                      oracle_info* info, oracle_history* hist);

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int oracle_threads(void);

#ifdef __cplusplus
}
#endif
#endif
