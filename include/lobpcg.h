/*
 * lobpcg.h - C ABI of the GB300 LOBPCG eigensolver.
 *
 * Finds the k lowest eigenpairs of a large real symmetric matrix A with the robust
 * LOBPCG method of "Robust and efficient LOBPCG for quantum chemistry" (arXiv
 * 2305.06668): Algorithm 1 (three-term recurrence in the orthonormal basis (X, W, P),
 * Sec. 3.1), Algorithm 2 (shifted, repeated Cholesky-QR, Sec. 3.2), Algorithm 3
 * (orthogonalisation against a block, Sec. 3.2), soft locking of converged pairs
 * (Sec. 3.1, "Locking") and the diagonal preconditioner (diag(A) - theta)^-1 (Sec. 2).
 *
 * Every compute step runs in CUDA kernels for sm_103a.  There is no CPU fallback: a
 * call that cannot run on the GPU returns an error status.
 *
 * Memory ownership
 *   - Pointers documented as "device" must point to CUDA device memory of the current
 *     device; "host" pointers to ordinary host memory.
 *   - Input pointers are borrowed: the caller owns them and keeps them valid (and
 *     unmodified) until lobpcg_destroy (matrix arrays) or until the call returns
 *     (initial block, outputs).  The context owns every derived copy and workspace.
 *   - Outputs are allocated by the caller.
 *
 * Errors
 *   - No C++ exception or abort crosses this interface.  Every function reports a
 *     lobpcg_status; lobpcg_last_error() returns a one-line description.
 *   - LOBPCG_ENOCONV still fills every output with the best approximation reached.
 *
 * Tracing: when the environment variable LOBPCG_TRACE names a file, lobpcg_solve appends
 * one JSON line per iteration (Ritz values, residual norms, active count).
 *
 * Threading: a context is used by one host thread at a time.  All work of a context
 * is issued on the stream given to lobpcg_create; calls return after that stream has
 * finished the work they issued.
 */
#ifndef LOBPCG_H
#define LOBPCG_H

#include <stdint.h>

#if defined(__GNUC__)
#define LOBPCG_API __attribute__((visibility("default")))
#else
#define LOBPCG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* lobpcg_stream; /* same type as cudaStream_t; NULL = legacy default stream */

typedef struct lobpcg_ctx lobpcg_ctx; /* opaque; owns derived copies and workspace */

typedef enum {
  LOBPCG_OK = 0,
  LOBPCG_EINVAL = 1,     /* invalid argument (sizes, NULL pointers, non-finite input) */
  LOBPCG_ENOMEM = 2,     /* device or host allocation failed */
  LOBPCG_ECUDA = 3,      /* a CUDA runtime call or kernel failed */
  LOBPCG_ENOCONV = 4,    /* maxiter reached before the first k pairs converged */
  LOBPCG_EBREAKDOWN = 5  /* the basis lost rank beyond what shifts / SVQB can repair */
} lobpcg_status;

typedef enum { LOBPCG_CSR = 0, LOBPCG_DENSE = 1 } lobpcg_format;

typedef enum {
  LOBPCG_PREC_NONE = 0,   /* W~ = R */
  LOBPCG_PREC_DIAG = 1,   /* W~_ij = R_ij / (d_i - lambda_j)  (Sec. 2), guarded near zero */
  LOBPCG_PREC_LEARNED = 2, /* diagonal preconditioner times a learned positive per-entry scale */
  LOBPCG_PREC_TRIDIAG = 3  /* W~_j = (T - lambda_j I)^{-1} R_j, T = the diagonal and first
                              off-diagonals of A (Sec. 4.4), partial pivoting, guarded pivots */
} lobpcg_precond;

typedef enum {
  LOBPCG_FP64 = 0, /* every step in FP64 */
  LOBPCG_MIXED = 1 /* FP32 storage / products until the residual stalls, then FP64 refinement */
} lobpcg_precision;

/* Symmetric input matrix.  Only the fields of the chosen format are read. */
typedef struct {
  lobpcg_format fmt;
  int64_t n;              /* order of A, n >= 3 (k + extra) */
  int64_t nnz;            /* CSR: number of stored entries (both triangles) */
  const int64_t* row_ptr; /* CSR, device, n + 1 entries, row_ptr[0] = 0 */
  const int32_t* col_idx; /* CSR, device, nnz column indices in [0, n) */
  const double* val;      /* CSR, device, nnz values; A must be symmetric */
  const double* dense;    /* DENSE, device, column-major n x n, both triangles stored */
  int64_t ld;             /* DENSE leading dimension, ld >= n */
  const double* diag;     /* device, length n, diag(A) (used by the preconditioner) */
} lobpcg_matrix;

typedef struct {
  int extra;                  /* block size m = k + extra (Sec. 2); default 0 */
  int maxiter;                /* main-loop iteration cap; default 1000 */
  int tol_kind;               /* 0: ||r_j||_2 <= tol (default); 1: rms(r_j) <= tol/10 and max|r_ij| <= tol (Sec. 4.1) */
  lobpcg_precond precond;     /* default LOBPCG_PREC_DIAG */
  lobpcg_precision precision; /* default LOBPCG_FP64 */
  double tau_ortho;           /* orthogonality threshold (Sec. 4: 1e-14); default 1e-14 */
  int ortho_cap;              /* Cholesky-QR passes per ortho(X), default 6 */
  int ortho2_cap;             /* projection passes per ortho(X, Y), default 4 */
  uint64_t seed;              /* seed of the random initial block when X0 == NULL */
  const float* mlp_weights;   /* host, lobpcg_mlp_num_params() learned-preconditioner parameters
                                 (LOBPCG_PREC_LEARNED); copied by lobpcg_create */
  int profile;                /* non-zero: fill lobpcg_info.phase_seconds (adds CUDA events) */
  double mixed_switch;        /* MIXED: leave FP32 once the k sought residuals are <= this;
                                 0 (default) = when the largest stops improving: once it is
                                 below 1% of its first value, two iterations in a row that
                                 cut it by less than 25% each after three that cut it by a
                                 factor <= 0.6 each on geometric average, or no 10% drop in
                                 2 iterations; at any level, no 10% drop in 5 iterations */
  int autotune;               /* non-zero: on the first solve with a given block width, time the
                                 CSR product kernel families on this matrix (a few products per
                                 precision, inside that solve) and keep the fastest.  Meant for
                                 contexts reused over many solves (serving, batches).  0
                                 (default): the built-in choice */
  int ortho_trim;             /* non-zero (default): the cost trims of Sec. 3.2.  Algorithm 2 skips
                                 its re-check Gram after an unshifted pass with ||L^-T||_2^2 <= 2
                                 (bounded from the scaled overlap I + F by 1 / (1 - ||F||_F));
                                 Algorithm 3 skips its test Gram when eps sqrt(q) times the growth
                                 factor of ortho (column amplification times that bound) is <=
                                 tau.  Applies to the FP64 phases (the FP32 phase's Grams are not
                                 accurate to a few eps).  0: the printed Algorithms 2 and 3 */
  int df_products;            /* arithmetic of the FP64 Grams and block updates (not in the paper).
                                 FP64 data and results either way; double-float forms each product
                                 and sum from pairs of floats with error-free transformations on
                                 the FP32 pipes (about 2^-48 per product, chunk sums in FP64).
                                 0 (default): double-float in the FP64 refinement of the MIXED
                                 form, FP64 fused multiply-adds in the FP64 form; 1: double-float
                                 in every FP64 phase; -1: FP64 fused multiply-adds everywhere */
  int tc_gram;                /* FP32 Gram matrices of the MIXED form: non-zero (default) on the
                                 tcgen05 tensor cores (lobpcg_gram_f32_tcgen05), 0 with warp-level
                                 mma.sync (lobpcg_gram_f32); both 3xTF32 */
  double precond_floor;       /* diagonal preconditioner (not in the paper; a damped-diagonal
                                 control for the learned one): the denominator d_i - theta_j is
                                 replaced by sign(d_i - theta_j) max(|d_i - theta_j|, floor) with
                                 this absolute floor (>= 0); 0 (default) = the guard of reading
                                 R6 only.  The learned preconditioner ignores it */
} lobpcg_options;

typedef struct {
  int iterations;        /* main-loop iterations, all precision phases together */
  int fp64_iterations;   /* of which in FP64 */
  int converged;         /* leading pairs locked at exit */
  int cholqr_passes_max; /* most Cholesky-QR passes in one ortho(X) */
  int ortho_passes_max;  /* most projection passes in one ortho(X, Y) */
  int shifts;            /* shifted Cholesky attempts */
  int svqb;              /* SVQB fallbacks */
  int cap_hits;          /* ortho loops stopped at their cap */
  int64_t spmm_columns;  /* columns multiplied by A */
  double seconds;        /* wall time of the solve on the stream (CUDA events) */
  double phase_seconds[6]; /* with opt.profile: A products, Rayleigh-Ritz Gram, Rayleigh-Ritz
                              eigensolve, basis update + lock, preconditioner, ortho(W; Y) */
  int64_t kernel_launches; /* CUDA kernels this call launched */
  int64_t spmm_launches;   /* of which products with A inside the iteration */
  int precond_fallback;    /* 1 if the learned preconditioner stalled and the diagonal one took over */
  double phase_seconds_fp64[6]; /* with opt.profile: the FP64 part of phase_seconds */
  int64_t spmm_launches_fp64;   /* products with A in FP64 */
  int64_t spmm_columns_fp64;    /* columns of those products */
  double update_fp64_seconds;   /* with opt.profile: summed duration of the FP64 block updates
                                   (X = V u, W -= Y C, W <- W L^-T, ...), CUDA events per launch */
  double update_fp64_flops;     /* their algorithmic flops, 2 n s q per product */
  int64_t update_fp64_launches; /* their number */
  int spmm_variant_fp32;        /* CSR product kernel in use: 0 default, 1 row-parallel,
                                   2 vector gather, 3 band window with global gathers,
                                   4 band window on the unpacked band part (split FP32) */
  int spmm_variant_fp64;
  int w_dropped;                /* W columns dropped after an ortho(W~; Y) pass cap (reading R16) */
  int p_dropped;                /* P columns dropped: x_j did not move (R14) or after a pass cap (R16) */
  int ortho_grams;              /* n-row Gram matrices formed by Algorithms 2 and 3 */
  int skipped_recheck;          /* Algorithm 2 re-check Grams skipped (ortho_trim) */
  int skipped_test;             /* Algorithm 3 test Grams skipped (ortho_trim) */
  int df_products;              /* 1 if the FP64 Grams and updates ran in double-float arithmetic */
  double rr_gram32_bytes;       /* algorithmic bytes of the FP32 Rayleigh-Ritz Grams (2 n s 4 each) */
  int64_t rr_gram32_count;      /* their number */
} lobpcg_info;

/* Fills *opt with the defaults listed above.  Returns LOBPCG_EINVAL if opt is NULL. */
LOBPCG_API lobpcg_status lobpcg_options_default(lobpcg_options* opt);

/* Creates a solver context for A (Algorithm 1 input "operator A").
 *   out    host, receives the context (NULL on failure)
 *   A      host struct describing device arrays (borrowed until lobpcg_destroy)
 *   opt    host, NULL selects the defaults
 *   stream CUDA stream every kernel of this context is issued on
 * Errors: EINVAL for a NULL/inconsistent description, ENOMEM, ECUDA. */
LOBPCG_API lobpcg_status lobpcg_create(lobpcg_ctx** out, const lobpcg_matrix* A, const lobpcg_options* opt,
                            lobpcg_stream stream);

/* Creates a solver context for the generalised problem A x = lambda B x with B symmetric
 * positive definite (Sec. 3.3).  The basis is kept B-orthonormal with B V carried along;
 * W~ (preconditioned residuals A x - lambda B x, diagonal (diag A - theta diag B)^-1) is
 * projected against an orthonormal basis of span(B X, B P) by Algorithms 2 and 3, then
 * orthonormalised in the B product by Cholesky-QR re-using the one application of B.
 *   A, B   host structs describing device arrays (borrowed until lobpcg_destroy); B->diag
 *          must hold diag(B)
 *   opt    precision LOBPCG_FP64, preconditioner NONE or DIAG, df_products <= 0
 * lobpcg_solve then returns eigenvectors with x^T B x = 1 and resnorms ||A x - lambda B x||.
 * Errors: EINVAL (inconsistent B, non-finite entries, unsupported options), ENOMEM, ECUDA. */
LOBPCG_API lobpcg_status lobpcg_create_gen(lobpcg_ctx** out, const lobpcg_matrix* A, const lobpcg_matrix* B,
                                           const lobpcg_options* opt, lobpcg_stream stream);

/* Runs Algorithm 1 for the k lowest eigenpairs.
 *   k         1 <= k, 3 (k + extra) <= n
 *   tol       residual tolerance (> 0), see tol_kind
 *   X0        device, column-major n x (k + extra) initial block, or NULL for a seeded
 *             N(0, 1) block (Philox4x32-10 keyed by opt.seed)
 *   evals     host, k ascending eigenvalues
 *   evecs     device, column-major n x k eigenvectors, unit 2-norm, largest-|.|
 *             entry positive
 *   resnorms  host, k values ||A x_j - lambda_j x_j||_2 recomputed with a fresh product
 *   info      host, optional (NULL)
 * Returns OK, ENOCONV (outputs hold the best approximation), EINVAL, ENOMEM, ECUDA,
 * EBREAKDOWN. */
LOBPCG_API lobpcg_status lobpcg_solve(lobpcg_ctx* ctx, int k, double tol, const double* X0, double* evals,
                           double* evecs, double* resnorms, lobpcg_info* info);

/* Solves nprob independent problems concurrently (the batched serving form; not in the
 * paper).  ctxs[i] is a context from lobpcg_create; give each its own stream so that the
 * problems' kernels run side by side.  A pool of nthreads host threads (<= 0: 32) runs
 * lobpcg_solve(ctxs[i], k[i], tol[i], X0 ? X0[i] : NULL, evals[i], evecs[i],
 * resnorms[i], infos ? &infos[i] : NULL), largest problems first; statuses[i] receives
 * each result.  Every problem's arithmetic is exactly that of lobpcg_solve, so the
 * results equal one-by-one solves.  Each context releases its block workspace when its
 * problem is done, so only the problems in flight hold it.  Returns OK when every
 * problem returned OK, else the first non-OK status in problem order.  Contexts must be
 * distinct. */
LOBPCG_API lobpcg_status lobpcg_solve_batched(lobpcg_ctx* const* ctxs, int nprob, const int* k, const double* tol,
                                              const double* const* X0, double* const* evals, double* const* evecs,
                                              double* const* resnorms, lobpcg_info* infos, lobpcg_status* statuses,
                                              int nthreads);

/* Releases the context and everything it owns.  NULL-safe. */
LOBPCG_API void lobpcg_destroy(lobpcg_ctx* ctx);

/* Description of the last error of ctx, or (ctx == NULL) of the calling thread's last
 * failed lobpcg_create or building-block call.  Never NULL; valid until the next call. */
LOBPCG_API const char* lobpcg_last_error(const lobpcg_ctx* ctx);

/* ------------------------------------------------------------------------------
 * Building blocks of Algorithm 1, exposed for unit checks and for callers that drive
 * their own iteration.  Blocks here are ROW-major: row i of an n x p block B starts at
 * B + i*ld (ld >= p).  All arrays are device arrays; work is issued on `stream` and
 * the call returns after the stream has finished it.
 * ------------------------------------------------------------------------------ */

/* Y = A X for CSR A (Algorithm 1, "AW = A W").  X: n x p (ldx), Y: n x p (ldy), p <= 32.
 * Returns EINVAL for p outside [1, 32] or NULL pointers. */
LOBPCG_API lobpcg_status lobpcg_spmm_csr_f64(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                  const double* val, int p, const double* X, int ldx, double* Y,
                                  int ldy, lobpcg_stream stream);

/* Y = A X for CSR A (nnz entries) like lobpcg_spmm_csr_f64, formed in double-float
 * arithmetic on the FP32 pipes (the FP64 refinement's product, see
 * lobpcg_options.df_products): values and X split into float pairs, compensated row sums,
 * FP64 result.  X, Y: 16-byte aligned, even row strides; p <= 32.  Allocates the split
 * copies on every call.  Not in the paper; the operation is Algorithm 1's A W. */
LOBPCG_API lobpcg_status lobpcg_spmm_csr_f64_df(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                                const double* val, int64_t nnz, int p, const double* X, int ldx,
                                                double* Y, int ldy, lobpcg_stream stream);

/* Y = A X in FP32 with A's values rounded to FP32: the product of the mixed form
 * (Algorithm 1, "AW = A W", with FP32 blocks).  X, Y: n x p float, row-major, 16-byte
 * aligned with ldx, ldy multiples of 4; p <= 32.  band = -1 picks the half-width b that
 * holds 80% of the entries (the choice lobpcg_create makes); band >= 0 forces b; band = -2
 * uses the unsplit product.  With b >= 0 the matrix is split into A_band (|col - row| <= b,
 * gathered from a shared-memory window of X) and A_lr (the rest, added by a second
 * kernel).  *band_used (nullable) receives b, or -1 for the unsplit product.  Allocates
 * its temporaries (the split copy of A) on every call.  EINVAL for bad sizes, NULL
 * pointers or misaligned blocks. */
LOBPCG_API lobpcg_status lobpcg_spmm_csr_f32(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                  const double* val, int64_t nnz, int p, const float* X, int ldx,
                                  float* Y, int ldy, int band, int* band_used, lobpcg_stream stream);

/* The rule by which the mixed form leaves FP32 (lobpcg_options.mixed_switch; with
 * switch_tol = 0 the rounding-floor rule), replayed on the host over a history rk[0..n) of
 * the largest sought residual norm per FP32 iteration: *leave_at receives the first i after
 * which the solver leaves FP32, or -1.  switch_tol > 0: the first i with rk[i] <= switch_tol.
 * switch_tol = 0: once rk[i] <= 1e-2 rk[0], the first i at which the residual fell by a
 * factor <= 0.6 per iteration over iterations i-5 .. i-2 and then by less than 25% at both
 * i-1 and i; or the first i at which the best rk so far has not improved by 10% for 2
 * iterations (best <= 1e-2 rk[0]) or for 5 iterations.  No device work.  EINVAL for a NULL
 * pointer (rk may be NULL when n == 0), n < 0 or switch_tol < 0. */
LOBPCG_API lobpcg_status lobpcg_mixed_switch_replay(const double* rk, int n, double switch_tol, int* leave_at);

/* Tridiagonal preconditioner (Sec. 4.4; the option LOBPCG_PREC_TRIDIAG): W[:, j] =
 * (T - shift[j] I)^{-1} R[:, j] for j < p, with T the tridiagonal matrix of sub-diagonal
 * dl (dl[i] = T[i+1][i]), diagonal d and super-diagonal du (du[i] = T[i][i+1]); dl, du hold
 * n - 1 entries (NULL allowed when n == 1).  R and W are row-major n x p with leading
 * dimensions ldr, ldw >= p; all arrays are device memory owned by the caller.  The solve
 * splits the rows into partitions (32 to 1024 rows, chosen from n and p), eliminates each
 * with partial pivoting (row interchanges between neighbours), then couples the partitions
 * through their first and last unknowns; pivots smaller than 1e-8 max(1, |shift[j]|) are replaced by that value
 * with their sign.  It computes in FP32 (a preconditioner shapes a search direction; the
 * solver orthonormalises the result in its own precision).  Allocates its scratch (about
 * 24 n p bytes) on every call.  EINVAL for n < 1, p outside [1, 32], ld < p or a NULL
 * array. */
LOBPCG_API lobpcg_status lobpcg_precond_tridiag(int64_t n, const double* dl, const double* d, const double* du,
                                                int p, const double* shift, const double* R, int ldr, double* W,
                                                int ldw, lobpcg_stream stream);

/* Y = A X for dense column-major symmetric A (lda >= n); X, Y as above, p <= 32. */
LOBPCG_API lobpcg_status lobpcg_spmm_dense_f64(int64_t n, const double* A, int64_t lda, int p,
                                    const double* X, int ldx, double* Y, int ldy,
                                    lobpcg_stream stream);

/* C = X^T Y (the Gram / projected matrices of Algorithm 1 and Eq. (CDOrtho)).
 * X: n x p (ldx), Y: n x q (ldy), p, q <= 96.  C: device, column-major p x q. */
LOBPCG_API lobpcg_status lobpcg_gram_f64(int64_t n, int p, const double* X, int ldx, int q, const double* Y,
                              int ldy, double* C, lobpcg_stream stream);

/* C = X^T Y like lobpcg_gram_f64, formed in double-float arithmetic on the FP32 pipes (the
 * arithmetic of the FP64 refinement, see lobpcg_options.df_products): each FP64 element is
 * split into two floats, products and sums are error-compensated, sums of ~128 rows are
 * added in FP64.  X, Y: 16-byte aligned, one even row stride (ldx == ldy).  Not in the
 * paper; the operation is Algorithm 1's Gram. */
LOBPCG_API lobpcg_status lobpcg_gram_f64_df(int64_t n, int p, const double* X, int ldx, int q, const double* Y,
                                            int ldy, double* C, lobpcg_stream stream);

/* The FP64 block update X = base + alpha [V_g] U (and AX, residual norms) in double-float
 * arithmetic; arguments as lobpcg_update_f32 with FP64 blocks (V_g, AV_g, base, X, AX:
 * double, row stride ld / ld_base / ld_out in doubles). */
LOBPCG_API lobpcg_status lobpcg_update_f64_df(int64_t n, int nseg, const double* const* V, const double* const* AV,
                                              const int* w, int ld, const double* U, int q, double alpha,
                                              const double* base, int ld_base, double* X, double* AX, int ld_out,
                                              const double* lam, double* resnorm, lobpcg_stream stream);

/* The block update of Algorithm 1 for FP32 blocks: X = base + alpha [V_0 .. V_{nseg-1}] U
 * and, with AV, AX = alpha [AV_0 ..] U (the basis and residual update X <- V u_x, AX <- AV u_x,
 * and P <- V u_p).  V_g, AV_g: device, n x w[g] row-major with row stride ld floats
 * (1 <= nseg <= 3, s = sum of w[g] <= 96, w[g] <= ld).  U: device FP64, s x q column-major,
 * q <= 32.  base (nullable, X only) and X, AX: device, row-major, strides ld_base, ld_out
 * >= q; X may alias base or V_0 (in place).  With resnorm (host, q doubles; needs AV, lam
 * and no base): resnorm[j] = || AX_j - lam_j X_j ||_2, lam device FP64 (q).  Products are
 * FP32 FMAs in the order of the rows of U.  Rows 16-byte aligned with ld a multiple of 4
 * take the staged kernel; other layouts a general one with the same arithmetic.
 * EINVAL for bad sizes or NULL pointers. */
LOBPCG_API lobpcg_status lobpcg_update_f32(int64_t n, int nseg, const float* const* V, const float* const* AV,
                                          const int* w, int ld, const double* U, int q, double alpha,
                                          const float* base, int ld_base, float* X, float* AX, int ld_out,
                                          const double* lam, double* resnorm, lobpcg_stream stream);

/* C = X^T Y for FP32 blocks, the Gram of the mixed form (Algorithm 1's projected matrices
 * with FP32 storage), with warp-level mma.sync (the solver's default is the tcgen05 kernel
 * of lobpcg_gram_f32_tcgen05, see lobpcg_options.tc_gram).  X: n x p float (ldx), Y: n x q float (ldy), p, q <= 96.  C: device,
 * FP64, column-major p x q.  When the rows are 16-byte aligned with ldx == ldy a multiple
 * of 4, it runs on the tensor cores: TF32 mma with the 3xTF32 split, x = x_hi + x_lo and
 * a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, which keeps ~21 bits per product.  Otherwise it
 * runs on the FP32 FMA units.  Sums are FP32 within a CTA, FP64 across CTAs (fixed
 * order). */
LOBPCG_API lobpcg_status lobpcg_gram_f32(int64_t n, int p, const float* X, int ldx, int q, const float* Y,
                              int ldy, double* C, lobpcg_stream stream);

/* The FP32 Gram of lobpcg_gram_f32 (3xTF32 products, FP32 sums within a CTA, FP64 across
 * CTAs) on the 5th-generation tensor cores: rows staged by TMA bulk copies, operands split
 * into TF32 hi / lo parts in shared memory, tcgen05.mma with the accumulator in tensor
 * memory, each 32- or 64-row chunk's sum added to FP32 running sums with round-to-nearest
 * adds.  X, Y: 16-byte aligned, one row stride (ldx == ldy, a multiple of 4); p, q <= 96.
 * Each copy reads the rows' full stride except for the last row, of which it reads the
 * used columns rounded up to 16 bytes (never past the 16-byte granule of the last
 * element).  EINVAL for other layouts; ECUDA if a CTA gave up waiting on a copy, an MMA
 * or a pipeline stage.  The operation is Algorithm 1's Gram; the kernel design is not
 * from the paper. */
LOBPCG_API lobpcg_status lobpcg_gram_f32_tcgen05(int64_t n, int p, const float* X, int ldx, int q, const float* Y,
                                                 int ldy, double* C, lobpcg_stream stream);

/* Symmetric eigen-decomposition of s x s column-major a (s <= 96) by parallel-order
 * Jacobi rotations in FP64 (the Rayleigh-Ritz solve of Algorithm 1).  lam: device, s
 * values ascending; U: device, column-major s x s eigenvectors. */
LOBPCG_API lobpcg_status lobpcg_syev_f64(int s, const double* a, double* lam, double* U, lobpcg_stream stream);

/* Same contract, two-stage method (the Rayleigh-Ritz solve of the FP32 phase of the mixed
 * form): FP32 Jacobi, one FP64 Cholesky-QR of its rotation matrix Q, then Jacobi on
 * Q^T a Q accumulated into Q until its off-diagonal mass is <= tol ||a||_F (tol = 0 means
 * 1e-15).  tol < 1e-12: FP64 rotations; eigenvalues and residuals to FP64 absolute accuracy
 * (~eps ||a||), U orthonormal to FP64 rounding.  1e-12 <= tol < 1e-6 (the solver uses
 * 1e-10): the rotations of that last stage update the small off-diagonal part in FP32
 * (diagonal and rotation product in FP64), good to about tol.  Exact zero couplings of a
 * are not kept.  EINVAL for tol outside [0, 1e-6). */
LOBPCG_API lobpcg_status lobpcg_syev2_f64(int s, const double* a, double tol, double* lam, double* U,
                                          lobpcg_stream stream);

/* Algorithm 2 in place on X (n x p row-major, ldx, p <= 32).  stats (host, optional):
 * [0] Cholesky-QR passes, [1] shifted attempts, [2] SVQB steps, [3] cap hit (0/1). */
LOBPCG_API lobpcg_status lobpcg_ortho_f64(int64_t n, int p, double* X, int ldx, double tau, int cap,
                               int* stats, lobpcg_stream stream);

/* Algorithm 3 in place: orthonormalise X (n x p, p <= 32) against orthonormal Y
 * (n x q, q <= 64).  stats (host, optional): [0] projection passes, [1] max
 * Cholesky-QR passes, [2] shifted attempts, [3] SVQB steps, [4] cap hits. */
LOBPCG_API lobpcg_status lobpcg_ortho_against_f64(int64_t n, int p, double* X, int ldx, int q,
                                       const double* Y, int ldy, double tau, int cap, int cap2,
                                       int* stats, lobpcg_stream stream);

/* ------------------------------------------------------------------------------
 * Learned preconditioner (LOBPCG_PREC_LEARNED).  Not in the paper; its preconditioner
 * study (Sec. 4.4, Table 1) motivates correcting the diagonal step of Sec. 2.  Per
 * (row i, active column j) a 3 -> 64 -> 64 -> 1 ReLU perceptron gives z and
 *     w_ij = softplus(z) r_ij / (d_i - theta_j)
 * for rows with |d_i - theta_j| <= 64 c (c = mean off-diagonal row 2-norm rho); other
 * rows keep the diagonal step.  Features: f1 = (d_i - theta_j) / (8 c), f2 = rho_i / c,
 * f3 = r_ij / max_i |r_ij|.  Weights and activations are BF16, sums FP32.  Parameter
 * vector (float, lobpcg_mlp_num_params() = 4481 entries, row-major out x in):
 *     W1[64][3] b1[64] W2[64][64] b2[64] W3[64] b3[1].
 * The entry points below train it; all arrays are device arrays and every call returns
 * after the stream has finished its work.
 * ------------------------------------------------------------------------------ */

/* Number of parameters of the perceptron (4481). */
LOBPCG_API int lobpcg_mlp_num_params(void);

/* s_i = softplus(MLP(F_i)) for N samples; F: N x 3 row-major.  bf16 != 0 rounds
 * weights, inputs and activations to BF16 as the solver does; bf16 == 0 keeps FP32
 * (only for checking the arithmetic). */
LOBPCG_API lobpcg_status lobpcg_mlp_forward(int64_t N, const float* F, const float* params, float* s, int bf16,
                                            lobpcg_stream stream);

/* grad += sum_i g_i ds_i / dparams, taken at the (BF16-rounded when bf16 != 0) parameters. */
LOBPCG_API lobpcg_status lobpcg_mlp_backward(int64_t N, const float* F, const float* params, const float* g,
                                             float* grad, int bf16, lobpcg_stream stream);

/* Training loss: samples grouped by column col[i] in [0, ncol); w_i = s_i q_i;
 * per column L_c = 1 - (w.e)^2 / (|w|^2 ee_c) with the fixed contributions far_we_c,
 * far_ww_c of the rows outside the learned region added to w.e and |w|^2.
 *   work: device, 2 ncol doubles;  loss: device double, mean of L_c;  dLds: dloss/ds_i. */
LOBPCG_API lobpcg_status lobpcg_mlp_loss(int64_t N, int ncol, const int32_t* col, const float* q, const float* e,
                                         const float* s, const double* far_we, const double* far_ww, const double* ee,
                                         double* work, float* dLds, double* loss, lobpcg_stream stream);

/* One Adam step on params (FP32 master copy) from grad, which is then zeroed.
 * np must equal lobpcg_mlp_num_params(); step >= 1 is the 1-based step count. */
LOBPCG_API lobpcg_status lobpcg_mlp_adam(int np, float* params, float* grad, float* m, float* v, int step, float lr,
                                         float beta1, float beta2, float eps, lobpcg_stream stream);

/* Training features of a block of Ritz pairs (row-major X, AX: n x p, ld): for every
 * (row i, column j): F (3 floats, as above), q = r_ij / guard(d_i - lam_j), e = XS_ij -
 * alpha_j X_ij (the exact correction made orthogonal to x_j when XS holds the aligned
 * exact eigenvector and alpha_j = x_j . XS_j), near flag; and per column (sums, 3 p
 * doubles): |e|^2 over all rows, then (q e) and q^2 summed over the rows outside the
 * learned region.  rho / cscale: from lobpcg_row_norms; colmax_j = max_i |r_ij|. */
LOBPCG_API lobpcg_status lobpcg_precond_features(int64_t n, int p, const double* X, const double* AX, int ld,
                                                 const double* lam, const double* diag, const float* rho, float cscale,
                                                 const double* colmax, const double* XS, const double* alpha, float* F,
                                                 float* q, float* e, int* near, double* sums, lobpcg_stream stream);

/* rho_i = off-diagonal 2-norm of row i of A (CSR, or dense column-major when dense != NULL);
 * *mean_out (host) = mean of rho. */
LOBPCG_API lobpcg_status lobpcg_row_norms(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                          const double* val, const double* dense, int64_t lda, float* rho,
                                          double* mean_out, lobpcg_stream stream);

/* C = X^T Y exactly like lobpcg_gram_f64, but without allocating any memory.  The paper
 * has no counterpart; this entry point exists for callers that cannot allocate device
 * memory: for example a serving loop that sizes all of its GPU memory at start-up and
 * must not call cudaMalloc afterwards (cudaMalloc can synchronise the device and can
 * fail under memory pressure), or code whose device memory is owned by another
 * allocator.  The split-row partial sums go to a fixed array in the library,
 * 152 x 1024 doubles (1.2 MB), which every GPU that loads the library holds until the
 * process exits.
 *   n >= 1; 1 <= p, q <= 96; p * q <= 1024 (else LOBPCG_EINVAL); X: n x p (ldx), Y: n x q (ldy),
 *   row-major, device; C: device, column-major p x q.
 * The first call on a device looks up that array's device address (cudaGetSymbolAddress)
 * with the device current; make that first call before any stream capture.  All calls
 * share the one array: calls whose work overlaps on the GPU (different streams or
 * threads) race and give wrong results; serialise them.  Every partial sum a call
 * reads is written by that same call, so nothing left by an earlier call leaks into
 * the result.  Returns after the stream has finished the work. */
LOBPCG_API lobpcg_status lobpcg_gram_f64_noalloc(int64_t n, int p, const double* X, int ldx, int q,
                                                 const double* Y, int ldy, double* C, lobpcg_stream stream);

/* ------------------------------------------------------------------------------
 * Measurement.  The paper has no counterpart: this measures the part the solver runs on.
 * ------------------------------------------------------------------------------ */

/* Peak rate of the FMA pipes of the current device in TFLOP/s (an FMA counts as 2 flops):
 * fp64 != 0 measures FP64 fused multiply-adds, fp64 == 0 FP32 ones.  Independent FMA
 * chains fill every SM; the launch is calibrated to about 50 ms and the best of 5 is
 * returned in *tflops (host).  This is the denominator of the rooflines of the kernels
 * bound by the FMA pipes.  Allocates a small output array; synchronises the stream.
 * EINVAL for a NULL tflops, ECUDA on a CUDA failure. */
LOBPCG_API lobpcg_status lobpcg_probe_fma_rate(int fp64, double* tflops, lobpcg_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* LOBPCG_H */
