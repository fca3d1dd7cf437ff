// Shared device helpers and the internal launch interface of the GB300 LOBPCG library.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>

namespace lobpcg {

constexpr int kMaxS = 96;     // largest Rayleigh-Ritz size s = m + 2 m_act (m <= 32)
constexpr int kMaxM = 32;     // largest block width m = k + extra
constexpr int kWarp = 32;

struct CudaError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

#define LB_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw ::lobpcg::CudaError(std::string(#call) + ": " + cudaGetErrorString(e_) + " (" + \
                                __FILE__ + ":" + std::to_string(__LINE__) + ")");          \
  } while (0)

// Every kernel launch of the library goes through LB_LAUNCH_CHECK, which also counts it.
long long& launch_counter();
#define LB_LAUNCH_CHECK()               \
  do {                                  \
    ++::lobpcg::launch_counter();       \
    LB_CUDA(cudaGetLastError());        \
  } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int round_up(int a, int b) { return (a + b - 1) / b * b; }
__host__ __device__ inline int64_t ceil_div_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

// A logical n x w block made of up to three row-major segments placed side by side
// (the expansion basis V = [X | P | W] and AV = [AX | AP | AW]).
template <class T>
struct Cols {
  const T* p[3];
  int ld[3];
  int w[3];
  int nseg;
  __host__ __device__ int width() const {
    int s = 0;
    for (int i = 0; i < nseg; ++i) s += w[i];
    return s;
  }
};

template <class T>
inline Cols<T> cols1(const T* p, int ld, int w) {
  Cols<T> c{};
  c.p[0] = p, c.ld[0] = ld, c.w[0] = w, c.nseg = w > 0 ? 1 : 0;
  return c;
}
template <class T>
inline Cols<T> cols_add(Cols<T> c, const T* p, int ld, int w) {
  if (w > 0) {
    c.p[c.nseg] = p, c.ld[c.nseg] = ld, c.w[c.nseg] = w;
    c.nseg++;
  }
  return c;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ----------------------------------------------------------------------------------
// Launch wrappers (host side).  All take the stream; none synchronises.
// ----------------------------------------------------------------------------------

// Y = A X, CSR, row-major blocks.  p <= 32.  band >= 0: half-width of the band that holds
// most non-zeros (from profile_band); the product then stages that window of X in
// shared memory.  pure: every entry satisfies |col - row| <= band (the band part of a
// split matrix), so no gather leaves the window.
// variant: kSpmmAuto picks by precision, alignment and band; the others force one kernel
// family (when the blocks allow it): the row-parallel kernel, the vector-gather kernel
// (no band window), or the band window kernel with global gathers outside the band.
// kSpmmWindow applies to the band part of a split matrix: the window kernel on its unpacked
// CSR arrays instead of the packed form (here it acts as kSpmmAuto).
enum { kSpmmAuto = 0, kSpmmRows = 1, kSpmmVec = 2, kSpmmBand = 3, kSpmmWindow = 4 };
template <class T, class V>
void launch_spmm_csr(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const V* val,
                     int p, const T* X, int ldx, T* Y, int ldy, cudaStream_t st, int band = -1,
                     bool pure = false, int variant = kSpmmAuto);
// Y += A X for a CSR matrix whose rows hold few, scattered entries (the long-range part of
// a band / long-range split).  Row-major 16-byte aligned blocks, p <= 32.
template <class T, class V>
void launch_spmm_csr_add(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const V* val, int p,
                         const T* X, int ldx, T* Y, int ldy, cudaStream_t st);
// Band / long-range split A = A_band + A_lr with A_band holding |col - row| <= band:
// per-row counts, exclusive scan of counts into row pointers (scratch: split_scan_scratch(n)
// int64), and the scatter of column indices and values (rounded to V).
void split_csr_count(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, int band, int32_t* cnt_band,
                     int32_t* cnt_lr, cudaStream_t st);
int64_t split_scan_scratch(int64_t n);
void split_csr_rowptr(int64_t n, const int32_t* cnt, int64_t* row_ptr_out, int64_t* scratch, cudaStream_t st);
template <class V>
void split_csr_scatter(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val, int band,
                       const int64_t* rp_band, int32_t* ci_band, V* v_band, const int64_t* rp_lr, int32_t* ci_lr,
                       V* v_lr, cudaStream_t st);
// Packed form of the band part (FP32): entries as (col - row, value bits) pairs with the
// column clamped into [row - band, row + band] and [0, n), rows padded to an even length
// with a (0, 0.0f) entry; row pointers from the scan of split_even_counts.  launch_spmm_band_packed computes Y = A_band X from it and returns
// false, without launching, when the blocks or the band do not fit its shared-memory window.
void split_even_counts(int64_t n, const int32_t* cnt, int32_t* out, cudaStream_t st);
void split_pack_band(int64_t n, int band, const int64_t* rp_band, const int32_t* ci_band, const float* v_band,
                     const int64_t* rp_packed, int2* packed, cudaStream_t st);
bool launch_spmm_band_packed(int64_t n, const int64_t* rp_packed, const int2* packed, int p, const float* X,
                             int ldx, float* Y, int ldy, int band, cudaStream_t st);
// Smallest half-width b in {16, ..., 2048} with 80% of the non-zeros at |col - row| <= b,
// or -1 (synchronises the stream).
int profile_band(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, int64_t nnz, cudaStream_t st);
// Y = A X, dense column-major symmetric A.
template <class T>
void launch_spmm_dense(int64_t n, const T* A, int64_t lda, int p, const T* X, int ldx, T* Y,
                       int ldy, cudaStream_t st);

// Gram partials: part[g][i + j*pa] = sum over CTA g's rows of a_ri * b_rj.
// upper: only i <= j entries are produced.  Returns the number of CTAs used.
template <class T>
int gram_partials(int64_t n, const Cols<T>& a, const Cols<T>& b, bool upper, double* part,
                  int max_ctas, cudaStream_t st);
// Pipelined variants (tiles.cu) for operands sharing one 16-byte aligned row stride;
// return 0 without launching when they do not apply.
template <class T>
int gram_partials_pipe(int64_t n, const Cols<T>& a, const Cols<T>& b, bool upper, double* part, int max_ctas,
                       cudaStream_t st);
template <class T>
struct UpdateJob;
template <class T>
int launch_update_pipe(int64_t n, const UpdateJob<T>& job, const double* U, int s, int q, double alpha,
                       const double* lam, double* norm_part, int max_ctas, cudaStream_t st);
// FP32 Gram partials on the 5th-generation tensor cores (tcgen05, TMA bulk copies, TMEM
// accumulator; 3xTF32 products); returns 0 without launching when the operands do not
// share one 16-byte aligned row stride or are wider than 96 columns.  umma_check reads and
// clears its give-up flag (synchronising the stream) and throws if a CTA gave up waiting.
int gram_partials_umma(int64_t n, const Cols<float>& a, const Cols<float>& b, bool upper, double* part,
                       int max_ctas, cudaStream_t st);
void umma_check(cudaStream_t st);
// out[e] = sum_g part[g][e] for e < count (FP64, fixed order).
void reduce_partials(const double* part, int nparts, int count, double* out, cudaStream_t st);

// out_t = base_t + alpha * in_t * U for t = 0..nprod-1 (U: s x q column-major FP64 on device).
// in_t: Cols of width s; out_t/base_t row-major (ld).  base_t may be null (then 0).
// When norm_part != null (nprod == 2, out0 = X, out1 = AX): also accumulates per-column
// partial sums of r_ij^2 and max |r_ij| with r = AX - X diag(lam) into norm_part[cta][2*q].
// unit_base (FP64 double-float path only): out = in + in (U - I) for an in-place square
// right-multiply (s == q, one segment), so the unchanged part of in is carried in FP64 and
// only the correction is formed from float pairs; the FP64 FMA path computes in U.
template <class T>
struct UpdateJob {
  Cols<T> in[2];
  T* out[2];
  int ld_out[2];
  const T* base[2];
  int ld_base[2];
  int nprod;
  int unit_base;
};
template <class T>
int launch_update(int64_t n, const UpdateJob<T>& job, const double* U, int s, int q, double alpha,
                  const double* lam, double* norm_part, int max_ctas, cudaStream_t st);

// The same FP64 products formed in double-float arithmetic on the FP32 pipes (FP64 data,
// FP64 results; every product and sum error-compensated, see dfloat.cuh).
// gram_partials_df returns 0 without launching when the operands do not share one
// aligned row stride.
int gram_partials_df(int64_t n, const Cols<double>& a, const Cols<double>& b, bool upper, double* part,
                     int max_ctas, cudaStream_t st);
int launch_update_df(int64_t n, const UpdateJob<double>& job, const double* U, int s, int q, double alpha,
                     const double* lam, double* norm_part, int max_ctas, cudaStream_t st);
// dst[i] = (hi, lo) split of src[i] (the double-float operands: matrix values, blocks).
void launch_split_df(int64_t count, const double* src, float2* dst, cudaStream_t st);
// Y = A X (FP64 result) from the split values vs (nnz) and the split block Xs (n x ldx
// pairs, row-major, ldx even, p <= 32); Y row-major FP64 (ldy even).
void launch_spmm_csr_df(int64_t n, const int64_t* rp, const int32_t* ci, const float2* vs, int p,
                        const float2* Xs, int ldx, double* Y, int ldy, cudaStream_t st);

// W~_ij = R_ij / guard(d_i - lam_{c0+j}) (precond 1) or R_ij (precond 0) with
// R = AX[:, c0+j] - lam_{c0+j} X[:, c0+j], j < a.  With diagB (generalised problem: pass B X
// as X) the denominator is d_i - lam diagB_i.  `floor` > 0 floors |denominator| at it (sign
// kept): the damped diagonal.
template <class T>
void launch_precond(int64_t n, const T* X, const T* AX, int ld, const double* lam, int c0, int a,
                    const double* diag, int precond, T* W, int ldw, cudaStream_t st,
                    const double* diagB = nullptr, double floor = 0.0);
// Tridiagonal preconditioner (tridiag.cu): W[:, c] = (T - lam[c0 + c] I)^{-1} r_{c0+c} for
// c < a, r = AX - X lam (or r = AX when X is NULL), T = (dl, d, du) in FP64; FP32 solve
// through tridiag_scratch_floats(n, a) floats of scratch.  tridiag_extract fills dl
// (A[i+1][i]) and du (A[i][i+1]) from CSR (duplicates summed) or dense column-major A.
int tridiag_partition_rows(int64_t n, int a);
int64_t tridiag_partitions(int64_t n);
size_t tridiag_scratch_floats(int64_t n, int a);
void tridiag_extract(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                     const double* dense, int64_t lda, double* dl, double* du, cudaStream_t st);
template <class T>
void launch_precond_tridiag(int64_t n, const T* X, const T* AX, int ld, const double* lam, int c0, int a,
                            const double* d, const double* dl, const double* du, T* W, int ldw, float* scratch,
                            cudaStream_t st);

// row-major (ld) <-> column-major (n x p) conversions, optional precision change.
template <class Tin, class Tout>
void launch_colmajor_to_rows(int64_t n, int p, const Tin* src, Tout* dst, int ld, cudaStream_t st);
template <class Tin, class Tout>
void launch_rows_to_colmajor(int64_t n, int p, const Tin* src, int ld, Tout* dst, cudaStream_t st);
// Seeded N(0,1) column-major block (Philox4x32-10 + Box-Muller).
void launch_gaussian(int64_t n, int p, uint64_t seed, double* dst, cudaStream_t st);
// dst[i] = (float) src[i]
void launch_to_float(int64_t count, const double* src, float* dst, cudaStream_t st);
// true if every entry is finite (result written to *flag on device as 0/1)
void launch_all_finite(int64_t count, const double* src, int* flag, cudaStream_t st);

// ---- small FP64 kernels (one CTA) ----
// Symmetric eigensolve: a (s x s, column-major; only the upper triangle is read when
// upper_only) -> lam ascending, U column-major.  sweeps_out: device int (may be null),
// FP64 sweeps.  two_stage: FP32 Jacobi, Cholesky-QR of its rotations, FP64 Jacobi on
// Q^T a Q (faster; absolute accuracy eps ||a||); else FP64 Jacobi from a.  The FP64
// Jacobi stops when its off-diagonal mass is <= tol64 ||a||_F.
void launch_syev(int s, const double* a, bool upper_only, double* lam, double* U, int* sweeps_out,
                 cudaStream_t st, bool two_stage = false, double tol64 = 1e-15);

// Cholesky-QR step on the reduced Gram matrix M (p x p, column-major):
//  ctl[0] <- 1 if max|M - I| <= tau (already orthonormal), else 0 and Linv <- L^{-T}
//  of chol(M + shift) (upper triangular, column-major p x p).  ctl[1] += shifted
//  attempts, ctl[2] += 1 if SVQB had to be used (then Linv holds the SVQB transform).
//  ctl[6] <- 1 if the pass was unshifted with ||D M D - I||_F <= 1/2 (reading R17);
//  with C (q x p, first call of an Algorithm 3 pass) ctl[7] <- 1 if the pass's growth
//  factor squared is <= growth2 (reading R18).
void launch_cholqr_small(int p, const double* M, double tau, double* Linv, int* ctl,
                         cudaStream_t st, const double* C = nullptr, int q = 0, double growth2 = 0.0);
// max |C - I| over a p x p matrix -> *out (device double)
void launch_maxabs_minus_identity(int p, const double* C, double* out, cudaStream_t st);
// max |C| over a p x q matrix -> *out (device double)
void launch_maxabs(int count, const double* C, double* out, cudaStream_t st);

// Lock decision + P coefficients (Algorithm 1, lock and u_p steps):
//  reads norm partials (nparts x 2m), lam (m), U (s x s), state -> writes resnorm (m),
//  new m_conv / m_act, done flag, and u_p (s x p_cols) = ortho(u~_p; u_x) over the active
//  columns whose projected coefficient vector is not negligible (state->p_cols of them).
struct LockState {
  int m_conv;
  int m_act;
  int done;
  int sp_shifts;
  int sp_passes;
  int p_cols;  // columns of u_p (the active ones whose Ritz vector moved)
};
void launch_lock_and_p(int s, int m, int k, int64_t n, const double* norm_part, int nparts,
                       const double* U, double tol, int tol_kind, double tau, LockState* state,
                       double* resnorm, double* colmax, double* up, bool build_p, cudaStream_t st);

}  // namespace lobpcg

namespace lobpcg {
// Per-column largest |x_ij| with its sign (ties: smallest row) for the first p columns
// of a row-major block; writes sign (+1/-1) per column into sgn (device double).
template <class T>
void launch_col_sign(int64_t n, int p, const T* X, int ld, double* part, int max_ctas, double* sgn,
                     cudaStream_t st);
// scale[j] = sgn[j] / sqrt(G[j + j*p]) written as a p x p diagonal matrix S (column-major).
void launch_scale_matrix(int p, const double* G, const double* sgn, double* S, cudaStream_t st);
}  // namespace lobpcg
