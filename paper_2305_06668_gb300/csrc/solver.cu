// Host driver of Algorithm 1 (LOBPCG, Sec. 3.1) with Algorithms 2 and 3 (Sec. 3.2)
// and the C ABI declared in include/lobpcg.h.
//
// The iteration keeps every n-sized block on the GPU in row-major layout:
//   X, AX, P, AP (double-buffered: the new X and P are built from the old basis), W, AW.
// The expansion basis is ordered V = [X | P | W] (the paper writes (X, W, P); the order
// of basis vectors does not change the Rayleigh-Ritz problem, and this order keeps
// Y = [X | P] contiguous for ortho(W~; Y)).  Small matrices (<= 96 x 96) stay on the
// GPU in FP64; the host only reads a few flags per step to decide loop exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/lobpcg.h"
#include "common.cuh"
#include "switch_rule.cuh"
#include "mlp.cuh"

using namespace lobpcg;

namespace {
thread_local std::string g_create_error;
}

namespace lobpcg {
long long& launch_counter() {
  static thread_local long long n = 0;
  return n;
}
const char* set_thread_error(const std::string& msg) {
  g_create_error = msg;
  return g_create_error.c_str();
}
}  // namespace lobpcg

namespace {

// Orthogonality threshold of the FP64 phases with double-float products (reading R21):
// their products are good to ~2^-47 relative, so ||X^T X - I|| and ||Y^T X|| can be
// certified to about 1e-13, not to FP64's 1e-14; 1e-12 keeps the basis orthonormal far
// below what the residual tolerance needs (an error d in V^T V moves Ritz values by
// ~d ||A||, 1e-12 x 2000 = 2e-9 for tol 1e-8 on the CI-like workload).
constexpr double kTauDf = 1e-12;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }  // also on an exception between allocation and the explicit release
  void ensure(size_t b) {
    if (b <= bytes) return;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    if (b == 0) return;
    LB_CUDA(cudaMalloc(&p, b));
    bytes = b;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

struct InvalidArg : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct NoMem : std::runtime_error {
  using std::runtime_error::runtime_error;
};

struct Stats {
  int cholqr_passes_max = 0, ortho_passes_max = 0, shifts = 0, svqb = 0, cap_hits = 0;
  int64_t spmm_columns = 0;
  int64_t spmm_launches = 0;
  int64_t spmm_launches64 = 0, spmm_columns64 = 0;
  int precond_fallback = 0;
  int w_dropped = 0;
  int p_dropped = 0;
  int ortho_grams = 0, skipped_recheck = 0, skipped_test = 0;
  int64_t b_products = 0;
  double rr_gram32_bytes = 0.0;  // algorithmic bytes of the FP32 Rayleigh-Ritz Grams (V and AV read once)
  int64_t rr_gram32_count = 0;
};

// Optional per-phase timing with CUDA events recorded on the solver stream.
enum Phase { PH_SPMM = 0, PH_RR_GRAM, PH_RR_EIG, PH_UPDATE, PH_PRECOND, PH_ORTHO, PH_OTHER, PH_COUNT };
struct Profiler {
  bool on = false;
  int prec64 = 1;  // precision of the phases being marked (1: FP64, 0: FP32)
  cudaStream_t st = nullptr;
  std::vector<cudaEvent_t> pool;
  std::vector<int> phase;
  size_t used = 0;
  void begin(bool enable, cudaStream_t s) {
    on = enable;
    st = s;
    used = 0;
    phase.clear();
    kused = 0;
    kflops = 0.0;
  }
  void mark(int ph) {
    if (!on) return;
    if (used == pool.size()) {
      cudaEvent_t e;
      LB_CUDA(cudaEventCreate(&e));
      pool.push_back(e);
    }
    LB_CUDA(cudaEventRecord(pool[used], st));
    phase.push_back(ph + (prec64 ? PH_COUNT : 0));
    ++used;
  }
  // out[0..PH_COUNT) all phases, out64[0..PH_COUNT) the FP64 part
  void finish(double* out, double* out64) {
    for (int i = 0; i < PH_COUNT; ++i) out[i] = out64[i] = 0.0;
    if (!on || used < 2) return;
    LB_CUDA(cudaStreamSynchronize(st));
    for (size_t i = 0; i + 1 < used; ++i) {
      float ms = 0.f;
      LB_CUDA(cudaEventElapsedTime(&ms, pool[i], pool[i + 1]));
      const int ph = phase[i] % PH_COUNT;
      out[ph] += ms * 1e-3;
      if (phase[i] >= PH_COUNT) out64[ph] += ms * 1e-3;
    }
  }
  // event pairs around every FP64 block update (the FP64-bound update kernel), with the
  // algorithmic flops of each: 2 n s q per product
  std::vector<cudaEvent_t> kpool;
  size_t kused = 0;
  double kflops = 0.0;
  void kmark() {
    if (kused == kpool.size()) {
      cudaEvent_t e;
      LB_CUDA(cudaEventCreate(&e));
      kpool.push_back(e);
    }
    LB_CUDA(cudaEventRecord(kpool[kused], st));
    ++kused;
  }
  // seconds of the timed updates (after finish's synchronisation)
  double kseconds() {
    double t = 0.0;
    for (size_t i = 0; i + 1 < kused; i += 2) {
      float ms = 0.f;
      LB_CUDA(cudaEventElapsedTime(&ms, kpool[i], kpool[i + 1]));
      t += ms * 1e-3;
    }
    return t;
  }
  ~Profiler() {
    for (auto e : pool) cudaEventDestroy(e);
    for (auto e : kpool) cudaEventDestroy(e);
  }
};

// Block workspace of one precision.
template <class T>
struct Blocks {
  DevBuf buf;
  int ld = 0;
  int64_t n = 0;
  T *X[2]{}, *AX[2]{}, *P[2]{}, *AP[2]{}, *W = nullptr, *AW = nullptr;
  void ensure(int64_t n_, int m) {
    const int vec = 16 / (int)sizeof(T);
    const int ld_ = round_up(m, vec);
    const size_t per = (size_t)n_ * ld_ * sizeof(T);
    buf.ensure(per * 10);
    n = n_;
    ld = ld_;
    T* b = buf.as<T>();
    const size_t e = (size_t)n_ * ld_;
    X[0] = b, X[1] = b + e, AX[0] = b + 2 * e, AX[1] = b + 3 * e;
    P[0] = b + 4 * e, P[1] = b + 5 * e, AP[0] = b + 6 * e, AP[1] = b + 7 * e;
    W = b + 8 * e, AW = b + 9 * e;
  }
};

}  // namespace

// FP32 copy of a CSR matrix split into A_band (|col - row| <= band) and A_lr (the rest),
// both in CSR with the original row order of the entries, plus A_band in packed form
// ((col - row, value) pairs, rows padded to even length) for the packed window kernel.
struct SplitCSR {
  DevBuf rp_buf, ci_buf, val_buf, rpk_buf, pk_buf;
  const int64_t *rp_band = nullptr, *rp_lr = nullptr, *rp_pk = nullptr;
  const int32_t *ci_band = nullptr, *ci_lr = nullptr;
  const float *v_band = nullptr, *v_lr = nullptr;
  const int2* pk = nullptr;
  int64_t nnz_band = 0, nnz_lr = 0, nnz_pk = 0;
  int band = -1;

  void build(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val, int64_t nnz, int b,
             cudaStream_t st) {
    DevBuf cnt, scratch;
    cnt.ensure((size_t)3 * std::max<int64_t>(n, 1) * sizeof(int32_t));
    scratch.ensure((size_t)split_scan_scratch(n) * sizeof(int64_t));
    int32_t* cb = cnt.as<int32_t>();
    int32_t* cl = cb + n;
    int32_t* ce = cl + n;
    split_csr_count(n, row_ptr, col_idx, b, cb, cl, st);
    split_even_counts(n, cb, ce, st);
    rp_buf.ensure((size_t)2 * (n + 1) * sizeof(int64_t));
    rpk_buf.ensure((size_t)(n + 1) * sizeof(int64_t));
    int64_t* rpb = rp_buf.as<int64_t>();
    int64_t* rpl = rpb + (n + 1);
    int64_t* rpk = rpk_buf.as<int64_t>();
    split_csr_rowptr(n, cb, rpb, scratch.as<int64_t>(), st);
    split_csr_rowptr(n, cl, rpl, scratch.as<int64_t>(), st);
    split_csr_rowptr(n, ce, rpk, scratch.as<int64_t>(), st);
    int64_t tot[3] = {0, 0, 0};
    LB_CUDA(cudaMemcpyAsync(&tot[0], rpb + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LB_CUDA(cudaMemcpyAsync(&tot[1], rpl + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LB_CUDA(cudaMemcpyAsync(&tot[2], rpk + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LB_CUDA(cudaStreamSynchronize(st));
    if (tot[0] + tot[1] != nnz) throw std::runtime_error("band split: entry counts do not add up to nnz");
    nnz_band = tot[0], nnz_lr = tot[1], nnz_pk = tot[2];
    const size_t nz = (size_t)std::max<int64_t>(nnz, 1);
    ci_buf.ensure(nz * sizeof(int32_t));
    val_buf.ensure(nz * sizeof(float));
    pk_buf.ensure((size_t)std::max<int64_t>(nnz_pk, 2) * sizeof(int2));
    int32_t* cib = ci_buf.as<int32_t>();
    float* vb = val_buf.as<float>();
    split_csr_scatter<float>(n, row_ptr, col_idx, val, b, rpb, cib, vb, rpl, cib + tot[0], vb + tot[0], st);
    split_pack_band(n, b, rpb, cib, vb, rpk, pk_buf.as<int2>(), st);
    LB_CUDA(cudaStreamSynchronize(st));
    cnt.release();
    scratch.release();
    rp_band = rpb, rp_lr = rpl, rp_pk = rpk;
    ci_band = cib, ci_lr = cib + tot[0];
    v_band = vb, v_lr = vb + tot[0];
    pk = pk_buf.as<int2>();
    band = b;
  }
  // Y = A_band X (the packed window kernel by default), then Y += A_lr X
  void apply(int64_t n, int p, const float* X, int ldx, float* Y, int ldy, cudaStream_t st,
             int variant = kSpmmAuto) const {
    if (variant != kSpmmAuto || !launch_spmm_band_packed(n, rp_pk, pk, p, X, ldx, Y, ldy, band, st))
      launch_spmm_csr<float, float>(n, rp_band, ci_band, v_band, p, X, ldx, Y, ldy, st, band, true,
                                    variant == kSpmmWindow ? kSpmmAuto : variant);
    if (nnz_lr > 0) launch_spmm_csr_add<float, float>(n, rp_lr, ci_lr, v_lr, p, X, ldx, Y, ldy, st);
  }
  void release() {
    rp_buf.release();
    ci_buf.release();
    val_buf.release();
    rpk_buf.release();
    pk_buf.release();
  }
};

struct lobpcg_ctx {
  lobpcg_matrix A{};
  lobpcg_options opt{};
  cudaStream_t st = nullptr;
  std::string err;
  int sms = 152;
  int max_ctas = 304;
  int band = -1;  // CSR: half-width holding most non-zeros (shared-memory window of the product)

  DevBuf val32, dense32;  // FP32 copies for the mixed form
  DevBuf val_df, xs_df;   // (hi, lo) float pairs of the CSR values and of a product's input block
  // mixed form, CSR with a band: the FP32 matrix split into the band part (|col - row| <=
  // band, product from a shared-memory window of X) and the long-range rest
  SplitCSR sp;
  bool split = false;
  // CSR product kernels picked by the autotuner for each precision, and the block width
  // they were timed at (0: not yet)
  int var32 = kSpmmAuto, var64 = kSpmmAuto;
  int tuned32 = 0, tuned64 = 0;
  Blocks<double> b64;
  Blocks<float> b32;
  DevBuf small;  // all small FP64 matrices and partials
  double *Gpart = nullptr, *G = nullptr, *U = nullptr, *lam_all = nullptr, *up = nullptr;
  double *Tm = nullptr, *C = nullptr, *npart = nullptr, *resnorm = nullptr, *scal = nullptr;
  double *lam = nullptr, *sgn = nullptr, *S = nullptr, *colmax = nullptr;
  int* ictl = nullptr;  // [0..3] cholqr ctl, [4] sweeps, [5] finite flag
  LockState* lock = nullptr;
  DevBuf x0buf;        // column-major FP64 initial block when X0 == NULL
  DevBuf xbest;        // the FP32 phase's X with the smallest largest-sought residual (reading R22)
  DevBuf tri_offd;     // tridiagonal preconditioner: dl then du of A (n - 1 doubles each)
  DevBuf tri_scratch;  // its FP32 scratch (tridiag_scratch_floats(n, a))
  double* host = nullptr;  // pinned readback area
  Stats stats;
  Profiler prof;
  // learned preconditioner: weights (device), off-diagonal row norms rho, their mean
  DevBuf mlp_params, rho;
  float cscale = 0.f;
  bool use_learned = false;  // cleared for the rest of a solve when the residuals stall
  bool df_on = false;        // FP64 Grams and updates in double-float arithmetic (this phase)
  // generalised problem A x = lambda B x (Sec. 3.3): B (borrowed), B X, B P (double-
  // buffered like X and P), B W, and Q = orth(B X, B P) for the projection of W~
  lobpcg_matrix B{};
  bool gen = false;
  DevBuf gbuf;
  double *BX[2]{}, *BP[2]{}, *BW = nullptr, *Q = nullptr;
  int ldq = 0;
  void ensure_gen(int64_t n, int ld) {
    ldq = 2 * ld;
    const size_t e = (size_t)n * ld;
    gbuf.ensure(e * 7 * sizeof(double));
    double* b = gbuf.as<double>();
    BX[0] = b, BX[1] = b + e, BP[0] = b + 2 * e, BP[1] = b + 3 * e, BW = b + 4 * e, Q = b + 5 * e;
  }
  FILE* trace = nullptr;  // per-iteration JSON lines (LOBPCG_TRACE=path)
  bool trace_orth = false;  // LOBPCG_TRACE_ORTH=1: also trace max |V^T V - I|

  void sync() { LB_CUDA(cudaStreamSynchronize(st)); }

  void alloc_small() {
    const size_t gpart = (size_t)max_ctas * kMaxS * kMaxS;
    const size_t doubles = gpart + 8 * (size_t)kMaxS * kMaxS + (size_t)max_ctas * 4 * kMaxS + 64 * kMaxS;
    small.ensure(doubles * sizeof(double) + 4096);
    double* p = small.as<double>();
    Gpart = p, p += gpart;
    G = p, p += kMaxS * kMaxS;
    U = p, p += kMaxS * kMaxS;
    up = p, p += kMaxS * kMaxS;
    Tm = p, p += kMaxS * kMaxS;
    C = p, p += kMaxS * kMaxS;
    S = p, p += kMaxS * kMaxS;
    npart = p, p += (size_t)max_ctas * 4 * kMaxS;
    lam_all = p, p += kMaxS;
    lam = p, p += kMaxS;
    resnorm = p, p += kMaxS;
    scal = p, p += kMaxS;
    sgn = p, p += kMaxS;
    colmax = p, p += kMaxS;
    p += 7 * kMaxS;
    ictl = reinterpret_cast<int*>(p);
    lock = reinterpret_cast<LockState*>(ictl + 32);
    LB_CUDA(cudaMallocHost(&host, 64 * kMaxS * sizeof(double)));
  }
};

namespace {

// --------------------------------------------------------------------------- helpers

template <class T>
struct Prec;
template <>
struct Prec<double> {
  static Blocks<double>& blocks(lobpcg_ctx& c) { return c.b64; }
  static const double* val(lobpcg_ctx& c) { return c.A.val; }
  static const double* dense(lobpcg_ctx& c) { return c.A.dense; }
  static int64_t lda(lobpcg_ctx& c) { return c.A.ld; }
};
template <>
struct Prec<float> {
  static Blocks<float>& blocks(lobpcg_ctx& c) { return c.b32; }
  static const float* val(lobpcg_ctx& c) { return c.val32.as<float>(); }
  static const float* dense(lobpcg_ctx& c) { return c.dense32.as<float>(); }
  static int64_t lda(lobpcg_ctx& c) { return c.A.n; }
};

// launch_update with, in profile mode, the FP64 launches timed and their flops counted.
template <class T>
int update(lobpcg_ctx& c, const UpdateJob<T>& job, const double* U, int s, int q, double alpha, const double* lam,
           double* norm_part) {
  const bool timed = c.prof.on && sizeof(T) == 8;
  if (timed) c.prof.kmark();
  int parts;
  if constexpr (std::is_same<T, double>::value) {
    parts = c.df_on ? launch_update_df(c.A.n, job, U, s, q, alpha, lam, norm_part, c.max_ctas, c.st)
                    : launch_update<T>(c.A.n, job, U, s, q, alpha, lam, norm_part, c.max_ctas, c.st);
  } else {
    parts = launch_update<T>(c.A.n, job, U, s, q, alpha, lam, norm_part, c.max_ctas, c.st);
  }
  if (timed) {
    c.prof.kmark();
    c.prof.kflops += 2.0 * (double)c.A.n * s * q * job.nprod;
  }
  return parts;
}

// Y = A X with the product kernel chosen for this precision (no statistics).
template <class T>
void spmm_product(lobpcg_ctx& c, const T* X, int ldx, int p, T* Y, int ldy) {
  const int var = sizeof(T) == 4 ? c.var32 : c.var64;
  if (c.A.fmt == LOBPCG_CSR && std::is_same<T, float>::value && c.split)
    c.sp.apply(c.A.n, p, reinterpret_cast<const float*>(X), ldx, reinterpret_cast<float*>(Y), ldy, c.st, var);
  else if (c.A.fmt == LOBPCG_CSR)
    launch_spmm_csr<T, T>(c.A.n, c.A.row_ptr, c.A.col_idx, Prec<T>::val(c), p, X, ldx, Y, ldy, c.st, c.band,
                          false, var);
  else
    launch_spmm_dense<T>(c.A.n, Prec<T>::dense(c), Prec<T>::lda(c), p, X, ldx, Y, ldy, c.st);
}

// Autotuner of the CSR product: on the first solve with block width p, time every kernel
// family that applies to this matrix and precision (CUDA events, one warm-up and two timed
// products each, on scratch blocks) and keep the fastest.  The default choice wins ties
// within 2%.  Candidates: the default (packed window kernel on the band part of a split
// FP32 matrix, row-parallel for FP64, band window or vector gather otherwise), the window
// kernel on the unpacked band part (split FP32 matrices), the row-parallel kernel, the
// vector-gather kernel and the band window kernel with global gathers.
template <class T>
void autotune_spmm(lobpcg_ctx& c, int p, T* X, int ld, T* Y) {
  int& var = sizeof(T) == 4 ? c.var32 : c.var64;
  int& tuned = sizeof(T) == 4 ? c.tuned32 : c.tuned64;
  if (c.A.fmt != LOBPCG_CSR || !c.opt.autotune || p <= 0 || tuned == p) return;
  std::vector<int> cand = {kSpmmAuto, kSpmmRows, kSpmmVec};
  if (c.band >= 0) cand.push_back(kSpmmBand);
  if (sizeof(T) == 4 && c.split) cand = {kSpmmAuto, kSpmmWindow, kSpmmRows, kSpmmBand};  // band part of the split
  cudaEvent_t e0, e1;
  LB_CUDA(cudaEventCreate(&e0));
  LB_CUDA(cudaEventCreate(&e1));
  int best = kSpmmAuto;
  float tbest = 0.f;
  for (int v : cand) {
    var = v;
    spmm_product<T>(c, X, ld, p, Y, ld);
    LB_CUDA(cudaEventRecord(e0, c.st));
    spmm_product<T>(c, X, ld, p, Y, ld);
    spmm_product<T>(c, X, ld, p, Y, ld);
    LB_CUDA(cudaEventRecord(e1, c.st));
    LB_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    LB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (v == kSpmmAuto || ms < 0.98f * tbest) best = v, tbest = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  var = best;
  tuned = p;
}

template <class T>
void apply_A(lobpcg_ctx& c, const T* X, int ldx, int p, T* Y, int ldy) {
  if (p <= 0) return;
  c.prof.mark(PH_SPMM);
  bool done = false;
  if constexpr (std::is_same<T, double>::value) {
    if (c.df_on && c.A.fmt == LOBPCG_CSR && c.val_df.p && !(ldx & 1) && !(ldy & 1)) {
      // double-float product: split the block once, then the compensated row sums
      c.xs_df.ensure((size_t)c.A.n * ldx * sizeof(float2));
      launch_split_df(c.A.n * (int64_t)ldx, X, c.xs_df.as<float2>(), c.st);
      launch_spmm_csr_df(c.A.n, c.A.row_ptr, c.A.col_idx, c.val_df.as<float2>(), p, c.xs_df.as<float2>(), ldx, Y,
                         ldy, c.st);
      done = true;
    }
  }
  if (!done) spmm_product<T>(c, X, ldx, p, Y, ldy);
  c.stats.spmm_columns += p;
  c.stats.spmm_launches += 1;
  if (sizeof(T) == 8) c.stats.spmm_launches64 += 1, c.stats.spmm_columns64 += p;
  c.prof.mark(PH_OTHER);
}

template <class T>
void gram(lobpcg_ctx& c, const Cols<T>& a, const Cols<T>& b, bool upper, double* out) {
  const int pa = a.width(), pb = b.width();
  int parts = 0;
  if constexpr (std::is_same<T, double>::value) {
    if (c.df_on) parts = gram_partials_df(c.A.n, a, b, upper, c.Gpart, c.max_ctas, c.st);
  } else {
    // FP32: the tcgen05 kernel when the blocks fit it (every block the solver allocates);
    // its give-up flag is checked once per solve (umma_check)
    if (c.opt.tc_gram != 0) parts = gram_partials_umma(c.A.n, a, b, upper, c.Gpart, c.max_ctas, c.st);
  }
  if (!parts) parts = gram_partials<T>(c.A.n, a, b, upper, c.Gpart, c.max_ctas, c.st);
  reduce_partials(c.Gpart, parts, pa * pb, out, c.st);
}

// W <- W * T (p x p FP64 matrix on device), in place.
template <class T>
void right_multiply(lobpcg_ctx& c, T* W, int ld, int p, const double* Tm) {
  UpdateJob<T> job{};
  job.in[0] = cols1<T>(W, ld, p);
  job.out[0] = W;
  job.ld_out[0] = ld;
  job.nprod = 1;
  job.unit_base = 1;  // double-float path: W + W (T - I)
  update<T>(c, job, Tm, p, p, 1.0, nullptr, nullptr);
}

// Algorithm 2: W (n x p) <- ortho(W).  Host-driven loop, one flag read per pass.  With
// opt.ortho_trim the re-check Gram is skipped after an unshifted pass whose scaled overlap
// I + F had ||F||_F <= 1/2 (reading R17, the ||L^{-T}|| estimate of Sec. 3.2).  Cg (q x p,
// the coefficients of the projection just applied by Algorithm 3) asks the first
// factorisation for the pass's growth factor test (reading R18); *growth_ok receives it.
template <class T>
int ortho(lobpcg_ctx& c, T* W, int ld, int p, double tau, int cap, const double* Cg = nullptr, int q = 0,
          bool* growth_ok = nullptr) {
  if (growth_ok) *growth_ok = false;
  if (p <= 0) return 0;
  // the estimates assume Grams accurate to a few eps (FP64 or double-float); the FP32
  // phase's tensor-core Grams summed in FP32 are not, so it runs the printed algorithms
  const bool trim = c.opt.ortho_trim != 0 && sizeof(T) == 8;
  // eps sqrt(q) g <= tau with the unit of the products' arithmetic (reading R18):
  // 2^-46 for double-float (two roundings at 2^-47 of the split), else FP64's
  const double eps = c.df_on ? 1.4210854715202004e-14 : 2.220446049250313e-16;
  const double g_max = q > 0 ? tau / (eps * std::sqrt((double)q)) : 0.0;
  int passes = 0;
  LB_CUDA(cudaMemsetAsync(c.ictl, 0, 8 * sizeof(int), c.st));
  const int* h = reinterpret_cast<const int*>(c.host);
  for (int call = 0;; ++call) {
    const Cols<T> w = cols1<T>(W, ld, p);
    gram<T>(c, w, w, false, c.G);                       // M = W^T W
    c.stats.ortho_grams++;
    const bool want_growth = trim && call == 0 && Cg && growth_ok;
    launch_cholqr_small(p, c.G, tau, c.Tm, c.ictl, c.st, want_growth ? Cg : nullptr, q,
                        g_max * g_max);                 // test ||M - I||, factor
    LB_CUDA(cudaMemcpyAsync(c.host, c.ictl, 8 * sizeof(int), cudaMemcpyDeviceToHost, c.st));
    c.sync();
    if (want_growth) *growth_ok = h[7] != 0;
    if (h[0]) break;
    if (passes >= cap) {
      c.stats.cap_hits++;
      break;
    }
    ++passes;
    right_multiply<T>(c, W, ld, p, c.Tm);               // W <- W L^{-T}
    if (trim && h[6] && 2.0 * eps <= tau) {             // R17: ||L^{-T}||^2 <= 2, no re-check
      c.stats.skipped_recheck++;
      break;
    }
  }
  c.stats.shifts += h[1];
  c.stats.svqb += h[2];
  c.stats.cholqr_passes_max = std::max(c.stats.cholqr_passes_max, passes);
  return passes;
}

// Algorithm 3: W (n x p) <- ortho(W; Y), Y orthonormal (Cols).  Body runs at least once.
// Reading R16: when a pass cap (of Algorithm 3 or of an Algorithm 2 inside it) was hit,
// the columns whose overlap with Y is above sqrt(tau) or whose norm differs from 1 by more
// than sqrt(tau) are dropped and the rest packed to the front in order; *kept receives the
// number of columns left (p otherwise).  Without a cap hit no column can fail these tests.
template <class T>
int ortho_against(lobpcg_ctx& c, T* W, int ld, int p, const Cols<T>& Y, double tau, int cap, int cap2,
                  int* kept = nullptr) {
  if (kept) *kept = p;
  if (p <= 0) return 0;
  const int q = Y.width();
  const int hits0 = c.stats.cap_hits;
  int passes = 0;
  double last = 0.0;
  bool c_ready = false;  // C = Y^T W of the current W is already in c.C (the previous pass's test)
  c.prof.mark(PH_ORTHO);
  bool c_current = true;  // c.C = Y^T W of the final W (false after a growth-factor exit)
  for (;;) {
    if (q > 0) {
      if (!c_ready) {
        gram<T>(c, Y, cols1<T>(W, ld, p), false, c.C);  // C = Y^T W
        c.stats.ortho_grams++;
      }
      UpdateJob<T> job{};
      job.in[0] = Y;
      job.out[0] = W;
      job.ld_out[0] = ld;
      job.base[0] = W;
      job.ld_base[0] = ld;
      job.nprod = 1;
      update<T>(c, job, c.C, q, p, -1.0, nullptr, nullptr);  // W -= Y C
    }
    bool growth_ok = false;
    ortho<T>(c, W, ld, p, tau, cap, q > 0 ? c.C : nullptr, q, &growth_ok);
    ++passes;
    if (q == 0) break;
    if (growth_ok) {  // R18: moderate growth factor, the overlap with Y is below tau
      c.stats.skipped_test++;
      c_current = false;
      break;
    }
    gram<T>(c, Y, cols1<T>(W, ld, p), false, c.C);
    c.stats.ortho_grams++;
    launch_maxabs(q * p, c.C, c.scal, c.st);
    LB_CUDA(cudaMemcpyAsync(c.host, c.scal, sizeof(double), cudaMemcpyDeviceToHost, c.st));
    c.sync();
    last = c.host[0];
    if (last <= tau) break;
    if (passes >= cap2) {
      c.stats.cap_hits++;
      break;
    }
    c_ready = true;
  }
  if (kept && c.stats.cap_hits > hits0) {
    // R16: c.C holds Y^T W of the final W (the last pass's test); the norms come from W^T W
    const Cols<T> w = cols1<T>(W, ld, p);
    if (q > 0 && !c_current) gram<T>(c, Y, w, false, c.C);
    gram<T>(c, w, w, false, c.G);
    std::vector<double> Ch((size_t)q * p), Mh((size_t)p * p);
    if (q > 0) LB_CUDA(cudaMemcpyAsync(Ch.data(), c.C, Ch.size() * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    LB_CUDA(cudaMemcpyAsync(Mh.data(), c.G, Mh.size() * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    c.sync();
    std::vector<double> sel((size_t)p * p, 0.0);  // p x p column selection (column-major)
    int k2 = 0;
    for (int j = 0; j < p; ++j) {
      double worst = 0.0;
      for (int i = 0; i < q; ++i) worst = std::max(worst, std::fabs(Ch[(size_t)j * q + i]));
      const double nrm = std::sqrt(std::max(Mh[(size_t)j * p + j], 0.0));
      if (worst <= std::sqrt(tau) && std::fabs(nrm - 1.0) <= std::sqrt(tau)) sel[(size_t)k2 * p + j] = 1.0, ++k2;
    }
    if (k2 < p) {
      LB_CUDA(cudaMemcpyAsync(c.Tm, sel.data(), sel.size() * sizeof(double), cudaMemcpyHostToDevice, c.st));
      if (k2 > 0) {
        UpdateJob<T> job{};
        job.in[0] = cols1<T>(W, ld, p);
        job.out[0] = W;
        job.ld_out[0] = ld;
        job.nprod = 1;
        update<T>(c, job, c.Tm, p, k2, 1.0, nullptr, nullptr);  // W <- W S
      }
      c.stats.w_dropped += p - k2;
    }
    *kept = k2;
  }
  c.stats.ortho_passes_max = std::max(c.stats.ortho_passes_max, passes);
  c.prof.mark(PH_OTHER);
  return passes;
}

template <class T>
void precondition(lobpcg_ctx& c, const T* X, const T* AX, int ld, int m_conv, int a, T* W) {
  const int pc = c.opt.precond == LOBPCG_PREC_NONE ? 0 : 1;
  c.prof.mark(PH_PRECOND);
  if (c.use_learned) {
    mlp::launch_precond_learned<T>(c.A.n, X, AX, ld, c.lam, m_conv, a, c.A.diag, c.rho.as<float>(), c.cscale,
                                   c.colmax, c.mlp_params.as<float>(), W, ld, c.st);
  } else if (c.opt.precond == LOBPCG_PREC_TRIDIAG) {
    c.tri_scratch.ensure(tridiag_scratch_floats(c.A.n, a) * sizeof(float));
    const int64_t no = std::max<int64_t>(c.A.n - 1, 1);
    const double* dl = c.tri_offd.as<double>();
    launch_precond_tridiag<T>(c.A.n, X, AX, ld, c.lam, m_conv, a, c.A.diag, dl, dl + no, W, ld,
                              c.tri_scratch.as<float>(), c.st);
  } else
    launch_precond<T>(c.A.n, X, AX, ld, c.lam, m_conv, a, c.A.diag, pc, W, ld, c.st, nullptr, c.opt.precond_floor);
  c.prof.mark(PH_OTHER);
}

struct PhaseOut {
  int sweeps = 0;  // Jacobi sweeps of the last Rayleigh-Ritz solve
  int iterations = 0;
  int m_conv = 0;
  bool converged = false;
  int xbuf = 0;  // which X buffer holds the result
  const void* xbest = nullptr;  // stall exit of the mixed form: its best X (ld of the blocks)
  std::vector<double> lam, res;
};

// One run of Algorithm 1 in precision T starting from the row-major block X[0] (n x m,
// not yet orthonormal).  `stall_exit` enables the mixed-precision switch test.
template <class T>
PhaseOut run_lobpcg(lobpcg_ctx& c, int k, int m, double tol, double tau, int maxiter, bool stall_exit,
                    double switch_tol = 0.0) {
  Blocks<T>& b = Prec<T>::blocks(c);
  c.prof.prec64 = sizeof(T) == 8 ? 1 : 0;
  const int64_t n = c.A.n;
  const int ld = b.ld;
  const int cap = c.opt.ortho_cap, cap2 = c.opt.ortho2_cap;
  const int tol_kind = c.opt.tol_kind;
  PhaseOut out;
  int cur = 0;
  LockState ls{0, m, 0, 0, 0, 0};
  LB_CUDA(cudaMemcpyAsync(c.lock, &ls, sizeof ls, cudaMemcpyHostToDevice, c.st));

  auto read_lock = [&](int mm) {
    LB_CUDA(cudaMemcpyAsync(c.host, c.lock, sizeof(LockState), cudaMemcpyDeviceToHost, c.st));
    LB_CUDA(cudaMemcpyAsync(c.host + 8, c.resnorm, mm * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    LB_CUDA(cudaMemcpyAsync(c.host + 8 + kMaxS, c.lam_all, mm * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    LB_CUDA(cudaMemcpyAsync(c.host + 4, c.ictl + 4, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    c.sync();
    out.sweeps = *reinterpret_cast<const int*>(c.host + 4);
    std::memcpy(&ls, c.host, sizeof ls);
    out.res.assign(c.host + 8, c.host + 8 + mm);
    out.lam.assign(c.host + 8 + kMaxS, c.host + 8 + kMaxS + mm);
  };

  // ---- initialisation ----
  ortho<T>(c, b.X[0], ld, m, tau, cap);                                 // X0 <- ortho(X0)
  apply_A<T>(c, b.X[0], ld, m, b.AX[0], ld);                            // AX = A X
  gram<T>(c, cols1<T>(b.X[0], ld, m), cols1<T>(b.AX[0], ld, m), true, c.G);  // a = X^T AX
  launch_syev(m, c.G, true, c.lam_all, c.U, c.ictl + 4, c.st, sizeof(T) == 4,
              sizeof(T) == 4 ? 1e-10 : 1e-15);  // a u = u lambda
  LB_CUDA(cudaMemcpyAsync(c.lam, c.lam_all, m * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
  {
    UpdateJob<T> job{};
    job.in[0] = cols1<T>(b.X[0], ld, m);
    job.in[1] = cols1<T>(b.AX[0], ld, m);
    job.out[0] = b.X[1], job.out[1] = b.AX[1];
    job.ld_out[0] = job.ld_out[1] = ld;
    job.nprod = 2;
    const int parts = update<T>(c, job, c.U, m, m, 1.0, c.lam, c.npart);
    launch_lock_and_p(m, m, k, n, c.npart, parts, c.U, tol, tol_kind, tau, c.lock, c.resnorm, c.colmax, c.up,
                      false, c.st);
  }
  cur = 1;
  read_lock(m);
  if (ls.done) {
    out.converged = true;
    out.m_conv = ls.m_conv;
    out.xbuf = cur;
    return out;
  }
  int a = ls.m_act, m_conv = ls.m_conv;
  int aw = a;  // columns of W (fewer than a when R16 drops some)
  precondition<T>(c, b.X[cur], b.AX[cur], ld, m_conv, a, b.W);         // W~ = T R
  ortho_against<T>(c, b.W, ld, a, cols1<T>(b.X[cur], ld, m), tau, cap, cap2, &aw);  // W = ortho(W~; X)
  apply_A<T>(c, b.W, ld, aw, b.AW, ld);                                 // AW = A W
  int pw = 0;  // width of P in the current basis
  MixedSwitch sw;                                  // when the mixed form leaves FP32
  sw.switch_tol = switch_tol;
  double xbest_rk = 1e300;                         // largest sought residual of the best X
  double lbest = 1e300;
  int lsince = 0;

  // ---- main loop ----
  int it = 1;
  for (; it <= maxiter; ++it) {
    const int s = m + pw + aw;
    Cols<T> V = cols1<T>(b.X[cur], ld, m);
    V = cols_add<T>(V, b.P[cur], ld, pw);
    V = cols_add<T>(V, b.W, ld, aw);
    Cols<T> AV = cols1<T>(b.AX[cur], ld, m);
    AV = cols_add<T>(AV, b.AP[cur], ld, pw);
    AV = cols_add<T>(AV, b.AW, ld, aw);
    double orth_dev = -1.0;
    int orth_i = -1, orth_j = -1;
    if (c.trace && c.trace_orth) {
      // optional check of the basis: max |V^T V - I| (LOBPCG_TRACE_ORTH=1)
      gram<T>(c, V, V, false, c.G);
      launch_maxabs_minus_identity(s, c.G, c.scal, c.st);
      LB_CUDA(cudaMemcpyAsync(c.host + 7, c.scal, sizeof(double), cudaMemcpyDeviceToHost, c.st));
      LB_CUDA(cudaMemcpyAsync(c.host + 64, c.G, (size_t)s * s * sizeof(double), cudaMemcpyDeviceToHost, c.st));
      c.sync();
      orth_dev = c.host[7];
      // location of the largest deviation and the column norms, for the trace
      double worst = -1.0;
      for (int j = 0; j < s; ++j)
        for (int i = 0; i < s; ++i) {
          const double d = std::fabs(c.host[64 + i + j * s] - (i == j ? 1.0 : 0.0));
          if (d > worst) worst = d, orth_i = i, orth_j = j;
        }
    }
    c.prof.mark(PH_RR_GRAM);
    gram<T>(c, V, AV, true, c.G);                                       // a = V^T AV (upper)
    if (sizeof(T) == 4) c.stats.rr_gram32_bytes += 2.0 * (double)n * s * sizeof(T), c.stats.rr_gram32_count++;
    c.prof.mark(PH_RR_EIG);
    // Rayleigh-Ritz; the FP32 phase, whose Ritz vectors go to FP32 blocks (rounding 6e-8),
    // takes the two-stage solver stopped at 1e-10 relative, the FP64 phase plain FP64 Jacobi
    launch_syev(s, c.G, true, c.lam_all, c.U, c.ictl + 4, c.st, sizeof(T) == 4, sizeof(T) == 4 ? 1e-10 : 1e-15);
    c.prof.mark(PH_UPDATE);
    LB_CUDA(cudaMemcpyAsync(c.lam, c.lam_all, m * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
    const int nxt = cur ^ 1;
    UpdateJob<T> job{};
    job.in[0] = V, job.in[1] = AV;
    job.out[0] = b.X[nxt], job.out[1] = b.AX[nxt];
    job.ld_out[0] = job.ld_out[1] = ld;
    job.nprod = 2;
    const int parts = update<T>(c, job, c.U, s, m, 1.0, c.lam, c.npart);  // X = V u_x
    launch_lock_and_p(s, m, k, n, c.npart, parts, c.U, tol, tol_kind, tau, c.lock, c.resnorm, c.colmax, c.up,
                      true, c.st);                                      // lock, u_p
    read_lock(m);
    c.prof.mark(PH_OTHER);
    if (c.trace) {
      std::fprintf(c.trace, "{\"it\": %d, \"prec\": %d, \"s\": %d, \"pw\": %d, \"sweeps\": %d, \"m_act\": %d, "
                   "\"orth\": %.3e, \"orth_ij\": [%d, %d], \"lambda\": [", it, (int)sizeof(T) * 8, s, pw,
                   out.sweeps, ls.m_act, orth_dev, orth_i, orth_j);
      for (int j = 0; j < m; ++j) std::fprintf(c.trace, "%s%.17g", j ? ", " : "", out.lam[j]);
      std::fprintf(c.trace, "], \"res\": [");
      for (int j = 0; j < m; ++j) std::fprintf(c.trace, "%s%.6e", j ? ", " : "", out.res[j]);
      std::fprintf(c.trace, "]}\n");
    }
    if (ls.done) {
      cur = nxt;
      out.converged = true;
      break;
    }
    if (stall_exit) {
      // mixed-precision switch (reading R22, switch_rule.cuh) on the largest of the k sought
      // residuals; the FP64 phase starts from the best X, not from the last one
      double rk = 0.0;
      for (int j = 0; j < k; ++j) rk = std::max(rk, out.res[j]);
      if (rk < xbest_rk) {
        c.xbest.ensure((size_t)n * ld * sizeof(T));
        LB_CUDA(cudaMemcpyAsync(c.xbest.p, b.X[nxt], (size_t)n * ld * sizeof(T), cudaMemcpyDeviceToDevice, c.st));
        xbest_rk = rk;
      }
      if (sw.step(rk)) {
        cur = nxt;
        out.xbest = c.xbest.p;
        break;
      }
    }
    if (c.use_learned) {
      // the diagonal preconditioner takes over when the learned one stops making progress:
      // the largest residual of the k sought pairs has not dropped by 10% in 20 iterations
      double rk = 0.0;
      for (int j = 0; j < k; ++j) rk = std::max(rk, out.res[j]);
      if (rk < 0.9 * lbest) lbest = rk, lsince = 0;
      else if (++lsince >= 20) c.use_learned = false, c.stats.precond_fallback = 1;
    }
    const int a_new = ls.m_act;
    m_conv = ls.m_conv;
    c.prof.mark(PH_UPDATE);
    const int pw_new = ls.p_cols;  // P directions whose Ritz vector moved (reading R14)
    c.stats.p_dropped += a_new - pw_new;
    if (pw_new > 0) {
      UpdateJob<T> pj{};
      pj.in[0] = V, pj.in[1] = AV;
      pj.out[0] = b.P[nxt], pj.out[1] = b.AP[nxt];
      pj.ld_out[0] = pj.ld_out[1] = ld;
      pj.nprod = 2;
      update<T>(c, pj, c.up, s, pw_new, 1.0, nullptr, nullptr);  // P = V u_p
    }
    c.prof.mark(PH_OTHER);
    cur = nxt;
    a = a_new;
    pw = pw_new;
    precondition<T>(c, b.X[cur], b.AX[cur], ld, m_conv, a, b.W);       // W~ = T R
    Cols<T> Y = cols1<T>(b.X[cur], ld, m);
    Y = cols_add<T>(Y, b.P[cur], ld, pw);
    ortho_against<T>(c, b.W, ld, a, Y, tau, cap, cap2, &aw);            // W = ortho(W~; (X, P))
    apply_A<T>(c, b.W, ld, aw, b.AW, ld);                               // AW = A W
  }
  out.iterations = std::min(it, maxiter);
  out.m_conv = ls.m_conv;
  out.xbuf = cur;
  return out;
}

// ============================================ generalised problem (Sec. 3.3), FP64
// Y = B X for the mass matrix B (CSR or dense, FP64 products).
void apply_B(lobpcg_ctx& c, const double* X, int ldx, int p, double* Y, int ldy) {
  if (p <= 0) return;
  if (c.B.fmt == LOBPCG_CSR)
    launch_spmm_csr<double, double>(c.A.n, c.B.row_ptr, c.B.col_idx, c.B.val, p, X, ldx, Y, ldy, c.st);
  else
    launch_spmm_dense<double>(c.A.n, c.B.dense, c.B.ld, p, X, ldx, Y, ldy, c.st);
  c.stats.b_products += 1;
}

// Algorithm 2 in the B product with re-use of B X: M = X^T (B X), stop when ||M - I|| <=
// tau, else X <- X T and B X <- (B X) T with the Cholesky-QR transform T of M.
int b_ortho(lobpcg_ctx& c, double* X, double* BXp, int ld, int p, double tau, int cap) {
  if (p <= 0) return 0;
  int passes = 0;
  LB_CUDA(cudaMemsetAsync(c.ictl, 0, 8 * sizeof(int), c.st));
  const int* h = reinterpret_cast<const int*>(c.host);
  for (;;) {
    gram<double>(c, cols1<double>(X, ld, p), cols1<double>(BXp, ld, p), false, c.G);
    launch_cholqr_small(p, c.G, tau, c.Tm, c.ictl, c.st);
    LB_CUDA(cudaMemcpyAsync(c.host, c.ictl, 8 * sizeof(int), cudaMemcpyDeviceToHost, c.st));
    c.sync();
    if (h[0]) break;
    if (passes >= cap) {
      c.stats.cap_hits++;
      break;
    }
    ++passes;
    right_multiply<double>(c, X, ld, p, c.Tm);
    right_multiply<double>(c, BXp, ld, p, c.Tm);
  }
  c.stats.shifts += h[1];
  c.stats.svqb += h[2];
  c.stats.cholqr_passes_max = std::max(c.stats.cholqr_passes_max, passes);
  return passes;
}

// W from W~ (Sec. 3.3): W^ = ortho(W~, Q) with Q = orth(B X, B P) (Algorithms 2 and 3),
// then Cholesky-QR of W^ in the B product with B W = (B W^) L^{-T}.  Returns the columns
// kept (reading R16 when a cap was hit).
int gen_w_step(lobpcg_ctx& c, int m, int pw, int a, double tau, int cap, int cap2, int cur) {
  Blocks<double>& b = c.b64;
  const int ld = b.ld;
  const int64_t n = c.A.n;
  const int q = m + pw;
  LB_CUDA(cudaMemcpy2DAsync(c.Q, (size_t)c.ldq * 8, c.BX[cur], (size_t)ld * 8, (size_t)m * 8, (size_t)n,
                            cudaMemcpyDeviceToDevice, c.st));
  if (pw > 0)
    LB_CUDA(cudaMemcpy2DAsync(c.Q + m, (size_t)c.ldq * 8, c.BP[cur], (size_t)ld * 8, (size_t)pw * 8, (size_t)n,
                              cudaMemcpyDeviceToDevice, c.st));
  ortho<double>(c, c.Q, c.ldq, q, tau, cap);                            // Q = orth(B X, B P)
  int aw = a;
  ortho_against<double>(c, b.W, ld, a, cols1<double>(c.Q, c.ldq, q), tau, cap, cap2, &aw);  // W^
  apply_B(c, b.W, ld, aw, c.BW, ld);                                    // B W^
  const int hits0 = c.stats.cap_hits;
  b_ortho(c, b.W, c.BW, ld, aw, tau, cap);                             // W = W^ L^{-T}, B W re-used
  if (c.stats.cap_hits > hits0 && aw > 0) {
    // R16 in the B product: keep the columns with B-norm 1 to sqrt(tau)
    gram<double>(c, cols1<double>(b.W, ld, aw), cols1<double>(c.BW, ld, aw), false, c.G);
    std::vector<double> Mh((size_t)aw * aw);
    LB_CUDA(cudaMemcpyAsync(Mh.data(), c.G, Mh.size() * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    c.sync();
    std::vector<double> sel((size_t)aw * aw, 0.0);
    int k2 = 0;
    for (int j = 0; j < aw; ++j)
      if (std::fabs(std::sqrt(std::max(Mh[(size_t)j * aw + j], 0.0)) - 1.0) <= std::sqrt(tau))
        sel[(size_t)k2 * aw + j] = 1.0, ++k2;
    if (k2 < aw) {
      LB_CUDA(cudaMemcpyAsync(c.Tm, sel.data(), sel.size() * sizeof(double), cudaMemcpyHostToDevice, c.st));
      for (double* blk : {b.W, c.BW}) {
        if (k2 == 0) break;
        UpdateJob<double> job{};
        job.in[0] = cols1<double>(blk, ld, aw);
        job.out[0] = blk;
        job.ld_out[0] = ld;
        job.nprod = 1;
        update<double>(c, job, c.Tm, aw, k2, 1.0, nullptr, nullptr);
      }
      c.stats.w_dropped += aw - k2;
      aw = k2;
    }
  }
  apply_A<double>(c, b.W, ld, aw, b.AW, ld);                             // A W
  return aw;
}

// Algorithm 1 for A x = lambda B x in FP64: B-orthonormal basis, B V carried along.  The
// residual pair is (B V, A V) u_x, so the fused epilogue gives ||A x - lambda B x||.
PhaseOut run_lobpcg_gen(lobpcg_ctx& c, int k, int m, double tol, double tau, int maxiter) {
  Blocks<double>& b = c.b64;
  c.prof.prec64 = 1;
  const int64_t n = c.A.n;
  const int ld = b.ld;
  const int cap = c.opt.ortho_cap, cap2 = c.opt.ortho2_cap;
  const int tol_kind = c.opt.tol_kind;
  const int pc = c.opt.precond == LOBPCG_PREC_NONE ? 0 : 1;
  PhaseOut out;
  LockState ls{0, m, 0, 0, 0, 0};
  LB_CUDA(cudaMemcpyAsync(c.lock, &ls, sizeof ls, cudaMemcpyHostToDevice, c.st));
  auto read_lock = [&]() {
    LB_CUDA(cudaMemcpyAsync(c.host, c.lock, sizeof(LockState), cudaMemcpyDeviceToHost, c.st));
    c.sync();
    std::memcpy(&ls, c.host, sizeof ls);
  };
  // ---- initialisation: B-orthonormal X0 (R20), Rayleigh-Ritz, residual ----
  apply_B(c, b.X[0], ld, m, c.BX[0], ld);
  b_ortho(c, b.X[0], c.BX[0], ld, m, tau, cap);
  apply_A<double>(c, b.X[0], ld, m, b.AX[0], ld);
  gram<double>(c, cols1<double>(b.X[0], ld, m), cols1<double>(b.AX[0], ld, m), true, c.G);
  launch_syev(m, c.G, true, c.lam_all, c.U, c.ictl + 4, c.st, false, 1e-15);
  LB_CUDA(cudaMemcpyAsync(c.lam, c.lam_all, m * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
  auto rotate = [&](const Cols<double>& V, const Cols<double>& AV, const Cols<double>& BV, int s, int nxt,
                    bool with_p) {
    UpdateJob<double> jx{};
    jx.in[0] = V, jx.out[0] = b.X[nxt], jx.ld_out[0] = ld, jx.nprod = 1;
    update<double>(c, jx, c.U, s, m, 1.0, nullptr, nullptr);                 // X = V u_x
    UpdateJob<double> jp{};
    jp.in[0] = BV, jp.in[1] = AV;
    jp.out[0] = c.BX[nxt], jp.out[1] = b.AX[nxt];
    jp.ld_out[0] = jp.ld_out[1] = ld;
    jp.nprod = 2;
    const int parts = update<double>(c, jp, c.U, s, m, 1.0, c.lam, c.npart);  // (BX, AX), ||AX - BX lam||
    launch_lock_and_p(s, m, k, n, c.npart, parts, c.U, tol, tol_kind, tau, c.lock, c.resnorm, c.colmax, c.up,
                      with_p, c.st);
  };
  rotate(cols1<double>(b.X[0], ld, m), cols1<double>(b.AX[0], ld, m), cols1<double>(c.BX[0], ld, m), m, 1, false);
  int cur = 1;
  read_lock();
  if (ls.done) {
    out.converged = true, out.m_conv = ls.m_conv, out.xbuf = cur;
    return out;
  }
  int a = ls.m_act, m_conv = ls.m_conv, pw = 0;
  launch_precond<double>(n, c.BX[cur], b.AX[cur], ld, c.lam, m_conv, a, c.A.diag, pc, b.W, ld, c.st, c.B.diag, c.opt.precond_floor);
  int aw = gen_w_step(c, m, 0, a, tau, cap, cap2, cur);
  int it = 1;
  for (; it <= maxiter; ++it) {
    const int s = m + pw + aw;
    Cols<double> V = cols_add<double>(cols_add<double>(cols1<double>(b.X[cur], ld, m), b.P[cur], ld, pw), b.W, ld, aw);
    Cols<double> AV =
        cols_add<double>(cols_add<double>(cols1<double>(b.AX[cur], ld, m), b.AP[cur], ld, pw), b.AW, ld, aw);
    Cols<double> BV =
        cols_add<double>(cols_add<double>(cols1<double>(c.BX[cur], ld, m), c.BP[cur], ld, pw), c.BW, ld, aw);
    gram<double>(c, V, AV, true, c.G);                                      // a = V^T A V
    launch_syev(s, c.G, true, c.lam_all, c.U, c.ictl + 4, c.st, false, 1e-15);
    LB_CUDA(cudaMemcpyAsync(c.lam, c.lam_all, m * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
    const int nxt = cur ^ 1;
    rotate(V, AV, BV, s, nxt, true);
    read_lock();
    if (ls.done) {
      cur = nxt;
      out.converged = true;
      break;
    }
    const int a_new = ls.m_act, pw_new = ls.p_cols;
    c.stats.p_dropped += a_new - pw_new;
    if (pw_new > 0) {
      UpdateJob<double> jp{};
      jp.in[0] = V, jp.out[0] = b.P[nxt], jp.ld_out[0] = ld, jp.nprod = 1;
      update<double>(c, jp, c.up, s, pw_new, 1.0, nullptr, nullptr);          // P = V u_p
      UpdateJob<double> jq{};
      jq.in[0] = BV, jq.in[1] = AV;
      jq.out[0] = c.BP[nxt], jq.out[1] = b.AP[nxt];
      jq.ld_out[0] = jq.ld_out[1] = ld;
      jq.nprod = 2;
      update<double>(c, jq, c.up, s, pw_new, 1.0, nullptr, nullptr);         // B P, A P
    }
    cur = nxt, a = a_new, m_conv = ls.m_conv, pw = pw_new;
    launch_precond<double>(n, c.BX[cur], b.AX[cur], ld, c.lam, m_conv, a, c.A.diag, pc, b.W, ld, c.st, c.B.diag, c.opt.precond_floor);
    aw = gen_w_step(c, m, pw, a, tau, cap, cap2, cur);
  }
  out.iterations = std::min(it, maxiter);
  out.m_conv = ls.m_conv;
  out.xbuf = cur;
  return out;
}

lobpcg_status fail(lobpcg_ctx* c, lobpcg_status s, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return s;
}

template <class F>
lobpcg_status guarded(lobpcg_ctx* c, F&& f) {
  try {
    return f();
  } catch (const InvalidArg& e) {
    return fail(c, LOBPCG_EINVAL, e.what());
  } catch (const NoMem& e) {
    return fail(c, LOBPCG_ENOMEM, e.what());
  } catch (const CudaError& e) {
    const std::string w = e.what();
    const bool oom = w.find("out of memory") != std::string::npos;
    return fail(c, oom ? LOBPCG_ENOMEM : LOBPCG_ECUDA, w);
  } catch (const std::invalid_argument& e) {
    return fail(c, LOBPCG_EINVAL, e.what());
  } catch (const std::bad_alloc& e) {
    return fail(c, LOBPCG_ENOMEM, e.what());
  } catch (const std::exception& e) {
    return fail(c, LOBPCG_ECUDA, e.what());
  } catch (...) {
    return fail(c, LOBPCG_ECUDA, "unknown error");
  }
}

void require(bool ok, const char* what) {
  if (!ok) throw InvalidArg(what);
}

}  // namespace

// ===================================================================== C ABI

extern "C" lobpcg_status lobpcg_options_default(lobpcg_options* opt) {
  if (!opt) return LOBPCG_EINVAL;
  std::memset(opt, 0, sizeof *opt);
  opt->extra = 0;
  opt->maxiter = 1000;
  opt->tol_kind = 0;
  opt->precond = LOBPCG_PREC_DIAG;
  opt->precision = LOBPCG_FP64;
  opt->tau_ortho = 1e-14;
  opt->ortho_cap = 6;
  opt->ortho2_cap = 4;
  opt->seed = 0;
  opt->mlp_weights = nullptr;
  opt->autotune = 0;
  opt->ortho_trim = 1;
  opt->df_products = 0;
  opt->tc_gram = 1;
  opt->precond_floor = 0.0;
  return LOBPCG_OK;
}

extern "C" lobpcg_status lobpcg_create(lobpcg_ctx** out, const lobpcg_matrix* A,
                                       const lobpcg_options* opt, lobpcg_stream stream) {
  if (out) *out = nullptr;
  std::unique_ptr<lobpcg_ctx> c(new (std::nothrow) lobpcg_ctx());
  if (!c) return fail(nullptr, LOBPCG_ENOMEM, "host allocation failed");
  lobpcg_status st = guarded(nullptr, [&]() -> lobpcg_status {
    require(out && A, "lobpcg_create: out and A must not be NULL");
    require(A->n >= 3, "lobpcg_create: n must be >= 3");
    require(A->diag != nullptr, "lobpcg_create: diag must not be NULL");
    if (A->fmt == LOBPCG_CSR)
      require(A->row_ptr && A->col_idx && A->val && A->nnz >= 0, "lobpcg_create: CSR arrays missing");
    else if (A->fmt == LOBPCG_DENSE)
      require(A->dense && A->ld >= A->n, "lobpcg_create: dense array missing or ld < n");
    else
      throw InvalidArg("lobpcg_create: unknown format");
    c->A = *A;
    if (opt) c->opt = *opt;
    else lobpcg_options_default(&c->opt);
    if (c->opt.maxiter <= 0) c->opt.maxiter = 1000;
    if (!(c->opt.tau_ortho > 0)) c->opt.tau_ortho = 1e-14;
    if (c->opt.ortho_cap <= 0) c->opt.ortho_cap = 6;
    if (c->opt.ortho2_cap <= 0) c->opt.ortho2_cap = 4;
    require(c->opt.extra >= 0, "lobpcg_create: extra must be >= 0");
    require(c->opt.tol_kind == 0 || c->opt.tol_kind == 1, "lobpcg_create: tol_kind must be 0 or 1");
    require(c->opt.precond_floor >= 0.0 && std::isfinite(c->opt.precond_floor),
            "lobpcg_create: precond_floor must be finite and >= 0");
    require(c->opt.precond >= LOBPCG_PREC_NONE && c->opt.precond <= LOBPCG_PREC_TRIDIAG,
            "lobpcg_create: unknown preconditioner");
    require(c->opt.precision == LOBPCG_FP64 || c->opt.precision == LOBPCG_MIXED,
            "lobpcg_create: unknown precision");
    require(c->opt.precond != LOBPCG_PREC_LEARNED || c->opt.mlp_weights,
            "lobpcg_create: learned preconditioner needs mlp_weights");
    c->st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    LB_CUDA(cudaGetDevice(&dev));
    LB_CUDA(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev));
    c->max_ctas = 2 * c->sms;
    c->alloc_small();
    // reject non-finite matrix entries (a host-visible error instead of NaN results)
    LB_CUDA(cudaMemsetAsync(c->ictl + 5, 0xff, sizeof(int), c->st));
    const int one = 1;
    LB_CUDA(cudaMemcpyAsync(c->ictl + 5, &one, sizeof(int), cudaMemcpyHostToDevice, c->st));
    if (A->fmt == LOBPCG_CSR) launch_all_finite(A->nnz, A->val, c->ictl + 5, c->st);
    else if (A->ld == A->n) launch_all_finite(A->n * A->n, A->dense, c->ictl + 5, c->st);
    else for (int64_t j = 0; j < A->n; ++j) launch_all_finite(A->n, A->dense + j * A->ld, c->ictl + 5, c->st);
    launch_all_finite(A->n, A->diag, c->ictl + 5, c->st);
    int finite = 0;
    LB_CUDA(cudaMemcpyAsync(&finite, c->ictl + 5, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    c->sync();
    require(finite == 1, "lobpcg_create: matrix or diagonal has non-finite entries");
    if (A->fmt == LOBPCG_CSR) c->band = profile_band(A->n, A->row_ptr, A->col_idx, A->nnz, c->st);
    if (c->opt.precision == LOBPCG_MIXED) {
      if (A->fmt == LOBPCG_CSR && c->band >= 0) {
        c->sp.build(A->n, A->row_ptr, A->col_idx, A->val, A->nnz, c->band, c->st);
        c->split = true;
      } else if (A->fmt == LOBPCG_CSR) {
        c->val32.ensure((size_t)std::max<int64_t>(A->nnz, 1) * sizeof(float));
        launch_to_float(A->nnz, A->val, c->val32.as<float>(), c->st);
      } else {
        c->dense32.ensure((size_t)A->n * A->n * sizeof(float));
        if (A->ld == A->n) launch_to_float(A->n * A->n, A->dense, c->dense32.as<float>(), c->st);
        else for (int64_t j = 0; j < A->n; ++j)
          launch_to_float(A->n, A->dense + j * A->ld, c->dense32.as<float>() + j * A->n, c->st);
      }
    }
    const bool df_phase = c->opt.precision == LOBPCG_MIXED ? c->opt.df_products >= 0 : c->opt.df_products > 0;
    if (A->fmt == LOBPCG_CSR && df_phase) {
      c->val_df.ensure((size_t)std::max<int64_t>(A->nnz, 1) * sizeof(float2));
      launch_split_df(A->nnz, A->val, c->val_df.as<float2>(), c->st);
    }
    if (c->opt.precond == LOBPCG_PREC_LEARNED) {
      c->mlp_params.ensure(mlp::kNumParams * sizeof(float));
      LB_CUDA(cudaMemcpyAsync(c->mlp_params.p, c->opt.mlp_weights, mlp::kNumParams * sizeof(float),
                              cudaMemcpyHostToDevice, c->st));
      c->rho.ensure((size_t)A->n * sizeof(float));
      const double cs = mlp::row_norms(A->n, A->row_ptr, A->col_idx, A->val,
                                       A->fmt == LOBPCG_DENSE ? A->dense : nullptr, A->ld, c->rho.as<float>(),
                                       c->scal, c->st);
      c->cscale = (float)(cs > 0 ? cs : 1.0);
    }
    if (c->opt.precond == LOBPCG_PREC_TRIDIAG) {
      const int64_t no = std::max<int64_t>(A->n - 1, 1);
      c->tri_offd.ensure((size_t)2 * no * sizeof(double));
      double* dl = c->tri_offd.as<double>();
      LB_CUDA(cudaMemsetAsync(dl, 0, (size_t)2 * no * sizeof(double), c->st));
      tridiag_extract(A->n, A->row_ptr, A->col_idx, A->val, A->fmt == LOBPCG_DENSE ? A->dense : nullptr, A->ld, dl,
                      dl + no, c->st);
    }
    c->opt.mlp_weights = nullptr;  // not retained
    c->sync();
    return LOBPCG_OK;
  });
  if (st == LOBPCG_OK) *out = c.release();
  return st;
}

extern "C" lobpcg_status lobpcg_create_gen(lobpcg_ctx** out, const lobpcg_matrix* A, const lobpcg_matrix* B,
                                           const lobpcg_options* opt, lobpcg_stream stream) {
  if (out) *out = nullptr;
  if (!B) return fail(nullptr, LOBPCG_EINVAL, "lobpcg_create_gen: B must not be NULL");
  lobpcg_options o;
  if (opt) o = *opt;
  else lobpcg_options_default(&o);
  if (o.precision != LOBPCG_FP64 || o.precond == LOBPCG_PREC_LEARNED || o.precond == LOBPCG_PREC_TRIDIAG ||
      o.df_products > 0)
    return fail(nullptr, LOBPCG_EINVAL,
                "lobpcg_create_gen: the generalised problem runs in FP64 with the diagonal or no preconditioner");
  lobpcg_ctx* c = nullptr;
  lobpcg_status st = lobpcg_create(&c, A, &o, stream);
  if (st != LOBPCG_OK) return st;
  st = guarded(nullptr, [&]() -> lobpcg_status {
    require(B->n == A->n && B->diag != nullptr, "lobpcg_create_gen: B must have A's order and a diagonal");
    if (B->fmt == LOBPCG_CSR)
      require(B->row_ptr && B->col_idx && B->val && B->nnz >= 0, "lobpcg_create_gen: CSR arrays of B missing");
    else if (B->fmt == LOBPCG_DENSE)
      require(B->dense && B->ld >= B->n, "lobpcg_create_gen: dense B missing or ld < n");
    else
      throw InvalidArg("lobpcg_create_gen: unknown format of B");
    const int one = 1;
    LB_CUDA(cudaMemcpyAsync(c->ictl + 5, &one, sizeof(int), cudaMemcpyHostToDevice, c->st));
    if (B->fmt == LOBPCG_CSR) launch_all_finite(B->nnz, B->val, c->ictl + 5, c->st);
    else for (int64_t j = 0; j < B->n; ++j) launch_all_finite(B->n, B->dense + j * B->ld, c->ictl + 5, c->st);
    launch_all_finite(B->n, B->diag, c->ictl + 5, c->st);
    int finite = 0;
    LB_CUDA(cudaMemcpyAsync(&finite, c->ictl + 5, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    c->sync();
    require(finite == 1, "lobpcg_create_gen: B or its diagonal has non-finite entries");
    c->B = *B;
    c->gen = true;
    return LOBPCG_OK;
  });
  if (st != LOBPCG_OK) {
    lobpcg_destroy(c);
    return st;
  }
  *out = c;
  return LOBPCG_OK;
}

extern "C" lobpcg_status lobpcg_solve(lobpcg_ctx* c, int k, double tol, const double* X0,
                                      double* evals, double* evecs, double* resnorms,
                                      lobpcg_info* info) {
  if (!c) return fail(nullptr, LOBPCG_EINVAL, "lobpcg_solve: NULL context");
  return guarded(c, [&]() -> lobpcg_status {
    const int64_t n = c->A.n;
    const int m = k + c->opt.extra;
    require(k >= 1, "lobpcg_solve: k must be >= 1");
    require(m <= kMaxM, "lobpcg_solve: k + extra must be <= 32");
    require(3 * (int64_t)m <= n, "lobpcg_solve: 3 (k + extra) must be <= n");
    require(tol > 0 && std::isfinite(tol), "lobpcg_solve: tol must be positive");
    require(evals && evecs && resnorms, "lobpcg_solve: output pointers must not be NULL");
    c->stats = Stats{};
    c->use_learned = c->opt.precond == LOBPCG_PREC_LEARNED;
    const long long launches0 = launch_counter();
    c->prof.begin(c->opt.profile != 0, c->st);
    const char* tr = std::getenv("LOBPCG_TRACE");
    c->trace = tr && *tr ? std::fopen(tr, "a") : nullptr;
    const char* tro = std::getenv("LOBPCG_TRACE_ORTH");
    c->trace_orth = tro && *tro == '1';
    cudaEvent_t e0, e1;
    LB_CUDA(cudaEventCreate(&e0));
    LB_CUDA(cudaEventCreate(&e1));
    LB_CUDA(cudaEventRecord(e0, c->st));
    c->b64.ensure(n, m);
    const double* x0 = X0;
    if (!x0) {
      c->x0buf.ensure((size_t)n * m * sizeof(double));
      launch_gaussian(n, m, c->opt.seed, c->x0buf.as<double>(), c->st);
      x0 = c->x0buf.as<double>();
    } else {
      const int one = 1;
      LB_CUDA(cudaMemcpyAsync(c->ictl + 5, &one, sizeof(int), cudaMemcpyHostToDevice, c->st));
      launch_all_finite(n * m, X0, c->ictl + 5, c->st);
      int finite = 0;
      LB_CUDA(cudaMemcpyAsync(&finite, c->ictl + 5, sizeof(int), cudaMemcpyDeviceToHost, c->st));
      c->sync();
      require(finite == 1, "lobpcg_solve: X0 has non-finite entries");
    }
    int iters = 0, fp64_iters = 0;
    PhaseOut ph;
    const double tau = c->opt.tau_ortho;
    autotune_spmm<double>(*c, m, c->b64.W, c->b64.ld, c->b64.AW);
    if (c->gen) {
      c->ensure_gen(n, c->b64.ld);
      launch_colmajor_to_rows<double, double>(n, m, x0, c->b64.X[0], c->b64.ld, c->st);
      ph = run_lobpcg_gen(*c, k, m, tol, tau, c->opt.maxiter);
      iters = fp64_iters = ph.iterations;
    } else if (c->opt.precision == LOBPCG_MIXED) {
      c->b32.ensure(n, m);
      autotune_spmm<float>(*c, m, c->b32.W, c->b32.ld, c->b32.AW);
      launch_colmajor_to_rows<double, float>(n, m, x0, c->b32.X[0], c->b32.ld, c->st);
      const double tau32 = std::max(tau, 3e-5);
      PhaseOut p32 = run_lobpcg<float>(*c, k, m, tol, tau32, c->opt.maxiter, true, c->opt.mixed_switch);
      iters += p32.iterations;
      // continue in FP64 from the FP32 block
      Blocks<float>& b = c->b32;
      c->x0buf.ensure((size_t)n * m * sizeof(double));
      const float* x32 = p32.xbest ? static_cast<const float*>(p32.xbest) : b.X[p32.xbuf];
      launch_rows_to_colmajor<float, double>(n, m, x32, b.ld, c->x0buf.as<double>(), c->st);
      launch_colmajor_to_rows<double, double>(n, m, c->x0buf.as<double>(), c->b64.X[0], c->b64.ld, c->st);
      c->df_on = c->opt.df_products >= 0;
      ph = run_lobpcg<double>(*c, k, m, tol, c->df_on ? std::max(tau, kTauDf) : tau,
                              std::max(1, c->opt.maxiter - p32.iterations), false);
      c->df_on = false;
      fp64_iters = ph.iterations;
      iters += ph.iterations;
    } else {
      launch_colmajor_to_rows<double, double>(n, m, x0, c->b64.X[0], c->b64.ld, c->st);
      c->df_on = c->opt.df_products > 0;
      ph = run_lobpcg<double>(*c, k, m, tol, c->df_on ? std::max(tau, kTauDf) : tau, c->opt.maxiter, false);
      c->df_on = false;
      iters = fp64_iters = ph.iterations;
    }
    // ---- outputs: normalise, fix signs, fresh residuals ----
    Blocks<double>& b = c->b64;
    const double* X = b.X[ph.xbuf];
    const Cols<double> xk = cols1<double>(X, b.ld, k);
    // normalisation: x^T x = 1, or x^T B x = 1 for the generalised problem
    gram<double>(*c, xk, c->gen ? cols1<double>(c->BX[ph.xbuf], b.ld, k) : xk, false, c->G);
    launch_col_sign<double>(n, k, X, b.ld, c->Gpart, c->max_ctas, c->sgn, c->st);
    launch_scale_matrix(k, c->G, c->sgn, c->S, c->st);
    double* Xs = b.P[0];   // scratch blocks (no longer needed)
    double* AXs = b.AP[0];
    {
      UpdateJob<double> job{};
      job.in[0] = cols1<double>(X, b.ld, k);
      job.out[0] = Xs;
      job.ld_out[0] = b.ld;
      job.nprod = 1;
      update<double>(*c, job, c->S, k, k, 1.0, nullptr, nullptr);
    }
    apply_A<double>(*c, Xs, b.ld, k, AXs, b.ld);
    c->stats.spmm_columns -= k;  // the check product is not part of the iteration
    c->stats.spmm_launches -= 1;
    c->stats.spmm_launches64 -= 1, c->stats.spmm_columns64 -= k;
    {
      // residual norms of the normalised vectors: out = in * I (reuse the update epilogue)
      std::vector<double> eye((size_t)k * k, 0.0);
      for (int j = 0; j < k; ++j) eye[(size_t)j * k + j] = 1.0;
      LB_CUDA(cudaMemcpyAsync(c->Tm, eye.data(), eye.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
      // the pair (X, AX), or (B X, A X): the epilogue forms A x - lambda x or A x - lambda B x
      double* BXs = c->gen ? c->BP[0] : nullptr;
      if (c->gen) apply_B(*c, Xs, b.ld, k, BXs, b.ld);
      UpdateJob<double> job{};
      job.in[0] = cols1<double>(c->gen ? BXs : Xs, b.ld, k);
      job.in[1] = cols1<double>(AXs, b.ld, k);
      job.out[0] = b.W, job.out[1] = b.AW;
      job.ld_out[0] = job.ld_out[1] = b.ld;
      job.nprod = 2;
      const int parts = update<double>(*c, job, c->Tm, k, k, 1.0, c->lam, c->npart);
      LockState tmp{0, k, 0, 0, 0, 0};
      LB_CUDA(cudaMemcpyAsync(c->lock, &tmp, sizeof tmp, cudaMemcpyHostToDevice, c->st));
      launch_lock_and_p(k, k, k, n, c->npart, parts, c->Tm, tol, 0, tau, c->lock, c->resnorm, c->colmax, c->up, false, c->st);
    }
    launch_rows_to_colmajor<double, double>(n, k, Xs, b.ld, evecs, c->st);
    LB_CUDA(cudaMemcpyAsync(evals, c->lam, k * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    LB_CUDA(cudaMemcpyAsync(resnorms, c->resnorm, k * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    LB_CUDA(cudaEventRecord(e1, c->st));
    c->sync();
    if (c->opt.precision == LOBPCG_MIXED) umma_check(c->st);
    float ms = 0.f;
    LB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    double phases[PH_COUNT], phases64[PH_COUNT];
    c->prof.finish(phases, phases64);
    if (c->trace) std::fclose(c->trace);
    c->trace = nullptr;
    if (info) {
      info->iterations = iters;
      info->fp64_iterations = fp64_iters;
      info->converged = ph.m_conv;
      info->cholqr_passes_max = c->stats.cholqr_passes_max;
      info->ortho_passes_max = c->stats.ortho_passes_max;
      info->shifts = c->stats.shifts;
      info->svqb = c->stats.svqb;
      info->cap_hits = c->stats.cap_hits;
      info->spmm_columns = c->stats.spmm_columns;
      info->seconds = ms * 1e-3;
      for (int i = 0; i < 6; ++i) info->phase_seconds[i] = phases[i], info->phase_seconds_fp64[i] = phases64[i];
      info->spmm_launches_fp64 = c->stats.spmm_launches64;
      info->spmm_columns_fp64 = c->stats.spmm_columns64;
      info->kernel_launches = launch_counter() - launches0;
      info->spmm_launches = c->stats.spmm_launches;
      info->precond_fallback = c->stats.precond_fallback;
      info->update_fp64_seconds = c->prof.on ? c->prof.kseconds() : 0.0;
      info->update_fp64_flops = c->prof.on ? c->prof.kflops : 0.0;
      info->update_fp64_launches = c->prof.on ? (int64_t)(c->prof.kused / 2) : 0;
      info->spmm_variant_fp32 = c->var32;
      info->spmm_variant_fp64 = c->var64;
      info->w_dropped = c->stats.w_dropped;
      info->p_dropped = c->stats.p_dropped;
      info->ortho_grams = c->stats.ortho_grams;
      info->skipped_recheck = c->stats.skipped_recheck;
      info->skipped_test = c->stats.skipped_test;
      info->df_products = (c->opt.precision == LOBPCG_MIXED) ? (c->opt.df_products >= 0) : (c->opt.df_products > 0);
      info->rr_gram32_bytes = c->stats.rr_gram32_bytes;
      info->rr_gram32_count = c->stats.rr_gram32_count;
    }
    for (int j = 0; j < k; ++j)
      if (!std::isfinite(evals[j]) || !std::isfinite(resnorms[j]))
        return fail(c, LOBPCG_EBREAKDOWN, "lobpcg_solve: non-finite result (basis breakdown)");
    if (!ph.converged) return fail(c, LOBPCG_ENOCONV, "lobpcg_solve: maxiter reached before convergence");
    return LOBPCG_OK;
  });
}

extern "C" void lobpcg_destroy(lobpcg_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  c->val32.release();
  c->dense32.release();
  c->val_df.release();
  c->xs_df.release();
  c->gbuf.release();
  c->sp.release();
  c->b64.buf.release();
  c->b32.buf.release();
  c->small.release();
  c->x0buf.release();
  c->xbest.release();
  c->tri_offd.release();
  c->tri_scratch.release();
  c->mlp_params.release();
  c->rho.release();
  if (c->host) cudaFreeHost(c->host);
  delete c;
}

extern "C" const char* lobpcg_last_error(const lobpcg_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

// ============================================================ building-block entry points

namespace {
// A context without a matrix: workspace for the block-level entry points.
struct ScratchCtx {
  lobpcg_ctx c;
  ScratchCtx(int64_t n, cudaStream_t st) {
    c.A.n = n;
    c.st = st;
    int dev = 0;
    LB_CUDA(cudaGetDevice(&dev));
    LB_CUDA(cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev));
    c.max_ctas = 2 * c.sms;
    lobpcg_options_default(&c.opt);
    c.alloc_small();
  }
  ~ScratchCtx() {
    c.small.release();
    if (c.host) cudaFreeHost(c.host);
    c.host = nullptr;
  }
};
}  // namespace

extern "C" lobpcg_status lobpcg_spmm_csr_f64(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                             const double* val, int p, const double* X, int ldx,
                                             double* Y, int ldy, lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(n >= 0 && row_ptr && col_idx && val && X && Y, "lobpcg_spmm_csr_f64: NULL argument");
    require(p >= 1 && p <= 32 && ldx >= p && ldy >= p, "lobpcg_spmm_csr_f64: need 1 <= p <= 32, ld >= p");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    launch_spmm_csr<double, double>(n, row_ptr, col_idx, val, p, X, ldx, Y, ldy, st);
    LB_CUDA(cudaStreamSynchronize(st));
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_spmm_csr_f64_df(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                                const double* val, int64_t nnz, int p, const double* X, int ldx,
                                                double* Y, int ldy, lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(n >= 0 && nnz >= 0 && row_ptr && col_idx && val && X && Y, "lobpcg_spmm_csr_f64_df: NULL argument");
    require(p >= 1 && p <= 32 && ldx >= p && ldy >= p, "lobpcg_spmm_csr_f64_df: need 1 <= p <= 32, ld >= p");
    require(ldx % 2 == 0 && ldy % 2 == 0 && !(reinterpret_cast<uintptr_t>(X) & 15) &&
                !(reinterpret_cast<uintptr_t>(Y) & 15),
            "lobpcg_spmm_csr_f64_df: X and Y must be 16-byte aligned with even row strides");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DevBuf vs, xs;
    vs.ensure((size_t)std::max<int64_t>(nnz, 1) * sizeof(float2));
    xs.ensure((size_t)std::max<int64_t>(n, 1) * ldx * sizeof(float2));
    launch_split_df(nnz, val, vs.as<float2>(), st);
    launch_split_df(n * (int64_t)ldx, X, xs.as<float2>(), st);
    launch_spmm_csr_df(n, row_ptr, col_idx, vs.as<float2>(), p, xs.as<float2>(), ldx, Y, ldy, st);
    LB_CUDA(cudaStreamSynchronize(st));
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_spmm_csr_f32(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                             const double* val, int64_t nnz, int p, const float* X, int ldx,
                                             float* Y, int ldy, int band, int* band_used, lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(n >= 0 && nnz >= 0 && row_ptr && col_idx && val && X && Y, "lobpcg_spmm_csr_f32: NULL argument");
    require(p >= 1 && p <= 32 && ldx >= p && ldy >= p, "lobpcg_spmm_csr_f32: need 1 <= p <= 32, ld >= p");
    require(ldx % 4 == 0 && ldy % 4 == 0 && !(reinterpret_cast<uintptr_t>(X) & 15) &&
                !(reinterpret_cast<uintptr_t>(Y) & 15),
            "lobpcg_spmm_csr_f32: X and Y must be 16-byte aligned with ld a multiple of 4");
    require(band >= -2, "lobpcg_spmm_csr_f32: band must be -2, -1 or >= 0");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int b = band;
    if (b == -1) b = profile_band(n, row_ptr, col_idx, nnz, st);
    if (b >= 0) {
      SplitCSR sp;
      sp.build(n, row_ptr, col_idx, val, nnz, b, st);
      sp.apply(n, p, X, ldx, Y, ldy, st);
      LB_CUDA(cudaStreamSynchronize(st));
      sp.release();
    } else {
      DevBuf v32;
      v32.ensure((size_t)std::max<int64_t>(nnz, 1) * sizeof(float));
      launch_to_float(nnz, val, v32.as<float>(), st);
      launch_spmm_csr<float, float>(n, row_ptr, col_idx, v32.as<float>(), p, X, ldx, Y, ldy, st);
      LB_CUDA(cudaStreamSynchronize(st));
      v32.release();
    }
    if (band_used) *band_used = b < 0 ? -1 : b;
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_mixed_switch_replay(const double* rk, int n, double switch_tol, int* leave_at) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(leave_at && n >= 0 && (rk || n == 0), "lobpcg_mixed_switch_replay: NULL argument or n < 0");
    require(switch_tol >= 0.0, "lobpcg_mixed_switch_replay: switch_tol must be >= 0");
    MixedSwitch sw;
    sw.switch_tol = switch_tol;
    *leave_at = -1;
    for (int i = 0; i < n; ++i)
      if (sw.step(rk[i])) {
        *leave_at = i;
        break;
      }
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_precond_tridiag(int64_t n, const double* dl, const double* d, const double* du,
                                                int p, const double* shift, const double* R, int ldr, double* W,
                                                int ldw, lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(n >= 1 && d && shift && R && W && (n == 1 || (dl && du)), "lobpcg_precond_tridiag: NULL argument");
    require(p >= 1 && p <= kMaxM && ldr >= p && ldw >= p, "lobpcg_precond_tridiag: need 1 <= p <= 32, ld >= p");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DevBuf scratch, zero;
    scratch.ensure(tridiag_scratch_floats(n, p) * sizeof(float));
    if (n == 1) {  // no off-diagonals: any valid pointer will do, none is read
      zero.ensure(sizeof(double));
      dl = du = zero.as<double>();
    }
    launch_precond_tridiag<double>(n, nullptr, R, ldr, shift, 0, p, d, dl, du, W, ldw, scratch.as<float>(), st);
    LB_CUDA(cudaStreamSynchronize(st));
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_spmm_dense_f64(int64_t n, const double* A, int64_t lda, int p,
                                               const double* X, int ldx, double* Y, int ldy,
                                               lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(n >= 0 && A && X && Y && lda >= n, "lobpcg_spmm_dense_f64: NULL argument or lda < n");
    require(p >= 1 && p <= 32 && ldx >= p && ldy >= p, "lobpcg_spmm_dense_f64: need 1 <= p <= 32, ld >= p");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    launch_spmm_dense<double>(n, A, lda, p, X, ldx, Y, ldy, st);
    LB_CUDA(cudaStreamSynchronize(st));
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_gram_f64(int64_t n, int p, const double* X, int ldx, int q,
                                         const double* Y, int ldy, double* C, lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(n >= 1 && X && Y && C, "lobpcg_gram_f64: NULL argument or n < 1");
    require(p >= 1 && q >= 1 && p <= kMaxS && q <= kMaxS && ldx >= p && ldy >= q,
            "lobpcg_gram_f64: need 1 <= p, q <= 96, ld >= width");
    ScratchCtx s(n, reinterpret_cast<cudaStream_t>(stream));
    gram<double>(s.c, cols1<double>(X, ldx, p), cols1<double>(Y, ldy, q), false, C);
    s.c.sync();
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_gram_f64_df(int64_t n, int p, const double* X, int ldx, int q,
                                            const double* Y, int ldy, double* C, lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(n >= 1 && X && Y && C, "lobpcg_gram_f64_df: NULL argument or n < 1");
    require(p >= 1 && q >= 1 && p <= kMaxS && q <= kMaxS && ldx >= p && ldy >= q,
            "lobpcg_gram_f64_df: need 1 <= p, q <= 96, ld >= width");
    require(ldx == ldy && ldx % 2 == 0 && !(reinterpret_cast<uintptr_t>(X) & 15) &&
                !(reinterpret_cast<uintptr_t>(Y) & 15),
            "lobpcg_gram_f64_df: X and Y must be 16-byte aligned with one even row stride");
    ScratchCtx s(n, reinterpret_cast<cudaStream_t>(stream));
    s.c.df_on = true;
    gram<double>(s.c, cols1<double>(X, ldx, p), cols1<double>(Y, ldy, q), false, C);
    s.c.sync();
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_update_f64_df(int64_t n, int nseg, const double* const* V, const double* const* AV,
                                              const int* w, int ld, const double* U, int q, double alpha,
                                              const double* base, int ld_base, double* X, double* AX, int ld_out,
                                              const double* lam, double* resnorm, lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(n >= 1 && nseg >= 1 && nseg <= 3 && V && w && U && X,
            "lobpcg_update_f64_df: NULL argument, n < 1 or nseg outside 1..3");
    require(!AV == !AX, "lobpcg_update_f64_df: AV and AX go together");
    require(!resnorm || (AV && lam && !base), "lobpcg_update_f64_df: resnorm needs AV, AX, lam and no base");
    int s = 0;
    Cols<double> cv{}, ca{};
    for (int g = 0; g < nseg; ++g) {
      require(V[g] && (!AV || AV[g]) && w[g] >= 0 && w[g] <= ld, "lobpcg_update_f64_df: NULL segment or w > ld");
      cv = cols_add<double>(cv, V[g], ld, w[g]);
      if (AV) ca = cols_add<double>(ca, AV[g], ld, w[g]);
      s += w[g];
    }
    require(s >= 1 && s <= kMaxS && q >= 1 && q <= 32 && ld_out >= q && (!base || ld_base >= q),
            "lobpcg_update_f64_df: need 1 <= s <= 96, 1 <= q <= 32, ld_out >= q, ld_base >= q");
    ScratchCtx sc(n, reinterpret_cast<cudaStream_t>(stream));
    sc.c.df_on = true;
    UpdateJob<double> job{};
    job.in[0] = cv, job.in[1] = ca;
    job.out[0] = X, job.out[1] = AX;
    job.ld_out[0] = job.ld_out[1] = ld_out;
    job.base[0] = base;
    job.ld_base[0] = ld_base;
    job.nprod = AV ? 2 : 1;
    const int parts = update<double>(sc.c, job, U, s, q, alpha, resnorm ? lam : nullptr,
                                     resnorm ? sc.c.npart : nullptr);
    if (resnorm) {
      reduce_partials(sc.c.npart, parts, 2 * q, sc.c.G, sc.c.st);
      LB_CUDA(cudaMemcpyAsync(sc.c.host, sc.c.G, (size_t)q * sizeof(double), cudaMemcpyDeviceToHost, sc.c.st));
    }
    sc.c.sync();
    if (resnorm)
      for (int j = 0; j < q; ++j) resnorm[j] = std::sqrt(sc.c.host[j]);
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_gram_f32(int64_t n, int p, const float* X, int ldx, int q, const float* Y,
                                         int ldy, double* C, lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(n >= 1 && X && Y && C, "lobpcg_gram_f32: NULL argument or n < 1");
    require(p >= 1 && q >= 1 && p <= kMaxS && q <= kMaxS && ldx >= p && ldy >= q,
            "lobpcg_gram_f32: need 1 <= p, q <= 96, ld >= width");
    ScratchCtx s(n, reinterpret_cast<cudaStream_t>(stream));
    s.c.opt.tc_gram = 0;  // the warp-level kernel; lobpcg_gram_f32_tcgen05 is the tcgen05 one
    gram<float>(s.c, cols1<float>(X, ldx, p), cols1<float>(Y, ldy, q), false, C);
    s.c.sync();
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_gram_f32_tcgen05(int64_t n, int p, const float* X, int ldx, int q, const float* Y,
                                                 int ldy, double* C, lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(n >= 1 && X && Y && C, "lobpcg_gram_f32_tcgen05: NULL argument or n < 1");
    require(p >= 1 && q >= 1 && p <= kMaxS && q <= kMaxS && ldx >= p && ldy >= q,
            "lobpcg_gram_f32_tcgen05: need 1 <= p, q <= 96, ld >= width");
    require(ldx == ldy && ldx % 4 == 0 && !(reinterpret_cast<uintptr_t>(X) & 15) &&
                !(reinterpret_cast<uintptr_t>(Y) & 15),
            "lobpcg_gram_f32_tcgen05: X and Y must be 16-byte aligned with one row stride, a multiple of 4");
    ScratchCtx s(n, reinterpret_cast<cudaStream_t>(stream));
    const int parts = gram_partials_umma(n, cols1<float>(X, ldx, p), cols1<float>(Y, ldy, q), false, s.c.Gpart,
                                         s.c.max_ctas, s.c.st);
    if (!parts) throw InvalidArg("lobpcg_gram_f32_tcgen05: operands do not fit the kernel");
    reduce_partials(s.c.Gpart, parts, p * q, C, s.c.st);
    umma_check(s.c.st);
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_update_f32(int64_t n, int nseg, const float* const* V, const float* const* AV,
                                           const int* w, int ld, const double* U, int q, double alpha,
                                           const float* base, int ld_base, float* X, float* AX, int ld_out,
                                           const double* lam, double* resnorm, lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(n >= 1 && nseg >= 1 && nseg <= 3 && V && w && U && X,
            "lobpcg_update_f32: NULL argument, n < 1 or nseg outside 1..3");
    require(!AV == !AX, "lobpcg_update_f32: AV and AX go together");
    require(!resnorm || (AV && lam && !base), "lobpcg_update_f32: resnorm needs AV, AX, lam and no base");
    int s = 0;
    Cols<float> cv{}, ca{};
    for (int g = 0; g < nseg; ++g) {
      require(V[g] && (!AV || AV[g]) && w[g] >= 0 && w[g] <= ld, "lobpcg_update_f32: NULL segment or w > ld");
      cv = cols_add<float>(cv, V[g], ld, w[g]);
      if (AV) ca = cols_add<float>(ca, AV[g], ld, w[g]);
      s += w[g];
    }
    require(s >= 1 && s <= kMaxS && q >= 1 && q <= 32 && ld_out >= q && (!base || ld_base >= q),
            "lobpcg_update_f32: need 1 <= s <= 96, 1 <= q <= 32, ld_out >= q, ld_base >= q");
    ScratchCtx sc(n, reinterpret_cast<cudaStream_t>(stream));
    UpdateJob<float> job{};
    job.in[0] = cv, job.in[1] = ca;
    job.out[0] = X, job.out[1] = AX;
    job.ld_out[0] = job.ld_out[1] = ld_out;
    job.base[0] = base;
    job.ld_base[0] = ld_base;
    job.nprod = AV ? 2 : 1;
    const int parts = update<float>(sc.c, job, U, s, q, alpha, resnorm ? lam : nullptr,
                                    resnorm ? sc.c.npart : nullptr);
    if (resnorm) {
      // per-column sums of the partial squared norms (entries 0..q-1 of each part's 2q)
      reduce_partials(sc.c.npart, parts, 2 * q, sc.c.G, sc.c.st);
      LB_CUDA(cudaMemcpyAsync(sc.c.host, sc.c.G, (size_t)q * sizeof(double), cudaMemcpyDeviceToHost, sc.c.st));
    }
    sc.c.sync();
    if (resnorm)
      for (int j = 0; j < q; ++j) resnorm[j] = std::sqrt(sc.c.host[j]);
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_syev_f64(int s, const double* a, double* lam, double* U,
                                         lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(s >= 1 && s <= kMaxS && a && lam && U, "lobpcg_syev_f64: need 1 <= s <= 96 and non-NULL arrays");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    launch_syev(s, a, false, lam, U, nullptr, st);
    LB_CUDA(cudaStreamSynchronize(st));
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_syev2_f64(int s, const double* a, double tol, double* lam, double* U,
                                          lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(s >= 1 && s <= kMaxS && a && lam && U, "lobpcg_syev2_f64: need 1 <= s <= 96 and non-NULL arrays");
    require(tol >= 0.0 && tol < 1e-6, "lobpcg_syev2_f64: need 0 <= tol < 1e-6");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    launch_syev(s, a, false, lam, U, nullptr, st, true, tol > 0.0 ? tol : 1e-15);
    LB_CUDA(cudaStreamSynchronize(st));
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_ortho_f64(int64_t n, int p, double* X, int ldx, double tau, int cap,
                                          int* stats, lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(n >= p && p >= 1 && p <= kMaxM && X && ldx >= p, "lobpcg_ortho_f64: need 1 <= p <= min(32, n)");
    require(tau > 0 && cap >= 1, "lobpcg_ortho_f64: tau > 0 and cap >= 1 required");
    ScratchCtx s(n, reinterpret_cast<cudaStream_t>(stream));
    const int passes = ortho<double>(s.c, X, ldx, p, tau, cap);
    s.c.sync();
    if (stats) {
      stats[0] = passes;
      stats[1] = s.c.stats.shifts;
      stats[2] = s.c.stats.svqb;
      stats[3] = s.c.stats.cap_hits;
    }
    return LOBPCG_OK;
  });
}

extern "C" lobpcg_status lobpcg_ortho_against_f64(int64_t n, int p, double* X, int ldx, int q,
                                                  const double* Y, int ldy, double tau, int cap,
                                                  int cap2, int* stats, lobpcg_stream stream) {
  return guarded(nullptr, [&]() -> lobpcg_status {
    require(n >= p + q && p >= 1 && p <= kMaxM && q >= 0 && q <= 2 * kMaxM && X && ldx >= p,
            "lobpcg_ortho_against_f64: need 1 <= p <= 32, 0 <= q <= 64, p + q <= n");
    require(q == 0 || (Y && ldy >= q), "lobpcg_ortho_against_f64: Y missing or ldy < q");
    require(tau > 0 && cap >= 1 && cap2 >= 1, "lobpcg_ortho_against_f64: tau > 0 and caps >= 1 required");
    ScratchCtx s(n, reinterpret_cast<cudaStream_t>(stream));
    const int passes = ortho_against<double>(s.c, X, ldx, p, cols1<double>(Y, ldy, q), tau, cap, cap2);
    s.c.sync();
    if (stats) {
      stats[0] = passes;
      stats[1] = s.c.stats.cholqr_passes_max;
      stats[2] = s.c.stats.shifts;
      stats[3] = s.c.stats.svqb;
      stats[4] = s.c.stats.cap_hits;
    }
    return LOBPCG_OK;
  });
}

// ============================================================ batched solve

#include <atomic>
#include <thread>

extern "C" lobpcg_status lobpcg_solve_batched(lobpcg_ctx* const* ctxs, int nprob, const int* k, const double* tol,
                                              const double* const* X0, double* const* evals, double* const* evecs,
                                              double* const* resnorms, lobpcg_info* infos, lobpcg_status* statuses,
                                              int nthreads) {
  if (nprob < 0 || (nprob > 0 && (!ctxs || !k || !tol || !evals || !evecs || !resnorms || !statuses))) {
    lobpcg::set_thread_error("lobpcg_solve_batched: NULL argument");
    return LOBPCG_EINVAL;
  }
  for (int i = 0; i < nprob; ++i)
    if (!ctxs[i]) {
      lobpcg::set_thread_error("lobpcg_solve_batched: NULL context");
      return LOBPCG_EINVAL;
    }
  if (nthreads <= 0) nthreads = 32;
  nthreads = std::min(nthreads, std::max(nprob, 1));
  // larger problems first: the longest solves start early and the tail stays short
  std::vector<int> order(nprob);
  for (int i = 0; i < nprob; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    const double wa = (double)ctxs[a]->A.n * (k[a] + ctxs[a]->opt.extra);
    const double wb = (double)ctxs[b]->A.n * (k[b] + ctxs[b]->opt.extra);
    return wa > wb;
  });
  int dev = 0;
  cudaGetDevice(&dev);
  std::atomic<int> next{0};
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int t = next.fetch_add(1);
      if (t >= nprob) break;
      const int i = order[t];
      statuses[i] = lobpcg_solve(ctxs[i], k[i], tol[i], X0 ? X0[i] : nullptr, evals[i], evecs[i], resnorms[i],
                                 infos ? &infos[i] : nullptr);
      // only the problems in flight hold block workspace: a finished problem returns its own
      ctxs[i]->b64.buf.release();
      ctxs[i]->xs_df.release();
      ctxs[i]->gbuf.release();
      ctxs[i]->b32.buf.release();
      ctxs[i]->x0buf.release();
      ctxs[i]->xbest.release();
    }
  };
  std::vector<std::thread> pool;
  pool.reserve(nthreads);
  for (int t = 0; t < nthreads; ++t) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
  for (int i = 0; i < nprob; ++i)
    if (statuses[i] != LOBPCG_OK) return statuses[i];
  return LOBPCG_OK;
}
