// Applications of A to a block (Algorithm 1: "AX = A X", "AW = A W").
//
// CSR: one warp per row.  The warp loads 32 (col, val) pairs of its row with one
// coalesced access, then broadcasts them by shuffle; groups of L lanes each take one
// non-zero and gather the matching row of the row-major block X, so every gather of a
// block row is a contiguous, coalesced L*8-byte access.  The G = 32/L partial sums of a
// column are combined with xor-shuffles at the end of the row.
//
// Dense: a warp owns RB rows of the symmetric column-major A (row i == column i, so a
// row is contiguous); lanes stride over the columns with coalesced loads of A and keep
// RB x PC partial sums, reduced by warp shuffles.
#include "common.cuh"

namespace lobpcg {
namespace {

template <class T, class V, int L, int CPL>
__global__ void __launch_bounds__(256) spmm_csr_kernel(int64_t n, const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ ci,
                                                       const V* __restrict__ val, int p,
                                                       const T* __restrict__ X, int ldx,
                                                       T* __restrict__ Y, int ldy) {
  constexpr int G = kWarp / L;
  const int lane = threadIdx.x & 31;
  const int g = lane / L, li = lane % L;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / kWarp);
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp; row < n;
       row += warps) {
    T acc[CPL];
#pragma unroll
    for (int t = 0; t < CPL; ++t) acc[t] = T(0);
    const int64_t e0 = rp[row], e1 = rp[row + 1];
    for (int64_t base = e0; base < e1; base += kWarp) {
      const int64_t e = base + lane;
      int c = 0;
      T v = T(0);
      if (e < e1) {
        c = ci[e];
        v = (T)val[e];
      }
      const int cnt = (e1 - base) < kWarp ? (int)(e1 - base) : kWarp;
      for (int j = 0; j < cnt; j += G) {
        const int src = j + g;  // <= 31 because j <= cnt - 1 - ((cnt - 1) % G) and g < G
        const int cc = __shfl_sync(0xffffffffu, c, src);
        const T vv = __shfl_sync(0xffffffffu, v, src);
        if (src < cnt) {
          const T* xr = X + (int64_t)cc * ldx;
#pragma unroll
          for (int t = 0; t < CPL; ++t) {
            const int col = li + L * t;
            if (col < p) acc[t] = fma(vv, xr[col], acc[t]);
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < CPL; ++t)
#pragma unroll
      for (int o = L; o < kWarp; o <<= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
    if (g == 0) {
      T* yr = Y + row * ldy;
#pragma unroll
      for (int t = 0; t < CPL; ++t) {
        const int col = li + L * t;
        if (col < p) yr[col] = acc[t];
      }
    }
  }
}

template <class T, class V, int L, int CPL>
void csr_launch(int64_t n, const int64_t* rp, const int32_t* ci, const V* val, int p, const T* X,
                int ldx, T* Y, int ldy, cudaStream_t st) {
  const int threads = 256;
  int64_t blocks = ceil_div(n, threads / kWarp);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  blocks = std::min<int64_t>(blocks, (int64_t)sms * 16);
  if (blocks < 1) blocks = 1;
  spmm_csr_kernel<T, V, L, CPL><<<(unsigned)blocks, threads, 0, st>>>(n, rp, ci, val, p, X, ldx, Y, ldy);
  LB_LAUNCH_CHECK();
}

// RB rows per warp, PC columns per pass.
template <class T, int RB, int PC>
__global__ void __launch_bounds__(256) spmm_dense_kernel(int64_t n, const T* __restrict__ A,
                                                         int64_t lda, int p, int c0,
                                                         const T* __restrict__ X, int ldx,
                                                         T* __restrict__ Y, int ldy) {
  const int lane = threadIdx.x & 31;
  const int64_t row0 = ((int64_t)blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp) * RB;
  if (row0 >= n) return;
  const int pc = min(PC, p - c0);
  T acc[RB][PC];
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int j = 0; j < PC; ++j) acc[r][j] = T(0);
  for (int64_t c = lane; c < n; c += kWarp) {
    T x[PC];
    const T* xr = X + c * ldx + c0;
#pragma unroll
    for (int j = 0; j < PC; ++j) x[j] = j < pc ? xr[j] : T(0);
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int64_t i = row0 + r;
      const T a = i < n ? A[c + i * lda] : T(0);  // a_ci = a_ic (A symmetric)
#pragma unroll
      for (int j = 0; j < PC; ++j) acc[r][j] = fma(a, x[j], acc[r][j]);
    }
  }
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int j = 0; j < PC; ++j) acc[r][j] = warp_sum(acc[r][j]);
  if (lane == 0) {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int64_t i = row0 + r;
      if (i < n)
#pragma unroll
        for (int j = 0; j < PC; ++j)
          if (j < pc) Y[i * ldy + c0 + j] = acc[r][j];
    }
  }
}

}  // namespace

template <class T, class V>
void launch_spmm_csr(int64_t n, const int64_t* rp, const int32_t* ci, const V* val, int p,
                     const T* X, int ldx, T* Y, int ldy, cudaStream_t st) {
  if (n <= 0 || p <= 0) return;
  if (p > 32) throw std::invalid_argument("spmm: p > 32");
  // L lanes per non-zero, CPL columns per lane: L = pow2 >= ceil(p / 2)
  if (p <= 2) csr_launch<T, V, 1, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
  else if (p <= 4) csr_launch<T, V, 2, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
  else if (p <= 8) csr_launch<T, V, 4, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
  else if (p <= 16) csr_launch<T, V, 8, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
  else csr_launch<T, V, 16, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
}

template <class T>
void launch_spmm_dense(int64_t n, const T* A, int64_t lda, int p, const T* X, int ldx, T* Y,
                       int ldy, cudaStream_t st) {
  if (n <= 0 || p <= 0) return;
  constexpr int RB = 4, PC = 8;
  const int threads = 256;
  const int64_t blocks = ceil_div(ceil_div(n, RB), threads / kWarp);
  for (int c0 = 0; c0 < p; c0 += PC) {
    spmm_dense_kernel<T, RB, PC><<<(unsigned)blocks, threads, 0, st>>>(n, A, lda, p, c0, X, ldx, Y, ldy);
    LB_LAUNCH_CHECK();
  }
}

template void launch_spmm_csr<double, double>(int64_t, const int64_t*, const int32_t*, const double*,
                                              int, const double*, int, double*, int, cudaStream_t);
template void launch_spmm_csr<float, float>(int64_t, const int64_t*, const int32_t*, const float*,
                                            int, const float*, int, float*, int, cudaStream_t);
template void launch_spmm_dense<double>(int64_t, const double*, int64_t, int, const double*, int,
                                        double*, int, cudaStream_t);
template void launch_spmm_dense<float>(int64_t, const float*, int64_t, int, const float*, int,
                                       float*, int, cudaStream_t);

}  // namespace lobpcg
