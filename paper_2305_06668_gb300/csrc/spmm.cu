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


// Vectorised variant for 16-byte aligned blocks: each lane of a group holds VEC
// consecutive columns (one 16-byte load per gathered row), and every lane issues UNR
// independent gathers before using them, so several rows of X are in flight per warp.
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};
__device__ __forceinline__ void vfma(float a, const float4& x, float* acc) {
  acc[0] = fmaf(a, x.x, acc[0]), acc[1] = fmaf(a, x.y, acc[1]), acc[2] = fmaf(a, x.z, acc[2]),
  acc[3] = fmaf(a, x.w, acc[3]);
}
__device__ __forceinline__ void vfma(double a, const double2& x, double* acc) {
  acc[0] = fma(a, x.x, acc[0]), acc[1] = fma(a, x.y, acc[1]);
}

template <class T, class V, int L, int UNR>
__global__ void __launch_bounds__(256) spmm_csr_vec_kernel(int64_t n, const int64_t* __restrict__ rp,
                                                           const int32_t* __restrict__ ci,
                                                           const V* __restrict__ val, int p,
                                                           const T* __restrict__ X, int ldx,
                                                           T* __restrict__ Y, int ldy, int64_t rows_per_cta) {
  using VT = typename Vec16<T>::type;
  constexpr int VEC = Vec16<T>::n;
  constexpr int G = kWarp / L;  // non-zeros handled side by side
  const int lane = threadIdx.x & 31;
  const int g = lane / L, li = lane % L;
  const int col0 = li * VEC;
  const bool has_cols = col0 < p;
  // the warps of a CTA sweep one contiguous range of rows together, so the rows of X
  // that neighbouring rows share (banded couplings) are reused from L1
  const int wpc = blockDim.x / kWarp;
  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = min(n, r_begin + rows_per_cta);
  int64_t row = r_begin + threadIdx.x / kWarp;
  int64_t e0 = 0, e1 = 0;
  if (row < r_end) e0 = rp[row], e1 = rp[row + 1];
  int c = 0;
  T v = T(0);
  if (row < r_end && e0 + lane < e1) c = ci[e0 + lane], v = (T)val[e0 + lane];
  while (row < r_end) {
    const int64_t nrow = row + wpc;
    int64_t ne0 = 0, ne1 = 0;
    if (nrow < r_end) ne0 = rp[nrow], ne1 = rp[nrow + 1];
    T acc[VEC];
#pragma unroll
    for (int t = 0; t < VEC; ++t) acc[t] = T(0);
    for (int64_t base = e0; base < e1; base += kWarp) {
      const int cnt = (e1 - base) < kWarp ? (int)(e1 - base) : kWarp;
      // prefetch the next chunk of this row, or the first chunk of the next row
      int c2 = 0;
      T v2 = T(0);
      {
        const int64_t nb = base + kWarp;
        if (nb < e1) {
          if (nb + lane < e1) c2 = ci[nb + lane], v2 = (T)val[nb + lane];
        } else if (nrow < r_end && ne0 + lane < ne1) {
          c2 = ci[ne0 + lane], v2 = (T)val[ne0 + lane];
        }
      }
      for (int j = 0; j < cnt; j += G * UNR) {
        VT xv[UNR];
        T vv[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          const int src = j + u * G + g;  // <= 31: j + G * UNR <= 32 whenever j < cnt
          const int cc = __shfl_sync(0xffffffffu, c, src & 31);
          vv[u] = __shfl_sync(0xffffffffu, v, src & 31);
          if (src < cnt && has_cols) {
            xv[u] = *reinterpret_cast<const VT*>(X + (int64_t)cc * ldx + col0);
          } else {
            xv[u] = VT{};
            vv[u] = T(0);
          }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) vfma(vv[u], xv[u], acc);
      }
      c = c2;
      v = v2;
    }
#pragma unroll
    for (int t = 0; t < VEC; ++t)
#pragma unroll
      for (int o = L; o < kWarp; o <<= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
    if (g == 0 && has_cols) {
      T* yr = Y + row * ldy + col0;
      if (col0 + VEC <= p) {
        VT out;
        T* po = reinterpret_cast<T*>(&out);
#pragma unroll
        for (int t = 0; t < VEC; ++t) po[t] = acc[t];
        *reinterpret_cast<VT*>(yr) = out;
      } else {
#pragma unroll
        for (int t = 0; t < VEC; ++t)
          if (col0 + t < p) yr[t] = acc[t];
      }
    }
    row = nrow;
    e0 = ne0;
    e1 = ne1;
  }
}

template <class T, class V, int L>
void csr_vec_launch(int64_t n, const int64_t* rp, const int32_t* ci, const V* val, int p, const T* X, int ldx,
                    T* Y, int ldy, cudaStream_t st) {
  const int threads = 256;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t ctas = std::min<int64_t>(ceil_div(n, 64), (int64_t)sms * 8);
  if (ctas < 1) ctas = 1;
  const int64_t rpc = ceil_div(n, ctas);
  ctas = ceil_div(n, rpc);
  constexpr int UNR = L < 8 ? L : 8;
  spmm_csr_vec_kernel<T, V, L, UNR><<<(unsigned)ctas, threads, 0, st>>>(n, rp, ci, val, p, X, ldx, Y, ldy, rpc);
  LB_LAUNCH_CHECK();
}


// Banded variant: the CTA owns rows [r0, r0 + R) and first copies rows [r0 - b, r0 + R + b)
// of X (the couplings inside the band) into shared memory with 16-byte cp.async; gathers
// that fall in that window read shared memory, the rest (long-range couplings) read
// global memory.  Each X row is then fetched from HBM/L2 about (R + 2b) / R times instead
// of once per non-zero.
__device__ __forceinline__ void cp_async16_sp(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}

__device__ __forceinline__ void cp_async4_sp(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}

// Issue the copy of the column indices and values of non-zeros [eb, ee) into shared memory.
template <class V>
__device__ __forceinline__ void stage_csr(const int32_t* __restrict__ ci, const V* __restrict__ val, int64_t eb,
                                          int64_t ee, int32_t* sc, V* sv) {
  static_assert(sizeof(V) == 4 || sizeof(V) == 8, "value type");
  const int cnt = (int)(ee - eb);
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    cp_async4_sp(sc + i, ci + eb + i);
    if (sizeof(V) == 4) {
      cp_async4_sp(sv + i, val + eb + i);
    } else {
      cp_async4_sp(reinterpret_cast<char*>(sv + i), reinterpret_cast<const char*>(val + eb + i));
      cp_async4_sp(reinterpret_cast<char*>(sv + i) + 4, reinterpret_cast<const char*>(val + eb + i) + 4);
    }
  }
}

// The CTA owns rows [r0, r0 + R).  It copies rows [r0 - band, r0 + R + band) of X into
// shared memory, then walks its rows in sub-blocks of RS rows whose (col, val) streams are
// double-buffered in shared memory with cp.async, so the HBM stream of the matrix stays
// in flight while the warps gather from shared memory.  A sub-block with more than `cap`
// non-zeros is read straight from global memory.
template <class T, class V, int L, int UNR, int RS, int NV>
__global__ void __launch_bounds__(512) spmm_csr_band_kernel(int64_t n, const int64_t* __restrict__ rp,
                                                            const int32_t* __restrict__ ci,
                                                            const V* __restrict__ val, int p,
                                                            const T* __restrict__ X, int ldx,
                                                            T* __restrict__ Y, int ldy, int R, int band,
                                                            int pp, int cap) {
  using VT = typename Vec16<T>::type;
  constexpr int VEC = Vec16<T>::n;
  constexpr int G = kWarp / L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int64_t r_end = min(n, r0 + R);
  const int64_t lo = max((int64_t)0, r0 - band), hi = min(n, r_end + band);
  const int win = (int)(hi - lo);
  T* tile = reinterpret_cast<T*>(smem_raw);
  V* sval = reinterpret_cast<V*>(smem_raw + (size_t)win * pp * sizeof(T));  // [2][cap]
  int32_t* scol = reinterpret_cast<int32_t*>(sval + 2 * cap);                   // [2][cap]
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x / kWarp, wpc = blockDim.x / kWarp;
  {
    const int vpr = pp / VEC;
    const int groups = blockDim.x / vpr;
    if (threadIdx.x < groups * vpr)
      for (int rr = threadIdx.x / vpr; rr < win; rr += groups)
        cp_async16_sp(tile + (int64_t)rr * pp + (threadIdx.x % vpr) * VEC,
                      X + (lo + rr) * ldx + (threadIdx.x % vpr) * VEC);
  }
  const int nsub = (int)((r_end - r0 + RS - 1) / RS);
  auto sub_range = [&](int k, int64_t& eb, int64_t& ee) {
    const int64_t a = r0 + (int64_t)k * RS, b = min(r_end, a + RS);
    eb = rp[a];
    ee = rp[b];
  };
  {
    int64_t eb, ee;
    sub_range(0, eb, ee);
    if (ee - eb <= cap) stage_csr<V>(ci, val, eb, ee, scol, sval);
  }
  asm volatile("cp.async.commit_group;\n" ::);
  const int g = lane / L, li = lane % L;
  const int col0 = li * VEC * NV;  // each lane owns NV consecutive 16-byte vectors of a row
  const bool has_cols = col0 < p;
  const T* tile_c = tile + col0;
  const T* X_c = X + col0;
  const unsigned uwin = (unsigned)win;
  const int ilo = (int)lo;
  for (int k = 0; k < nsub; ++k) {
    const int buf = k & 1;
    int64_t eb, ee;
    sub_range(k, eb, ee);
    const bool staged = ee - eb <= cap;
    if (k + 1 < nsub) {
      int64_t nb, ne;
      sub_range(k + 1, nb, ne);
      // the buffer being refilled was last read in sub-block k - 1 (finished at the barrier below)
      if (ne - nb <= cap) stage_csr<V>(ci, val, nb, ne, scol + (buf ^ 1) * cap, sval + (buf ^ 1) * cap);
    }
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 1;\n" ::);
    __syncthreads();
    // column indices / values of this sub-block: shared memory, or global memory when the
    // sub-block was too large to stage (both indexed by e - eb)
    const int32_t* sc = staged ? scol + buf * cap : ci + eb;
    const V* sv = staged ? sval + buf * cap : val + eb;
    const int64_t rb = r0 + (int64_t)k * RS, re = min(r_end, rb + RS);
    for (int64_t row = rb + wid; row < re; row += wpc) {
      const int le0 = (int)(rp[row] - eb), le1 = (int)(rp[row + 1] - eb);
      T acc[NV][VEC];
#pragma unroll
      for (int w = 0; w < NV; ++w)
#pragma unroll
        for (int t = 0; t < VEC; ++t) acc[w][t] = T(0);
      for (int lj = le0; lj < le1; lj += G * UNR) {
        VT xv[UNR][NV];
        T vv[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          const int le = lj + u * G + g;
          const bool valid = le < le1 && has_cols;
          const int c = valid ? sc[le] : ilo;
          vv[u] = valid ? (T)sv[le] : T(0);
          // band couplings read the shared-memory window, the others global memory; one
          // generic load for both keeps the lanes of a warp on one path
          const unsigned o = (unsigned)(c - ilo);
          const VT* src = reinterpret_cast<const VT*>(o < uwin ? tile_c + (int64_t)o * pp : X_c + (int64_t)c * ldx);
#pragma unroll
          for (int w = 0; w < NV; ++w) xv[u][w] = valid ? src[w] : VT{};
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u)
#pragma unroll
          for (int w = 0; w < NV; ++w) vfma(vv[u], xv[u][w], acc[w]);
      }
#pragma unroll
      for (int w = 0; w < NV; ++w)
#pragma unroll
        for (int t = 0; t < VEC; ++t)
#pragma unroll
          for (int o = L; o < kWarp; o <<= 1) acc[w][t] += __shfl_xor_sync(0xffffffffu, acc[w][t], o);
      if (g == 0 && has_cols) {
        T* yr = Y + row * ldy + col0;
#pragma unroll
        for (int w = 0; w < NV; ++w) {
          const int cw = col0 + w * VEC;
          if (cw + VEC <= p) {
            VT out;
            T* po = reinterpret_cast<T*>(&out);
#pragma unroll
            for (int t = 0; t < VEC; ++t) po[t] = acc[w][t];
            *reinterpret_cast<VT*>(yr + w * VEC) = out;
          } else {
#pragma unroll
            for (int t = 0; t < VEC; ++t)
              if (cw + t < p) yr[w * VEC + t] = acc[w][t];
          }
        }
      }
    }
    __syncthreads();  // buffer `buf` is refilled in the next iteration's prefetch
  }
  asm volatile("cp.async.wait_group 0;\n" ::);
}

template <class T, class V, int L, int NV>
bool csr_band_launch(int64_t n, const int64_t* rp, const int32_t* ci, const V* val, int p, const T* X, int ldx,
                     T* Y, int ldy, int band, cudaStream_t st) {
  constexpr int VEC = 16 / sizeof(T);
  constexpr int RS = 64;
  const int pp = round_up(p, VEC * NV);
  if (ldx < pp) return false;  // the window rows and X rows are read NV vectors at a time
  const size_t row_bytes = (size_t)pp * sizeof(T);
  const int cap = 5120;  // non-zeros per staged sub-block of RS rows (about 33 KB of the matrix in flight)
  const size_t csr_bytes = (size_t)2 * cap * (sizeof(V) + sizeof(int32_t));
  const size_t budget = 210 * 1024;
  if (budget <= csr_bytes) return false;
  // rows per CTA: as many as fit beside the two band halos, at least 2 band widths
  int64_t R = (int64_t)((budget - csr_bytes) / row_bytes) - 2 * (int64_t)band;
  if (R < 2 * (int64_t)band || R < 256) return false;
  R = std::min<int64_t>(R, std::max<int64_t>(256, ceil_div(n, 152)));
  R = (R + RS - 1) / RS * RS;
  const int64_t win = std::min<int64_t>(n, R + 2 * (int64_t)band);
  const size_t smem = (size_t)win * row_bytes + csr_bytes;
  if (smem > 220 * 1024) return false;
  constexpr int UNR = (L < 4 ? L : 4);
  // set once per process; function-local statics initialise thread-safely
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(spmm_csr_band_kernel<T, V, L, UNR, RS, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 225 * 1024));
    return true;
  }();
  (void)attr;
  const int64_t ctas = ceil_div(n, R);
  spmm_csr_band_kernel<T, V, L, UNR, RS, NV><<<(unsigned)ctas, 512, smem, st>>>(n, rp, ci, val, p, X, ldx, Y, ldy,
                                                                              (int)R, band, pp, cap);
  LB_LAUNCH_CHECK();
  return true;
}

// Fraction of non-zeros with |col - row| <= b for b in kBands (one pass over the rows).
__global__ void band_profile_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                    unsigned long long* counts, int nb, const int* bands) {
  __shared__ unsigned long long sc[16];
  if (threadIdx.x < 16) sc[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long loc[16] = {};
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x)
    for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
      const int64_t d = ci[e] > row ? ci[e] - row : row - ci[e];
      for (int k = 0; k < nb; ++k) loc[k] += d <= bands[k];
    }
  for (int k = 0; k < nb; ++k) atomicAdd(&sc[k], loc[k]);
  __syncthreads();
  if (threadIdx.x < nb) atomicAdd(&counts[threadIdx.x], sc[threadIdx.x]);
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
                     const T* X, int ldx, T* Y, int ldy, cudaStream_t st, int band) {
  if (n <= 0 || p <= 0) return;
  if (p > 32) throw std::invalid_argument("spmm: p > 32");
  constexpr int VEC = 16 / sizeof(T);
  const bool vec_ok = (ldx % VEC == 0) && (ldy % VEC == 0) && ldx >= round_up(p, VEC) &&
                      !(reinterpret_cast<uintptr_t>(X) & 15) && !(reinterpret_cast<uintptr_t>(Y) & 15);
  if (vec_ok && band >= 0) {
    // two 16-byte vectors per lane halve the index work per gathered value
    const int lanes = (p + 2 * VEC - 1) / (2 * VEC);
    bool done = false;
    if (lanes <= 1) done = csr_band_launch<T, V, 1, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, band, st);
    else if (lanes <= 2) done = csr_band_launch<T, V, 2, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, band, st);
    else if (lanes <= 4) done = csr_band_launch<T, V, 4, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, band, st);
    else if (lanes <= 8) done = csr_band_launch<T, V, 8, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, band, st);
    else done = csr_band_launch<T, V, 16, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, band, st);
    if (done) return;
  }
  if (vec_ok) {
    // L lanes per non-zero, each holding VEC columns: L = pow2 >= ceil(p / VEC)
    const int lanes = (p + VEC - 1) / VEC;
    if (lanes <= 1) csr_vec_launch<T, V, 1>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
    else if (lanes <= 2) csr_vec_launch<T, V, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
    else if (lanes <= 4) csr_vec_launch<T, V, 4>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
    else if (lanes <= 8) csr_vec_launch<T, V, 8>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
    else csr_vec_launch<T, V, 16>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
    return;
  }
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
                                              int, const double*, int, double*, int, cudaStream_t, int);
template void launch_spmm_csr<float, float>(int64_t, const int64_t*, const int32_t*, const float*,
                                            int, const float*, int, float*, int, cudaStream_t, int);

int profile_band(int64_t n, const int64_t* rp, const int32_t* ci, int64_t nnz, cudaStream_t st) {
  if (n <= 0 || nnz <= 0) return -1;
  const int nb = 8;
  const int bands[nb] = {16, 32, 64, 128, 256, 512, 1024, 2048};
  int* dbands = nullptr;
  unsigned long long* dcounts = nullptr;
  LB_CUDA(cudaMallocAsync(&dbands, sizeof(bands), st));
  LB_CUDA(cudaMallocAsync(&dcounts, nb * sizeof(unsigned long long), st));
  LB_CUDA(cudaMemcpyAsync(dbands, bands, sizeof(bands), cudaMemcpyHostToDevice, st));
  LB_CUDA(cudaMemsetAsync(dcounts, 0, nb * sizeof(unsigned long long), st));
  band_profile_kernel<<<std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 1216)), 256, 0, st>>>(n, rp, ci, dcounts, nb, dbands);
  LB_LAUNCH_CHECK();
  unsigned long long counts[nb];
  LB_CUDA(cudaMemcpyAsync(counts, dcounts, sizeof(counts), cudaMemcpyDeviceToHost, st));
  LB_CUDA(cudaStreamSynchronize(st));
  cudaFreeAsync(dbands, st);
  cudaFreeAsync(dcounts, st);
  // the smallest band that holds 80% of the non-zeros (if the whole matrix is narrow, n)
  for (int k = 0; k < nb; ++k)
    if (counts[k] >= 0.8 * (double)nnz) return bands[k];
  return -1;
}
template void launch_spmm_dense<double>(int64_t, const double*, int64_t, int, const double*, int,
                                        double*, int, cudaStream_t);
template void launch_spmm_dense<float>(int64_t, const float*, int64_t, int, const float*, int,
                                       float*, int, cudaStream_t);

}  // namespace lobpcg
