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
#include <type_traits>

#include "common.cuh"
#include "dfloat.cuh"

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

__device__ __forceinline__ void cp_async8_sp(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}

// Shared-memory loads by 32-bit shared-window address.
__device__ __forceinline__ int2 lds_s32x2(unsigned addr) {
  int2 r;
  asm volatile("ld.shared.v2.s32 {%0, %1}, [%2];\n" : "=r"(r.x), "=r"(r.y) : "r"(addr));
  return r;
}
__device__ __forceinline__ float4 lds_f32x4(unsigned addr) {
  float4 r;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "r"(addr));
  return r;
}

// Sum of a lane's V values over the G = 32/L lane groups of a warp, left scattered over
// the lanes (a transpose reduction): at each xor level a lane keeps half of its values
// (the upper half when its level bit is set) and adds the partner's copy of that half, so
// the levels exchange V/2 + V/4 + ... values instead of V each.  On return the lane holds
// in acc[0 .. Scatter<L, V>::keep) the sums of its chunk's values [off, off + keep);
// `owner` is false on the lanes that hold a duplicate (levels after the count turned odd).
template <int L, int V>
struct Scatter {
  static constexpr int kept() {
    int cur = V;
    for (int o = L; o < kWarp; o <<= 1)
      if (cur > 1 && (cur & 1) == 0) cur >>= 1;
    return cur;
  }
  static constexpr int keep = kept();
};
template <int L, int V, class T>
__device__ __forceinline__ int reduce_scatter(T (&acc)[V], int lane, bool& owner) {
  int off = 0;
  owner = true;
#pragma unroll
  for (int o = L, cur = V; o < kWarp; o <<= 1) {
    const bool up = (lane & o) != 0;
    if (cur > 1 && (cur & 1) == 0) {
      const int half = cur >> 1;
#pragma unroll
      for (int i = 0; i < V / 2; ++i)
        if (i < half) {
          const T send = up ? acc[i] : acc[i + half];
          const T keep = up ? acc[i + half] : acc[i];
          acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      if (up) off += half;
      cur = half;
    } else {
      // odd count: plain butterfly on what is left; the upper lane becomes a duplicate
#pragma unroll
      for (int i = 0; i < V; ++i)
        if (i < cur) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
      if (up) owner = false;
    }
  }
  return off;
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

constexpr int kWindowPad = 64;  // staged entries beyond a sub-block that a batch may read

// Band part of a split matrix (every entry has |col - row| <= band), FP32.  The CTA owns
// rows [r0, r0 + R) and keeps rows [r0 - band, r0 + R + band) of X in shared memory (row
// stride pp = p rounded up to 16 bytes), plus one zero row that the lanes past the end
// of a row read instead of masking their data.  The matrix streams through in sub-blocks
// of RS rows: row pointers and interleaved (column, value) pairs are double-buffered in
// shared memory with cp.async one sub-block ahead.  A group of L lanes takes one
// non-zero and reads its row of X as L consecutive 16-byte vectors, so each quarter-warp
// phase of a gather reads one contiguous row (free of bank conflicts); G = 32/L non-zeros
// per warp step, UNR steps in flight, and a transpose reduction over the G groups.
template <class T, class V, int L, int UNR, int RS>
__global__ void __launch_bounds__(512, 1) spmm_csr_window_kernel(int64_t n, const int64_t* __restrict__ rp,
                                                              const int32_t* __restrict__ ci,
                                                              const V* __restrict__ val, int p,
                                                              const T* __restrict__ X, int ldx,
                                                              T* __restrict__ Y, int ldy, int R, int band,
                                                              int pp, int cap) {
  static_assert(sizeof(V) == 4 && sizeof(T) == 4, "FP32 blocks, interleaved 4-byte values");
  using VT = typename Vec16<T>::type;
  constexpr int VEC = Vec16<T>::n;
  constexpr int G = kWarp / L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int64_t r_end = min(n, r0 + R);
  const int64_t lo = max((int64_t)0, r0 - band), hi = min(n, r_end + band);
  const int win = (int)(hi - lo);
  const int nvec = pp / VEC;
  T* tile = reinterpret_cast<T*>(smem_raw);                                                 // [win + 1][pp]
  int64_t* srp = reinterpret_cast<int64_t*>(smem_raw + (size_t)(win + 1) * pp * sizeof(T));  // [2][RS + 1]
  static_assert(G * UNR <= kWindowPad, "a batch may read kWindowPad entries past a sub-block's end");
  const int cpad = cap + kWindowPad;  // entries read past a sub-block's end stay in the buffer
  int2* scv = reinterpret_cast<int2*>(srp + 2 * (RS + 1));                                // [2][cpad]
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x / kWarp, wpc = blockDim.x / kWarp;
  for (int e = threadIdx.x; e < win * nvec; e += blockDim.x) {
    const int rr = e / nvec, w = e - rr * nvec;
    cp_async16_sp(tile + (int64_t)rr * pp + w * VEC, X + (lo + rr) * ldx + w * VEC);
  }
  for (int e = threadIdx.x; e < pp; e += blockDim.x) tile[(int64_t)win * pp + e] = T(0);
  for (int e = threadIdx.x; e < 2 * cpad; e += blockDim.x) scv[e] = make_int2(0, 0);
  __syncthreads();  // zeroed entries before any cp.async lands on them
  const unsigned row_bytes = (unsigned)(pp * sizeof(T));
  const unsigned zoff = (unsigned)win * row_bytes;
  const int nsub = (int)((r_end - r0 + RS - 1) / RS);
  auto bounds = [&](int k, int64_t& eb, int64_t& ee) {
    const int64_t a = r0 + (int64_t)k * RS, b = min(r_end, a + RS);
    eb = rp[a];
    ee = rp[b];
  };
  auto stage = [&](int k, int buf, int64_t eb, int64_t ee) {
    const int64_t a = r0 + (int64_t)k * RS;
    const int rows = (int)(min(r_end, a + RS) - a);
    for (int i = threadIdx.x; i <= rows; i += blockDim.x) cp_async8_sp(srp + buf * (RS + 1) + i, rp + a + i);
    if (ee - eb <= cap) {
      int2* d = scv + buf * cpad;
      for (int i = threadIdx.x; i < (int)(ee - eb); i += blockDim.x) {
        cp_async4_sp(&d[i].x, ci + eb + i);
        cp_async4_sp(&d[i].y, val + eb + i);
      }
    }
  };
  int64_t eb, ee, nb = 0, ne = 0;
  bounds(0, eb, ee);
  stage(0, 0, eb, ee);
  asm volatile("cp.async.commit_group;\n" ::);
  if (nsub > 1) bounds(1, nb, ne);
  const int g = lane / L, li = lane % L;
  const bool has_vec = li < nvec;
  const char* tile_b = reinterpret_cast<const char*>(tile + li * VEC);
  const unsigned tile_s = (unsigned)__cvta_generic_to_shared(tile_b);
  const int ilo = (int)lo;
  for (int k = 0; k < nsub; ++k) {
    const int buf = k & 1;
    if (k + 1 < nsub) stage(k + 1, buf ^ 1, nb, ne);  // buffer buf^1 was last read in k - 1
    asm volatile("cp.async.commit_group;\n" ::);
    int64_t fb = 0, fe = 0;
    if (k + 2 < nsub) bounds(k + 2, fb, fe);  // in flight during this sub-block
    asm volatile("cp.async.wait_group 1;\n" ::);
    if (ee - eb <= cap) {
      // this thread's copies of sub-block k have landed: column index -> byte offset of
      // its row in the window (clamped, so a malformed index stays in bounds)
      int2* d = scv + buf * cpad;
      for (int i = threadIdx.x; i < (int)(ee - eb); i += blockDim.x)
        d[i].x = (int)(min((unsigned)(d[i].x - ilo), (unsigned)win) * row_bytes);
    }
    __syncthreads();
    const bool staged = ee - eb <= cap;
    const int2* sp = scv + buf * cpad;
    const unsigned sp_s = (unsigned)__cvta_generic_to_shared(sp);
    const int64_t* brp = srp + buf * (RS + 1);
    const int64_t rb = r0 + (int64_t)k * RS;
    const int rows = (int)(min(r_end, rb + RS) - rb);
    for (int r = wid; r < rows; r += wpc) {
      const int le0 = (int)(brp[r] - eb), le1 = (int)(brp[r + 1] - eb);
      T acc[VEC];
#pragma unroll
      for (int t = 0; t < VEC; ++t) acc[t] = T(0);
      if (staged) {
        // branch-free: entries hold window byte offsets; lanes past the row end read the
        // zero row (their value is a finite stale or zero entry)
        for (int lj = le0; lj < le1; lj += G * UNR) {
          const unsigned ea = sp_s + (unsigned)(lj + g) * 8u;  // entry address of step 0
          const int rem = le1 - lj - g;                          // steps with u * G < rem are in the row
          float4 xv[UNR];
          float vv[UNR];
#pragma unroll
          for (int u = 0; u < UNR; ++u) {
            const int2 cv = lds_s32x2(ea + u * G * 8);
            const unsigned off = u * G < rem ? (unsigned)cv.x : zoff;
            vv[u] = __int_as_float(cv.y);
            xv[u] = lds_f32x4(tile_s + off);
          }
#pragma unroll
          for (int u = 0; u < UNR; ++u) vfma(vv[u], xv[u], acc);
        }
      } else {
        for (int lj = le0; lj < le1; lj += G * UNR) {
          VT xv[UNR];
          T vv[UNR];
#pragma unroll
          for (int u = 0; u < UNR; ++u) {
            const int le = lj + u * G + g;
            unsigned off = zoff;
            T v = T(0);
            if (le < le1) {
              // in the window by construction (the clamp keeps a malformed index in bounds)
              off = min((unsigned)(ci[eb + le] - ilo), (unsigned)win) * row_bytes;
              v = (T)val[eb + le];
            }
            vv[u] = v;
            xv[u] = *reinterpret_cast<const VT*>(tile_b + off);
          }
#pragma unroll
          for (int u = 0; u < UNR; ++u) vfma(vv[u], xv[u], acc);
        }
      }
      bool owner;
      const int off = reduce_scatter<L, VEC>(acc, lane, owner);
      if (owner && has_vec) {
        T* yr = Y + (rb + r) * ldy + li * VEC + off;
#pragma unroll
        for (int t = 0; t < Scatter<L, VEC>::keep; ++t)
          if (li * VEC + off + t < p) yr[t] = acc[t];
      }
    }
    eb = nb, ee = ne, nb = fb, ne = fe;
    __syncthreads();  // buffer `buf` is refilled in the next iteration's prefetch
  }
  asm volatile("cp.async.wait_group 0;\n" ::);
}

template <class T, class V, int L>
bool csr_window_launch(int64_t n, const int64_t* rp, const int32_t* ci, const V* val, int p, const T* X, int ldx,
                       T* Y, int ldy, int band, cudaStream_t st) {
  constexpr int VEC = 16 / sizeof(T);
  constexpr int RS = 64;
  constexpr int UNR = 2 * L;  // G * UNR = 64 non-zeros per batch (a typical band row)
  const int pp = round_up(p, VEC);
  if (ldx < pp || pp > L * VEC) return false;
  const size_t row_bytes = (size_t)pp * sizeof(T);
  const int cap = 4096;  // non-zeros per staged sub-block of RS rows
  const size_t fixed = (size_t)2 * (cap + kWindowPad) * sizeof(int2) + (size_t)2 * (RS + 1) * sizeof(int64_t);
  const size_t budget = 216 * 1024;
  if (budget <= fixed + row_bytes) return false;
  // rows per CTA: as many as fit beside the two band halos and the zero row
  int64_t R = (int64_t)((budget - fixed) / row_bytes) - 1 - 2 * (int64_t)band;
  R = R / RS * RS;
  if (R < RS) return false;
  R = std::min<int64_t>(R, std::max<int64_t>(RS, ceil_div(ceil_div(n, 152), RS) * RS));
  const int64_t win = std::min<int64_t>(n, R + 2 * (int64_t)band);
  const size_t smem = (size_t)(win + 1) * row_bytes + fixed;
  if (smem > 220 * 1024) return false;
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(spmm_csr_window_kernel<T, V, L, UNR, RS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024));
    return true;
  }();
  (void)attr;
  const int64_t ctas = ceil_div(n, R);
  spmm_csr_window_kernel<T, V, L, UNR, RS><<<(unsigned)ctas, 512, smem, st>>>(n, rp, ci, val, p, X, ldx, Y, ldy,
                                                                            (int)R, band, pp, cap);
  LB_LAUNCH_CHECK();
  return true;
}

__device__ __forceinline__ int4 lds_s32x4(unsigned addr) {
  int4 r;
  asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];\n" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "r"(addr));
  return r;
}

// Band part of a split matrix in packed form, FP32.  Each entry is one 8-byte pair
// (col - row, value bits) with the column already inside [row - band, row + band] and
// [0, n), and every row holds an even number of entries (a zero entry pads odd rows), so a
// row starts on a 16-byte boundary and a lane reads two entries with one 16-byte load.  The
// CTA owns rows [r0, r0 + R) and keeps rows [r0 - band, r0 + R + band) of X in shared
// memory (row stride pp = p rounded up to 16 bytes).  Row pointers and entry pairs of
// sub-blocks of RS rows are double-buffered in shared memory with 16-byte cp.async, one
// sub-block ahead.  A group of L lanes takes two entries of a row per step and reads the
// two gathered rows of X as L consecutive 16-byte vectors each.  Full batches of 2 G UNR
// entries issue all their entry loads, then all their gathers; the rest of the row goes
// in steps of 2 G entries, where pairs past the row's end read a zero pair (value 0, the
// row's own X row), so no lane needs a predicate.  A transpose reduction sums the G groups.
template <int L, int UNR, int RS>
__global__ void __launch_bounds__(512, 1) spmm_band_packed_kernel(int64_t n, const int64_t* __restrict__ rpk,
                                                               const int2* __restrict__ pk, int p,
                                                               const float* __restrict__ X, int ldx,
                                                               float* __restrict__ Y, int ldy, int R, int band,
                                                               int pp, int cap) {
  constexpr int VEC = 4;
  constexpr int G = kWarp / L;
  constexpr int BATCH = 2 * G * UNR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int64_t r_end = min(n, r0 + R);
  const int64_t lo = max((int64_t)0, r0 - band), hi = min(n, r_end + band);
  const int win = (int)(hi - lo);
  const int nvec = pp / VEC;
  float* tile = reinterpret_cast<float*>(smem_raw);                                        // [win][pp]
  int64_t* srp = reinterpret_cast<int64_t*>(smem_raw + (size_t)win * pp * sizeof(float));  // [2][RS + 1]
  int2* spk = reinterpret_cast<int2*>(srp + 2 * (RS + 1));                                 // [2][cap] + zero pair
  int2* zpair = spk + 2 * cap;
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x / kWarp, wpc = blockDim.x / kWarp;
  for (int e = threadIdx.x; e < win * nvec; e += blockDim.x) {
    const int rr = e / nvec, w = e - rr * nvec;
    cp_async16_sp(tile + (int64_t)rr * pp + w * VEC, X + (lo + rr) * ldx + w * VEC);
  }
  if (threadIdx.x < 2) zpair[threadIdx.x] = make_int2(0, 0);
  const unsigned row_bytes = (unsigned)(pp * sizeof(float));
  const int nsub = (int)((r_end - r0 + RS - 1) / RS);
  auto bounds = [&](int k, int64_t& eb, int64_t& ee) {
    const int64_t a = r0 + (int64_t)k * RS, b = min(r_end, a + RS);
    eb = rpk[a];
    ee = rpk[b];
  };
  // row pointers and, when they fit, the entries of sub-block k (eb, ee even: 16-byte
  // aligned source and size)
  auto stage = [&](int k, int buf, int64_t eb, int64_t ee) {
    const int64_t a = r0 + (int64_t)k * RS;
    const int rows = (int)(min(r_end, a + RS) - a);
    for (int i = threadIdx.x; i <= rows; i += blockDim.x) cp_async8_sp(srp + buf * (RS + 1) + i, rpk + a + i);
    if (ee - eb <= cap) {
      int2* d = spk + buf * cap;
      for (int i = threadIdx.x; 2 * i < (int)(ee - eb); i += blockDim.x) cp_async16_sp(d + 2 * i, pk + eb + 2 * i);
    }
  };
  int64_t eb, ee, nb = 0, ne = 0;
  bounds(0, eb, ee);
  stage(0, 0, eb, ee);
  asm volatile("cp.async.commit_group;\n" ::);
  if (nsub > 1) bounds(1, nb, ne);
  const int g = lane / L, li = lane % L;
  const bool has_vec = li < nvec;
  const unsigned tile_s = (unsigned)__cvta_generic_to_shared(tile + li * VEC);
  const unsigned zero_s = (unsigned)__cvta_generic_to_shared(zpair);
  for (int k = 0; k < nsub; ++k) {
    const int buf = k & 1;
    if (k + 1 < nsub) stage(k + 1, buf ^ 1, nb, ne);  // buffer buf^1 was last read in k - 1
    asm volatile("cp.async.commit_group;\n" ::);
    int64_t fb = 0, fe = 0;
    if (k + 2 < nsub) bounds(k + 2, fb, fe);  // in flight during this sub-block
    asm volatile("cp.async.wait_group 1;\n" ::);
    __syncthreads();
    const bool staged = ee - eb <= cap;
    const unsigned sp_s = (unsigned)__cvta_generic_to_shared(spk + buf * cap);
    const int64_t* brp = srp + buf * (RS + 1);
    const int64_t rb = r0 + (int64_t)k * RS;
    const int rows = (int)(min(r_end, rb + RS) - rb);
    for (int r = wid; r < rows; r += wpc) {
      const int le0 = (int)(brp[r] - eb), le1 = (int)(brp[r + 1] - eb);
      // this lane's vector of the row's own window row; an entry (d, v) gathers row + d
      const unsigned rbase = tile_s + (unsigned)(rb + r - lo) * row_bytes;
      float acc[VEC] = {0.f, 0.f, 0.f, 0.f};
      int lj = le0;
      if (staged) {
        for (; lj + BATCH <= le1; lj += BATCH) {
          int4 q[UNR];
#pragma unroll
          for (int u = 0; u < UNR; ++u) q[u] = lds_s32x4(sp_s + (unsigned)(lj + 2 * (u * G + g)) * 8u);
          float4 xa[UNR], xb[UNR];
#pragma unroll
          for (int u = 0; u < UNR; ++u) {
            xa[u] = lds_f32x4(rbase + (unsigned)(q[u].x * (int)row_bytes));
            xb[u] = lds_f32x4(rbase + (unsigned)(q[u].z * (int)row_bytes));
          }
#pragma unroll
          for (int u = 0; u < UNR; ++u) {
            vfma(__int_as_float(q[u].y), xa[u], acc);
            vfma(__int_as_float(q[u].w), xb[u], acc);
          }
        }
        for (; lj < le1; lj += 2 * G) {
          const int e = lj + 2 * g;  // even: entries e and e + 1 are both in the row
          const int4 q = lds_s32x4(e < le1 ? sp_s + (unsigned)e * 8u : zero_s);
          const float4 xa = lds_f32x4(rbase + (unsigned)(q.x * (int)row_bytes));
          const float4 xb = lds_f32x4(rbase + (unsigned)(q.z * (int)row_bytes));
          vfma(__int_as_float(q.y), xa, acc);
          vfma(__int_as_float(q.w), xb, acc);
        }
      } else {
        for (; lj < le1; lj += 2 * G) {
          const int e = lj + 2 * g;
          const int4 q = e < le1 ? __ldg(reinterpret_cast<const int4*>(pk + eb + e)) : make_int4(0, 0, 0, 0);
          const float4 xa = lds_f32x4(rbase + (unsigned)(q.x * (int)row_bytes));
          const float4 xb = lds_f32x4(rbase + (unsigned)(q.z * (int)row_bytes));
          vfma(__int_as_float(q.y), xa, acc);
          vfma(__int_as_float(q.w), xb, acc);
        }
      }
      bool owner;
      const int off = reduce_scatter<L, VEC>(acc, lane, owner);
      if (owner && has_vec) {
        float* yr = Y + (rb + r) * ldy + li * VEC + off;
#pragma unroll
        for (int t = 0; t < Scatter<L, VEC>::keep; ++t)
          if (li * VEC + off + t < p) yr[t] = acc[t];
      }
    }
    eb = nb, ee = ne, nb = fb, ne = fe;
    __syncthreads();  // buffer `buf` is refilled in the next iteration's prefetch
  }
  asm volatile("cp.async.wait_group 0;\n" ::);
}

template <int L>
bool band_packed_launch(int64_t n, const int64_t* rpk, const int2* pk, int p, const float* X, int ldx, float* Y,
                        int ldy, int band, cudaStream_t st) {
  constexpr int VEC = 4;
  constexpr int RS = 32;
  constexpr int UNR = 16 / (kWarp / L);  // 2 G UNR = 32 entries per step of the warp
  const int pp = round_up(p, VEC);
  if (ldx < pp || pp > L * VEC || band < 0) return false;
  const size_t row_bytes = (size_t)pp * sizeof(float);
  const int cap = 2048;  // entries per staged sub-block of RS rows (even)
  const size_t fixed = (size_t)(2 * cap + 2) * sizeof(int2) + (size_t)2 * (RS + 1) * sizeof(int64_t);
  const size_t budget = 216 * 1024;
  if (budget <= fixed + row_bytes) return false;
  // rows per CTA: as many as fit beside the two band halos, then evened out over whole
  // waves of 152 CTAs
  int64_t R = (int64_t)((budget - fixed) / row_bytes) - 2 * (int64_t)band;
  R = R / RS * RS;
  if (R < RS) return false;
  const int64_t waves = ceil_div(ceil_div(n, R), 152);
  R = std::min<int64_t>(R, ceil_div(ceil_div(n, 152 * waves), RS) * RS);
  const int64_t win = std::min<int64_t>(n, R + 2 * (int64_t)band);
  const size_t smem = (size_t)win * row_bytes + fixed;
  if (smem > 220 * 1024) return false;
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(spmm_band_packed_kernel<L, UNR, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 225 * 1024));
    return true;
  }();
  (void)attr;
  const int64_t ctas = ceil_div(n, R);
  spmm_band_packed_kernel<L, UNR, RS><<<(unsigned)ctas, 512, smem, st>>>(n, rpk, pk, p, X, ldx, Y, ldy, (int)R,
                                                                         band, pp, cap);
  LB_LAUNCH_CHECK();
  return true;
}

// Row-parallel product, Y += A X (ACC) or Y = A X.  Each group of L lanes owns one row of
// Y (NV 16-byte vectors per lane, no cross-lane reduction) and walks that row's entries
// UNR at a time, issuing all UNR gathers before using them; a warp thus keeps G = 32/L
// rows x UNR gathers in flight.  Used for the long-range part of a split product (few,
// scattered entries per row) and for FP64 products, which are bound by the FP64 FMA rate:
// here nearly every lane of every FMA instruction does useful work.
template <class T, class V, int L, int NV, int UNR, bool ACC>
__global__ void __launch_bounds__(256) spmm_csr_add_kernel(int64_t n, const int64_t* __restrict__ rp,
                                                           const int32_t* __restrict__ ci,
                                                           const V* __restrict__ val, int p,
                                                           const T* __restrict__ X, int ldx,
                                                           T* __restrict__ Y, int ldy) {
  using VT = typename Vec16<T>::type;
  constexpr int VEC = Vec16<T>::n;
  constexpr int G = kWarp / L;
  const int lane = threadIdx.x & 31;
  const int g = lane / L, li = lane % L;
  const int col0 = li * VEC * NV;
  const bool has_cols = col0 < p;
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / kWarp) * G;
  for (int64_t row = ((int64_t)blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp) * G + g; row < n;
       row += groups) {
    const int64_t e0 = rp[row], e1 = rp[row + 1];
    if ((ACC && e0 == e1) || !has_cols) continue;
    T acc[NV][VEC];
#pragma unroll
    for (int w = 0; w < NV; ++w)
#pragma unroll
      for (int t = 0; t < VEC; ++t) acc[w][t] = T(0);
    for (int64_t e = e0; e < e1; e += UNR) {
      VT xv[UNR][NV];
      T vv[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const bool valid = e + u < e1;
        const int c = valid ? ci[e + u] : 0;
        vv[u] = valid ? (T)val[e + u] : T(0);
        const VT* src = reinterpret_cast<const VT*>(X + (int64_t)c * ldx + col0);
#pragma unroll
        for (int w = 0; w < NV; ++w) xv[u][w] = (valid && col0 + w * VEC < p) ? __ldg(src + w) : VT{};
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u)
#pragma unroll
        for (int w = 0; w < NV; ++w) vfma(vv[u], xv[u][w], acc[w]);
    }
    T* yr = Y + row * ldy + col0;
#pragma unroll
    for (int w = 0; w < NV; ++w) {
      const int cw = col0 + w * VEC;
      if (cw + VEC <= p) {
        VT y = ACC ? *reinterpret_cast<const VT*>(yr + w * VEC) : VT{};
        T* py = reinterpret_cast<T*>(&y);
#pragma unroll
        for (int t = 0; t < VEC; ++t) py[t] += acc[w][t];
        *reinterpret_cast<VT*>(yr + w * VEC) = y;
      } else {
#pragma unroll
        for (int t = 0; t < VEC; ++t)
          if (cw + t < p) yr[w * VEC + t] = ACC ? yr[w * VEC + t] + acc[w][t] : acc[w][t];
      }
    }
  }
}

template <class T, class V, int L, int NV, bool ACC>
void csr_add_launch(int64_t n, const int64_t* rp, const int32_t* ci, const V* val, int p, const T* X, int ldx,
                    T* Y, int ldy, cudaStream_t st) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256;
  constexpr int G = kWarp / L;
  int64_t ctas = std::min<int64_t>(ceil_div(n, (threads / kWarp) * G), (int64_t)sms * 6);
  if (ctas < 1) ctas = 1;
  spmm_csr_add_kernel<T, V, L, NV, 4, ACC><<<(unsigned)ctas, threads, 0, st>>>(n, rp, ci, val, p, X, ldx, Y, ldy);
  LB_LAUNCH_CHECK();
}

// L lanes x NV vectors cover the row: nvec 16-byte vectors per row of X
template <class T, class V, bool ACC>
void csr_rows_dispatch(int64_t n, const int64_t* rp, const int32_t* ci, const V* val, int p, const T* X, int ldx,
                       T* Y, int ldy, cudaStream_t st) {
  constexpr int VEC = 16 / sizeof(T);
  const int nvec = (p + VEC - 1) / VEC;
  if (nvec <= 2) csr_add_launch<T, V, 1, 2, ACC>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
  else if (nvec <= 3) csr_add_launch<T, V, 1, 3, ACC>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
  else if (nvec <= 4) csr_add_launch<T, V, 1, 4, ACC>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
  else if (nvec <= 6) csr_add_launch<T, V, 2, 3, ACC>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
  else if (nvec <= 8) csr_add_launch<T, V, 2, 4, ACC>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
  else if (nvec <= 12) csr_add_launch<T, V, 4, 3, ACC>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
  else csr_add_launch<T, V, 4, 4, ACC>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
}

// ---- FP64 product in double-float arithmetic (the refinement phase, dfloat.cuh) ----
// Y = A X with A's values and X given as (hi, lo) float pairs (split once: the matrix at
// create time, X before the product).  A group of L lanes owns a row; each lane holds NV
// 16-byte vectors (2 columns each) and keeps UNR gathers in flight, as the row-parallel
// FP64 kernel does.  Each term is a compensated double-float product-sum; Y is FP64.
template <int L, int NV, int UNR>
__global__ void __launch_bounds__(256) spmm_csr_df_kernel(int64_t n, const int64_t* __restrict__ rp,
                                                          const int32_t* __restrict__ ci,
                                                          const float2* __restrict__ vs, int p,
                                                          const float2* __restrict__ Xs, int ldx,
                                                          double* __restrict__ Y, int ldy) {
  constexpr int G = kWarp / L;
  const int lane = threadIdx.x & 31;
  const int g = lane / L, li = lane % L;
  const int col0 = li * 2 * NV;
  const bool has_cols = col0 < p;
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / kWarp) * G;
  for (int64_t row = ((int64_t)blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp) * G + g; row < n;
       row += groups) {
    const int64_t e0 = rp[row], e1 = rp[row + 1];
    if (!has_cols) continue;
    DfAcc acc[NV][2];
#pragma unroll
    for (int w = 0; w < NV; ++w) df_zero(acc[w][0]), df_zero(acc[w][1]);
    for (int64_t e = e0; e < e1; e += UNR) {
      float4 xv[UNR][NV];
      float2 vv[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const bool valid = e + u < e1;
        const int c = valid ? ci[e + u] : 0;
        vv[u] = valid ? vs[e + u] : make_float2(0.f, 0.f);
        const float4* src = reinterpret_cast<const float4*>(Xs + (int64_t)c * ldx + col0);
#pragma unroll
        for (int w = 0; w < NV; ++w)
          xv[u][w] = (valid && col0 + 2 * w < p) ? __ldg(src + w) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u)
#pragma unroll
        for (int w = 0; w < NV; ++w) {
          df_fma(acc[w][0], vv[u], make_float2(xv[u][w].x, xv[u][w].y));
          df_fma(acc[w][1], vv[u], make_float2(xv[u][w].z, xv[u][w].w));
        }
    }
    double* yr = Y + row * ldy + col0;
#pragma unroll
    for (int w = 0; w < NV; ++w) {
      const int cw = col0 + 2 * w;
      if (cw + 2 <= p) {
        *reinterpret_cast<double2*>(yr + 2 * w) = make_double2(df_value(acc[w][0]), df_value(acc[w][1]));
      } else if (cw < p) {
        yr[2 * w] = df_value(acc[w][0]);
      }
    }
  }
}

__global__ void split_df_kernel(int64_t count, const double* __restrict__ src, float2* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = df_split(src[i]);
}

template <int L, int NV>
void csr_df_launch(int64_t n, const int64_t* rp, const int32_t* ci, const float2* vs, int p, const float2* Xs,
                   int ldx, double* Y, int ldy, cudaStream_t st) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256;
  constexpr int G = kWarp / L;
  int64_t ctas = std::min<int64_t>(ceil_div(n, (threads / kWarp) * G), (int64_t)sms * 6);
  if (ctas < 1) ctas = 1;
  spmm_csr_df_kernel<L, NV, 4><<<(unsigned)ctas, threads, 0, st>>>(n, rp, ci, vs, p, Xs, ldx, Y, ldy);
  LB_LAUNCH_CHECK();
}

// ---- band / long-range split of a CSR matrix (once, when the solver is created) ----

// Per row: number of entries with |col - row| <= band (cb) and the rest (cl).
__global__ void split_count_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                   int band, int32_t* __restrict__ cb, int32_t* __restrict__ cl) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * blockDim.x) {
    int b = 0, l = 0;
    for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
      const int64_t d = ci[e] > row ? ci[e] - row : row - ci[e];
      if (d <= band) ++b;
      else ++l;
    }
    cb[row] = b;
    cl[row] = l;
  }
}

// Exclusive prefix sum of n int32 counts into n + 1 int64 row pointers, in three passes:
// per-tile sums, one CTA scanning the tile sums, per-tile rescan with the tile offset.
constexpr int kScanThreads = 256, kScanPer = 16, kScanTile = kScanThreads * kScanPer;

__global__ void __launch_bounds__(kScanThreads) scan_tile_sums_kernel(int64_t n, const int32_t* __restrict__ cnt,
                                                                      int64_t* __restrict__ tsum) {
  __shared__ int64_t red[kScanThreads / kWarp];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t s = 0;
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    const int64_t j = base + i;
    if (j < n) s += cnt[j];
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / kWarp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kScanThreads / kWarp; ++w) t += red[w];
    tsum[blockIdx.x] = t;
  }
}

// In-place exclusive scan of the tile sums by one CTA of 1024 threads, 1024 at a time.
__global__ void __launch_bounds__(1024) scan_tile_offsets_kernel(int64_t ntiles, int64_t* __restrict__ tsum) {
  __shared__ int64_t wsum[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x / kWarp;
  for (int64_t base = 0; base < ntiles; base += 1024) {
    const int64_t j = base + threadIdx.x;
    const int64_t v = j < ntiles ? tsum[j] : 0;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int64_t wo = 0;
    for (int i = 0; i < w; ++i) wo += wsum[i];
    const int64_t c = carry;
    if (j < ntiles) tsum[j] = c + wo + x - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = c + wo + x;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_write_kernel(int64_t n, const int32_t* __restrict__ cnt,
                                                                  const int64_t* __restrict__ toff,
                                                                  int64_t* __restrict__ out) {
  __shared__ int64_t wsum[kScanThreads / kWarp];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int64_t v[kScanPer];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    const int64_t j = base + i;
    v[i] = j < n ? cnt[j] : 0;
    s += v[i];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x / kWarp;
  int64_t x = s;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  int64_t wo = 0;
  for (int i = 0; i < w; ++i) wo += wsum[i];
  int64_t run = toff[blockIdx.x] + wo + x - s;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    const int64_t j = base + i;
    if (j < n) out[j] = run;
    run += v[i];
  }
  if (base <= n - 1 && n - 1 < base + kScanPer) out[n] = run;
}

// Copies each entry into the band or the long-range matrix (keeping the row order), with
// the values rounded to V.
template <class V>
__global__ void split_scatter_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const double* __restrict__ val, int band, const int64_t* __restrict__ rpb,
                                     int32_t* __restrict__ cib, V* __restrict__ vb, const int64_t* __restrict__ rpl,
                                     int32_t* __restrict__ cil, V* __restrict__ vl) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = rpb[row], l = rpl[row];
    for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
      const int c = ci[e];
      const int64_t d = c > row ? c - row : row - c;
      if (d <= band) cib[b] = c, vb[b] = (V)val[e], ++b;
      else cil[l] = c, vl[l] = (V)val[e], ++l;
    }
  }
}

// Row lengths of the packed band part: each count rounded up to even.
__global__ void even_counts_kernel(int64_t n, const int32_t* __restrict__ cnt, int32_t* __restrict__ out) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x)
    out[row] = cnt[row] + (cnt[row] & 1);
}

// Packed band part: entry e of row i of A_band becomes (col - i, value bits) at rpk[i] + e;
// an odd row gets a trailing (0, 0.0f) entry.  One warp per row (coalesced copies).
__global__ void pack_band_kernel(int64_t n, int band, const int64_t* __restrict__ rpb,
                                 const int32_t* __restrict__ cib, const float* __restrict__ vb,
                                 const int64_t* __restrict__ rpk, int2* __restrict__ pk) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * blockDim.x / kWarp;
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kWarp; row < n; row += nw) {
    const int64_t b0 = rpb[row], b1 = rpb[row + 1], o = rpk[row];
    // a column outside [0, n) (malformed input) is clamped so the product's gathers stay in
    // its window; valid columns are unchanged
    const int64_t cmin = max((int64_t)0, row - band), cmax = min(n - 1, row + band);
    for (int64_t e = b0 + lane; e < b1; e += kWarp) {
      const int64_t c = min(max((int64_t)cib[e], cmin), cmax);
      pk[o + (e - b0)] = make_int2((int)(c - row), __float_as_int(vb[e]));
    }
    if (lane == 0 && ((b1 - b0) & 1)) pk[o + (b1 - b0)] = make_int2(0, 0);
  }
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

// Y[:, c0 : c0 + pc] = A X[:, c0 : c0 + pc] for a dense symmetric A (column-major, lda):
// column i of A is row i of A, so row i of Y is the dot product of A's column i (contiguous)
// with X.  A CTA of 8 warps owns 8 RB consecutive columns (RB per warp); X's rows stream
// through shared memory in slabs of kDenseSlab rows that all warps of the CTA share (row
// stride padded so a quarter-warp's 16-byte reads hit distinct banks); lane l of a warp takes
// slab rows l, l + 32, .. and reads A[c, i] coalesced across the warp, the four rows of a
// slab unrolled so their loads are in flight together.  Partial sums are reduced across the
// warp at the end in a fixed order.  A is read once per pass; X once per CTA.
constexpr int kDenseSlab = 128;
template <class T, int RB, int PC>
__global__ void __launch_bounds__(256) spmm_dense_kernel(int64_t n, const T* __restrict__ A, int64_t lda, int p,
                                                         int c0, const T* __restrict__ X, int ldx,
                                                         T* __restrict__ Y, int ldy) {
  // 16-byte reads at a row stride of 4 (mod 8) words (PC >= 16 bytes; narrower rows are read
  // element by element)
  constexpr int XS = sizeof(T) == 8 ? PC + 2 : PC + 4;
  constexpr int VE = 16 / sizeof(T);                    // elements per 16-byte read
  __shared__ __align__(16) T xs[kDenseSlab * XS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i0 = ((int64_t)blockIdx.x * 8 + warp) * RB;  // this warp's columns of A
  const int pc = min(PC, p - c0);
  T acc[RB][PC];
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int j = 0; j < PC; ++j) acc[r][j] = T(0);
  for (int64_t cs = 0; cs < n; cs += kDenseSlab) {
    __syncthreads();  // the previous slab is consumed
    for (int e = threadIdx.x; e < kDenseSlab * PC; e += blockDim.x) {
      const int cc = e / PC, j = e - cc * PC;
      const int64_t c = cs + cc;
      xs[cc * XS + j] = c < n && j < pc ? X[c * ldx + c0 + j] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kDenseSlab / 32; ++u) {
      const int cc = lane + 32 * u;
      const int64_t c = cs + cc;
      T a[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) a[r] = c < n && i0 + r < n ? A[c + (i0 + r) * lda] : T(0);
      T x[PC];
      if constexpr (PC % VE != 0) {
#pragma unroll
        for (int j = 0; j < PC; ++j) x[j] = xs[cc * XS + j];
      }
#pragma unroll
      for (int v = 0; v < (PC % VE == 0 ? PC / VE : 0); ++v) {
        if constexpr (sizeof(T) == 8) {
          const double2 t = *reinterpret_cast<const double2*>(xs + cc * XS + VE * v);
          x[VE * v] = t.x, x[VE * v + 1] = t.y;
        } else {
          const float4 t = *reinterpret_cast<const float4*>(xs + cc * XS + VE * v);
          x[VE * v] = t.x, x[VE * v + 1] = t.y, x[VE * v + 2] = t.z, x[VE * v + 3] = t.w;
        }
      }
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int j = 0; j < PC; ++j) acc[r][j] = fma(a[r], x[j], acc[r][j]);
    }
  }
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int j = 0; j < PC; ++j) acc[r][j] = warp_sum(acc[r][j]);
  if (lane == 0) {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int64_t i = i0 + r;
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
                     const T* X, int ldx, T* Y, int ldy, cudaStream_t st, int band, bool pure, int variant) {
  if (n <= 0 || p <= 0) return;
  if (p > 32) throw std::invalid_argument("spmm: p > 32");
  constexpr int VEC = 16 / sizeof(T);
  const bool vec_ok = (ldx % VEC == 0) && (ldy % VEC == 0) && ldx >= round_up(p, VEC) &&
                      !(reinterpret_cast<uintptr_t>(X) & 15) && !(reinterpret_cast<uintptr_t>(Y) & 15);
  // a kernel chosen by the caller (the solver's autotuner); kSpmmAuto: the default choice
  if (vec_ok && variant == kSpmmRows) {
    csr_rows_dispatch<T, V, false>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
    return;
  }
  if (variant == kSpmmBand) pure = false;
  if (variant == kSpmmVec) band = -1;
  if constexpr (std::is_same<T, double>::value) {
    if (vec_ok && variant == kSpmmAuto) {
      // FP64 is bound by the FMA rate: the row-parallel kernel keeps every lane busy
      csr_rows_dispatch<T, V, false>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
      return;
    }
  }
  if (vec_ok && band >= 0) {
    // two 16-byte vectors per lane halve the index work per gathered value
    const int lanes = (p + 2 * VEC - 1) / (2 * VEC);
    bool done = false;
    if constexpr (std::is_same<T, float>::value && sizeof(V) == 4) {
      if (pure) {
        // L lanes per non-zero, one 16-byte vector each: L = pow2 >= nvec
        const int nvec = (p + VEC - 1) / VEC;
        if (nvec <= 2) done = csr_window_launch<T, V, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, band, st);
        else if (nvec <= 4) done = csr_window_launch<T, V, 4>(n, rp, ci, val, p, X, ldx, Y, ldy, band, st);
        else done = csr_window_launch<T, V, 8>(n, rp, ci, val, p, X, ldx, Y, ldy, band, st);
      }
    }
    if (!done) {
      if (lanes <= 1) done = csr_band_launch<T, V, 1, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, band, st);
      else if (lanes <= 2) done = csr_band_launch<T, V, 2, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, band, st);
      else if (lanes <= 4) done = csr_band_launch<T, V, 4, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, band, st);
      else if (lanes <= 8) done = csr_band_launch<T, V, 8, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, band, st);
      else done = csr_band_launch<T, V, 16, 2>(n, rp, ci, val, p, X, ldx, Y, ldy, band, st);
    }
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
  // one pass over A for p <= 32 columns: RB x PC = 32 accumulators per thread
  const int threads = 256;
  // columns past p cost FMAs (the FP64 product is bound by the FP64 FMA rate): the
  // narrowest width that holds p
  const unsigned g32 = (unsigned)ceil_div(n, 32);
  if (p <= 2) {
    spmm_dense_kernel<T, 4, 2><<<g32, threads, 0, st>>>(n, A, lda, p, 0, X, ldx, Y, ldy);
  } else if (p <= 4) {
    spmm_dense_kernel<T, 4, 4><<<g32, threads, 0, st>>>(n, A, lda, p, 0, X, ldx, Y, ldy);
  } else if (p <= 8) {
    spmm_dense_kernel<T, 4, 8><<<g32, threads, 0, st>>>(n, A, lda, p, 0, X, ldx, Y, ldy);
  } else if (p <= 16) {
    spmm_dense_kernel<T, 2, 16><<<(unsigned)ceil_div(n, 16), threads, 0, st>>>(n, A, lda, p, 0, X, ldx, Y, ldy);
  } else {
    for (int c0 = 0; c0 < p; c0 += 32)
      spmm_dense_kernel<T, 1, 32><<<(unsigned)ceil_div(n, 8), threads, 0, st>>>(n, A, lda, p, c0, X, ldx, Y, ldy);
  }
  LB_LAUNCH_CHECK();
}

template void launch_spmm_csr<double, double>(int64_t, const int64_t*, const int32_t*, const double*,
                                              int, const double*, int, double*, int, cudaStream_t, int, bool, int);
template void launch_spmm_csr<float, float>(int64_t, const int64_t*, const int32_t*, const float*,
                                            int, const float*, int, float*, int, cudaStream_t, int, bool, int);

template <class T, class V>
void launch_spmm_csr_add(int64_t n, const int64_t* rp, const int32_t* ci, const V* val, int p, const T* X, int ldx,
                         T* Y, int ldy, cudaStream_t st) {
  if (n <= 0 || p <= 0) return;
  if (p > 32) throw std::invalid_argument("spmm: p > 32");
  constexpr int VEC = 16 / sizeof(T);
  const bool vec_ok = (ldx % VEC == 0) && (ldy % VEC == 0) && ldx >= round_up(p, VEC) &&
                      !(reinterpret_cast<uintptr_t>(X) & 15) && !(reinterpret_cast<uintptr_t>(Y) & 15);
  if (!vec_ok) throw std::invalid_argument("spmm add: blocks must be 16-byte aligned");
  csr_rows_dispatch<T, V, true>(n, rp, ci, val, p, X, ldx, Y, ldy, st);
}
template void launch_spmm_csr_add<float, float>(int64_t, const int64_t*, const int32_t*, const float*, int,
                                                const float*, int, float*, int, cudaStream_t);

void split_csr_count(int64_t n, const int64_t* rp, const int32_t* ci, int band, int32_t* cb, int32_t* cl,
                     cudaStream_t st) {
  if (n <= 0) return;
  split_count_kernel<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 4864), 256, 0, st>>>(n, rp, ci, band, cb, cl);
  LB_LAUNCH_CHECK();
}

int64_t split_scan_scratch(int64_t n) { return ceil_div(std::max<int64_t>(n, 1), kScanTile); }

void split_csr_rowptr(int64_t n, const int32_t* cnt, int64_t* out, int64_t* scratch, cudaStream_t st) {
  if (n <= 0) {
    LB_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
    return;
  }
  const int64_t ntiles = ceil_div(n, kScanTile);
  scan_tile_sums_kernel<<<(unsigned)ntiles, kScanThreads, 0, st>>>(n, cnt, scratch);
  LB_LAUNCH_CHECK();
  scan_tile_offsets_kernel<<<1, 1024, 0, st>>>(ntiles, scratch);
  LB_LAUNCH_CHECK();
  scan_write_kernel<<<(unsigned)ntiles, kScanThreads, 0, st>>>(n, cnt, scratch, out);
  LB_LAUNCH_CHECK();
}

template <class V>
void split_csr_scatter(int64_t n, const int64_t* rp, const int32_t* ci, const double* val, int band,
                       const int64_t* rpb, int32_t* cib, V* vb, const int64_t* rpl, int32_t* cil, V* vl,
                       cudaStream_t st) {
  if (n <= 0) return;
  split_scatter_kernel<V><<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 4864), 256, 0, st>>>(
      n, rp, ci, val, band, rpb, cib, vb, rpl, cil, vl);
  LB_LAUNCH_CHECK();
}
template void split_csr_scatter<float>(int64_t, const int64_t*, const int32_t*, const double*, int, const int64_t*,
                                       int32_t*, float*, const int64_t*, int32_t*, float*, cudaStream_t);

void split_even_counts(int64_t n, const int32_t* cnt, int32_t* out, cudaStream_t st) {
  if (n <= 0) return;
  even_counts_kernel<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 4864), 256, 0, st>>>(n, cnt, out);
  LB_LAUNCH_CHECK();
}

void split_pack_band(int64_t n, int band, const int64_t* rpb, const int32_t* cib, const float* vb,
                     const int64_t* rpk, int2* pk, cudaStream_t st) {
  if (n <= 0) return;
  pack_band_kernel<<<(unsigned)std::min<int64_t>(ceil_div(n, 8), 152 * 32), 256, 0, st>>>(n, band, rpb, cib, vb,
                                                                                          rpk, pk);
  LB_LAUNCH_CHECK();
}

bool launch_spmm_band_packed(int64_t n, const int64_t* rpk, const int2* pk, int p, const float* X, int ldx,
                             float* Y, int ldy, int band, cudaStream_t st) {
  if (n <= 0 || p <= 0) return true;
  if (p > 32) throw std::invalid_argument("spmm: p > 32");
  const bool vec_ok = (ldx % 4 == 0) && (ldy % 4 == 0) && ldx >= round_up(p, 4) &&
                      !(reinterpret_cast<uintptr_t>(X) & 15) && !(reinterpret_cast<uintptr_t>(Y) & 15) &&
                      !(reinterpret_cast<uintptr_t>(pk) & 15);
  if (!vec_ok) return false;
  // L lanes per gathered row, one 16-byte vector each: L = pow2 >= nvec
  const int nvec = (p + 3) / 4;
  if (nvec <= 2) return band_packed_launch<2>(n, rpk, pk, p, X, ldx, Y, ldy, band, st);
  if (nvec <= 4) return band_packed_launch<4>(n, rpk, pk, p, X, ldx, Y, ldy, band, st);
  return band_packed_launch<8>(n, rpk, pk, p, X, ldx, Y, ldy, band, st);
}

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

void launch_split_df(int64_t count, const double* src, float2* dst, cudaStream_t st) {
  if (count <= 0) return;
  split_df_kernel<<<(unsigned)std::min<int64_t>(ceil_div(count, 256), 152 * 16), 256, 0, st>>>(count, src, dst);
  LB_LAUNCH_CHECK();
}

void launch_spmm_csr_df(int64_t n, const int64_t* rp, const int32_t* ci, const float2* vs, int p,
                        const float2* Xs, int ldx, double* Y, int ldy, cudaStream_t st) {
  if (n <= 0 || p <= 0) return;
  if (p > 32 || (ldx & 1) || (ldy & 1)) throw std::invalid_argument("spmm df: p <= 32 and even row strides required");
  const int nvec = (p + 1) / 2;  // 16-byte vectors (2 columns) per row
  if (nvec <= 2) csr_df_launch<1, 2>(n, rp, ci, vs, p, Xs, ldx, Y, ldy, st);
  else if (nvec <= 4) csr_df_launch<2, 2>(n, rp, ci, vs, p, Xs, ldx, Y, ldy, st);
  else if (nvec <= 6) csr_df_launch<2, 3>(n, rp, ci, vs, p, Xs, ldx, Y, ldy, st);
  else if (nvec <= 8) csr_df_launch<4, 2>(n, rp, ci, vs, p, Xs, ldx, Y, ldy, st);
  else if (nvec <= 12) csr_df_launch<4, 3>(n, rp, ci, vs, p, Xs, ldx, Y, ldy, st);
  else csr_df_launch<8, 2>(n, rp, ci, vs, p, Xs, ldx, Y, ldy, st);
}

}  // namespace lobpcg
