// Tall-skinny block kernels of Algorithm 1: Gram / projected matrices (a = V^T AV,
// Y^T W, W^T W), basis updates (X = V u_x, P = V u_p, W - Y C, W L^{-T}), the fused
// residual-norm epilogue, the diagonal preconditioner, layout conversions and the
// seeded Gaussian initial block.
//
// Blocks are row-major (row i of an n x p block is contiguous), so a CTA stages a tile
// of R consecutive rows of every operand into shared memory with coalesced loads and
// then works only from shared memory.
#include <algorithm>

#include "common.cuh"
#include "dfloat.cuh"

namespace lobpcg {
namespace {

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms;
}

// Copy rows [r0, r0 + R) of the logical block `c` into s[r][0..w) (row stride sld),
// zero-filling rows at or past `rend`.
template <class T, int R>
__device__ __forceinline__ void stage_rows(const Cols<T>& c, int64_t r0, int64_t rend, T* s, int sld) {
  int off = 0;
  for (int g = 0; g < c.nseg; ++g) {
    const int w = c.w[g];
    const T* p = c.p[g];
    const int ld = c.ld[g];
    for (int e = threadIdx.x; e < R * w; e += blockDim.x) {
      const int r = e / w, j = e - r * w;
      const int64_t row = r0 + r;
      s[r * sld + off + j] = row < rend ? p[row * ld + j] : T(0);
    }
    off += w;
  }
}

// ---------------------------------------------------------------- Gram partials
// Each thread owns a TI x TJ tile of C = A^T B (upper: only tiles that reach i <= j);
// `groups` thread groups split the rows of every staged tile; group sums are combined
// in a fixed order, then one FP64 partial per CTA is written.
template <class T, int TI, int TJ, int R>
__global__ void __launch_bounds__(512) gram_kernel(int64_t n, Cols<T> A, Cols<T> B, int upper,
                                                   int ntiles, int groups,
                                                   double* __restrict__ part, int64_t rows_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ short tile_i[kMaxS * kMaxS / 16], tile_j[kMaxS * kMaxS / 16];
  const int pa = A.width(), pb = B.width();
  const int nti = (pa + TI - 1) / TI, ntj = (pb + TJ - 1) / TJ;
  const int pa_pad = nti * TI, pb_pad = ntj * TJ;
  T* sA = reinterpret_cast<T*>(smem_raw);
  T* sB = sA + R * pa_pad;
  if (threadIdx.x == 0) {
    int idx = 0;
    for (int tj = 0; tj < ntj; ++tj)
      for (int ti = 0; ti < nti; ++ti)
        if (!upper || ti * TI <= tj * TJ + TJ - 1) tile_i[idx] = (short)ti, tile_j[idx] = (short)tj, ++idx;
  }
  const int t = threadIdx.x % ntiles, grp = threadIdx.x / ntiles;
  const bool active = grp < groups;
  // zero the padding columns once
  for (int e = threadIdx.x; e < R * pa_pad; e += blockDim.x)
    if (e % pa_pad >= pa) sA[e] = T(0);
  for (int e = threadIdx.x; e < R * pb_pad; e += blockDim.x)
    if (e % pb_pad >= pb) sB[e] = T(0);
  __syncthreads();
  const int my_ti = tile_i[t], my_tj = tile_j[t];

  T acc[TI][TJ];
#pragma unroll
  for (int i = 0; i < TI; ++i)
#pragma unroll
    for (int j = 0; j < TJ; ++j) acc[i][j] = T(0);

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = min(n, r_begin + rows_per_cta);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += R) {
    __syncthreads();
    stage_rows<T, R>(A, r0, r_end, sA, pa_pad);
    stage_rows<T, R>(B, r0, r_end, sB, pb_pad);
    __syncthreads();
    if (active) {
      for (int r = grp; r < R; r += groups) {
        T a[TI], b[TJ];
#pragma unroll
        for (int i = 0; i < TI; ++i) a[i] = sA[r * pa_pad + my_ti * TI + i];
#pragma unroll
        for (int j = 0; j < TJ; ++j) b[j] = sB[r * pb_pad + my_tj * TJ + j];
#pragma unroll
        for (int i = 0; i < TI; ++i)
#pragma unroll
          for (int j = 0; j < TJ; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    }
  }
  __syncthreads();
  // combine the groups in a fixed order through shared memory (FP64)
  double* scratch = reinterpret_cast<double*>(smem_raw);
  constexpr int per = TI * TJ;
  if (active) {
#pragma unroll
    for (int i = 0; i < TI; ++i)
#pragma unroll
      for (int j = 0; j < TJ; ++j) scratch[(grp * ntiles + t) * per + i * TJ + j] = (double)acc[i][j];
  }
  __syncthreads();
  double* out = part + (int64_t)blockIdx.x * pa * pb;
  for (int e = threadIdx.x; e < ntiles * per; e += blockDim.x) {
    const int tt = e / per, ij = e % per;
    double s = 0.0;
    for (int g = 0; g < groups; ++g) s += scratch[(g * ntiles + tt) * per + ij];
    const int i = tile_i[tt] * TI + ij / TJ, j = tile_j[tt] * TJ + ij % TJ;
    if (i < pa && j < pb && (!upper || i <= j)) out[i + j * pa] = s;
  }
}

// out[e] = sum over g in order of part[g][e].  The loads of eight partials are issued before
// their adds (which stay in order), so the chain waits on memory once per eight.
__global__ void reduce_kernel(const double* __restrict__ part, int nparts, int count,
                              double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    int g = 0;
    for (; g + 8 <= nparts; g += 8) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldg(part + (int64_t)(g + u) * count + e);
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; g < nparts; ++g) s += part[(int64_t)g * count + e];
    out[e] = s;
  }
}

// ---------------------------------------------------------------- block update
// out_t = base_t + alpha * in_t * U.  Thread (rr, cj) computes CJ consecutive output
// columns of rows rr, rr + rows_per_pass, ... of the staged tile.
template <class T, int CJ, int R>
__global__ void __launch_bounds__(256) update_kernel(int64_t n, UpdateJob<T> job,
                                                     const double* __restrict__ U, int s, int q,
                                                     double alpha, const double* __restrict__ lam,
                                                     double* __restrict__ norm_part,
                                                     int64_t rows_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int qpad = (q + CJ - 1) / CJ * CJ;
  T* sU = reinterpret_cast<T*>(smem_raw);  // s x qpad, row-major
  T* sIn = sU + s * qpad;                   // nprod x R x s
  double* sNorm = reinterpret_cast<double*>(sIn + job.nprod * R * s);  // [rows_per_pass][2*qpad]
  for (int e = threadIdx.x; e < s * qpad; e += blockDim.x) {
    const int l = e / qpad, j = e % qpad;
    sU[e] = j < q ? (T)U[l + j * s] : T(0);
  }
  const int tpr = qpad / CJ;
  const int rows_per_pass = blockDim.x / tpr;
  const int rr = threadIdx.x / tpr, cj = threadIdx.x % tpr;
  const bool active = rr < rows_per_pass;
  double nsum[CJ], nmax[CJ];
#pragma unroll
  for (int j = 0; j < CJ; ++j) nsum[j] = 0.0, nmax[j] = 0.0;

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = min(n, r_begin + rows_per_cta);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += R) {
    __syncthreads();
    for (int t = 0; t < job.nprod; ++t) stage_rows<T, R>(job.in[t], r0, r_end, sIn + t * R * s, s);
    __syncthreads();
    if (!active) continue;
    for (int r = rr; r < R; r += rows_per_pass) {
      const int64_t row = r0 + r;
      if (row >= r_end) break;
      T res[2][CJ];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        if (t >= job.nprod) break;
        T acc[CJ];
#pragma unroll
        for (int j = 0; j < CJ; ++j) acc[j] = T(0);
        const T* x = sIn + (t * R + r) * s;
        for (int l = 0; l < s; ++l) {
          const T xv = x[l];
#pragma unroll
          for (int j = 0; j < CJ; ++j) acc[j] = fma(xv, sU[l * qpad + cj * CJ + j], acc[j]);
        }
        T* o = job.out[t] + row * job.ld_out[t];
        const T* b = job.base[t] ? job.base[t] + row * job.ld_base[t] : nullptr;
#pragma unroll
        for (int j = 0; j < CJ; ++j) {
          const int col = cj * CJ + j;
          T v = (T)alpha * acc[j];
          if (b && col < q) v = b[col] + v;
          res[t][j] = v;
          if (col < q) o[col] = v;
        }
      }
      if (norm_part) {
#pragma unroll
        for (int j = 0; j < CJ; ++j) {
          const int col = cj * CJ + j;
          if (col < q) {
            const double rij = (double)fma(-(T)lam[col], res[0][j], res[1][j]);  // AX - lam X, one rounding
            nsum[j] = fma(rij, rij, nsum[j]);
            nmax[j] = fmax(nmax[j], fabs(rij));
          }
        }
      }
    }
  }
  if (!norm_part) return;
  __syncthreads();
  if (active) {
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
      sNorm[rr * 2 * qpad + cj * CJ + j] = nsum[j];
      sNorm[rr * 2 * qpad + qpad + cj * CJ + j] = nmax[j];
    }
  }
  __syncthreads();
  for (int col = threadIdx.x; col < q; col += blockDim.x) {
    double s2 = 0.0, mx = 0.0;
    for (int g = 0; g < rows_per_pass; ++g) {
      s2 += sNorm[g * 2 * qpad + col];
      mx = fmax(mx, sNorm[g * 2 * qpad + qpad + col]);
    }
    norm_part[(int64_t)blockIdx.x * 2 * q + col] = s2;
    norm_part[(int64_t)blockIdx.x * 2 * q + q + col] = mx;
  }
}

// ---------------------------------------------------------- block update, double-float
// The FP64 update out_t = base_t + alpha * in_t * U formed on the FP32 pipes (dfloat.cuh):
// alpha U is split once per CTA into (hi, lo) pairs, each staged row element is split on
// its way into shared memory, every output element is a compensated double-float sum of
// its s products plus the base term, widened to FP64 once.  Thread layout, staging and
// the residual-norm epilogue (in FP64) are those of update_kernel.
template <int R>
__device__ __forceinline__ void stage_rows_split(const Cols<double>& c, int64_t r0, int64_t rend, float2* s, int sld) {
  int off = 0;
  for (int g = 0; g < c.nseg; ++g) {
    const int w = c.w[g];
    const double* p = c.p[g];
    const int ld = c.ld[g];
    for (int e = threadIdx.x; e < R * w; e += blockDim.x) {
      const int r = e / w, j = e - r * w;
      const int64_t row = r0 + r;
      s[r * sld + off + j] = row < rend ? df_split(p[row * ld + j]) : make_float2(0.f, 0.f);
    }
    off += w;
  }
}

template <int CJ, int R>
__global__ void __launch_bounds__(256, 3) update_df_kernel(int64_t n, UpdateJob<double> job,
                                                        const double* __restrict__ U, int s, int q,
                                                        double alpha, const double* __restrict__ lam,
                                                        double* __restrict__ norm_part, int64_t rows_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int qpad = (q + CJ - 1) / CJ * CJ;
  float2* sU = reinterpret_cast<float2*>(smem_raw);  // s x qpad, row-major: alpha U split
  float2* sIn = sU + s * qpad;                       // nprod x R x s
  double* sNorm = reinterpret_cast<double*>(sIn + job.nprod * R * s);  // [rows_per_pass][2*qpad]
  const bool unit = job.unit_base != 0;
  for (int e = threadIdx.x; e < s * qpad; e += blockDim.x) {
    const int l = e / qpad, j = e % qpad;
    sU[e] = j < q ? df_split(alpha * U[l + j * s] - (unit && l == j ? 1.0 : 0.0)) : make_float2(0.f, 0.f);
  }
  const int tpr = qpad / CJ;
  const int rows_per_pass = blockDim.x / tpr;
  const int rr = threadIdx.x / tpr, cj = threadIdx.x % tpr;
  const bool active = rr < rows_per_pass;
  double nsum[CJ], nmax[CJ];
#pragma unroll
  for (int j = 0; j < CJ; ++j) nsum[j] = 0.0, nmax[j] = 0.0;

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = min(n, r_begin + rows_per_cta);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += R) {
    __syncthreads();
    for (int t = 0; t < job.nprod; ++t) stage_rows_split<R>(job.in[t], r0, r_end, sIn + t * R * s, s);
    __syncthreads();
    if (!active) continue;
    for (int r = rr; r < R; r += rows_per_pass) {
      const int64_t row = r0 + r;
      if (row >= r_end) break;
      double res[2][CJ];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        if (t >= job.nprod) break;
        DfAcc acc[CJ];
#pragma unroll
        for (int j = 0; j < CJ; ++j) df_zero(acc[j]);
        const float2* x = sIn + (t * R + r) * s;
        for (int l = 0; l < s; ++l) {
          const float2 xv = x[l];
#pragma unroll
          for (int j = 0; j < CJ; ++j) df_fma(acc[j], xv, sU[l * qpad + cj * CJ + j]);
        }
        double* o = job.out[t] + row * job.ld_out[t];
        // the base is added in FP64 (one add per output): a base re-rounded to a float
        // pair would lose its bits past 2^-47 (e.g. the part of W along Y in W - Y C)
        const double* b = unit ? job.in[0].p[0] + row * job.in[0].ld[0]
                               : (job.base[t] ? job.base[t] + row * job.ld_base[t] : nullptr);
#pragma unroll
        for (int j = 0; j < CJ; ++j) {
          const int col = cj * CJ + j;
          double v = df_value(acc[j]);
          if (b && col < q) v = b[col] + v;
          res[t][j] = v;
          if (col < q) o[col] = v;
        }
      }
      if (norm_part) {
#pragma unroll
        for (int j = 0; j < CJ; ++j) {
          const int col = cj * CJ + j;
          if (col < q) {
            const double rij = fma(-lam[col], res[0][j], res[1][j]);  // AX - lam X, one rounding
            nsum[j] = fma(rij, rij, nsum[j]);
            nmax[j] = fmax(nmax[j], fabs(rij));
          }
        }
      }
    }
  }
  if (!norm_part) return;
  __syncthreads();
  if (active) {
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
      sNorm[rr * 2 * qpad + cj * CJ + j] = nsum[j];
      sNorm[rr * 2 * qpad + qpad + cj * CJ + j] = nmax[j];
    }
  }
  __syncthreads();
  for (int col = threadIdx.x; col < q; col += blockDim.x) {
    double s2 = 0.0, mx = 0.0;
    for (int g = 0; g < rows_per_pass; ++g) {
      s2 += sNorm[g * 2 * qpad + col];
      mx = fmax(mx, sNorm[g * 2 * qpad + qpad + col]);
    }
    norm_part[(int64_t)blockIdx.x * 2 * q + col] = s2;
    norm_part[(int64_t)blockIdx.x * 2 * q + q + col] = mx;
  }
}

// 16-byte cp.async global -> shared; zero-filled (nothing read) when !valid
__device__ __forceinline__ void cp_async16_df(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0));
}

// update_df_kernel with the next slab of rows in flight while the current one is computed.
// Slab rows (FP64, each segment padded to an even width so every row piece is whole 16-byte
// units) go to `raw` by cp.async; they are split into float pairs (sIn) once they land, and
// the copies of the following slab start as soon as raw is free, so the global-load latency
// overlaps the double-float products.  R = rows per slab = rows of one thread pass, so every
// thread has a row.  Needs 16-byte aligned segments and even row strides (checked by the
// launcher).  Arithmetic, order of the products and the FP64 epilogue as in update_df_kernel.
template <int CJ>
__global__ void __launch_bounds__(256, 2) update_df_async_kernel(int64_t n, UpdateJob<double> job,
                                                              const double* __restrict__ U, int s, int q,
                                                              double alpha, const double* __restrict__ lam,
                                                              double* __restrict__ norm_part, int64_t rows_per_cta,
                                                              int R, int sraw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int qpad = (q + CJ - 1) / CJ * CJ;
  const int nprod = job.nprod;
  float2* sU = reinterpret_cast<float2*>(smem_raw);    // s x qpad, row-major: alpha U split
  float2* sIn = sU + s * qpad;                         // nprod x R x s
  double* raw = reinterpret_cast<double*>(sIn + (nprod * R * s + 1) / 2 * 2);  // nprod x R x sraw, 16-byte aligned
  // column l -> offset in a raw row, past the raw slab (or the norm partials if larger)
  int* lraw = reinterpret_cast<int*>(raw + max(nprod * R * sraw, norm_part ? R * 2 * qpad : 0));
  const bool unit = job.unit_base != 0;
  for (int e = threadIdx.x; e < s * qpad; e += blockDim.x) {
    const int l = e / qpad, j = e % qpad;
    sU[e] = j < q ? df_split(alpha * U[l + j * s] - (unit && l == j ? 1.0 : 0.0)) : make_float2(0.f, 0.f);
  }
  if (threadIdx.x == 0) {
    int l = 0, roff = 0;
    for (int g = 0; g < job.in[0].nseg; ++g) {
      const int w = job.in[0].w[g];
      for (int j = 0; j < w; ++j) lraw[l++] = roff + j;
      roff += w + (w & 1);
    }
  }
  const int tpr = qpad / CJ;
  const int rows_per_pass = blockDim.x / tpr;
  const int rr = threadIdx.x / tpr, cj = threadIdx.x % tpr;
  const bool active = rr < rows_per_pass && rr < R;
  double nsum[CJ], nmax[CJ];
#pragma unroll
  for (int j = 0; j < CJ; ++j) nsum[j] = 0.0, nmax[j] = 0.0;

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = min(n, r_begin + rows_per_cta);
  auto issue = [&](int64_t r0) {
    for (int t = 0; t < nprod; ++t) {
      const Cols<double>& c = job.in[t];
      int roff = 0;
      for (int g = 0; g < c.nseg; ++g) {
        const int w = c.w[g], units = (w + 1) / 2, ld = c.ld[g];
        const double* p = c.p[g];
        for (int e = threadIdx.x; e < R * units; e += blockDim.x) {
          const int r = e / units, u = e - r * units;
          const int64_t row = r0 + r;
          const bool ok = row < r_end;
          cp_async16_df(raw + (t * R + r) * sraw + roff + 2 * u, p + (ok ? row : r0) * ld + 2 * u, ok);
        }
        roff += 2 * units;
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };
  if (r_begin < r_end) issue(r_begin);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += R) {
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();  // the slab landed (every thread's copies) and the previous slab is consumed
    for (int t = 0; t < nprod; ++t)
      for (int e = threadIdx.x; e < R * s; e += blockDim.x) {
        const int r = e / s, l = e - r * s;
        sIn[(t * R + r) * s + l] = r0 + r < r_end ? df_split(raw[(t * R + r) * sraw + lraw[l]]) : make_float2(0.f, 0.f);
      }
    __syncthreads();  // raw is free: the next slab's copies overlap this slab's products
    if (r0 + R < r_end) issue(r0 + R);
    if (!active) continue;
    const int r = rr;
    const int64_t row = r0 + r;
    if (row >= r_end) continue;
    double res[2][CJ];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (t >= nprod) break;
      DfAcc acc[CJ];
#pragma unroll
      for (int j = 0; j < CJ; ++j) df_zero(acc[j]);
      const float2* x = sIn + (t * R + r) * s;
      for (int l = 0; l < s; ++l) {
        const float2 xv = x[l];
#pragma unroll
        for (int j = 0; j < CJ; ++j) df_fma(acc[j], xv, sU[l * qpad + cj * CJ + j]);
      }
      double* o = job.out[t] + row * job.ld_out[t];
      // the base is added in FP64 (one add per output), as in update_df_kernel
      const double* b = unit ? job.in[0].p[0] + row * job.in[0].ld[0]
                             : (job.base[t] ? job.base[t] + row * job.ld_base[t] : nullptr);
#pragma unroll
      for (int j = 0; j < CJ; ++j) {
        const int col = cj * CJ + j;
        double v = df_value(acc[j]);
        if (b && col < q) v = b[col] + v;
        res[t][j] = v;
        if (col < q) o[col] = v;
      }
    }
    if (norm_part) {
#pragma unroll
      for (int j = 0; j < CJ; ++j) {
        const int col = cj * CJ + j;
        if (col < q) {
          const double rij = fma(-lam[col], res[0][j], res[1][j]);  // AX - lam X, one rounding
          nsum[j] = fma(rij, rij, nsum[j]);
          nmax[j] = fmax(nmax[j], fabs(rij));
        }
      }
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::);
  if (!norm_part) return;
  __syncthreads();
  double* sNorm = raw;  // [rows_per_pass][2 * qpad], in the idle slab buffer
  if (active) {
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
      sNorm[rr * 2 * qpad + cj * CJ + j] = nsum[j];
      sNorm[rr * 2 * qpad + qpad + cj * CJ + j] = nmax[j];
    }
  }
  __syncthreads();
  for (int col = threadIdx.x; col < q; col += blockDim.x) {
    double s2 = 0.0, mx = 0.0;
    for (int g = 0; g < min(rows_per_pass, R); ++g) {
      s2 += sNorm[g * 2 * qpad + col];
      mx = fmax(mx, sNorm[g * 2 * qpad + qpad + col]);
    }
    norm_part[(int64_t)blockIdx.x * 2 * q + col] = s2;
    norm_part[(int64_t)blockIdx.x * 2 * q + q + col] = mx;
  }
}

template <class T>
__global__ void precond_kernel(int64_t n, const T* __restrict__ X, const T* __restrict__ AX, int ld,
                               const double* __restrict__ lam, int c0, int a,
                               const double* __restrict__ diag, int precond, T* __restrict__ W,
                               int ldw, const double* __restrict__ diagB, double floor) {
  // a 2-D walk (row, column) without 64-bit divisions: a warp covers 32 / a rows
  const int a_pad = a <= 1 ? 1 : (a <= 2 ? 2 : (a <= 4 ? 4 : (a <= 8 ? 8 : (a <= 16 ? 16 : 32))));
  const int rows_per_block = blockDim.x / a_pad;
  const int j = threadIdx.x % a_pad;
  const int rl = threadIdx.x / a_pad;
  if (j >= a) return;
  const double l = lam[c0 + j];
  const T fl = (T)fmax(1e-8 * fmax(1.0, fabs(l)), floor);  // reading R6, or the damping floor
  for (int64_t i = (int64_t)blockIdx.x * rows_per_block + rl; i < n; i += (int64_t)gridDim.x * rows_per_block) {
    const T r = AX[i * ld + c0 + j] - (T)l * X[i * ld + c0 + j];
    T w = r;
    if (precond == 1) {
      // computed in the block's precision: FP64 path exact, FP32 path keeps the FP64 units free
      // generalised problem (diagB): X holds B X and the denominator is d_A - theta d_B
      T delta = diagB ? (T)(diag[i] - l * diagB[i]) : (T)diag[i] - (T)l;
      if (fabs(delta) < fl) delta = delta >= T(0) ? fl : -fl;
      w = r / delta;
    }
    W[i * ldw + j] = w;
  }
}

template <class Tin, class Tout>
__global__ void col_to_rows_kernel(int64_t n, int p, const Tin* __restrict__ src,
                                   Tout* __restrict__ dst, int ld) {
  const int64_t total = n * p;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / n);
    const int64_t i = e - (int64_t)j * n;
    dst[i * ld + j] = (Tout)src[e];
  }
}

template <class Tin, class Tout>
__global__ void rows_to_col_kernel(int64_t n, int p, const Tin* __restrict__ src, int ld,
                                   Tout* __restrict__ dst) {
  const int64_t total = n * p;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / n);
    const int64_t i = e - (int64_t)j * n;
    dst[e] = (Tout)src[i * ld + j];
  }
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter-based generator.
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint2 key) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, ctr.x), lo0 = M0 * ctr.x;
    const uint32_t hi1 = __umulhi(M1, ctr.z), lo1 = M1 * ctr.z;
    ctr = make_uint4(hi1 ^ ctr.y ^ key.x, lo1, hi0 ^ ctr.w ^ key.y, lo0);
    key.x += W0;
    key.y += W1;
  }
  return ctr;
}

__global__ void gaussian_kernel(int64_t total, uint64_t seed, double* __restrict__ dst) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)e, (uint32_t)(e >> 32), 0x5eedu, 0u), key);
    const uint64_t a = ((uint64_t)r.x << 21) ^ (uint64_t)r.y;  // 53 random bits
    const uint64_t b = ((uint64_t)r.z << 21) ^ (uint64_t)r.w;
    const double u1 = ((double)(a & ((1ull << 53) - 1)) + 1.0) * (1.0 / 9007199254740992.0);  // (0, 1]
    const double u2 = (double)(b & ((1ull << 53) - 1)) * (1.0 / 9007199254740992.0);          // [0, 1)
    dst[e] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}

__global__ void to_float_kernel(int64_t count, const double* __restrict__ src, float* __restrict__ dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (float)src[e];
}

__global__ void finite_kernel(int64_t count, const double* __restrict__ src, int* flag) {
  bool ok = true;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    ok &= isfinite(src[e]);
  if (!__all_sync(0xffffffffu, ok) && (threadIdx.x & 31) == 0) atomicExch(flag, 0);
}

unsigned grid_for(int64_t total, int threads) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, threads), (int64_t)num_sms() * 8));
}

int count_tiles(int pa, int pb, int TI, int TJ, bool upper) {
  const int nti = (pa + TI - 1) / TI, ntj = (pb + TJ - 1) / TJ;
  int ntiles = 0;
  for (int tj = 0; tj < ntj; ++tj)
    for (int ti = 0; ti < nti; ++ti)
      if (!upper || ti * TI <= tj * TJ + TJ - 1) ++ntiles;
  return ntiles;
}

template <class T, int TI, int TJ, int R>
int gram_launch(int64_t n, const Cols<T>& a, const Cols<T>& b, bool upper, double* part,
                int max_ctas, cudaStream_t st) {
  const int pa = a.width(), pb = b.width();
  const int pa_pad = round_up(pa, TI), pb_pad = round_up(pb, TJ);
  const int ntiles = count_tiles(pa, pb, TI, TJ, upper);
  const int threads = 512;
  constexpr int per = TI * TJ;
  const int groups = std::max(1, std::min(threads / ntiles, (int)(65536 / ((size_t)ntiles * per * sizeof(double)))));
  const size_t stage = (size_t)R * (pa_pad + pb_pad) * sizeof(T);
  const size_t red = (size_t)groups * ntiles * per * sizeof(double);
  const size_t smem = std::max(stage, red);
  // set once per process; function-local statics initialise thread-safely
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(gram_kernel<T, TI, TJ, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    return true;
  }();
  (void)attr;
  // rows per CTA: multiple of R, at most max_ctas CTAs
  int64_t ctas = std::min<int64_t>(max_ctas, ceil_div(n, R));
  if (ctas < 1) ctas = 1;
  const int64_t rpc = (ceil_div(n, ctas) + R - 1) / R * R;
  ctas = std::max<int64_t>(1, ceil_div(n, rpc));
  gram_kernel<T, TI, TJ, R><<<(unsigned)ctas, threads, smem, st>>>(n, a, b, upper ? 1 : 0, ntiles, groups, part, rpc);
  LB_LAUNCH_CHECK();
  return (int)ctas;
}

}  // namespace

template <class T>
int gram_partials(int64_t n, const Cols<T>& a, const Cols<T>& b, bool upper, double* part,
                  int max_ctas, cudaStream_t st) {
  const int pa = a.width(), pb = b.width();
  if (pa > kMaxS || pb > kMaxS) throw std::invalid_argument("gram: width > 96");
  if (const int parts = gram_partials_pipe<T>(n, a, b, upper, part, max_ctas, st)) return parts;
  if (count_tiles(pa, pb, 4, 4, upper) <= 512)
    return gram_launch<T, 4, 4, 32>(n, a, b, upper, part, max_ctas, st);
  return gram_launch<T, 8, 8, 32>(n, a, b, upper, part, max_ctas, st);
}

void reduce_partials(const double* part, int nparts, int count, double* out, cudaStream_t st) {
  if (count <= 0) return;
  reduce_kernel<<<(count + 255) / 256, 256, 0, st>>>(part, nparts, count, out);
  LB_LAUNCH_CHECK();
}

template <class T>
int launch_update(int64_t n, const UpdateJob<T>& job, const double* U, int s, int q, double alpha,
                  const double* lam, double* norm_part, int max_ctas, cudaStream_t st) {
  if (q <= 0 || n <= 0) return 0;
  if (const int parts = launch_update_pipe<T>(n, job, U, s, q, alpha, lam, norm_part, max_ctas, st)) return parts;
  constexpr int CJ = 4, R = 32;
  const int qpad = round_up(q, CJ);
  const int threads = 256;
  const int tpr = qpad / CJ;
  const int rows_per_pass = threads / tpr;
  const size_t smem = (size_t)s * qpad * sizeof(T) + (size_t)job.nprod * R * s * sizeof(T) +
                      (norm_part ? (size_t)rows_per_pass * 2 * qpad * sizeof(double) : 0) + 16;
  // set once per process; function-local statics initialise thread-safely
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(update_kernel<T, CJ, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    return true;
  }();
  (void)attr;
  int64_t ctas = std::min<int64_t>(max_ctas, ceil_div(n, R));
  if (ctas < 1) ctas = 1;
  const int64_t rpc = (ceil_div(n, ctas) + R - 1) / R * R;
  ctas = std::max<int64_t>(1, ceil_div(n, rpc));
  update_kernel<T, CJ, R><<<(unsigned)ctas, threads, smem, st>>>(n, job, U, s, q, alpha, lam, norm_part, rpc);
  LB_LAUNCH_CHECK();
  return (int)ctas;
}

// The asynchronous-staging form of the double-float update when the layout allows it
// (segments 16-byte aligned, even row strides); 0 otherwise.
int launch_update_df_async(int64_t n, const UpdateJob<double>& job, const double* U, int s, int q, double alpha,
                           const double* lam, double* norm_part, int max_ctas, cudaStream_t st) {
  constexpr int CJ = 4;
  int sraw = 0;
  for (int t = 0; t < job.nprod; ++t) {
    int sr = 0;
    for (int g = 0; g < job.in[t].nseg; ++g) {
      if ((reinterpret_cast<uintptr_t>(job.in[t].p[g]) & 15) || (job.in[t].ld[g] & 1)) return 0;
      sr += job.in[t].w[g] + (job.in[t].w[g] & 1);
      if (t > 0 && job.in[t].w[g] != job.in[0].w[g]) return 0;
    }
    if (t > 0 && job.in[t].nseg != job.in[0].nseg) return 0;
    sraw = sr;
  }
  const int qpad = round_up(q, CJ);
  const int threads = 256;
  const int tpr = qpad / CJ;
  const int R = threads / tpr;  // one row per thread pass
  const size_t in_bytes = (size_t)(job.nprod * R * s + 1) / 2 * 2 * sizeof(float2);
  const size_t raw_bytes = (size_t)job.nprod * R * sraw * sizeof(double);
  const size_t norm = norm_part ? (size_t)R * 2 * qpad * sizeof(double) : 0;
  // sU, sIn, then raw (reused for the norm partials at the end), then the column table
  const size_t smem = (size_t)s * qpad * sizeof(float2) + in_bytes + std::max(raw_bytes, norm) +
                      (size_t)kMaxS * sizeof(int) + 16;
  if (smem > 110 * 1024) return 0;  // two CTAs per SM
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(update_df_async_kernel<CJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 110 * 1024));
    return true;
  }();
  (void)attr;
  const int64_t max_df = std::max<int64_t>(max_ctas, 2 * (int64_t)num_sms());
  int64_t ctas = std::min<int64_t>(max_df, ceil_div(n, R));
  if (ctas < 1) ctas = 1;
  const int64_t rpc = (ceil_div(n, ctas) + R - 1) / R * R;
  ctas = std::max<int64_t>(1, ceil_div(n, rpc));
  update_df_async_kernel<CJ><<<(unsigned)ctas, threads, smem, st>>>(n, job, U, s, q, alpha, lam, norm_part, rpc, R,
                                                                    sraw);
  LB_LAUNCH_CHECK();
  return (int)ctas;
}

int launch_update_df(int64_t n, const UpdateJob<double>& job, const double* U, int s, int q, double alpha,
                     const double* lam, double* norm_part, int max_ctas, cudaStream_t st) {
  if (q <= 0 || n <= 0) return 0;
  if (const int parts = launch_update_df_async(n, job, U, s, q, alpha, lam, norm_part, max_ctas, st)) return parts;
  constexpr int CJ = 4, R = 32;
  const int qpad = round_up(q, CJ);
  const int threads = 256;
  const int tpr = qpad / CJ;
  const int rows_per_pass = threads / tpr;
  const size_t smem = (size_t)s * qpad * sizeof(float2) + (size_t)job.nprod * R * s * sizeof(float2) +
                      (norm_part ? (size_t)rows_per_pass * 2 * qpad * sizeof(double) : 0) + 16;
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(update_df_kernel<CJ, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    return true;
  }();
  (void)attr;
  // three CTAs per SM (registers and shared memory allow it): while one waits at its
  // staging barrier the others keep the FP32 pipes busy (two per SM left them 60% idle)
  const int64_t max_df = std::max<int64_t>(max_ctas, 3 * (int64_t)num_sms());
  int64_t ctas = std::min<int64_t>(max_df, ceil_div(n, R));
  if (ctas < 1) ctas = 1;
  const int64_t rpc = (ceil_div(n, ctas) + R - 1) / R * R;
  ctas = std::max<int64_t>(1, ceil_div(n, rpc));
  update_df_kernel<CJ, R><<<(unsigned)ctas, threads, smem, st>>>(n, job, U, s, q, alpha, lam, norm_part, rpc);
  LB_LAUNCH_CHECK();
  return (int)ctas;
}

template <class T>
void launch_precond(int64_t n, const T* X, const T* AX, int ld, const double* lam, int c0, int a,
                    const double* diag, int precond, T* W, int ldw, cudaStream_t st, const double* diagB,
                    double floor) {
  if (a <= 0 || n <= 0) return;
  precond_kernel<T><<<grid_for(n * a, 256), 256, 0, st>>>(n, X, AX, ld, lam, c0, a, diag, precond, W, ldw,
                                                         diagB, floor);
  LB_LAUNCH_CHECK();
}

template <class Tin, class Tout>
void launch_colmajor_to_rows(int64_t n, int p, const Tin* src, Tout* dst, int ld, cudaStream_t st) {
  if (n * p <= 0) return;
  col_to_rows_kernel<Tin, Tout><<<grid_for(n * p, 256), 256, 0, st>>>(n, p, src, dst, ld);
  LB_LAUNCH_CHECK();
}
template <class Tin, class Tout>
void launch_rows_to_colmajor(int64_t n, int p, const Tin* src, int ld, Tout* dst, cudaStream_t st) {
  if (n * p <= 0) return;
  rows_to_col_kernel<Tin, Tout><<<grid_for(n * p, 256), 256, 0, st>>>(n, p, src, ld, dst);
  LB_LAUNCH_CHECK();
}

void launch_gaussian(int64_t n, int p, uint64_t seed, double* dst, cudaStream_t st) {
  if (n * p <= 0) return;
  gaussian_kernel<<<grid_for(n * p, 256), 256, 0, st>>>(n * p, seed, dst);
  LB_LAUNCH_CHECK();
}

void launch_to_float(int64_t count, const double* src, float* dst, cudaStream_t st) {
  if (count <= 0) return;
  to_float_kernel<<<grid_for(count, 256), 256, 0, st>>>(count, src, dst);
  LB_LAUNCH_CHECK();
}

void launch_all_finite(int64_t count, const double* src, int* flag, cudaStream_t st) {
  if (count <= 0) return;
  finite_kernel<<<grid_for(count, 256), 256, 0, st>>>(count, src, flag);
  LB_LAUNCH_CHECK();
}

template int gram_partials<double>(int64_t, const Cols<double>&, const Cols<double>&, bool, double*, int, cudaStream_t);
template int gram_partials<float>(int64_t, const Cols<float>&, const Cols<float>&, bool, double*, int, cudaStream_t);
template int launch_update<double>(int64_t, const UpdateJob<double>&, const double*, int, int, double, const double*, double*, int, cudaStream_t);
template int launch_update<float>(int64_t, const UpdateJob<float>&, const double*, int, int, double, const double*, double*, int, cudaStream_t);
template void launch_precond<double>(int64_t, const double*, const double*, int, const double*, int, int, const double*, int, double*, int, cudaStream_t, const double*, double);
template void launch_precond<float>(int64_t, const float*, const float*, int, const double*, int, int, const double*, int, float*, int, cudaStream_t, const double*, double);
template void launch_colmajor_to_rows<double, double>(int64_t, int, const double*, double*, int, cudaStream_t);
template void launch_colmajor_to_rows<double, float>(int64_t, int, const double*, float*, int, cudaStream_t);
template void launch_rows_to_colmajor<double, double>(int64_t, int, const double*, int, double*, cudaStream_t);
template void launch_rows_to_colmajor<float, double>(int64_t, int, const float*, int, double*, cudaStream_t);

}  // namespace lobpcg

namespace lobpcg {
namespace {
template <class T>
__global__ void col_absmax_kernel(int64_t n, int p, const T* __restrict__ X, int ld,
                                  double* __restrict__ part) {
  // part[cta][j] = signed value of the largest |x_ij| in this CTA's rows (ties: first row)
  __shared__ double best_v[256];
  __shared__ int64_t best_i[256];
  const int64_t rows = ceil_div_dev(n, gridDim.x);
  const int64_t r0 = blockIdx.x * rows, r1 = min(n, r0 + rows);
  for (int j = 0; j < p; ++j) {
    double bv = 0.0;
    int64_t bi = INT64_MAX;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const double v = (double)X[i * ld + j];
      if (fabs(v) > fabs(bv) || (fabs(v) == fabs(bv) && i < bi)) bv = v, bi = i;
    }
    best_v[threadIdx.x] = bv;
    best_i[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        const double v = best_v[threadIdx.x + o];
        const int64_t i = best_i[threadIdx.x + o];
        if (fabs(v) > fabs(best_v[threadIdx.x]) ||
            (fabs(v) == fabs(best_v[threadIdx.x]) && i < best_i[threadIdx.x]))
          best_v[threadIdx.x] = v, best_i[threadIdx.x] = i;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      part[(int64_t)blockIdx.x * 2 * p + 2 * j] = best_v[0];
      part[(int64_t)blockIdx.x * 2 * p + 2 * j + 1] = (double)(best_i[0] == INT64_MAX ? -1 : best_i[0]);
    }
    __syncthreads();
  }
}

__global__ void col_sign_combine_kernel(int p, int nparts, const double* __restrict__ part,
                                        double* __restrict__ sgn) {
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    double bv = 0.0, bi = 1e300;
    for (int g = 0; g < nparts; ++g) {
      const double v = part[(int64_t)g * 2 * p + 2 * j], i = part[(int64_t)g * 2 * p + 2 * j + 1];
      if (i < 0) continue;
      if (fabs(v) > fabs(bv) || (fabs(v) == fabs(bv) && i < bi)) bv = v, bi = i;
    }
    sgn[j] = bv < 0.0 ? -1.0 : 1.0;
  }
}

__global__ void scale_matrix_kernel(int p, const double* __restrict__ G, const double* __restrict__ sgn,
                                    double* __restrict__ S) {
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e % p, j = e / p;
    S[e] = i == j ? sgn[j] / sqrt(G[j + j * p]) : 0.0;
  }
}
}  // namespace

template <class T>
void launch_col_sign(int64_t n, int p, const T* X, int ld, double* part, int max_ctas, double* sgn,
                     cudaStream_t st) {
  const int ctas = (int)std::max<int64_t>(1, std::min<int64_t>(max_ctas, ceil_div(n, 256)));
  col_absmax_kernel<T><<<ctas, 256, 0, st>>>(n, p, X, ld, part);
  LB_LAUNCH_CHECK();
  col_sign_combine_kernel<<<1, 64, 0, st>>>(p, ctas, part, sgn);
  LB_LAUNCH_CHECK();
}
template void launch_col_sign<double>(int64_t, int, const double*, int, double*, int, double*, cudaStream_t);

void launch_scale_matrix(int p, const double* G, const double* sgn, double* S, cudaStream_t st) {
  scale_matrix_kernel<<<1, 256, 0, st>>>(p, G, sgn, S);
  LB_LAUNCH_CHECK();
}
}  // namespace lobpcg
