// Pipelined tall-skinny kernels for row-major blocks whose segments share one 16-byte
// aligned row stride (every block the solver allocates): the Gram / projected
// matrices C = A^T B of Algorithm 1 and Eq. (CDOrtho), and the basis updates
// out = base + alpha * in * U (X = V u_x, P = V u_p, W - Y C, W L^{-T}).
//
// Each CTA streams its rows in chunks of R rows.  A chunk of every segment is a
// contiguous R x ld range in global memory, copied with 16-byte cp.async into a
// multi-stage shared-memory ring (row stride ld + VEC to spread banks), so the loads
// of chunk k+S-1 overlap the arithmetic on chunk k.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "dfloat.cuh"

namespace lobpcg {
namespace {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int bytes = valid ? 16 : 0;  // 0 source bytes: the 16 destination bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Issue the copies of rows [r0, r0 + R) of every segment of `c` into dst[seg][R][lds].
template <class T, int R>
__device__ __forceinline__ void issue_chunk(const Cols<T>& c, int ld, int lds, int64_t r0, int64_t rend,
                                            T* dst) {
  constexpr int VEC = 16 / sizeof(T);
  const int vpr = ld / VEC;  // 16-byte vectors per row
  const int total = R * vpr;
  for (int g = 0; g < c.nseg; ++g) {
    const T* src = c.p[g];
    T* d = dst + g * R * lds;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int r = i / vpr, v = i - r * vpr;
      const int64_t row = r0 + r;
      const bool ok = row < rend;
      cp_async16(d + r * lds + v * VEC, src + (ok ? row : 0) * ld + v * VEC, ok);
    }
  }
}

// Padded shared-memory row stride: a multiple of 16 bytes (cp.async destinations) that is
// an odd multiple of 4 banks, so 8 consecutive rows start in 8 different bank groups.
template <class T>
__host__ __device__ __forceinline__ int padded_ld(int ld) {
  constexpr int VEC = 16 / sizeof(T);
  int lds = (ld + VEC - 1) / VEC * VEC;
  while (((lds * (int)sizeof(T) / 4) & 7) != 4) lds += VEC;
  return lds;
}

// Shared-memory offset (within one stage) of logical column `col` of `c`, or -1.
template <class T>
__device__ __forceinline__ int col_offset(const Cols<T>& c, int col, int R, int lds) {
  int base = 0;
  for (int g = 0; g < c.nseg; ++g) {
    if (col < base + c.w[g]) return g * R * lds + (col - base);
    base += c.w[g];
  }
  return -1;
}

// ------------------------------------------------------------------------ Gram
template <class T, int TI, int TJ, int R, int S>
__global__ void __launch_bounds__(256) gram_pipe_kernel(int64_t n, Cols<T> A, Cols<T> B, int ld, int upper,
                                                        int ntiles, int groups, double* __restrict__ part,
                                                        int64_t rows_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lds = padded_ld<T>(ld);
  const int stageA = A.nseg * R * lds, stageB = B.nseg * R * lds;
  const int stage = stageA + stageB;
  T* ring = reinterpret_cast<T*>(smem_raw);
  __shared__ short tile_i[kMaxS * kMaxS / 16], tile_j[kMaxS * kMaxS / 16];
  const int pa = A.width(), pb = B.width();
  const int nti = (pa + TI - 1) / TI, ntj = (pb + TJ - 1) / TJ;
  if (threadIdx.x == 0) {
    int idx = 0;
    for (int tj = 0; tj < ntj; ++tj)
      for (int ti = 0; ti < nti; ++ti)
        if (!upper || ti * TI <= tj * TJ + TJ - 1) tile_i[idx] = (short)ti, tile_j[idx] = (short)tj, ++idx;
  }
  __syncthreads();
  const int t = threadIdx.x % ntiles, grp = threadIdx.x / ntiles;
  const bool active = grp < groups;
  int offA[TI], offB[TJ];
#pragma unroll
  for (int i = 0; i < TI; ++i) offA[i] = col_offset(A, tile_i[t] * TI + i, R, lds);
#pragma unroll
  for (int j = 0; j < TJ; ++j) offB[j] = col_offset(B, tile_j[t] * TJ + j, R, lds);

  T acc[TI][TJ];
#pragma unroll
  for (int i = 0; i < TI; ++i)
#pragma unroll
    for (int j = 0; j < TJ; ++j) acc[i][j] = T(0);

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = min(n, r_begin + rows_per_cta);
  const int nchunks = (int)((r_end - r_begin + R - 1) / R);
#pragma unroll
  for (int k = 0; k < S - 1; ++k) {
    if (k < nchunks) {
      issue_chunk<T, R>(A, ld, lds, r_begin + (int64_t)k * R, r_end, ring + k * stage);
      issue_chunk<T, R>(B, ld, lds, r_begin + (int64_t)k * R, r_end, ring + k * stage + stageA);
    }
    cp_async_commit();
  }
  for (int k = 0; k < nchunks; ++k) {
    cp_async_wait<S - 2>();
    __syncthreads();
    {
      const int kn = k + S - 1;
      if (kn < nchunks) {
        T* dst = ring + (kn % S) * stage;
        issue_chunk<T, R>(A, ld, lds, r_begin + (int64_t)kn * R, r_end, dst);
        issue_chunk<T, R>(B, ld, lds, r_begin + (int64_t)kn * R, r_end, dst + stageA);
      }
      cp_async_commit();
    }
    if (active) {
      const T* sa = ring + (k % S) * stage;
      const T* sb = sa + stageA;
      for (int r = grp; r < R; r += groups) {
        T a[TI], b[TJ];
#pragma unroll
        for (int i = 0; i < TI; ++i) a[i] = offA[i] >= 0 ? sa[offA[i] + r * lds] : T(0);
#pragma unroll
        for (int j = 0; j < TJ; ++j) b[j] = offB[j] >= 0 ? sb[offB[j] + r * lds] : T(0);
#pragma unroll
        for (int i = 0; i < TI; ++i)
#pragma unroll
          for (int j = 0; j < TJ; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  // groups add their sums into shared memory one after another (fixed order)
  double* scratch = reinterpret_cast<double*>(smem_raw);
  constexpr int per = TI * TJ;
  for (int g = 0; g < groups; ++g) {
    if (active && grp == g) {
#pragma unroll
      for (int i = 0; i < TI; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) {
          double& dst = scratch[t * per + i * TJ + j];
          dst = (g == 0 ? 0.0 : dst) + (double)acc[i][j];
        }
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.x * pa * pb;
  for (int e = threadIdx.x; e < ntiles * per; e += blockDim.x) {
    const int tt = e / per, ij = e % per;
    const int i = tile_i[tt] * TI + ij / TJ, j = tile_j[tt] * TJ + ij % TJ;
    if (i < pa && j < pb && (!upper || i <= j)) out[i + j * pa] = scratch[e];
  }
}

// ------------------------------------------------------------------ Gram, double-float
// FP64 Gram C = A^T B formed on the FP32 pipes (dfloat.cuh): the staged FP64 rows are
// split in place into (hi, lo) float pairs (same 8 bytes), each thread sums its TI x TJ
// tile with the compensated double-float product-sum, and every `flush` chunks the pairs
// are added to FP64 sums (a few rows' worth of FP64 adds per 100+ rows of products).
// Tiles, groups and the fixed-order group combination are those of gram_pipe_kernel.
template <int TI, int TJ, int R, int S>
__global__ void __launch_bounds__(512) gram_df_kernel(int64_t n, Cols<double> A, Cols<double> B, int ld, int upper,
                                                      int ntiles, int groups, int flush, double* __restrict__ part,
                                                      int64_t rows_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lds = padded_ld<double>(ld);
  const int stageA = A.nseg * R * lds, stageB = B.nseg * R * lds;
  const int stage = stageA + stageB;
  double* ring = reinterpret_cast<double*>(smem_raw);
  __shared__ short tile_i[kMaxS * kMaxS / 16], tile_j[kMaxS * kMaxS / 16];
  const int pa = A.width(), pb = B.width();
  const int nti = (pa + TI - 1) / TI, ntj = (pb + TJ - 1) / TJ;
  if (threadIdx.x == 0) {
    int idx = 0;
    for (int tj = 0; tj < ntj; ++tj)
      for (int ti = 0; ti < nti; ++ti)
        if (!upper || ti * TI <= tj * TJ + TJ - 1) tile_i[idx] = (short)ti, tile_j[idx] = (short)tj, ++idx;
  }
  __syncthreads();
  const int t = threadIdx.x % ntiles, grp = threadIdx.x / ntiles;
  const bool active = grp < groups;
  int offA[TI], offB[TJ];
#pragma unroll
  for (int i = 0; i < TI; ++i) offA[i] = col_offset(A, tile_i[t] * TI + i, R, lds);
#pragma unroll
  for (int j = 0; j < TJ; ++j) offB[j] = col_offset(B, tile_j[t] * TJ + j, R, lds);

  DfAcc acc[TI][TJ];
  double sum[TI][TJ];
#pragma unroll
  for (int i = 0; i < TI; ++i)
#pragma unroll
    for (int j = 0; j < TJ; ++j) df_zero(acc[i][j]), sum[i][j] = 0.0;

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = min(n, r_begin + rows_per_cta);
  const int nchunks = (int)((r_end - r_begin + R - 1) / R);
#pragma unroll
  for (int k = 0; k < S - 1; ++k) {
    if (k < nchunks) {
      issue_chunk<double, R>(A, ld, lds, r_begin + (int64_t)k * R, r_end, ring + k * stage);
      issue_chunk<double, R>(B, ld, lds, r_begin + (int64_t)k * R, r_end, ring + k * stage + stageA);
    }
    cp_async_commit();
  }
  const int vals = A.nseg + B.nseg;  // segments staged per chunk, each R x ld
  for (int k = 0; k < nchunks; ++k) {
    cp_async_wait<S - 2>();
    __syncthreads();
    {
      const int kn = k + S - 1;
      if (kn < nchunks) {
        double* dst = ring + (kn % S) * stage;
        issue_chunk<double, R>(A, ld, lds, r_begin + (int64_t)kn * R, r_end, dst);
        issue_chunk<double, R>(B, ld, lds, r_begin + (int64_t)kn * R, r_end, dst + stageA);
      }
      cp_async_commit();
    }
    // split the landed chunk in place: each double becomes its (hi, lo) float pair
    double* cur = ring + (k % S) * stage;
    for (int e = threadIdx.x; e < vals * R * ld; e += blockDim.x) {
      const int g = e / (R * ld), rem = e - g * R * ld;
      const int r = rem / ld, c = rem - r * ld;
      double* slot = cur + (size_t)g * R * lds + r * lds + c;
      const float2 h = df_split(*slot);
      *reinterpret_cast<float2*>(slot) = h;
    }
    __syncthreads();
    if (active) {
      const float2* sa = reinterpret_cast<const float2*>(cur);
      const float2* sb = sa + stageA;
      for (int r = grp; r < R; r += groups) {
        float2 a[TI], b[TJ];
#pragma unroll
        for (int i = 0; i < TI; ++i) a[i] = offA[i] >= 0 ? sa[offA[i] + r * lds] : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < TJ; ++j) b[j] = offB[j] >= 0 ? sb[offB[j] + r * lds] : make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < TI; ++i)
#pragma unroll
          for (int j = 0; j < TJ; ++j) df_fma(acc[i][j], a[i], b[j]);
      }
      if ((k + 1) % flush == 0 || k + 1 == nchunks) {
#pragma unroll
        for (int i = 0; i < TI; ++i)
#pragma unroll
          for (int j = 0; j < TJ; ++j) sum[i][j] += df_value(acc[i][j]), df_zero(acc[i][j]);
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  double* scratch = reinterpret_cast<double*>(smem_raw);
  constexpr int per = TI * TJ;
  for (int g = 0; g < groups; ++g) {
    if (active && grp == g) {
#pragma unroll
      for (int i = 0; i < TI; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) {
          double& dst = scratch[t * per + i * TJ + j];
          dst = (g == 0 ? 0.0 : dst) + sum[i][j];
        }
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.x * pa * pb;
  for (int e = threadIdx.x; e < ntiles * per; e += blockDim.x) {
    const int tt = e / per, ij = e % per;
    const int i = tile_i[tt] * TI + ij / TJ, j = tile_j[tt] * TJ + ij % TJ;
    if (i < pa && j < pb && (!upper || i <= j)) out[i + j * pa] = scratch[e];
  }
}

// ------------------------------------------------------------------ Gram, tensor cores
// FP32 Gram C = A^T B on the tensor cores (mma.sync m16n8k8, TF32 inputs, FP32
// accumulation) with the 3xTF32 split: x = x_hi + x_lo, both TF32, and
// a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, so each product keeps about 21 bits: FP32-level
// accuracy for the mixed form.  Each 8-row step is summed by the tensor core from zero and
// added to the running FP32 sums with ordinary round-to-nearest adds.  Rows are staged as in gram_pipe_kernel; a warp owns up to
// BPW output blocks of 16 x 32 (one M tile, four N tiles) and, when there are fewer blocks
// than warps, a share of the 8-row k steps of every chunk.  The groups of warps that split
// the k steps are summed in a fixed order.
__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(hi) : "f"(x));
  const float r = x - __uint_as_float(hi);
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(lo) : "f"(r));
}
__device__ __forceinline__ void mma_tf32(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Shared-memory row stride for the tensor-core Gram: >= ld, a multiple of 4 floats, and
// 8 (mod 32) floats, so the 4 k-rows x 8 columns of a fragment load hit 32 banks.
__host__ __device__ __forceinline__ int tc_lds(int ld) {
  int lds = (ld + 3) / 4 * 4;
  while (lds % 32 != 8) lds += 4;
  return lds;
}

template <int R, int S, int BPW>
__global__ void __launch_bounds__(256) gram_tc_kernel(int64_t n, Cols<float> A, Cols<float> B, int ld, int upper,
                                                      int mt, int nbk, int kgroups, double* __restrict__ part,
                                                      int64_t rows_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lds = tc_lds(ld);
  const int stageA = A.nseg * R * lds, stageB = B.nseg * R * lds;
  const int stage = stageA + stageB;
  float* ring = reinterpret_cast<float*>(smem_raw);
  const int pa = A.width(), pb = B.width();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gid = lane >> 2, t4 = lane & 3;
  const int nblocks = mt * nbk;
  const int used = nblocks < 8 ? nblocks * kgroups : 8;  // warps with work
  const bool active = wid < used;
  const int kg = nblocks < 8 ? wid / nblocks : 0;
  // fragment offsets (within one stage) of the rows / columns this lane reads; -1: zero
  int offA[BPW][2], offB[BPW][4];
  int blk[BPW];
#pragma unroll
  for (int b = 0; b < BPW; ++b) {
    blk[b] = nblocks < 8 ? (wid % nblocks) : wid + 8 * b;
    const bool ok = active && blk[b] < nblocks && (nblocks < 8 ? b == 0 : true);
    int mi = ok ? blk[b] / nbk : 0, nj = ok ? blk[b] % nbk : 0;
    // upper: a block wholly below the diagonal is not needed
    const bool need = !(upper && mi * 16 > nj * 32 + 31);
    mi = need ? mi : 0, nj = need ? nj : 0;
    offA[b][0] = ok && need ? col_offset(A, mi * 16 + gid, R, lds) : -1;
    offA[b][1] = ok && need ? col_offset(A, mi * 16 + gid + 8, R, lds) : -1;
#pragma unroll
    for (int t = 0; t < 4; ++t) offB[b][t] = ok && need ? col_offset(B, nj * 32 + t * 8 + gid, R, lds) : -1;
    if (!ok || !need) blk[b] = -1;
  }
  float acc[BPW][4][4];
#pragma unroll
  for (int b = 0; b < BPW; ++b)
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[b][t][e] = 0.f;

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = min(n, r_begin + rows_per_cta);
  const int nchunks = (int)((r_end - r_begin + R - 1) / R);
#pragma unroll
  for (int k = 0; k < S - 1; ++k) {
    if (k < nchunks) {
      issue_chunk<float, R>(A, ld, lds, r_begin + (int64_t)k * R, r_end, ring + k * stage);
      issue_chunk<float, R>(B, ld, lds, r_begin + (int64_t)k * R, r_end, ring + k * stage + stageA);
    }
    cp_async_commit();
  }
  for (int k = 0; k < nchunks; ++k) {
    cp_async_wait<S - 2>();
    __syncthreads();
    {
      const int kn = k + S - 1;
      if (kn < nchunks) {
        float* dst = ring + (kn % S) * stage;
        issue_chunk<float, R>(A, ld, lds, r_begin + (int64_t)kn * R, r_end, dst);
        issue_chunk<float, R>(B, ld, lds, r_begin + (int64_t)kn * R, r_end, dst + stageA);
      }
      cp_async_commit();
    }
    if (active) {
      const float* sa = ring + (k % S) * stage;
      const float* sb = sa + stageA;
      for (int st = kg; st < R / 8; st += kgroups) {
        const int r0 = st * 8 + t4, r1 = r0 + 4;
#pragma unroll
        for (int b = 0; b < BPW; ++b) {
          if (blk[b] < 0) continue;
          unsigned ah[4], al[4];
          split_tf32(offA[b][0] >= 0 ? sa[offA[b][0] + r0 * lds] : 0.f, ah[0], al[0]);
          split_tf32(offA[b][1] >= 0 ? sa[offA[b][1] + r0 * lds] : 0.f, ah[1], al[1]);
          split_tf32(offA[b][0] >= 0 ? sa[offA[b][0] + r1 * lds] : 0.f, ah[2], al[2]);
          split_tf32(offA[b][1] >= 0 ? sa[offA[b][1] + r1 * lds] : 0.f, ah[3], al[3]);
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            unsigned bh[2], bl[2];
            split_tf32(offB[b][t] >= 0 ? sb[offB[b][t] + r0 * lds] : 0.f, bh[0], bl[0]);
            split_tf32(offB[b][t] >= 0 ? sb[offB[b][t] + r1 * lds] : 0.f, bh[1], bl[1]);
            // the step's three products from a zero accumulator, then one round-to-nearest
            // FP32 add per element: the tensor core's own accumulation is not carried across
            // the hundreds of steps of a CTA (its rounding would bias the running sum)
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            mma_tf32(d, al, bh);
            mma_tf32(d, ah, bl);
            mma_tf32(d, ah, bh);
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[b][t][e] += d[e];
          }
        }
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  // sum the k groups in order into an (mt*16) x (nbk*32) FP64 scratch (reusing the ring)
  double* scratch = reinterpret_cast<double*>(smem_raw);
  const int SM = mt * 16, SN = nbk * 32;
  for (int e = threadIdx.x; e < SM * SN; e += blockDim.x) scratch[e] = 0.0;
  __syncthreads();
  for (int g = 0; g < (nblocks < 8 ? kgroups : 1); ++g) {
    if (active && kg == g) {
#pragma unroll
      for (int b = 0; b < BPW; ++b) {
        if (blk[b] < 0) continue;
        const int mi = blk[b] / nbk, nj = blk[b] % nbk;
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int i = mi * 16 + gid + (e >> 1) * 8;
            const int j = nj * 32 + t * 8 + 2 * t4 + (e & 1);
            scratch[i + j * SM] += (double)acc[b][t][e];
          }
      }
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.x * pa * pb;
  for (int e = threadIdx.x; e < pa * pb; e += blockDim.x) {
    const int i = e % pa, j = e / pa;
    if (!upper || i <= j) out[i + j * pa] = scratch[i + j * SM];
  }
}

template <int R, int S, int BPW>
int gram_tc_launch(int64_t n, const Cols<float>& a, const Cols<float>& b, int ld, bool upper, double* part,
                   int max_ctas, cudaStream_t st) {
  const int pa = a.width(), pb = b.width();
  const int mt = (pa + 15) / 16, nbk = (pb + 31) / 32;
  const int nblocks = mt * nbk;
  const int kgroups = nblocks < 8 ? std::min(8 / nblocks, R / 8) : 1;
  const int lds = tc_lds(ld);
  const size_t ring = (size_t)S * (a.nseg + b.nseg) * R * lds * sizeof(float);
  const size_t scr = (size_t)mt * 16 * nbk * 32 * sizeof(double);
  const size_t smem = std::max(ring, scr);
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(gram_tc_kernel<R, S, BPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    return true;
  }();
  (void)attr;
  int64_t ctas = std::min<int64_t>(max_ctas, ceil_div(n, R));
  if (ctas < 1) ctas = 1;
  const int64_t rpc = (ceil_div(n, ctas) + R - 1) / R * R;
  ctas = std::max<int64_t>(1, ceil_div(n, rpc));
  gram_tc_kernel<R, S, BPW><<<(unsigned)ctas, 256, smem, st>>>(n, a, b, ld, upper ? 1 : 0, mt, nbk, kgroups, part,
                                                               rpc);
  LB_LAUNCH_CHECK();
  return (int)ctas;
}

// ------------------------------------------------------------------------ update
// Thread (rg, cg) computes RJ rows x CJ columns of every product of the job.
template <class T, int RJ, int CJ, int R, int S>
__global__ void __launch_bounds__(256) update_pipe_kernel(int64_t n, UpdateJob<T> job, int ld,
                                                          const double* __restrict__ U, int s, int q,
                                                          double alpha, const double* __restrict__ lam,
                                                          double* __restrict__ norm_part, int64_t rows_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lds = padded_ld<T>(ld);
  const int qpad = (q + CJ - 1) / CJ * CJ;
  T* sU = reinterpret_cast<T*>(smem_raw);                        // s x qpad
  int* offs = reinterpret_cast<int*>(sU + ((s * qpad + 3) / 4) * 4);  // s column offsets
  T* ring = reinterpret_cast<T*>(offs + ((s + 3) / 4) * 4);
  const int stage_in = job.in[0].nseg * R * lds;
  const int stage = job.nprod * stage_in;
  for (int e = threadIdx.x; e < s * qpad; e += blockDim.x) {
    const int l = e / qpad, j = e % qpad;
    sU[e] = j < q ? (T)U[l + j * s] : T(0);
  }
  for (int l = threadIdx.x; l < s; l += blockDim.x) offs[l] = col_offset(job.in[0], l, R, lds);
  const int cgs = qpad / CJ, rgs = R / RJ;
  const int cg = threadIdx.x % cgs, rg = threadIdx.x / cgs;
  const bool active = rg < rgs;
  double nsum[CJ], nmax[CJ];
#pragma unroll
  for (int j = 0; j < CJ; ++j) nsum[j] = 0.0, nmax[j] = 0.0;

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = min(n, r_begin + rows_per_cta);
  const int nchunks = (int)((r_end - r_begin + R - 1) / R);
#pragma unroll
  for (int k = 0; k < S - 1; ++k) {
    if (k < nchunks)
      for (int t = 0; t < job.nprod; ++t)
        issue_chunk<T, R>(job.in[t], ld, lds, r_begin + (int64_t)k * R, r_end, ring + k * stage + t * stage_in);
    cp_async_commit();
  }
  for (int k = 0; k < nchunks; ++k) {
    cp_async_wait<S - 2>();
    __syncthreads();
    {
      const int kn = k + S - 1;
      if (kn < nchunks)
        for (int t = 0; t < job.nprod; ++t)
          issue_chunk<T, R>(job.in[t], ld, lds, r_begin + (int64_t)kn * R, r_end,
                            ring + (kn % S) * stage + t * stage_in);
      cp_async_commit();
    }
    if (!active) continue;
    const int64_t row0 = r_begin + (int64_t)k * R + rg;  // rows row0 + r * rgs, r < RJ
    T res[2][RJ][CJ];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (t >= job.nprod) break;
      const T* sin = ring + (k % S) * stage + t * stage_in + rg * lds;
      T acc[RJ][CJ];
#pragma unroll
      for (int r = 0; r < RJ; ++r)
#pragma unroll
        for (int j = 0; j < CJ; ++j) acc[r][j] = T(0);
      for (int l = 0; l < s; ++l) {
        const int o = offs[l];
        T u[CJ];
#pragma unroll
        for (int j = 0; j < CJ; ++j) u[j] = sU[l * qpad + cg * CJ + j];
#pragma unroll
        for (int r = 0; r < RJ; ++r) {
          const T x = sin[o + r * rgs * lds];
#pragma unroll
          for (int j = 0; j < CJ; ++j) acc[r][j] = fma(x, u[j], acc[r][j]);
        }
      }
#pragma unroll
      for (int r = 0; r < RJ; ++r) {
        const int64_t row = row0 + (int64_t)r * rgs;
        if (row >= r_end) continue;
        T* o = job.out[t] + row * job.ld_out[t];
        const T* b = job.base[t] ? job.base[t] + row * job.ld_base[t] : nullptr;
#pragma unroll
        for (int j = 0; j < CJ; ++j) {
          const int col = cg * CJ + j;
          T v = (T)alpha * acc[r][j];
          if (b && col < q) v = b[col] + v;
          res[t][r][j] = v;
          if (col < q) o[col] = v;
        }
      }
    }
    if (norm_part) {
#pragma unroll
      for (int r = 0; r < RJ; ++r) {
        if (row0 + (int64_t)r * rgs >= r_end) continue;
#pragma unroll
        for (int j = 0; j < CJ; ++j) {
          const int col = cg * CJ + j;
          if (col < q) {
            const T rij = fma(-(T)lam[col], res[0][r][j], res[1][r][j]);  // AX - lam X, one rounding
            nsum[j] = fma((double)rij, (double)rij, nsum[j]);
            nmax[j] = fmax(nmax[j], (double)fabs(rij));
          }
        }
      }
    }
  }
  cp_async_wait<0>();
  if (!norm_part) return;
  __syncthreads();
  double* sN = reinterpret_cast<double*>(ring);  // [rgs][2 * qpad]
  if (active)
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
      sN[rg * 2 * qpad + cg * CJ + j] = nsum[j];
      sN[rg * 2 * qpad + qpad + cg * CJ + j] = nmax[j];
    }
  __syncthreads();
  for (int col = threadIdx.x; col < q; col += blockDim.x) {
    double s2 = 0.0, mx = 0.0;
    for (int g = 0; g < rgs; ++g) {
      s2 += sN[g * 2 * qpad + col];
      mx = fmax(mx, sN[g * 2 * qpad + qpad + col]);
    }
    norm_part[(int64_t)blockIdx.x * 2 * q + col] = s2;
    norm_part[(int64_t)blockIdx.x * 2 * q + q + col] = mx;
  }
}


// ------------------------------------------------------------------------ update, one row per thread
// out_t = base_t + alpha * in_t * U with U (s x q, q <= QMAX) broadcast from shared memory
// and each thread streaming its own input row with 16-byte loads (the row's lines stay
// in L1 while the thread walks them).  The FP32 fallback of update_stage_kernel (products
// whose segments differ in width, or the norm form with a base).
template <class T>
struct V16;
template <>
struct V16<float> {
  using type = float4;
};
template <>
struct V16<double> {
  using type = double2;
};

template <class T, int QMAX>
__global__ void __launch_bounds__(256) update_row_kernel(int64_t n, UpdateJob<T> job, int ld,
                                                         const double* __restrict__ U, int s, int q,
                                                         double alpha, const double* __restrict__ lam,
                                                         double* __restrict__ norm_part, int64_t rows_per_cta) {
  using VT = typename V16<T>::type;
  constexpr int VEC = 16 / sizeof(T);
  constexpr int QV = QMAX / VEC;  // vectors per U row
  extern __shared__ __align__(16) unsigned char smem_raw[];
  VT* sU = reinterpret_cast<VT*>(smem_raw);  // s rows of QV vectors
  for (int e = threadIdx.x; e < s * QMAX; e += blockDim.x) {
    const int l = e / QMAX, j = e % QMAX;
    reinterpret_cast<T*>(sU)[e] = j < q ? (T)U[l + j * s] : T(0);
  }
  __syncthreads();
  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = min(n, r_begin + rows_per_cta);
  T nsum[QMAX], nmax[QMAX];  // per-thread partial column sums of r^2 and max |r|
  if (norm_part)
#pragma unroll
    for (int j = 0; j < QMAX; ++j) nsum[j] = T(0), nmax[j] = T(0);
  for (int64_t row = r_begin + threadIdx.x; row < r_end; row += blockDim.x) {
    T res[2][QMAX];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (t >= job.nprod) break;
      const Cols<T>& in = job.in[t];
#pragma unroll
      for (int j = 0; j < QMAX; ++j) res[t][j] = T(0);
      int l0 = 0;
      for (int g = 0; g < in.nseg; ++g) {
        const T* xr = in.p[g] + row * ld;
        const int w = in.w[g];
        for (int c = 0; c < w; c += VEC) {
          const VT xv = *reinterpret_cast<const VT*>(xr + c);
          const T* xs = reinterpret_cast<const T*>(&xv);
#pragma unroll
          for (int i = 0; i < VEC; ++i) {
            if (c + i >= w) break;
            const T x = xs[i];
            const VT* ur = sU + (l0 + c + i) * QV;
#pragma unroll
            for (int jv = 0; jv < QV; ++jv) {
              const VT u = ur[jv];
              const T* us = reinterpret_cast<const T*>(&u);
#pragma unroll
              for (int k = 0; k < VEC; ++k) res[t][jv * VEC + k] = fma(x, us[k], res[t][jv * VEC + k]);
            }
          }
        }
        l0 += w;
      }
      T* o = job.out[t] + row * job.ld_out[t];
      const T* b = job.base[t] ? job.base[t] + row * job.ld_base[t] : nullptr;
#pragma unroll
      for (int j = 0; j < QMAX; ++j) {
        if (j < q) {
          T v = (T)alpha * res[t][j];
          if (b) v = b[j] + v;
          res[t][j] = v;
          o[j] = v;
        }
      }
    }
    if (norm_part) {
#pragma unroll
      for (int j = 0; j < QMAX; ++j) {
        if (j < q) {
          const T rij = fma(-(T)lam[j], res[0][j], res[1][j]);  // AX - lam X, one rounding
          nsum[j] = fma(rij, rij, nsum[j]);
          nmax[j] = fmax(nmax[j], fabs(rij));
        }
      }
    }
  }
  if (!norm_part) return;
  // CTA reduction of the per-column partial norms: warp shuffles, then warps in order
  __syncthreads();
  double* red = reinterpret_cast<double*>(smem_raw);  // [warps][2 * QMAX]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < QMAX; ++j) {
    if (j >= q) break;
    const double a = warp_sum((double)nsum[j]);
    const double m = warp_max((double)nmax[j]);
    if (lane == 0) red[wid * 2 * QMAX + j] = a, red[wid * 2 * QMAX + QMAX + j] = m;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < q; j += blockDim.x) {
    double a = 0.0, m = 0.0;
    for (int w2 = 0; w2 < nw; ++w2) a += red[w2 * 2 * QMAX + j], m = fmax(m, red[w2 * 2 * QMAX + QMAX + j]);
    norm_part[(int64_t)blockIdx.x * 2 * q + j] = a;
    norm_part[(int64_t)blockIdx.x * 2 * q + q + j] = m;
  }
}

template <class T, int QMAX>
int update_row_launch(int64_t n, const UpdateJob<T>& job, int ld, const double* U, int s, int q, double alpha,
                      const double* lam, double* norm_part, int max_ctas, cudaStream_t st) {
  const int threads = 256;
  const size_t smem = std::max((size_t)s * QMAX * sizeof(T), (size_t)(threads / 32) * 2 * QMAX * sizeof(double));
  // set once per process; function-local statics initialise thread-safely
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(update_row_kernel<T, QMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 64 * 1024));
    return true;
  }();
  (void)attr;
  int64_t ctas = std::min<int64_t>(max_ctas, ceil_div(n, threads));
  if (ctas < 1) ctas = 1;
  const int64_t rpc = ceil_div(n, ctas);
  ctas = std::max<int64_t>(1, ceil_div(n, rpc));
  update_row_kernel<T, QMAX><<<(unsigned)ctas, threads, smem, st>>>(n, job, ld, U, s, q, alpha, lam, norm_part, rpc);
  LB_LAUNCH_CHECK();
  return (int)ctas;
}

// ------------------------------------------------------------------------ update, staged slabs
// out_t = base_t + alpha * in_t * U for FP32 blocks, q <= QMAX: the arithmetic of
// update_row_kernel (same rows per thread, the same FMA chain in the order of the rows of
// U), with the memory traffic and the instruction stream reorganised.
//  - The CTA's rows pass through shared memory in slabs of kStageRows rows x one input
//    segment of one product: cp.async copies the slabs kStageSlabs - 1 ahead of use
//    (coalesced 16-byte reads, in flight while the FMAs run).  Columns past the segment's
//    width are zero-filled, and U's rows sit in shared memory with each segment padded to a
//    multiple of 4 zero rows, so the inner loop runs over whole 16-byte vectors of x with no
//    bounds test (the padding adds exact zeros to the sums).
//  - Thread r multiplies row r of each slab by U (16-byte broadcasts), writes its results
//    over its own row of the product's last slab, and the CTA stores the slab's rows with
//    16-byte stores, 4 rows per warp pass.
// With NORM (nprod == 2, no base) the per-column partial sums of r_ij^2 and max |r_ij|,
// r = AX - X diag(lam), go to norm_part[cta][2q].
constexpr int kStageRows = 256, kStageSlabs = 3;

template <class T>
__device__ __forceinline__ const T* seg_ptr(const Cols<T>& c, int g) {
  return g == 0 ? c.p[0] : (g == 1 ? c.p[1] : c.p[2]);
}
template <class T>
__device__ __forceinline__ int seg_w(const Cols<T>& c, int g) {
  return g == 0 ? c.w[0] : (g == 1 ? c.w[1] : c.w[2]);
}
__host__ __device__ __forceinline__ int padded_rows(int w) { return (w + 3) / 4 * 4; }

template <int QMAX, bool NORM>
__global__ void __launch_bounds__(kStageRows, 2) update_stage_kernel(int64_t n, UpdateJob<float> job, int ld,
                                                                     int lds, const double* __restrict__ U, int s,
                                                                     int q, double alpha,
                                                                     const double* __restrict__ lam,
                                                                     double* __restrict__ norm_part,
                                                                     int64_t rows_per_cta) {
  constexpr int QV = QMAX / 4;  // float4 vectors per U row
  constexpr int R = kStageRows, S = kStageSlabs;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nseg = job.in[0].nseg;
  int sp = 0;  // padded rows of U
  for (int g = 0; g < nseg; ++g) sp += padded_rows(seg_w(job.in[0], g));
  float4* sU = reinterpret_cast<float4*>(smem_raw);  // sp rows of QV vectors
  float* ring = reinterpret_cast<float*>(sU + sp * QV);  // S slabs of R rows, row stride lds
  {
    float* su = reinterpret_cast<float*>(sU);
    int l0 = 0, p0 = 0;
    for (int g = 0; g < nseg; ++g) {
      const int w = seg_w(job.in[0], g), wp = padded_rows(w);
      for (int e = threadIdx.x; e < wp * QMAX; e += blockDim.x) {
        const int l = e / QMAX, j = e % QMAX;
        su[(p0 + l) * QMAX + j] = (l < w && j < q) ? (float)U[l0 + l + j * s] : 0.f;
      }
      l0 += w, p0 += wp;
    }
  }
  const int per_chunk = job.nprod * nseg;
  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_end = min(n, r_begin + rows_per_cta);
  const int nchunks = (int)((r_end - r_begin + R - 1) / R);
  const int total = nchunks * per_chunk;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // copy slab v (rows of chunk v / per_chunk; product, segment from v % per_chunk) to its
  // slot: a warp copies 32 / nv whole rows per pass, lane (rr, c) the c-th 16 bytes of row
  // rr, zero-filling the columns past w and the rows past the end
  auto issue = [&](int v) {
    const int k = v / per_chunk, u = v - k * per_chunk;
    const int t = u / nseg, g = u - t * nseg;
    const Cols<float>& in = t == 0 ? job.in[0] : job.in[1];
    const float* src = seg_ptr(in, g);
    const int w = seg_w(in, g);
    const int nv = (w + 3) / 4;  // 1..24 (w <= 96)
    if (nv == 0) return;
    const int rpi = 32 / nv, rr = lane / nv, c = lane - rr * nv;
    if (rr >= rpi) return;
    const int bytes = min(4, w - 4 * c) * 4;
    float* dst = ring + (v % S) * R * lds + c * 4;
    const int64_t r0 = r_begin + (int64_t)k * R;
    for (int r = wid * rpi + rr; r < R; r += nw * rpi) {
      const int64_t row = r0 + r;
      const bool ok = row < r_end;
      const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + r * lds);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa),
                   "l"(src + (ok ? row : 0) * ld + c * 4), "r"(ok ? bytes : 0));
    }
  };
  float nsum[NORM ? QMAX : 1], nmax[NORM ? QMAX : 1];  // per-thread partial column sums of r^2, max |r|
  if (NORM)
#pragma unroll
    for (int j = 0; j < QMAX; ++j) nsum[j] = 0.f, nmax[j] = 0.f;
#pragma unroll
  for (int v = 0; v < S - 1; ++v) {
    if (v < total) issue(v);
    cp_async_commit();
  }
  const int qv = (q + 3) / 4;
  const int fr = lane >> 3, fc = (lane & 7) * 4;  // write-back: row fr of 4, columns fc..fc+3
  int v = 0;
  for (int k = 0; k < nchunks; ++k) {
    const int64_t r0 = r_begin + (int64_t)k * R;
    const bool live = r0 + threadIdx.x < r_end;
    float x_res[NORM ? QMAX : 1];  // this row's X result, kept for the residual of AX
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (t >= job.nprod) break;
      const Cols<float>& in = job.in[t];
      float acc[QMAX];
#pragma unroll
      for (int j = 0; j < QMAX; ++j) acc[j] = 0.f;
      float* slab = ring;
      const float4* useg = sU;
      for (int g = 0; g < nseg; ++g, ++v) {
        cp_async_wait<S - 2>();
        __syncthreads();
        if (v + S - 1 < total) issue(v + S - 1);
        cp_async_commit();
        slab = ring + (v % S) * R * lds;
        const float* xr = slab + threadIdx.x * lds;
        const int nv = (seg_w(in, g) + 3) / 4;
        for (int c = 0; c < nv; ++c) {
          const float4 xv = *reinterpret_cast<const float4*>(xr + 4 * c);
          const float4* ur = useg + 4 * c * QV;
          const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int jv = 0; jv < QV; ++jv) {
              const float4 u = ur[i * QV + jv];
              acc[jv * 4 + 0] = fmaf(xs[i], u.x, acc[jv * 4 + 0]);
              acc[jv * 4 + 1] = fmaf(xs[i], u.y, acc[jv * 4 + 1]);
              acc[jv * 4 + 2] = fmaf(xs[i], u.z, acc[jv * 4 + 2]);
              acc[jv * 4 + 3] = fmaf(xs[i], u.w, acc[jv * 4 + 3]);
            }
          }
        }
        useg += 4 * nv * QV;
      }
      // this thread's results over its own row of the last slab (only thread r reads row r)
      float* own = slab + threadIdx.x * lds;
#pragma unroll
      for (int jv = 0; jv < QV; ++jv) {
        if (jv < qv) {
          float4 o;
          o.x = (float)alpha * acc[jv * 4 + 0];
          o.y = (float)alpha * acc[jv * 4 + 1];
          o.z = (float)alpha * acc[jv * 4 + 2];
          o.w = (float)alpha * acc[jv * 4 + 3];
          *reinterpret_cast<float4*>(own + 4 * jv) = o;
        }
      }
      if (NORM) {
#pragma unroll
        for (int j = 0; j < QMAX; ++j) {
          const float val = (float)alpha * acc[j];
          if (t == 0) {
            x_res[j] = val;
          } else if (live && j < q) {
            const float rij = fmaf(-(float)lam[j], x_res[j], val);  // AX - lam X, one rounding
            nsum[j] = fmaf(rij, rij, nsum[j]);
            nmax[j] = fmaxf(nmax[j], fabsf(rij));
          }
        }
      }
      __syncthreads();
      // the slab's rows back to out_t (+ base_t): 4 rows x 8 lanes of 4 columns per pass
      float* out = job.out[t];
      const float* base = job.base[t];
      const int ldo = job.ld_out[t], ldb = job.ld_base[t];
      const bool vec = !(ldo & 3) && !(reinterpret_cast<uintptr_t>(out) & 15) &&
                       (!base || (!(ldb & 3) && !(reinterpret_cast<uintptr_t>(base) & 15)));
      if (fc < q) {
        for (int r = wid * 4 + fr; r < R; r += nw * 4) {
          const int64_t row = r0 + r;
          if (row >= r_end) break;
          const float* sv = slab + r * lds + fc;
          float* o = out + row * ldo + fc;
          const float* b = base ? base + row * ldb + fc : nullptr;
          if (vec && fc + 4 <= q) {
            float4 val = *reinterpret_cast<const float4*>(sv);
            if (b) {
              const float4 bv = *reinterpret_cast<const float4*>(b);
              val.x = bv.x + val.x, val.y = bv.y + val.y, val.z = bv.z + val.z, val.w = bv.w + val.w;
            }
            *reinterpret_cast<float4*>(o) = val;
          } else {
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
              if (fc + jj < q) o[jj] = b ? b[jj] + sv[jj] : sv[jj];
          }
        }
      }
    }
  }
  cp_async_wait<0>();
  if (!NORM) return;
  // CTA reduction of the per-column partial norms: warp shuffles, then warps in order
  __syncthreads();
  double* red = reinterpret_cast<double*>(ring);  // [warps][2 * QMAX]
#pragma unroll
  for (int j = 0; j < QMAX; ++j) {
    if (j >= q) break;
    const double a = warp_sum((double)nsum[j]);
    const double m = warp_max((double)nmax[j]);
    if (lane == 0) red[wid * 2 * QMAX + j] = a, red[wid * 2 * QMAX + QMAX + j] = m;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < q; j += blockDim.x) {
    double a = 0.0, m = 0.0;
    for (int w2 = 0; w2 < nw; ++w2) a += red[w2 * 2 * QMAX + j], m = fmax(m, red[w2 * 2 * QMAX + QMAX + j]);
    norm_part[(int64_t)blockIdx.x * 2 * q + j] = a;
    norm_part[(int64_t)blockIdx.x * 2 * q + q + j] = m;
  }
}

// padded rows of U for the segments of `c`
inline int stage_u_rows(const Cols<float>& c) {
  int sp = 0;
  for (int g = 0; g < c.nseg; ++g) sp += padded_rows(c.w[g]);
  return sp;
}

inline size_t stage_smem(const Cols<float>& c, int qmax, int ld) {
  return (size_t)stage_u_rows(c) * qmax * sizeof(float) +
         (size_t)kStageSlabs * kStageRows * padded_ld<float>(ld) * sizeof(float);
}

template <int QMAX, bool NORM>
int update_stage_launch(int64_t n, const UpdateJob<float>& job, int ld, const double* U, int s, int q, double alpha,
                        const double* lam, double* norm_part, int max_ctas, cudaStream_t st) {
  const int lds = padded_ld<float>(ld);
  const size_t smem = stage_smem(job.in[0], QMAX, ld);
  // set once per process; function-local statics initialise thread-safely
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(update_stage_kernel<QMAX, NORM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024));
    return true;
  }();
  (void)attr;
  // the rows of each CTA and thread as in update_row_launch
  int64_t ctas = std::min<int64_t>(max_ctas, ceil_div(n, kStageRows));
  if (ctas < 1) ctas = 1;
  const int64_t rpc = ceil_div(n, ctas);
  ctas = std::max<int64_t>(1, ceil_div(n, rpc));
  update_stage_kernel<QMAX, NORM><<<(unsigned)ctas, kStageRows, smem, st>>>(n, job, ld, lds, U, s, q, alpha, lam,
                                                                           norm_part, rpc);
  LB_LAUNCH_CHECK();
  return (int)ctas;
}

template <bool NORM>
int update_stage_dispatch(int64_t n, const UpdateJob<float>& job, int ld, const double* U, int s, int q,
                          double alpha, const double* lam, double* norm_part, int max_ctas, cudaStream_t st) {
  if (q <= 8) return update_stage_launch<8, NORM>(n, job, ld, U, s, q, alpha, lam, norm_part, max_ctas, st);
  if (q <= 16) return update_stage_launch<16, NORM>(n, job, ld, U, s, q, alpha, lam, norm_part, max_ctas, st);
  if (q <= 24) return update_stage_launch<24, NORM>(n, job, ld, U, s, q, alpha, lam, norm_part, max_ctas, st);
  return update_stage_launch<32, NORM>(n, job, ld, U, s, q, alpha, lam, norm_part, max_ctas, st);
}

int count_tiles(int pa, int pb, int TI, int TJ, bool upper) {
  const int nti = (pa + TI - 1) / TI, ntj = (pb + TJ - 1) / TJ;
  int ntiles = 0;
  for (int tj = 0; tj < ntj; ++tj)
    for (int ti = 0; ti < nti; ++ti)
      if (!upper || ti * TI <= tj * TJ + TJ - 1) ++ntiles;
  return ntiles;
}

template <class T>
bool aligned(const Cols<T>& c, int ld) {
  for (int g = 0; g < c.nseg; ++g)
    if (c.ld[g] != ld || (reinterpret_cast<uintptr_t>(c.p[g]) & 15)) return false;
  return (ld * sizeof(T)) % 16 == 0;
}

template <class T, int TI, int TJ, int R, int S>
int gram_pipe_launch(int64_t n, const Cols<T>& a, const Cols<T>& b, int ld, bool upper, double* part,
                     int max_ctas, cudaStream_t st) {
  const int pa = a.width(), pb = b.width();
  const int ntiles = count_tiles(pa, pb, TI, TJ, upper);
  const int threads = 256;
  const int groups = std::max(1, threads / ntiles);
  const int lds = padded_ld<T>(ld);
  const size_t ring = (size_t)S * (a.nseg + b.nseg) * R * lds * sizeof(T);
  const size_t red = (size_t)ntiles * TI * TJ * sizeof(double);
  const size_t smem = std::max(ring, red);
  // set once per process; function-local statics initialise thread-safely
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(gram_pipe_kernel<T, TI, TJ, R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024));
    return true;
  }();
  (void)attr;
  int64_t ctas = std::min<int64_t>(max_ctas, ceil_div(n, R));
  if (ctas < 1) ctas = 1;
  const int64_t rpc = (ceil_div(n, ctas) + R - 1) / R * R;
  ctas = std::max<int64_t>(1, ceil_div(n, rpc));
  gram_pipe_kernel<T, TI, TJ, R, S><<<(unsigned)ctas, threads, smem, st>>>(n, a, b, ld, upper ? 1 : 0, ntiles,
                                                                          groups, part, rpc);
  LB_LAUNCH_CHECK();
  return (int)ctas;
}

template <int TI, int TJ, int R, int S>
int gram_df_launch(int64_t n, const Cols<double>& a, const Cols<double>& b, int ld, bool upper, double* part,
                   int max_ctas, cudaStream_t st) {
  const int pa = a.width(), pb = b.width();
  const int ntiles = count_tiles(pa, pb, TI, TJ, upper);
  const int threads = ntiles > 128 ? 512 : 256;
  const int groups = std::max(1, threads / ntiles);
  // about 128 rows per thread between the FP64 flushes of its double-float sums
  const int flush = std::max(1, 128 * groups / R);
  const int lds = padded_ld<double>(ld);
  const size_t ring = (size_t)S * (a.nseg + b.nseg) * R * lds * sizeof(double);
  const size_t red = (size_t)ntiles * TI * TJ * sizeof(double);
  const size_t smem = std::max(ring, red);
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(gram_df_kernel<TI, TJ, R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024));
    return true;
  }();
  (void)attr;
  int64_t ctas = std::min<int64_t>(max_ctas, ceil_div(n, R));
  if (ctas < 1) ctas = 1;
  const int64_t rpc = (ceil_div(n, ctas) + R - 1) / R * R;
  ctas = std::max<int64_t>(1, ceil_div(n, rpc));
  gram_df_kernel<TI, TJ, R, S><<<(unsigned)ctas, threads, smem, st>>>(n, a, b, ld, upper ? 1 : 0, ntiles, groups,
                                                                      flush, part, rpc);
  LB_LAUNCH_CHECK();
  return (int)ctas;
}

}  // namespace

// Double-float FP64 Gram partials (same layout and contract as gram_partials_pipe<double>);
// returns 0 when the operands do not share one aligned row stride or do not fit.
int gram_partials_df(int64_t n, const Cols<double>& a, const Cols<double>& b, bool upper, double* part,
                     int max_ctas, cudaStream_t st) {
  if (a.nseg == 0 || b.nseg == 0) return 0;
  const int ld = a.ld[0];
  if (!aligned(a, ld) || !aligned(b, ld)) return 0;
  const int pa = a.width(), pb = b.width();
  if (pa > kMaxS || pb > kMaxS) return 0;
  const size_t ring = (size_t)2 * (a.nseg + b.nseg) * 32 * padded_ld<double>(ld) * sizeof(double);
  if (ring > 190 * 1024) return 0;
  if (count_tiles(pa, pb, 4, 4, upper) <= 512) return gram_df_launch<4, 4, 32, 2>(n, a, b, ld, upper, part, max_ctas, st);
  return 0;
}

// Pipelined Gram partials; returns 0 (nothing launched) when the operands do not share
// one aligned row stride, so the caller can use the general kernel instead.
template <class T>
int gram_partials_pipe(int64_t n, const Cols<T>& a, const Cols<T>& b, bool upper, double* part, int max_ctas,
                       cudaStream_t st) {
  if (a.nseg == 0 || b.nseg == 0) return 0;
  const int ld = a.ld[0];
  if (!aligned(a, ld) || !aligned(b, ld)) return 0;
  const int pa = a.width(), pb = b.width();
  const size_t ring_per_stage = (size_t)(a.nseg + b.nseg) * 32 * padded_ld<T>(ld) * sizeof(T);
  if (ring_per_stage * 2 > 190 * 1024) return 0;
  if constexpr (std::is_same<T, float>::value) {
    // tensor cores (3xTF32) when the blocks fit: ring <= 200 KB at 64 rows x 2 stages
    const size_t tc_ring = (size_t)2 * (a.nseg + b.nseg) * 64 * tc_lds(ld) * sizeof(float);
    const int nblocks = ((pa + 15) / 16) * ((pb + 31) / 32);
    if (pa <= kMaxS && pb <= kMaxS && tc_ring <= 190 * 1024 && nblocks <= 24) {
      if (nblocks <= 8) return gram_tc_launch<64, 2, 1>(n, a, b, ld, upper, part, max_ctas, st);
      if (nblocks <= 16) return gram_tc_launch<64, 2, 2>(n, a, b, ld, upper, part, max_ctas, st);
      return gram_tc_launch<64, 2, 3>(n, a, b, ld, upper, part, max_ctas, st);
    }
  }
  if (sizeof(T) == 4 && pa >= 16 && pb >= 16 && count_tiles(pa, pb, 8, 8, upper) <= 256) {
    // long stages: enough rows per thread group between barriers
    const size_t stage128 = (size_t)(a.nseg + b.nseg) * 128 * padded_ld<T>(ld) * sizeof(T);
    if (stage128 * 2 <= 190 * 1024) return gram_pipe_launch<T, 8, 8, 128, 2>(n, a, b, ld, upper, part, max_ctas, st);
    return gram_pipe_launch<T, 8, 8, 32, 3>(n, a, b, ld, upper, part, max_ctas, st);
  }
  // FP64: 2 x 4 tiles (more threads on the FP64 units) when they fit the CTA, e.g. the
  // Grams of Algorithms 2 and 3; measured ~4% faster there than 4 x 4
  if (sizeof(T) == 8 && count_tiles(pa, pb, 2, 4, upper) <= 256)
    return gram_pipe_launch<T, 2, 4, 32, 2>(n, a, b, ld, upper, part, max_ctas, st);
  if (count_tiles(pa, pb, 4, 4, upper) <= 256)
    return gram_pipe_launch<T, 4, 4, 32, 2>(n, a, b, ld, upper, part, max_ctas, st);
  return 0;
}

template <class T>
int launch_update_pipe(int64_t n, const UpdateJob<T>& job, const double* U, int s, int q, double alpha,
                       const double* lam, double* norm_part, int max_ctas, cudaStream_t st) {
  if (job.in[0].nseg == 0) return 0;
  // FP64 updates are bound by the FP64 units, where the general kernel does as well
  if (sizeof(T) == 8) return 0;
  const int ld = job.in[0].ld[0];
  for (int t = 0; t < job.nprod; ++t)
    if (!aligned(job.in[t], ld) || job.in[t].nseg != job.in[0].nseg) return 0;
  // staged slabs (FP32): outputs no wider than a slab row and 32 columns, the products'
  // segments of equal widths, the norm form as the solver uses it
  if constexpr (sizeof(T) == 4) {
    bool same_w = true;
    for (int t = 1; t < job.nprod; ++t)
      for (int g = 0; g < job.in[0].nseg; ++g) same_w = same_w && job.in[t].w[g] == job.in[0].w[g];
    if (same_w && q <= 32 && q <= padded_ld<T>(ld) && s <= kMaxS && stage_smem(job.in[0], 32, ld) <= 200 * 1024) {
      if (!norm_part)
        return update_stage_dispatch<false>(n, job, ld, U, s, q, alpha, lam, norm_part, max_ctas, st);
      if (job.nprod == 2 && !job.base[0] && !job.base[1])
        return update_stage_dispatch<true>(n, job, ld, U, s, q, alpha, lam, norm_part, max_ctas, st);
    }
  }
  if (q <= 8) return update_row_launch<T, 8>(n, job, ld, U, s, q, alpha, lam, norm_part, max_ctas, st);
  if (q <= 16) return update_row_launch<T, 16>(n, job, ld, U, s, q, alpha, lam, norm_part, max_ctas, st);
  if (q <= 24) return update_row_launch<T, 24>(n, job, ld, U, s, q, alpha, lam, norm_part, max_ctas, st);
  if (q <= 32) return update_row_launch<T, 32>(n, job, ld, U, s, q, alpha, lam, norm_part, max_ctas, st);
  constexpr int RJ = 4, CJ = 4, R = 64, S = 2;
  const int lds = padded_ld<T>(ld);
  const int qpad = round_up(q, CJ);
  if (qpad / CJ * (R / RJ) > 256) return 0;
  const size_t head = (size_t)((s * qpad + 3) / 4 * 4) * sizeof(T) + (size_t)((s + 3) / 4 * 4) * sizeof(int);
  const size_t ring = (size_t)S * job.nprod * job.in[0].nseg * R * lds * sizeof(T);
  const size_t red = norm_part ? (size_t)(R / RJ) * 2 * qpad * sizeof(double) : 0;
  const size_t smem = head + std::max(ring, red) + 16;
  if (smem > 200 * 1024) return 0;
  // set once per process; function-local statics initialise thread-safely
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(update_pipe_kernel<T, RJ, CJ, R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024));
    return true;
  }();
  (void)attr;
  int64_t ctas = std::min<int64_t>(max_ctas, ceil_div(n, R));
  if (ctas < 1) ctas = 1;
  const int64_t rpc = (ceil_div(n, ctas) + R - 1) / R * R;
  ctas = std::max<int64_t>(1, ceil_div(n, rpc));
  update_pipe_kernel<T, RJ, CJ, R, S><<<(unsigned)ctas, 256, smem, st>>>(n, job, ld, U, s, q, alpha, lam, norm_part,
                                                                        rpc);
  LB_LAUNCH_CHECK();
  return (int)ctas;
}

template int gram_partials_pipe<double>(int64_t, const Cols<double>&, const Cols<double>&, bool, double*, int,
                                        cudaStream_t);
template int gram_partials_pipe<float>(int64_t, const Cols<float>&, const Cols<float>&, bool, double*, int,
                                       cudaStream_t);
template int launch_update_pipe<double>(int64_t, const UpdateJob<double>&, const double*, int, int, double,
                                        const double*, double*, int, cudaStream_t);
template int launch_update_pipe<float>(int64_t, const UpdateJob<float>&, const double*, int, int, double,
                                       const double*, double*, int, cudaStream_t);

}  // namespace lobpcg
