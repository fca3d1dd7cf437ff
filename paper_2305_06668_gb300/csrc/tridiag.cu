// Tridiagonal preconditioner (Sec. 4.4): W[:, c] = (T - lambda_{c0+c} I)^{-1} r_{c0+c}, with
// T the diagonal and first off-diagonals of A and r = AX - X lambda formed on the fly.
//
// The n-row solve is split into partitions of L rows (a SPIKE-type scheme, Polizzi and
// Sameh, 2006), L a power of two from 32 to 1024, the largest that still gives every SM
// a few warps of (partition, column) threads.  With M = T - lambda I and M_p the block of partition p:
//   1. per (partition, column): Gaussian elimination with partial pivoting of M_p (the
//      scheme of LAPACK's tridiagonal solver, rows interchanged with their neighbour, a
//      second super-diagonal as fill-in) for three right-hand sides: r_p, a_p e_1 and
//      c_p e_L, where a_p = M[s, s-1] and c_p = M[e-1, e] couple the partition [s, e) to
//      its neighbours.  The solutions y, v, w give x_p = y - x_{s-1} v - x_e w.
//   2. per column: the interface unknowns z_k = (x_last(k), x_first(k+1)) satisfy a block
//      tridiagonal system with 2 x 2 blocks, solved by block elimination in order.
//   3. per (row, column): x = y - x_{s-1} v - x_e w.
// Pivots below 1e-8 max(1, |lambda|) in magnitude are replaced by that value with their
// sign (the guard of the diagonal preconditioner).  The solve runs in FP32 in both
// precisions: a preconditioner only shapes the search direction W~, which Algorithm 3
// then orthonormalises in the block's precision.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace lobpcg {
namespace {

constexpr int kTriLMin = 32, kTriLMax = 1024;  // rows per partition
constexpr int64_t kTriThreads = 152 * 128;     // (partition, column) threads wanted

__device__ __forceinline__ float guard(float v, float fl) { return fabsf(v) < fl ? (v >= 0.f ? fl : -fl) : v; }

// scratch layout, per row i and column c: slot t in [0, 6) at S[(i * 6 + t) * a + c];
// during the elimination slots hold (pivot, u1, u2, rhs0, rhs1, rhs2), after the back
// substitution slots 3..5 hold (y, v, w)
template <class T>
__global__ void __launch_bounds__(256) tri_partition_kernel(int64_t n, int64_t P, int L, const T* __restrict__ X,
                                                            const T* __restrict__ AX, int ld,
                                                            const double* __restrict__ lam, int c0, int a,
                                                            const double* __restrict__ d,
                                                            const double* __restrict__ dl,
                                                            const double* __restrict__ du, float* __restrict__ S,
                                                            float* __restrict__ tips) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= P * a) return;
  const int c = (int)(tid % a);
  const int64_t p = tid / a;
  const int64_t s0 = p * L, e0 = min(n, s0 + L);
  const double th = lam[c0 + c];
  const float fl = (float)(1e-8 * fmax(1.0, fabs(th)));
  auto res = [&](int64_t i) -> float {
    const T ax = AX[i * ld + c0 + c];
    return X ? (float)(ax - (T)th * X[i * ld + c0 + c]) : (float)ax;
  };
  float* Sc = S + c;
  const int64_t sa = 6 * (int64_t)a;
  // current row (columns i, i+1; its column i+2 entry is zero) and its right-hand sides
  float piv = (float)(d[s0] - th);
  float u1 = s0 + 1 < e0 ? (float)du[s0] : 0.f;
  float r0 = res(s0), r1 = p > 0 ? (float)dl[s0 - 1] : 0.f, r2 = 0.f;
  const float cp = e0 < n ? (float)du[e0 - 1] : 0.f;
  if (e0 - s0 == 1) r2 = cp;
  for (int64_t i = s0; i + 1 < e0; ++i) {
    // next row i+1: (sub, nd, nu1) in columns (i, i+1, i+2)
    const float sub = (float)dl[i];
    float nd = (float)(d[i + 1] - th);
    float nu1 = i + 2 < e0 ? (float)du[i + 1] : 0.f;
    float q0 = res(i + 1), q1 = 0.f, q2 = i + 2 == e0 ? cp : 0.f;
    float fp, fu1, fu2, f0, f1, f2;  // final row i
    if (fabsf(piv) >= fabsf(sub)) {
      piv = guard(piv, fl);
      const float f = sub / piv;
      fp = piv, fu1 = u1, fu2 = 0.f, f0 = r0, f1 = r1, f2 = r2;
      nd = fmaf(-f, u1, nd);
      q0 = fmaf(-f, r0, q0), q1 = fmaf(-f, r1, q1), q2 = fmaf(-f, r2, q2);
    } else {
      // interchange: row i becomes (sub, nd, nu1), the old row i minus f times it follows
      const float pv = guard(sub, fl);
      const float f = piv / pv;
      fp = pv, fu1 = nd, fu2 = nu1, f0 = q0, f1 = q1, f2 = q2;
      const float t0 = r0, t1 = r1, t2 = r2;
      nd = fmaf(-f, nd, u1);
      nu1 = -f * nu1;
      q0 = fmaf(-f, f0, t0), q1 = fmaf(-f, f1, t1), q2 = fmaf(-f, f2, t2);
    }
    float* row = Sc + i * sa;
    row[0] = fp, row[a] = fu1, row[2 * a] = fu2, row[3 * a] = f0, row[4 * a] = f1, row[5 * a] = f2;
    piv = nd, u1 = nu1, r0 = q0, r1 = q1, r2 = q2;
  }
  piv = guard(piv, fl);
  // back substitution, last row first
  float x0 = r0 / piv, x1 = r1 / piv, x2 = r2 / piv;  // row e0-1
  {
    float* row = Sc + (e0 - 1) * sa;
    row[3 * a] = x0, row[4 * a] = x1, row[5 * a] = x2;
  }
  float y0n = x0, y1n = x1, y2n = x2;     // solution at row i+1
  float y0nn = 0.f, y1nn = 0.f, y2nn = 0.f;  // at row i+2
  for (int64_t i = e0 - 2; i >= s0; --i) {
    float* row = Sc + i * sa;
    const float pp = row[0], a1 = row[a], a2 = row[2 * a];
    const float z0 = (row[3 * a] - a1 * y0n - a2 * y0nn) / pp;
    const float z1 = (row[4 * a] - a1 * y1n - a2 * y1nn) / pp;
    const float z2 = (row[5 * a] - a1 * y2n - a2 * y2nn) / pp;
    row[3 * a] = z0, row[4 * a] = z1, row[5 * a] = z2;
    y0nn = y0n, y1nn = y1n, y2nn = y2n;
    y0n = z0, y1n = z1, y2n = z2;
  }
  // tips: y, v, w at the first and the last row of the partition
  float* tp = tips + (p * a + c) * 6;
  const float* first = Sc + s0 * sa;
  const float* last = Sc + (e0 - 1) * sa;
  tp[0] = first[3 * a], tp[1] = last[3 * a];
  tp[2] = first[4 * a], tp[3] = last[4 * a];
  tp[4] = first[5 * a], tp[5] = last[5 * a];
}

// Reduced system of one column c (one CTA per column): for k = 0 .. P-2, z_k = (u_k,
// t_{k+1}) = (x at the last row of partition k, x at the first row of partition k+1):
//   u_k + wL_k t_{k+1} + vL_k u_{k-1}         = yL_k
//   v0_{k+1} u_k + t_{k+1} + w0_{k+1} t_{k+2} = y0_{k+1}
// (L: last row of partition k, 0: first row of partition k+1).  Block elimination in order
// keeps B'_k = [[1, b01], [b10, 1]] and f'_k (fwd: b01, b10, f'_k[0]; f'_k[1] waits in z),
// then the back substitution z_k = B'_k^{-1} (f'_k - (0, w0_{k+1} t_{k+2})).  The CTA stages
// chunks of kRedChunk interfaces in shared memory and one thread runs the recurrence.
constexpr int kRedChunk = 256;

__device__ __forceinline__ float safe_det(float b01, float b10) {
  const float det = 1.f - b01 * b10;
  return fabsf(det) < 1e-30f ? (det >= 0.f ? 1e-30f : -1e-30f) : det;
}

__global__ void __launch_bounds__(256) tri_reduced_kernel(int64_t P, int a, const float* __restrict__ tips,
                                                          float* __restrict__ fwd, float* __restrict__ z) {
  __shared__ float sh[(kRedChunk + 1) * 6];
  const int c = blockIdx.x;
  const int64_t K = P - 1;  // interfaces
  float ib00 = 0.f, ib01 = 0.f, fp0 = 0.f, fp1 = 0.f;  // first row of B'_{k-1}^{-1}, and f'_{k-1}
  for (int64_t k0 = 0; k0 < K; k0 += kRedChunk) {
    const int cnt = (int)min((int64_t)kRedChunk, K - k0);  // interfaces k0 .. k0 + cnt - 1
    for (int t = threadIdx.x; t < (cnt + 1) * 6; t += blockDim.x)
      sh[t] = tips[((k0 + t / 6) * a + c) * 6 + t % 6];  // partitions k0 .. k0 + cnt
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int j = 0; j < cnt; ++j) {
        const int64_t k = k0 + j;
        const float* tk = sh + j * 6;        // partition k
        const float* tn = sh + (j + 1) * 6;  // partition k+1
        float b01 = tk[5], f0 = tk[1];
        const float b10 = tn[2], f1 = tn[0];
        if (k > 0) {
          const float al = tk[3], ga = tk[4];  // vL_k (coefficient of u_{k-1}); w0_k
          b01 = fmaf(-al * ib01, ga, b01);
          f0 = f0 - al * (ib00 * fp0 + ib01 * fp1);
        }
        const float det = safe_det(b01, b10);
        ib00 = 1.f / det, ib01 = -b01 / det;
        fp0 = f0, fp1 = f1;
        float* fw = fwd + (k * a + c) * 3;
        fw[0] = b01, fw[1] = b10, fw[2] = f0;
        z[(k * a + c) * 2 + 1] = f1;
      }
    }
    __syncthreads();
  }
  // back substitution, chunks from the end; each chunk needs fwd, f'_k[1] and w0_{k+1}
  float tnext = 0.f;  // t_{k+2}
  for (int64_t k1 = K; k1 > 0; k1 -= kRedChunk) {
    const int64_t k0 = max((int64_t)0, k1 - kRedChunk);
    const int cnt = (int)(k1 - k0);
    for (int t = threadIdx.x; t < cnt * 5; t += blockDim.x) {
      const int64_t k = k0 + t / 5;
      const int q = t % 5;
      float v;
      if (q < 3) v = fwd[(k * a + c) * 3 + q];
      else if (q == 3) v = z[(k * a + c) * 2 + 1];
      else v = tips[((k + 1) * a + c) * 6 + 4];  // w0_{k+1}
      sh[t] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int j = cnt - 1; j >= 0; --j) {
        const int64_t k = k0 + j;
        const float* e = sh + j * 5;
        const float b01 = e[0], b10 = e[1], f0 = e[2];
        float f1 = e[3];
        if (k + 2 < P) f1 -= e[4] * tnext;
        const float det = safe_det(b01, b10);
        const float u = (f0 - b01 * f1) / det, t = (f1 - b10 * f0) / det;
        z[(k * a + c) * 2 + 0] = u;
        z[(k * a + c) * 2 + 1] = t;
        tnext = t;
      }
    }
    __syncthreads();
  }
}

// x = y - u_{p-1} v - t_{p+1} w for every (row, column).
template <class T>
__global__ void tri_combine_kernel(int64_t n, int64_t P, int L, int a, const float* __restrict__ S,
                                   const float* __restrict__ z, T* __restrict__ W, int ldw) {
  const int64_t total = n * a;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / a;
    const int c = (int)(e - i * a);
    const int64_t p = i / L;
    const float* row = S + i * 6 * (int64_t)a + c;
    float x = row[3 * a];
    if (p > 0) x -= z[((p - 1) * a + c) * 2 + 0] * row[4 * a];
    if (p + 1 < P) x -= z[(p * a + c) * 2 + 1] * row[5 * a];
    W[i * ldw + c] = (T)x;
  }
}

__global__ void tri_extract_csr_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                       const double* __restrict__ val, double* __restrict__ dl,
                                       double* __restrict__ du) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i + 1 < n; i += (int64_t)gridDim.x * blockDim.x) {
    double lo = 0.0, up = 0.0;
    for (int64_t e = rp[i + 1]; e < rp[i + 2]; ++e)
      if (ci[e] == i) lo += val[e];
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
      if (ci[e] == i + 1) up += val[e];
    dl[i] = lo;
    du[i] = up;
  }
}

__global__ void tri_extract_dense_kernel(int64_t n, const double* __restrict__ A, int64_t lda,
                                         double* __restrict__ dl, double* __restrict__ du) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i + 1 < n; i += (int64_t)gridDim.x * blockDim.x) {
    dl[i] = A[i * lda + (i + 1)];  // column i, row i+1 (column-major)
    du[i] = A[(i + 1) * lda + i];  // column i+1, row i
  }
}

unsigned blocks_for(int64_t work, int threads) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, 152 * 64));
}

}  // namespace

// Partition length for n rows and a columns: halved from kTriLMax while fewer than
// kTriThreads (partition, column) pairs result, down to kTriLMin.
int tridiag_partition_rows(int64_t n, int a) {
  int L = kTriLMax;
  while (L > kTriLMin && (n + L - 1) / L * a < kTriThreads) L /= 2;
  return L;
}

int64_t tridiag_partitions(int64_t n) { return (n + kTriLMin - 1) / kTriLMin; }  // the most there can be

size_t tridiag_scratch_floats(int64_t n, int a) {
  const int64_t P = tridiag_partitions(n);
  return (size_t)n * 6 * a + (size_t)P * a * (6 + 3 + 2);
}

void tridiag_extract(int64_t n, const int64_t* rp, const int32_t* ci, const double* val, const double* dense,
                     int64_t lda, double* dl, double* du, cudaStream_t st) {
  if (n < 2) return;
  if (dense)
    tri_extract_dense_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, dense, lda, dl, du);
  else
    tri_extract_csr_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, rp, ci, val, dl, du);
  LB_LAUNCH_CHECK();
}

template <class T>
void launch_precond_tridiag(int64_t n, const T* X, const T* AX, int ld, const double* lam, int c0, int a,
                            const double* d, const double* dl, const double* du, T* W, int ldw, float* scratch,
                            cudaStream_t st) {
  if (n <= 0 || a <= 0) return;
  const int L = tridiag_partition_rows(n, a);
  const int64_t P = (n + L - 1) / L;
  float* S = scratch;
  float* tips = S + (size_t)n * 6 * a;
  float* fwd = tips + (size_t)P * a * 6;
  float* z = fwd + (size_t)P * a * 3;
  const int64_t work = P * a;
  tri_partition_kernel<T><<<(unsigned)((work + 127) / 128), 128, 0, st>>>(n, P, L, X, AX, ld, lam, c0, a, d, dl,
                                                                        du, S, tips);
  LB_LAUNCH_CHECK();
  if (P > 1) {
    tri_reduced_kernel<<<(unsigned)a, 256, 0, st>>>(P, a, tips, fwd, z);
    LB_LAUNCH_CHECK();
  }
  tri_combine_kernel<T><<<blocks_for(n * a, 256), 256, 0, st>>>(n, P, L, a, S, z, W, ldw);
  LB_LAUNCH_CHECK();
}

template void launch_precond_tridiag<double>(int64_t, const double*, const double*, int, const double*, int, int,
                                             const double*, const double*, const double*, double*, int, float*,
                                             cudaStream_t);
template void launch_precond_tridiag<float>(int64_t, const float*, const float*, int, const double*, int, int,
                                            const double*, const double*, const double*, float*, int, float*,
                                            cudaStream_t);

}  // namespace lobpcg
