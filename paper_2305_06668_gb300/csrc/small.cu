// Small FP64 kernels, one CTA each: the Rayleigh-Ritz eigensolve (parallel-order
// Jacobi), the Cholesky-QR step with level shift / SVQB fallback (Algorithm 2, Sec. 3.2),
// the lock decision and the P coefficients u_p = ortho(u~_p; u_x) (Algorithm 1, Sec.
// 3.1), all in shared memory.
#include <cfloat>

#include "common.cuh"

namespace lobpcg {
namespace {

constexpr int kSmallThreads = 512;
constexpr int kMaxCholP = 64;  // largest block orthonormalised by the Cholesky-QR kernel

// Block-wide reductions (all threads must call; result returned to every thread).
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}
__device__ double block_max(double v, double* red) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s = fmax(s, red[i]);
  __syncthreads();
  return s;
}

// Pairs of one parallel-order round (circle method, player N-1 fixed): pair i of round r
// is (p, q) with p < q; q may be the dummy player s when s is odd.
__device__ __forceinline__ void round_pair(int N, int r, int i, int& p, int& q) {
  const int M = N - 1;  // r < M, 0 < i < N / 2: one correction brings r +- i into [0, M)
  if (i == 0) {
    p = M, q = r;
  } else {
    p = r + i, q = r - i;
    if (p >= M) p -= M;
    if (q < 0) q += M;
  }
  if (p > q) { const int t = p; p = q; q = t; }
}

// Pair blocks of a round: item e -> (i1, i2), i1 <= i2, the upper triangle of the
// half x half grid of pair blocks in row-major order, as i1 << 8 | i2 (table filled once
// per call; half <= 48).
constexpr int kMaxBlk = (kMaxS / 2) * (kMaxS / 2 + 1) / 2;
__shared__ unsigned short g_blk[kMaxBlk];  // one per CTA, shared by the Jacobi routines of a kernel
__device__ void fill_blocks(int half, unsigned short* blk) {
  for (int i1 = threadIdx.x; i1 < half; i1 += blockDim.x) {
    const int base = i1 * half - i1 * (i1 - 1) / 2;  // items of the rows before i1
    for (int i2 = i1; i2 < half; ++i2) blk[base + i2 - i1] = (unsigned short)(i1 << 8 | i2);
  }
  __syncthreads();
}

// Parallel-order (round-robin) cyclic Jacobi on the symmetric s x s matrix a (column-
// major, leading dimension lda, overwritten by its rotated form) accumulating the
// rotations in V (s x s, ldv; set to the identity first when init_v).  Each round applies
// s/2 disjoint rotations (classical smaller-angle rotation of Golub & Van Loan, Sec. 8.5)
// as J^T A J, in the arithmetic of T.  A round is two phases: the rotation of every pair,
// then one pass that maps every 2 x 2 block of a between two pairs (rows of pair i1,
// columns of pair i2; the upper triangle of blocks, mirrored, so a stays exactly
// symmetric) to R_i1^T a_blk R_i2, rows first then columns, with the pair's own
// off-diagonal entry set to zero, together with columns p, q of V.  Stops when
// off(a) <= rel_tol * ||a||_F.  Returns the number of sweeps, or -1 without convergence
// in max_sweeps.
template <class T>
__device__ int jacobi_sweeps(int s, T* a, int lda, T* V, int ldv, T* rot, double* red, double rel_tol,
                             int max_sweeps, bool init_v) {
  const int N = s + (s & 1);
  const int half = N / 2;
  const int nblk = half * (half + 1) / 2;
  unsigned short* blk = g_blk;
  fill_blocks(half, blk);
  __shared__ int rpq[kMaxS / 2];
  // (pair, row) items of V as e = pair * sp + row with sp = pow2 >= s (shifts, no division)
  const int sh = s <= 32 ? 5 : (s <= 64 ? 6 : 7), sp = 1 << sh;
  if (init_v)
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
      const int i = e % s, j = e / s;
      V[i + j * ldv] = i == j ? T(1) : T(0);
    }
  double f2 = 0.0;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const double v = a[(e % s) + (e / s) * lda];
    f2 += v * v;
  }
  const double fro = sqrt(block_sum(f2, red));
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double o2 = 0.0;
    for (int e = threadIdx.x; e < (s << sh); e += blockDim.x) {
      const int i = e & (sp - 1), j = e >> sh;
      if (i < s && i != j) {
        const double v = a[i + j * lda];
        o2 += v * v;
      }
    }
    const double off = sqrt(block_sum(o2, red));
    if (off <= rel_tol * fro || off == 0.0) return sweep;
    for (int r = 0; r < N - 1; ++r) {
      // phase A: rotation of every pair of this round (identity for a dummy or zero pair);
      // rpq[i] = p << 8 | q, bit 16 set when the pair rotates
      for (int i = threadIdx.x; i < half; i += blockDim.x) {
        int p, q;
        round_pair(N, r, i, p, q);
        T c = T(1), sn = T(0);
        bool rotate = false;
        if (q < s) {
          const T apq = a[p + q * lda];
          if (apq != T(0)) {
            const T tau = (a[q + q * lda] - a[p + p * lda]) / (T(2) * apq);
            const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
            c = T(1) / sqrt(T(1) + t * t);
            sn = t * c;
            rotate = true;
          }
        }
        rpq[i] = p << 8 | q | (rotate ? 1 << 16 : 0);
        rot[2 * i + 0] = c;
        rot[2 * i + 1] = sn;
      }
      __syncthreads();
      // phase B: the blocks of a, then columns p, q of V (V J).  Items touch disjoint
      // entries, so in FP64 a thread loads all of its (up to four) items before it stores
      // any (the loads overlap the long FP64 latencies); in FP32 one item at a time is
      // faster (measured at s = 63: 3.4k against 5.2k cycles per round)
      const int total = nblk + (half << sh);
      if constexpr (sizeof(T) == 4) {
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
          if (e < nblk) {
            const int i1 = blk[e] >> 8, i2 = blk[e] & 255;
            const int m1 = rpq[i1], m2 = rpq[i2];
            if (!((m1 | m2) & (1 << 16))) continue;
            const int p1 = (m1 >> 8) & 255, q1 = m1 & 255, p2 = (m2 >> 8) & 255, q2 = m2 & 255;
            const T c1 = rot[2 * i1], s1 = rot[2 * i1 + 1], c2 = rot[2 * i2], s2 = rot[2 * i2 + 1];
            const bool v1 = q1 < s, v2 = q2 < s;
            const T x00 = a[p1 + p2 * lda], x01 = v2 ? a[p1 + q2 * lda] : T(0);
            const T x10 = v1 ? a[q1 + p2 * lda] : T(0), x11 = v1 && v2 ? a[q1 + q2 * lda] : T(0);
            const T r00 = c1 * x00 - s1 * x10, r01 = c1 * x01 - s1 * x11;
            const T r10 = s1 * x00 + c1 * x10, r11 = s1 * x01 + c1 * x11;
            T n00 = c2 * r00 - s2 * r01, n01 = s2 * r00 + c2 * r01;
            T n10 = c2 * r10 - s2 * r11, n11 = s2 * r10 + c2 * r11;
            if (i1 == i2) {
              n01 = n10 = T(0);
              a[p1 + p1 * lda] = n00;
              if (v1) a[q1 + q1 * lda] = n11, a[p1 + q1 * lda] = n01, a[q1 + p1 * lda] = n10;
              continue;
            }
            a[p1 + p2 * lda] = n00, a[p2 + p1 * lda] = n00;
            if (v2) a[p1 + q2 * lda] = n01, a[q2 + p1 * lda] = n01;
            if (v1) a[q1 + p2 * lda] = n10, a[p2 + q1 * lda] = n10;
            if (v1 && v2) a[q1 + q2 * lda] = n11, a[q2 + q1 * lda] = n11;
          } else {
            const int f = e - nblk, i = f >> sh, j = f & (sp - 1);
            const int m = rpq[i];
            if (j >= s || !(m & (1 << 16))) continue;
            const int p = (m >> 8) & 255, q = m & 255;
            const T c = rot[2 * i], sn = rot[2 * i + 1];
            const T vjp = V[j + p * ldv], vjq = V[j + q * ldv];
            V[j + p * ldv] = c * vjp - sn * vjq;
            V[j + q * ldv] = sn * vjp + c * vjq;
          }
        }
      } else
      for (int e0 = threadIdx.x; e0 < total; e0 += 4 * blockDim.x) {
        int kind[4], m1[4], m2[4];
        T x[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int e = e0 + k * blockDim.x;
          kind[k] = 0;
          if (e < nblk) {
            const int i1 = blk[e] >> 8, i2 = blk[e] & 255;
            m1[k] = rpq[i1], m2[k] = rpq[i2];
            if (!((m1[k] | m2[k]) & (1 << 16))) continue;  // both identity
            kind[k] = 1 + (i1 == i2);
            const int p1 = (m1[k] >> 8) & 255, q1 = m1[k] & 255, p2 = (m2[k] >> 8) & 255, q2 = m2[k] & 255;
            const bool v1 = q1 < s, v2 = q2 < s;
            x[k][0] = a[p1 + p2 * lda];
            x[k][1] = v2 ? a[p1 + q2 * lda] : T(0);
            x[k][2] = v1 ? a[q1 + p2 * lda] : T(0);
            x[k][3] = v1 && v2 ? a[q1 + q2 * lda] : T(0);
            m1[k] |= i1 << 17, m2[k] |= i2 << 17;
          } else if (e < total) {
            const int f = e - nblk, i = f >> sh, j = f & (sp - 1);
            m1[k] = rpq[i];
            if (j >= s || !(m1[k] & (1 << 16))) continue;
            kind[k] = 3;
            const int p = (m1[k] >> 8) & 255, q = m1[k] & 255;
            x[k][0] = V[j + p * ldv], x[k][1] = V[j + q * ldv];
            m1[k] |= i << 17, m2[k] = j;
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (kind[k] == 0) continue;
          if (kind[k] == 3) {
            const int i = m1[k] >> 17, j = m2[k], p = (m1[k] >> 8) & 255, q = m1[k] & 255;
            const T c = rot[2 * i], sn = rot[2 * i + 1];
            V[j + p * ldv] = c * x[k][0] - sn * x[k][1];
            V[j + q * ldv] = sn * x[k][0] + c * x[k][1];
            continue;
          }
          const int i1 = m1[k] >> 17, i2 = m2[k] >> 17;
          const int p1 = (m1[k] >> 8) & 255, q1 = m1[k] & 255, p2 = (m2[k] >> 8) & 255, q2 = m2[k] & 255;
          const T c1 = rot[2 * i1], s1 = rot[2 * i1 + 1], c2 = rot[2 * i2], s2 = rot[2 * i2 + 1];
          const bool v1 = q1 < s, v2 = q2 < s;
          // rows (J_1^T), then columns (J_2)
          const T r00 = c1 * x[k][0] - s1 * x[k][2], r01 = c1 * x[k][1] - s1 * x[k][3];
          const T r10 = s1 * x[k][0] + c1 * x[k][2], r11 = s1 * x[k][1] + c1 * x[k][3];
          T n00 = c2 * r00 - s2 * r01, n01 = s2 * r00 + c2 * r01;
          T n10 = c2 * r10 - s2 * r11, n11 = s2 * r10 + c2 * r11;
          if (kind[k] == 2) {  // the pair's own block: its off-diagonal entry is annihilated
            if (m1[k] & (1 << 16)) n01 = n10 = T(0);
            a[p1 + p1 * lda] = n00;
            if (v1) a[q1 + q1 * lda] = n11, a[p1 + q1 * lda] = n01, a[q1 + p1 * lda] = n10;
            continue;
          }
          a[p1 + p2 * lda] = n00, a[p2 + p1 * lda] = n00;
          if (v2) a[p1 + q2 * lda] = n01, a[q2 + p1 * lda] = n01;
          if (v1) a[q1 + p2 * lda] = n10, a[p2 + q1 * lda] = n10;
          if (v1 && v2) a[q1 + q2 * lda] = n11, a[q2 + q1 * lda] = n11;
        }
      }
      __syncthreads();
    }
  }
  return -1;
}

// Jacobi polish of a nearly diagonal symmetric matrix a = diag(d) + E, |E| small against
// ||a||: the rotations run in FP32 on E (ld lde), which stays small whatever the angle, so
// FP32 adds errors of order 6e-8 |E| there.  The diagonal d, the rotation parameters and
// Dl = V - I (ld ldd), the rotation product accumulated so far, stay in FP64.  Dl must be
// FP64 because the angles inside a cluster of eigenvalues are not small.  Dl must hold
// zeros on entry.  Rounds as in jacobi_sweeps: the pair rotations (with d updated), then
// one pass over the 2 x 2 blocks of E between different pairs and columns p, q of Dl.
// Stops when off(E) <= rel_tol * fro.  Returns the sweeps done, or -1.
__device__ int jacobi_polish(int s, double* d, float* E, int lde, double* Dl, int ldd, double* rot, double* red,
                             double rel_tol, double fro, int max_sweeps) {
  const int N = s + (s & 1);
  const int half = N / 2;
  const int nblk = half * (half + 1) / 2;
  unsigned short* blk = g_blk;
  fill_blocks(half, blk);
  __shared__ int rpq[kMaxS / 2];
  __shared__ float rcs[kMaxS];
  const int sh = s <= 32 ? 5 : (s <= 64 ? 6 : 7), sp = 1 << sh;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double o2 = 0.0;
    for (int e = threadIdx.x; e < (s << sh); e += blockDim.x) {
      const int i = e & (sp - 1), j = e >> sh;
      if (i < s && i != j) {
        const double v = E[i + j * lde];
        o2 += v * v;
      }
    }
    const double off = sqrt(block_sum(o2, red));
    if (off <= rel_tol * fro || off == 0.0) return sweep;
    for (int r = 0; r < N - 1; ++r) {
      // rpq[i] = p << 8 | q (bit 16: the pair rotates); rot[3i ..] = c - 1, c, s in FP64 and
      // rcs[2i ..] = c, s in FP32; the diagonal is updated here
      for (int i = threadIdx.x; i < half; i += blockDim.x) {
        int p, q;
        round_pair(N, r, i, p, q);
        double c = 1.0, sn = 0.0, cm1 = 0.0;
        bool rotate = false;
        if (q < s) {
          const double apq = (double)E[p + q * lde];
          if (apq != 0.0) {
            const double tau = (d[q] - d[p]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
            d[p] -= t * apq;
            d[q] += t * apq;
            cm1 = -sn * sn / (1.0 + c);  // c - 1 without cancellation, once per pair
            rotate = true;
          }
        }
        rpq[i] = p << 8 | q | (rotate ? 1 << 16 : 0);
        rot[3 * i + 0] = cm1;
        rot[3 * i + 1] = c;
        rot[3 * i + 2] = sn;
        rcs[2 * i + 0] = (float)c;
        rcs[2 * i + 1] = (float)sn;
      }
      __syncthreads();
      // blocks of E between different pairs (the pair's own entry is annihilated; d was
      // updated above), then columns p, q of Dl; loads of up to four items before stores
      const int total = nblk + (half << sh);
      for (int e0 = threadIdx.x; e0 < total; e0 += 4 * blockDim.x) {
        int kind[4], m1[4], m2[4];
        float x[4][4];
        double y[4][2];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int e = e0 + k * blockDim.x;
          kind[k] = 0;
          if (e < nblk) {
            const int i1 = blk[e] >> 8, i2 = blk[e] & 255;
            m1[k] = rpq[i1], m2[k] = rpq[i2];
            if (!((m1[k] | m2[k]) & (1 << 16))) continue;
            const int p1 = (m1[k] >> 8) & 255, q1 = m1[k] & 255, p2 = (m2[k] >> 8) & 255, q2 = m2[k] & 255;
            m1[k] |= i1 << 17, m2[k] |= i2 << 17;
            if (i1 == i2) {
              kind[k] = 2;
              continue;
            }
            kind[k] = 1;
            const bool v1 = q1 < s, v2 = q2 < s;
            x[k][0] = E[p1 + p2 * lde];
            x[k][1] = v2 ? E[p1 + q2 * lde] : 0.f;
            x[k][2] = v1 ? E[q1 + p2 * lde] : 0.f;
            x[k][3] = v1 && v2 ? E[q1 + q2 * lde] : 0.f;
          } else if (e < total) {
            const int f = e - nblk, i = f >> sh, j = f & (sp - 1);
            m1[k] = rpq[i];
            if (j >= s || !(m1[k] & (1 << 16))) continue;
            kind[k] = 3;
            const int p = (m1[k] >> 8) & 255, q = m1[k] & 255;
            y[k][0] = Dl[j + p * ldd], y[k][1] = Dl[j + q * ldd];
            m1[k] |= i << 17, m2[k] = j;
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (kind[k] == 0) continue;
          if (kind[k] == 3) {
            // V' = V J with V = I + Dl
            const int i = m1[k] >> 17, j = m2[k], p = (m1[k] >> 8) & 255, q = m1[k] & 255;
            const double cm1 = rot[3 * i], cd = rot[3 * i + 1], sd = rot[3 * i + 2];
            double np = cd * y[k][0] - sd * y[k][1], nq = sd * y[k][0] + cd * y[k][1];
            if (j == p) np += cm1, nq += sd;
            if (j == q) np -= sd, nq += cm1;
            Dl[j + p * ldd] = np;
            Dl[j + q * ldd] = nq;
            continue;
          }
          const int p1 = (m1[k] >> 8) & 255, q1 = m1[k] & 255;
          if (kind[k] == 2) {
            E[p1 + q1 * lde] = 0.f, E[q1 + p1 * lde] = 0.f;
            continue;
          }
          const int i1 = m1[k] >> 17, i2 = m2[k] >> 17, p2 = (m2[k] >> 8) & 255, q2 = m2[k] & 255;
          const float c1 = rcs[2 * i1], s1 = rcs[2 * i1 + 1], c2 = rcs[2 * i2], s2 = rcs[2 * i2 + 1];
          const bool v1 = q1 < s, v2 = q2 < s;
          const float r00 = c1 * x[k][0] - s1 * x[k][2], r01 = c1 * x[k][1] - s1 * x[k][3];
          const float r10 = s1 * x[k][0] + c1 * x[k][2], r11 = s1 * x[k][1] + c1 * x[k][3];
          const float n00 = c2 * r00 - s2 * r01, n01 = s2 * r00 + c2 * r01;
          const float n10 = c2 * r10 - s2 * r11, n11 = s2 * r10 + c2 * r11;
          E[p1 + p2 * lde] = n00, E[p2 + p1 * lde] = n00;
          if (v2) E[p1 + q2 * lde] = n01, E[q2 + p1 * lde] = n01;
          if (v1) E[q1 + p2 * lde] = n10, E[p2 + q1 * lde] = n10;
          if (v1 && v2) E[q1 + q2 * lde] = n11, E[q2 + q1 * lde] = n11;
        }
      }
      __syncthreads();
    }
  }
  return -1;
}

__device__ int jacobi_cta(int s, double* a, int lda, double* V, int ldv, double* rot, double* red) {
  return jacobi_sweeps<double>(s, a, lda, V, ldv, rot, red, 1e-15, 40, true);
}

__device__ int chol_cta(int p, double* L, int ld, int* flag);

// Rayleigh-Ritz eigensolve of the symmetric s x s matrix a; eigenvalues ascending (ties
// keep index order) with their eigenvector columns.
//
// TWO_STAGE = false: FP64 parallel-order Jacobi from a (the oracle's method).
//
// TWO_STAGE = true, in two precisions: FP32 Jacobi first diagonalises a (FP32 runs at
// about 60x the FP64 rate on this part); its rotation matrix, made orthonormal in FP64 by
// one Cholesky-QR step, gives Q with Q^T a Q diagonal up to ~1e-4 relative.  FP64 Jacobi
// then finishes on Q^T a Q, accumulating its rotations into Q, in about 2 sweeps instead of
// the ~7 it takes from a.  Off-diagonal mass ends <= 1e-15 ||a||_F with Q orthonormal to
// FP64 rounding, but forming Q^T a Q puts absolute errors of order eps ||a|| in every entry,
// so exact zero couplings (and the relative accuracy plain Jacobi keeps for small
// eigenvalues of a graded matrix) are not preserved.
template <bool TWO_STAGE>
__global__ void __launch_bounds__(kSmallThreads) syev_kernel(int s, const double* __restrict__ a_in,
                                                             int upper_only, double* __restrict__ lam,
                                                             double* __restrict__ U, int* sweeps_out,
                                                             double tol32, double tol64) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ double rot[4 * (kMaxS / 2 + 1)];
  __shared__ int rank[kMaxS];
  __shared__ double dsh[kMaxS];
  __shared__ int flag;
  const int ld = s | 1;  // odd stride: the row accesses of a round hit distinct banks
  double* A = sm;
  double* B = A + s * ld;
  double* C = B + s * ld;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int i = e % s, j = e / s;
    double v;
    if (upper_only) v = i <= j ? a_in[i + j * s] : a_in[j + i * s];
    else v = 0.5 * (a_in[i + j * s] + a_in[j + i * s]);
    A[i + j * ld] = v;
  }
  int sw;
  if (!TWO_STAGE) {
    __syncthreads();
    sw = jacobi_sweeps<double>(s, A, ld, B, ld, rot, red, tol64, 40, true);
  } else {
    // ---- FP32 pass (a32 and its rotations share the C buffer)
    float* a32 = reinterpret_cast<float*>(C);
    float* v32 = a32 + s * ld;
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) a32[(e % s) + (e / s) * ld] = (float)A[(e % s) + (e / s) * ld];
    __syncthreads();
    jacobi_sweeps<float>(s, a32, ld, v32, ld, reinterpret_cast<float*>(rot), red, tol32, 20, true);
    __syncthreads();
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) B[(e % s) + (e / s) * ld] = (double)v32[(e % s) + (e / s) * ld];
    __syncthreads();
    // ---- Q = B L^{-T} with L L^T = B^T B (Cholesky-QR in FP64)
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
      const int i = e % s, j = e / s;
      if (i >= j) {
        double acc = 0.0;
        for (int r = 0; r < s; ++r) acc += B[r + i * ld] * B[r + j * ld];
        C[i + j * ld] = acc;
      }
    }
    __syncthreads();
    const int bad = chol_cta(s, C, ld, &flag);
    if (bad) {
      // cannot happen for a rotation product; start the FP64 pass from the identity instead
      for (int e = threadIdx.x; e < s * s; e += blockDim.x) B[(e % s) + (e / s) * ld] = (e % s) == (e / s) ? 1.0 : 0.0;
    } else {
      for (int r = threadIdx.x; r < s; r += blockDim.x)  // row r of B solves x L^T = b
        for (int j = 0; j < s; ++j) {
          double acc = B[r + j * ld];
          for (int i = 0; i < j; ++i) acc -= B[r + i * ld] * C[j + i * ld];
          B[r + j * ld] = acc / C[j + j * ld];
        }
    }
    __syncthreads();
    // ---- A <- Q^T a Q (C = a Q, then the upper triangle of Q^T C, mirrored)
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
      const int i = e % s, j = e / s;
      double acc = 0.0;
      for (int t = 0; t < s; ++t) acc += A[i + t * ld] * B[t + j * ld];
      C[i + j * ld] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
      const int i = e % s, j = e / s;
      if (i <= j) {
        double acc = 0.0;
        for (int t = 0; t < s; ++t) acc += B[t + i * ld] * C[t + j * ld];
        A[i + j * ld] = acc;
        A[j + i * ld] = acc;
      }
    }
    __syncthreads();
    if (tol64 >= 1e-12) {
      // ---- polish to tol64 with FP32 rotations on the small off-diagonal part (E); the
      // rotation product minus the identity (Dl) in FP64; U = Q (I + Dl) at the end
      float* E = reinterpret_cast<float*>(C);
      double* Dl = A;  // A is read into d and E first
      double f2 = 0.0;
      for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
        const int i = e % s, j = e / s;
        const double v = A[i + j * ld];
        f2 += v * v;
        E[i + j * ld] = i == j ? 0.f : (float)v;
        if (i == j) dsh[i] = v;
      }
      const double fro = sqrt(block_sum(f2, red));  // ends with a barrier: A fully read
      for (int e = threadIdx.x; e < s * s; e += blockDim.x) Dl[(e % s) + (e / s) * ld] = 0.0;
      __syncthreads();
      sw = jacobi_polish(s, dsh, E, ld, Dl, ld, rot, red, tol64, fro, 20);
      __syncthreads();
      for (int i = threadIdx.x; i < s; i += blockDim.x) {
        const double li = dsh[i];
        int r = 0;
        for (int j = 0; j < s; ++j) {
          const double lj = dsh[j];
          r += (lj < li) || (lj == li && j < i);
        }
        rank[i] = r;
        lam[r] = li;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
        const int r = e % s, i = e / s;
        double acc = B[r + i * ld];
        for (int t = 0; t < s; ++t) acc += B[r + t * ld] * Dl[t + i * ld];
        U[r + rank[i] * s] = acc;
      }
      if (threadIdx.x == 0 && sweeps_out) *sweeps_out = sw;
      return;
    }
    // ---- FP64 pass, rotations accumulated into Q
    sw = jacobi_sweeps<double>(s, A, ld, B, ld, rot, red, tol64, 40, false);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    const double li = A[i + i * ld];
    int r = 0;
    for (int j = 0; j < s; ++j) {
      const double lj = A[j + j * ld];
      r += (lj < li) || (lj == li && j < i);
    }
    rank[i] = r;
    lam[r] = li;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int r = e % s, i = e / s;
    U[r + rank[i] * s] = B[r + i * ld];
  }
  if (threadIdx.x == 0 && sweeps_out) *sweeps_out = sw;
}

// In-place right-looking Cholesky of the p x p matrix L (lower part, ld).  Returns 0 or
// j+1 for the first non-positive pivot (same value in every thread).
__device__ int chol_cta(int p, double* L, int ld, int* flag) {
  if (threadIdx.x == 0) *flag = 0;
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    if (threadIdx.x == 0) {
      const double d = L[j + j * ld];
      if (!(d > 0.0)) *flag = j + 1;
      else L[j + j * ld] = sqrt(d);
    }
    __syncthreads();
    if (*flag) break;
    const double ljj = L[j + j * ld];
    for (int i = j + 1 + threadIdx.x; i < p; i += blockDim.x) L[i + j * ld] /= ljj;
    __syncthreads();
    const int rem = p - j - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int i = j + 1 + e % rem, l = j + 1 + e / rem;
      if (l <= i) L[i + l * ld] -= L[i + j * ld] * L[l + j * ld];
    }
    __syncthreads();
  }
  const int f = *flag;
  __syncthreads();
  return f;
}

// Shifted Cholesky of M (p x p, ld): tries M, then M + sigma I with sigma = 100 eps
// trace(M) * 10^t, t = 0..7.  L receives the factor.  Returns 0 on success.
__device__ int shifted_chol_cta(int p, const double* M, int ldm, double* L, int ld, int* flag,
                                int* shifts, double* red) {
  double tr = 0.0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) tr += M[i + i * ldm];
  tr = block_sum(tr, red);
  int fail = 1;
  for (int t = -1; t < 8 && fail; ++t) {
    const double sigma = t < 0 ? 0.0 : 100.0 * DBL_EPSILON * tr * pow(10.0, (double)t);
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
      const int i = e % p, j = e / p;
      L[i + j * ld] = M[i + j * ldm] + (i == j ? sigma : 0.0);
    }
    __syncthreads();
    if (t >= 0 && threadIdx.x == 0) ++*shifts;
    fail = chol_cta(p, L, ld, flag);
  }
  return fail;
}

// T = L^{-T} (upper triangular p x p, column-major, ldt) from the lower factor L.
__device__ void inv_lower_transpose_cta(int p, const double* L, int ld, double* T, int ldt) {
  // column j of L^{-1} by forward substitution; written transposed into row j of T
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    for (int i = 0; i < p; ++i) T[j + i * ldt] = 0.0;
    for (int i = j; i < p; ++i) {
      double s = i == j ? 1.0 : 0.0;
      for (int l = j; l < i; ++l) s -= L[i + l * ld] * T[j + l * ldt];
      T[j + i * ldt] = s / L[i + i * ld];
    }
  }
  __syncthreads();
}

// SVQB transform T = D Z Theta^{-1/2} for Gram M (Stathopoulos & Wu).  Uses B (p x p,
// ldb) and Z as scratch.
__device__ void svqb_cta(int p, const double* M, int ldm, double* B, double* Z, int ldb, double* T,
                         int ldt, double* rot, double* red, double* theta) {
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e % p, j = e / p;
    const double di = M[i + i * ldm] > 0.0 ? rsqrt(M[i + i * ldm]) : 0.0;
    const double dj = M[j + j * ldm] > 0.0 ? rsqrt(M[j + j * ldm]) : 0.0;
    B[i + j * ldb] = di * M[i + j * ldm] * dj;
  }
  __syncthreads();
  jacobi_cta(p, B, ldb, Z, ldb, rot, red);
  __syncthreads();
  double tmax = 0.0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) tmax = fmax(tmax, B[i + i * ldb]);
  tmax = block_max(tmax, red);
  for (int i = threadIdx.x; i < p; i += blockDim.x) theta[i] = fmax(B[i + i * ldb], DBL_EPSILON * tmax);
  __syncthreads();
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e % p, j = e / p;
    const double di = M[i + i * ldm] > 0.0 ? rsqrt(M[i + i * ldm]) : 0.0;
    T[i + j * ldt] = di * Z[i + j * ldb] / sqrt(theta[j]);
  }
  __syncthreads();
}

// ctl[6] <- 1 when this pass factored an unshifted scaled overlap I + F with ||F||_F <= 1/2
// (||L^{-T}||_2^2 <= 2: the re-check Gram of Algorithm 2 can be skipped, reading R17).
// With C (q x p, column-major, the projection coefficients of this Algorithm 3 pass; only
// on the first call of the pass): ctl[7] <- 1 when the growth factor satisfies
// max_j (||C_j||^2 + M_jj) / M_jj * ||L^{-T}||^2 <= growth2 (reading R18).
__global__ void __launch_bounds__(kSmallThreads) cholqr_small_kernel(int p, const double* __restrict__ Min,
                                                                     double tau, double* __restrict__ Tout,
                                                                     int* ctl, const double* __restrict__ C,
                                                                     int q, double growth2) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ double rot[4 * (kMaxS / 2 + 1)];
  __shared__ double theta[kMaxS];
  __shared__ int flag, shifts;
  const int ld = p | 1;  // odd stride: row accesses hit distinct banks
  double* M = sm;
  double* L = M + p * ld;
  double* T = L + p * ld;
  double* Z = T + p * ld;
  double dev = 0.0;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e % p, j = e / p;
    const double v = Min[e];
    M[i + j * ld] = v;
    const double d = fabs(v - (i == j ? 1.0 : 0.0));
    dev = (d <= dev) ? dev : d;  // NaN counts as large
    if (d != d) dev = INFINITY;
  }
  if (threadIdx.x == 0) shifts = 0;
  dev = block_max(dev, red);
  // growth factor of the Algorithm 3 pass (R18): amplification ||x~_j|| / ||x_proj,j|| of
  // column j times the bound on ||L^{-T}||; here the squared column term, the bound below
  double g2 = 0.0;
  if (C) {
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
      double c2 = 0.0;
      for (int i = 0; i < q; ++i) c2 += C[i + j * q] * C[i + j * q];
      const double mjj = M[j + j * ld];
      const double gj = mjj > 0.0 ? (c2 + mjj) / mjj : INFINITY;
      g2 = (gj <= g2) ? g2 : gj;
    }
    g2 = block_max(g2, red);
  }
  if (dev <= tau) {
    if (threadIdx.x == 0) {
      ctl[0] = 1;
      ctl[6] = 0;
      if (C) ctl[7] = g2 <= growth2 ? 1 : 0;
    }
    return;
  }
  // scaled Cholesky-QR: factor D M D with D = diag(M)^{-1/2}, transform T = D L^{-T}
  for (int i = threadIdx.x; i < p; i += blockDim.x) theta[i] = M[i + i * ld] > 0.0 ? rsqrt(M[i + i * ld]) : 1.0;
  __syncthreads();
  double fro = 0.0;  // ||F||_F of the scaled overlap D M D = I + F
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e % p, j = e / p;
    const double z = theta[i] * M[i + j * ld] * theta[j];
    Z[i + j * ld] = z;
    const double f = z - (i == j ? 1.0 : 0.0);
    fro += f * f;
  }
  fro = sqrt(block_sum(fro, red));
  __syncthreads();
  const int fail = shifted_chol_cta(p, Z, ld, L, ld, &flag, &shifts, red);
  if (!fail) {
    inv_lower_transpose_cta(p, L, ld, T, ld);
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
      const int i = e % p, j = e / p;
      T[i + j * ld] *= theta[i];
    }
    __syncthreads();
  } else {
    svqb_cta(p, M, ld, L, Z, ld, T, ld, rot, red, theta);
  }
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) Tout[e] = T[(e % p) + (e / p) * ld];
  if (threadIdx.x == 0) {
    const bool clean = !fail && shifts == 0;
    ctl[0] = 0;
    ctl[1] += shifts;
    ctl[2] += fail ? 1 : 0;
    ctl[6] = clean && fro <= 0.5 ? 1 : 0;
    if (C) {
      const double l2 = clean && fro < 1.0 ? 1.0 / (1.0 - fro) : INFINITY;
      ctl[7] = g2 * l2 <= growth2 ? 1 : 0;
    }
  }
}

__global__ void maxabs_kernel(int count, const double* __restrict__ C, double* out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int e = threadIdx.x; e < count; e += blockDim.x) {
    const double v = fabs(C[e]);
    m = (v <= m) ? m : v;
    if (v != v) m = INFINITY;
  }
  m = block_max(m, red);
  if (threadIdx.x == 0) *out = m;
}

// ---- Algorithm 2 / 3 in the small s-dimensional space (for u_p) -----------------------
// X: s x a (column-major, ldx), Y: s x q (ldy); everything in shared memory.
__device__ void small_ortho(int s, int a, double* X, int ldx, double tau, int cap, double* M,
                            double* L, double* Tm, double* Z, int ld, double* rot, double* red,
                            double* theta, int* flag, int* shifts) {
  for (int pass = 0;; ++pass) {
    for (int e = threadIdx.x; e < a * a; e += blockDim.x) {
      const int i = e % a, j = e / a;
      double acc = 0.0;
      for (int r = 0; r < s; ++r) acc += X[r + i * ldx] * X[r + j * ldx];
      M[i + j * ld] = acc;
    }
    __syncthreads();
    double dev = 0.0;
    for (int e = threadIdx.x; e < a * a; e += blockDim.x) {
      const double d = fabs(M[(e % a) + (e / a) * ld] - ((e % a) == (e / a) ? 1.0 : 0.0));
      dev = (d <= dev) ? dev : d;
      if (d != d) dev = INFINITY;
    }
    dev = block_max(dev, red);
    if (dev <= tau || pass >= cap) return;
    // scaled Cholesky-QR (D M D, D = diag(M)^{-1/2}), as in the n-dimensional ortho
    for (int i = threadIdx.x; i < a; i += blockDim.x) theta[i] = M[i + i * ld] > 0.0 ? rsqrt(M[i + i * ld]) : 1.0;
    __syncthreads();
    for (int e = threadIdx.x; e < a * a; e += blockDim.x) {
      const int i = e % a, j = e / a;
      Z[i + j * ld] = theta[i] * M[i + j * ld] * theta[j];
    }
    __syncthreads();
    const int fail = shifted_chol_cta(a, Z, ld, L, ld, flag, shifts, red);
    if (!fail) {
      inv_lower_transpose_cta(a, L, ld, Tm, ld);
      for (int e = threadIdx.x; e < a * a; e += blockDim.x) Tm[(e % a) + (e / a) * ld] *= theta[e % a];
      __syncthreads();
    } else {
      svqb_cta(a, M, ld, L, Z, ld, Tm, ld, rot, red, theta);
    }
    // X <- X Tm, row by row (each thread owns rows of X)
    for (int r = threadIdx.x; r < s; r += blockDim.x) {
      double row[kMaxM];
      for (int j = 0; j < a; ++j) row[j] = X[r + j * ldx];
      for (int j = 0; j < a; ++j) {
        double acc = 0.0;
        for (int l = 0; l < a; ++l) acc += row[l] * Tm[l + j * ld];
        X[r + j * ldx] = acc;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSmallThreads) lock_p_kernel(int s, int m, int k, int64_t n,
                                                               const double* __restrict__ norm_part,
                                                               int nparts, const double* __restrict__ U,
                                                               double tol, int tol_kind, double tau,
                                                               LockState* state, double* __restrict__ resnorm,
                                                               double* __restrict__ colmax,
                                                               double* __restrict__ up, int build_p) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ double rot[4 * (kMaxS / 2 + 1)];
  __shared__ double theta[kMaxS];
  __shared__ int conv[kMaxM];
  __shared__ int flag, shifts, s_mconv, s_mact, s_done, s_pw;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double s2 = 0.0, mx = 0.0;
    for (int g = 0; g < nparts; ++g) {
      s2 += norm_part[(int64_t)g * 2 * m + j];
      mx = fmax(mx, norm_part[(int64_t)g * 2 * m + m + j]);
    }
    const double nr = sqrt(s2);
    resnorm[j] = nr;
    colmax[j] = mx;
    conv[j] = tol_kind == 1 ? (nr / sqrt((double)n) <= 0.1 * tol && mx <= tol) : (nr <= tol);
  }
  if (threadIdx.x == 0) shifts = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    // longest converged prefix in the new Ritz order (recomputed every step: a lower,
    // unconverged Ritz vector can move in front of a converged one)
    int mc = 0;
    while (mc < m && conv[mc]) ++mc;
    s_mconv = mc;
    s_mact = m - mc;
    s_done = mc >= k;
    state->m_conv = mc;
    state->m_act = m - mc;
    state->done = s_done;
  }
  __syncthreads();
  if (!build_p || s_done) return;
  const int mc = s_mconv, a = s_mact;
  const int ld = kMaxS + 1;        // s-dimensional columns
  const int lds = kMaxM + 1;       // a x a / m x a matrices
  double* X = sm;                  // s x a   (ld)
  double* Y = X + kMaxM * ld;      // s x m   (ld), u_x
  double* C = Y + kMaxM * ld;      // m x a   (lds)
  double* M = C + kMaxM * lds;     // a x a   (lds) and scratch
  double* L = M + kMaxM * lds;
  double* Tm = L + kMaxM * lds;
  double* Z = Tm + kMaxM * lds;
  for (int e = threadIdx.x; e < s * a; e += blockDim.x) {
    const int r = e % s, c = e / s;
    X[r + c * ld] = U[r + (mc + c) * s] - (r == mc + c ? 1.0 : 0.0);  // u~_p = u_x[:,act] - E_act
  }
  for (int e = threadIdx.x; e < s * m; e += blockDim.x) Y[(e % s) + (e / s) * ld] = U[e];
  __syncthreads();
  // A P direction exists only where x_j moved: drop column c when (I - u_x u_x^T) u~_p_c
  // vanishes exactly (a zero vector cannot be normalised and would give a spurious Ritz
  // value 0 in V); pack the kept columns to the front.
  __shared__ int keep[kMaxM];
  for (int c = threadIdx.x; c < a; c += blockDim.x) {
    double cf[kMaxM];
    for (int i = 0; i < m; ++i) {
      double d = 0.0;
      for (int r = 0; r < s; ++r) d += Y[r + i * ld] * X[r + c * ld];
      cf[i] = d;
    }
    double nrm = 0.0;
    for (int r = 0; r < s; ++r) {
      double v = X[r + c * ld];
      for (int i = 0; i < m; ++i) v -= Y[r + i * ld] * cf[i];
      nrm += v * v;
    }
    keep[c] = sqrt(nrm) > 1e-200 ? 1 : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int kept = 0;
    for (int c = 0; c < a; ++c)
      if (keep[c]) {
        if (kept != c)
          for (int r = 0; r < s; ++r) X[r + kept * ld] = X[r + c * ld];
        ++kept;
      }
    s_pw = kept;
  }
  __syncthreads();
  const int ap = s_pw;
  if (threadIdx.x == 0) state->p_cols = ap;
  if (ap == 0) return;
  const int cap = 6, cap2 = 4;
  int passes = 0;
  for (;;) {
    // C = Y^T X, X <- X - Y C
    for (int e = threadIdx.x; e < m * ap; e += blockDim.x) {
      const int i = e % m, j = e / m;
      double acc = 0.0;
      for (int r = 0; r < s; ++r) acc += Y[r + i * ld] * X[r + j * ld];
      C[i + j * lds] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < s * ap; e += blockDim.x) {
      const int r = e % s, j = e / s;
      double acc = 0.0;
      for (int i = 0; i < m; ++i) acc += Y[r + i * ld] * C[i + j * lds];
      X[r + j * ld] -= acc;
    }
    __syncthreads();
    small_ortho(s, ap, X, ld, tau, cap, M, L, Tm, Z, lds, rot, red, theta, &flag, &shifts);
    ++passes;
    double mx = 0.0;
    for (int e = threadIdx.x; e < m * ap; e += blockDim.x) {
      const int i = e % m, j = e / m;
      double acc = 0.0;
      for (int r = 0; r < s; ++r) acc += Y[r + i * ld] * X[r + j * ld];
      const double v = fabs(acc);
      mx = (v <= mx) ? mx : v;
      if (v != v) mx = INFINITY;
    }
    mx = block_max(mx, red);
    if (mx <= tau || passes >= cap2) break;
  }
  // drop columns that could not be made orthonormal against u_x (more P directions than
  // the complement of u_x holds, e.g. after a column was unlocked); pack the rest
  for (int c = threadIdx.x; c < ap; c += blockDim.x) {
    double worst = 0.0, nrm = 0.0;
    for (int i = 0; i < m; ++i) {
      double d = 0.0;
      for (int r = 0; r < s; ++r) d += Y[r + i * ld] * X[r + c * ld];
      worst = fmax(worst, fabs(d));
    }
    for (int r = 0; r < s; ++r) nrm += X[r + c * ld] * X[r + c * ld];
    keep[c] = (worst <= sqrt(tau) && fabs(sqrt(nrm) - 1.0) <= sqrt(tau)) ? 1 : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int kept = 0;
    for (int c = 0; c < ap; ++c)
      if (keep[c]) {
        if (kept != c)
          for (int r = 0; r < s; ++r) X[r + kept * ld] = X[r + c * ld];
        ++kept;
      }
    s_pw = kept;
    state->p_cols = kept;
  }
  __syncthreads();
  const int ap2 = s_pw;
  for (int e = threadIdx.x; e < s * ap2; e += blockDim.x) up[e] = X[(e % s) + (e / s) * ld];
  if (threadIdx.x == 0) {
    state->sp_shifts += shifts;
    state->sp_passes = passes;
  }
}

}  // namespace

void launch_syev(int s, const double* a, bool upper_only, double* lam, double* U, int* sweeps_out,
                 cudaStream_t st, bool two_stage, double tol64) {
  if (s <= 0) return;
  if (s > kMaxS) throw std::invalid_argument("syev: s > 96");
  const size_t smem = (size_t)(two_stage ? 3 : 2) * s * (s + 1) * sizeof(double);
  // set once per process; function-local statics initialise thread-safely
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(syev_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 2 * kMaxS * (kMaxS + 1) * 8));
    LB_CUDA(cudaFuncSetAttribute(syev_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 3 * kMaxS * (kMaxS + 1) * 8));
    return true;
  }();
  (void)attr;
  const double tol32 = 1e-4;  // measured: the stopping point of this stage hardly changes the total
  if (two_stage)
    syev_kernel<true><<<1, kSmallThreads, smem, st>>>(s, a, upper_only ? 1 : 0, lam, U, sweeps_out, tol32, tol64);
  else
    syev_kernel<false><<<1, kSmallThreads, smem, st>>>(s, a, upper_only ? 1 : 0, lam, U, sweeps_out, tol32, tol64);
  LB_LAUNCH_CHECK();
}

void launch_cholqr_small(int p, const double* M, double tau, double* Linv, int* ctl, cudaStream_t st,
                         const double* C, int q, double growth2) {
  if (p <= 0) return;
  if (p > kMaxCholP) throw std::invalid_argument("cholqr: p > 64");
  const size_t smem = (size_t)4 * p * (p + 1) * sizeof(double);
  // set once per process; function-local statics initialise thread-safely
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(cholqr_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * kMaxCholP * (kMaxCholP + 1) * 8));
    return true;
  }();
  (void)attr;
  cholqr_small_kernel<<<1, kSmallThreads, smem, st>>>(p, M, tau, Linv, ctl, C, q, growth2);
  LB_LAUNCH_CHECK();
}

namespace {
__global__ void maxabs_minus_identity_kernel(int p, const double* __restrict__ C, double* out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const double v = fabs(C[e] - ((e % p) == (e / p) ? 1.0 : 0.0));
    m = (v <= m) ? m : v;
    if (v != v) m = INFINITY;
  }
  m = block_max(m, red);
  if (threadIdx.x == 0) *out = m;
}
}  // namespace

void launch_maxabs_minus_identity(int p, const double* C, double* out, cudaStream_t st) {
  maxabs_minus_identity_kernel<<<1, 256, 0, st>>>(p, C, out);
  LB_LAUNCH_CHECK();
}

void launch_maxabs(int count, const double* C, double* out, cudaStream_t st) {
  maxabs_kernel<<<1, 256, 0, st>>>(count, C, out);
  LB_LAUNCH_CHECK();
}

void launch_lock_and_p(int s, int m, int k, int64_t n, const double* norm_part, int nparts,
                       const double* U, double tol, int tol_kind, double tau, LockState* state,
                       double* resnorm, double* colmax, double* up, bool build_p, cudaStream_t st) {
  const size_t smem = ((size_t)2 * kMaxM * (kMaxS + 1) + (size_t)5 * kMaxM * (kMaxM + 1)) * sizeof(double);
  // set once per process; function-local statics initialise thread-safely
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(lock_p_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return true;
  }();
  (void)attr;
  lock_p_kernel<<<1, kSmallThreads, smem, st>>>(s, m, k, n, norm_part, nparts, U, tol, tol_kind, tau,
                                                 state, resnorm, colmax, up, build_p ? 1 : 0);
  LB_LAUNCH_CHECK();
}

}  // namespace lobpcg
