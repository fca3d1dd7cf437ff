// Learned preconditioner scale (not in the paper; motivated by its preconditioner study,
// Sec. 4.4): a 3 -> 64 -> 64 -> 1 ReLU perceptron per (row, active column) whose
// softplus output s > 0 scales the diagonal step of Sec. 2:
//     w_ij = s_ij r_ij / (d_i - theta_j),
// so the preconditioner stays positive.  Weights and activations are rounded to BF16,
// sums are accumulated in FP32.  The correction is applied in the "near" region
// |d_i - theta_j| <= 64 c (c = mean off-diagonal row norm); elsewhere the diagonal
// step is already accurate to first order and s = 1.
//
// Features: f1 = (d_i - theta_j) / (8 c), f2 = rho_i / c, f3 = r_ij / max_i |r_ij|.
// Parameter layout (4481 floats): W1[64][3] b1[64] W2[64][64] b2[64] W3[64] b3.
#include <cuda_bf16.h>

#include <algorithm>
#include <string>

#include "../../include/lobpcg.h"
#include "common.cuh"
#include "mlp.cuh"

namespace lobpcg {
namespace mlp {
namespace {

constexpr int H = kHidden;
constexpr int OFF_W1 = 0, OFF_B1 = H * 3, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H, OFF_W3 = OFF_B2 + H,
              OFF_B3 = OFF_W3 + H;

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
// Rounding of weights / activations: BF16 in the solver and in training; FP32 (no
// rounding) only to check the kernels' arithmetic against the FP64 definition.
__device__ __forceinline__ float rnd(float x, bool b) { return b ? bf(x) : x; }
__device__ __forceinline__ float softplusf(float z) { return z > 20.f ? z : log1pf(expf(z)); }
__device__ __forceinline__ float sigmoidf(float z) { return 1.f / (1.f + expf(-z)); }

// Copies the parameters into shared memory rounded to BF16 (kept as float for FMA).
__device__ void load_params(const float* __restrict__ P, float* sP, bool b = true) {
  for (int i = threadIdx.x; i < kNumParams; i += blockDim.x) sP[i] = rnd(P[i], b);
  __syncthreads();
}

// Forward pass of one sample with parameters in shared memory; returns z.
__device__ __forceinline__ float forward_z(const float* sP, float f1, float f2, float f3, float* h1, bool b = true) {
  f1 = rnd(f1, b), f2 = rnd(f2, b), f3 = rnd(f3, b);
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const float a = sP[OFF_B1 + i] + sP[OFF_W1 + 3 * i] * f1 + sP[OFF_W1 + 3 * i + 1] * f2 + sP[OFF_W1 + 3 * i + 2] * f3;
    h1[i] = rnd(fmaxf(a, 0.f), b);
  }
  float z = sP[OFF_B3];
  for (int i = 0; i < H; ++i) {
    const float4* w = reinterpret_cast<const float4*>(sP + OFF_W2 + i * H);
    float a = sP[OFF_B2 + i];
#pragma unroll
    for (int k4 = 0; k4 < H / 4; ++k4) {
      const float4 wv = w[k4];
      a = fmaf(wv.x, h1[4 * k4], a);
      a = fmaf(wv.y, h1[4 * k4 + 1], a);
      a = fmaf(wv.z, h1[4 * k4 + 2], a);
      a = fmaf(wv.w, h1[4 * k4 + 3], a);
    }
    z = fmaf(sP[OFF_W3 + i], rnd(fmaxf(a, 0.f), b), z);
  }
  return z;
}

__global__ void __launch_bounds__(256) forward_kernel(int64_t N, const float* __restrict__ F,
                                                      const float* __restrict__ P, float* __restrict__ s, bool b) {
  __shared__ __align__(16) float sP[kNumParams + 3];
  load_params(P, sP, b);
  float h1[H];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    s[i] = softplusf(forward_z(sP, F[3 * i], F[3 * i + 1], F[3 * i + 2], h1, b));
}

// Backward over tiles of 128 samples: every thread rebuilds its sample's activations
// and deltas into shared memory, then the CTA forms the weight-gradient outer products
// over the tile and adds them to grad with atomics.
constexpr int TB = 128;
__global__ void __launch_bounds__(TB) backward_kernel(int64_t N, const float* __restrict__ F,
                                                      const float* __restrict__ P, const float* __restrict__ g,
                                                      float* __restrict__ grad, bool b) {
  extern __shared__ __align__(16) float sm[];
  float* sP = sm;                      // kNumParams (+pad)
  float* sH1 = sP + kNumParams + 3;    // [TB][H+1] post-ReLU layer-1 activations
  float* sD2 = sH1 + TB * (H + 1);     // [TB][H+1] layer-2 deltas
  float* sD1 = sD2 + TB * (H + 1);     // [TB][H+1] layer-1 deltas
  float* sF = sD1 + TB * (H + 1);      // [TB][3]
  float* sH2 = sF + TB * 3;            // [TB][H+1]
  float* sDZ = sH2 + TB * (H + 1);     // [TB]
  load_params(P, sP, b);
  const int LD = H + 1;
  for (int64_t t0 = (int64_t)blockIdx.x * TB; t0 < N; t0 += (int64_t)gridDim.x * TB) {
    const int64_t i = t0 + threadIdx.x;
    const int r = threadIdx.x;
    {
      float h1[H];
      float f1 = 0.f, f2 = 0.f, f3 = 0.f, gi = 0.f;
      if (i < N) f1 = F[3 * i], f2 = F[3 * i + 1], f3 = F[3 * i + 2], gi = g[i];
      f1 = rnd(f1, b), f2 = rnd(f2, b), f3 = rnd(f3, b);
      sF[3 * r] = f1, sF[3 * r + 1] = f2, sF[3 * r + 2] = f3;
      float a1[H];
#pragma unroll 8
      for (int k = 0; k < H; ++k) {
        a1[k] = sP[OFF_B1 + k] + sP[OFF_W1 + 3 * k] * f1 + sP[OFF_W1 + 3 * k + 1] * f2 + sP[OFF_W1 + 3 * k + 2] * f3;
        h1[k] = rnd(fmaxf(a1[k], 0.f), b);
        sH1[r * LD + k] = h1[k];
      }
      float z = sP[OFF_B3];
      for (int k = 0; k < H; ++k) {
        float a = sP[OFF_B2 + k];
        for (int l = 0; l < H; ++l) a = fmaf(sP[OFF_W2 + k * H + l], h1[l], a);
        const float h2 = rnd(fmaxf(a, 0.f), b);
        sH2[r * LD + k] = h2;
        sD2[r * LD + k] = a > 0.f ? 1.f : 0.f;  // ReLU mask, scaled below
        z = fmaf(sP[OFF_W3 + k], h2, z);
      }
      const float dz = i < N ? gi * sigmoidf(z) : 0.f;
      sDZ[r] = dz;
      for (int k = 0; k < H; ++k) sD2[r * LD + k] *= dz * sP[OFF_W3 + k];
      for (int l = 0; l < H; ++l) {
        float acc = 0.f;
        for (int k = 0; k < H; ++k) acc = fmaf(sP[OFF_W2 + k * H + l], sD2[r * LD + k], acc);
        sD1[r * LD + l] = a1[l] > 0.f ? acc : 0.f;
      }
    }
    __syncthreads();
    // outer products over the tile
    for (int e = threadIdx.x; e < kNumParams; e += blockDim.x) {
      float acc = 0.f;
      if (e < OFF_B1) {  // W1[k][c]
        const int k = e / 3, c = e % 3;
        for (int r2 = 0; r2 < TB; ++r2) acc = fmaf(sD1[r2 * LD + k], sF[3 * r2 + c], acc);
      } else if (e < OFF_W2) {  // b1
        const int k = e - OFF_B1;
        for (int r2 = 0; r2 < TB; ++r2) acc += sD1[r2 * LD + k];
      } else if (e < OFF_B2) {  // W2[k][l]
        const int k = (e - OFF_W2) / H, l = (e - OFF_W2) % H;
        for (int r2 = 0; r2 < TB; ++r2) acc = fmaf(sD2[r2 * LD + k], sH1[r2 * LD + l], acc);
      } else if (e < OFF_W3) {  // b2
        const int k = e - OFF_B2;
        for (int r2 = 0; r2 < TB; ++r2) acc += sD2[r2 * LD + k];
      } else if (e < OFF_B3) {  // W3
        const int k = e - OFF_W3;
        for (int r2 = 0; r2 < TB; ++r2) acc = fmaf(sDZ[r2], sH2[r2 * LD + k], acc);
      } else {  // b3
        for (int r2 = 0; r2 < TB; ++r2) acc += sDZ[r2];
      }
      atomicAdd(grad + e, acc);
    }
    __syncthreads();
  }
}

// Column sums: we[c] += w e, ww[c] += w^2 over the samples (w = s q).
__global__ void col_sums_kernel(int64_t N, const int32_t* __restrict__ col, const float* __restrict__ q,
                                const float* __restrict__ e, const float* __restrict__ s, double* we, double* ww) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double w = (double)s[i] * q[i];
    atomicAdd(we + col[i], w * e[i]);
    atomicAdd(ww + col[i], w * w);
  }
}

__global__ void loss_grad_kernel(int64_t N, int ncol, const int32_t* __restrict__ col, const float* __restrict__ q,
                                 const float* __restrict__ e, const float* __restrict__ s, const double* __restrict__ we,
                                 const double* __restrict__ ww, const double* __restrict__ ee, float* __restrict__ dLds,
                                 double* loss) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double L = 0.0;
    for (int c = 0; c < ncol; ++c) L += 1.0 - we[c] * we[c] / (ww[c] * ee[c]);
    *loss = L / ncol;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = col[i];
    const double w = (double)s[i] * q[i];
    const double dLdw = -2.0 * we[c] * e[i] / (ww[c] * ee[c]) + 2.0 * we[c] * we[c] * w / (ww[c] * ww[c] * ee[c]);
    dLds[i] = (float)(dLdw * q[i] / ncol);
  }
}

__global__ void adam_kernel(int np, float* __restrict__ P, float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    const float gi = grad[i];
    m[i] = b1 * m[i] + (1.f - b1) * gi;
    v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
    P[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
    grad[i] = 0.f;
  }
}

}  // namespace

// ---- learned preconditioner step inside the solver ----------------------------------------
// Two passes.  The diagonal step w = r / guard(d - theta) over every (row, column) is a
// light elementwise kernel; the MLP scale applies only where |d - theta| <= 64 c, a few
// rows around each Ritz value, and its register-heavy forward pass runs in a second
// kernel that recomputes those entries (the same expression, so the result is the same as
// one fused pass).
template <class T>
__global__ void __launch_bounds__(256) precond_diag_kernel(int64_t n, const T* __restrict__ X,
                                                           const T* __restrict__ AX, int ld,
                                                           const double* __restrict__ lam, int c0, int a,
                                                           const double* __restrict__ diag, T* __restrict__ W,
                                                           int ldw) {
  // 2-D walk (row, column) without 64-bit divisions: a_pad = pow2 >= a lanes per row
  const int a_pad = a <= 1 ? 1 : (a <= 2 ? 2 : (a <= 4 ? 4 : (a <= 8 ? 8 : (a <= 16 ? 16 : 32))));
  const int rows_per_block = blockDim.x / a_pad;
  const int j = threadIdx.x % a_pad;
  const int rl = threadIdx.x / a_pad;
  if (j >= a) return;
  const double l = lam[c0 + j];
  const T fl = (T)(1e-8 * fmax(1.0, fabs(l)));
  const T lt = (T)l;
  for (int64_t i = (int64_t)blockIdx.x * rows_per_block + rl; i < n; i += (int64_t)gridDim.x * rows_per_block) {
    const T r = AX[i * ld + c0 + j] - lt * X[i * ld + c0 + j];
    // in the block's precision: exact for FP64, and the FP64 units stay free in the FP32 phase
    T delta = (T)diag[i] - lt;
    if (fabs(delta) < fl) delta = delta >= T(0) ? fl : -fl;
    W[i * ldw + j] = r * T(1) / delta;
  }
}

template <class T>
__global__ void precond_learned_kernel(int64_t n, const T* __restrict__ X, const T* __restrict__ AX, int ld,
                                       const double* __restrict__ lam, int c0, int a, const double* __restrict__ diag,
                                       const float* __restrict__ rho, float cscale, const double* __restrict__ colmax,
                                       const float* __restrict__ P, T* __restrict__ W, int ldw) {
  __shared__ __align__(16) float sP[kNumParams + 3];
  load_params(P, sP);
  float h1[H];
  const T band = (T)(64.0 * cscale);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T di = (T)diag[i];
    for (int j = 0; j < a; ++j) {
      const double l = lam[c0 + j];
      const T lt = (T)l;
      const T dd = di - lt;
      if (!(fabs(dd) <= band)) continue;
      const T fl = (T)(1e-8 * fmax(1.0, fabs(l)));
      const float g = (float)colmax[c0 + j];
      const T r = AX[i * ld + c0 + j] - lt * X[i * ld + c0 + j];
      T delta = dd;
      if (fabs(delta) < fl) delta = delta >= T(0) ? fl : -fl;
      const float f3 = g > 0.f ? (float)r / g : 0.f;
      const T scale = (T)softplusf(forward_z(sP, (float)dd / (float)(8.0 * cscale), rho[i] / cscale, f3, h1));
      W[i * ldw + j] = r * scale / delta;
    }
  }
}

// Features / targets of a block for training (same feature definition as above).
// For each (row, column j < p): q = r / guard(d - theta), near flag, f (3), and
// e_perp = xs - alpha_j x (exact correction made orthogonal to x, xs = aligned x*).
// Column sums over ALL rows (double atomics): ee = |e_perp|^2, far_we, far_ww.
__global__ void features_kernel(int64_t n, int p, const double* __restrict__ X, const double* __restrict__ AX, int ld,
                                const double* __restrict__ lam, const double* __restrict__ diag,
                                const float* __restrict__ rho, float cscale, const double* __restrict__ colmax,
                                const double* __restrict__ XS, const double* __restrict__ alpha, float* __restrict__ Fout,
                                float* __restrict__ qout, float* __restrict__ eout, int* __restrict__ near,
                                double* __restrict__ ee, double* __restrict__ far_we, double* __restrict__ far_ww) {
  const int64_t total = n * p;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / p;
    const int j = (int)(e - i * p);
    const double l = lam[j];
    const double x = X[i * ld + j];
    const double r = AX[i * ld + j] - l * x;
    const double dd = diag[i] - l;
    double delta = dd;
    const double fl = 1e-8 * fmax(1.0, fabs(l));
    if (fabs(delta) < fl) delta = delta >= 0.0 ? fl : -fl;
    const double q = r / delta;
    const double ep = XS[i * ld + j] - alpha[j] * x;
    const bool nr = fabs(dd) <= 64.0 * cscale;
    Fout[3 * e] = (float)(dd / (8.0 * cscale));
    Fout[3 * e + 1] = rho[i] / cscale;
    Fout[3 * e + 2] = colmax[j] > 0.0 ? (float)(r / colmax[j]) : 0.f;
    qout[e] = (float)q;
    eout[e] = (float)ep;
    near[e] = nr ? 1 : 0;
    atomicAdd(ee + j, ep * ep);
    if (!nr) {
      atomicAdd(far_we + j, q * ep);
      atomicAdd(far_ww + j, q * q);
    }
  }
}

// Off-diagonal row 2-norms of a CSR matrix.
__global__ void rho_csr_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const double* __restrict__ val, float* __restrict__ rho) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
      if (ci[e] != i) s += val[e] * val[e];
    rho[i] = (float)sqrt(s);
  }
}
// Off-diagonal row 2-norms of a dense symmetric column-major matrix (row i == column i).
__global__ void rho_dense_kernel(int64_t n, const double* __restrict__ A, int64_t lda, float* __restrict__ rho) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; i < n;
       i += ((int64_t)gridDim.x * blockDim.x) / 32) {
    double s = 0.0;
    for (int64_t c = lane; c < n; c += 32)
      if (c != i) s += A[c + i * lda] * A[c + i * lda];
    s = warp_sum(s);
    if (lane == 0) rho[i] = (float)sqrt(s);
  }
}
__global__ void mean_kernel(int64_t n, const float* __restrict__ v, double* out) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) s += v[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s / (double)n);
}

unsigned grid(int64_t total, int threads) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, threads), 152 * 16));
}

void launch_forward(int64_t N, const float* F, const float* P, float* s, bool b, cudaStream_t st) {
  if (N <= 0) return;
  forward_kernel<<<grid(N, 256), 256, 0, st>>>(N, F, P, s, b);
  LB_LAUNCH_CHECK();
}

void launch_backward(int64_t N, const float* F, const float* P, const float* g, float* grad, bool b,
                     cudaStream_t st) {
  if (N <= 0) return;
  const size_t smem = (size_t)(kNumParams + 3 + 4 * TB * (H + 1) + TB * 3 + TB) * sizeof(float);
  // set once per process; function-local statics initialise thread-safely
  static const bool attr = [&] {
    LB_CUDA(cudaFuncSetAttribute(backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return true;
  }();
  (void)attr;
  backward_kernel<<<(unsigned)std::min<int64_t>(ceil_div(N, TB), 152 * 4), TB, smem, st>>>(N, F, P, g, grad, b);
  LB_LAUNCH_CHECK();
}

template <class T>
void launch_precond_learned(int64_t n, const T* X, const T* AX, int ld, const double* lam, int c0, int a,
                            const double* diag, const float* rho, float cscale, const double* colmax, const float* P,
                            T* W, int ldw, cudaStream_t st) {
  if (n <= 0 || a <= 0) return;
  precond_diag_kernel<T><<<grid(n * a, 256), 256, 0, st>>>(n, X, AX, ld, lam, c0, a, diag, W, ldw);
  LB_LAUNCH_CHECK();
  precond_learned_kernel<T><<<grid(n, 256), 256, 0, st>>>(n, X, AX, ld, lam, c0, a, diag, rho, cscale, colmax, P,
                                                          W, ldw);
  LB_LAUNCH_CHECK();
}
template void launch_precond_learned<double>(int64_t, const double*, const double*, int, const double*, int, int,
                                             const double*, const float*, float, const double*, const float*, double*,
                                             int, cudaStream_t);
template void launch_precond_learned<float>(int64_t, const float*, const float*, int, const double*, int, int,
                                            const double*, const float*, float, const double*, const float*, float*,
                                            int, cudaStream_t);

double row_norms(int64_t n, const int64_t* rp, const int32_t* ci, const double* val, const double* dense,
                 int64_t lda, float* rho, double* scratch, cudaStream_t st) {
  if (dense) rho_dense_kernel<<<grid(n * 32, 256), 256, 0, st>>>(n, dense, lda, rho);
  else rho_csr_kernel<<<grid(n, 256), 256, 0, st>>>(n, rp, ci, val, rho);
  LB_LAUNCH_CHECK();
  LB_CUDA(cudaMemsetAsync(scratch, 0, sizeof(double), st));
  mean_kernel<<<grid(n, 256), 256, 0, st>>>(n, rho, scratch);
  LB_LAUNCH_CHECK();
  double c = 0.0;
  LB_CUDA(cudaMemcpyAsync(&c, scratch, sizeof(double), cudaMemcpyDeviceToHost, st));
  LB_CUDA(cudaStreamSynchronize(st));
  return c;
}

}  // namespace mlp
}  // namespace lobpcg

// ===================================================================== C ABI (training)
using namespace lobpcg;

namespace lobpcg {
const char* set_thread_error(const std::string& msg);
}

#define MLP_GUARD(...)                                \
  try {                                               \
    __VA_ARGS__;                                      \
    return LOBPCG_OK;                                 \
  } catch (const std::exception& ex) {                \
    lobpcg::set_thread_error(ex.what());              \
    return LOBPCG_ECUDA;                              \
  }

extern "C" int lobpcg_mlp_num_params(void) { return mlp::kNumParams; }

extern "C" lobpcg_status lobpcg_mlp_forward(int64_t N, const float* F, const float* params, float* s, int bf16,
                                            lobpcg_stream stream) {
  if (N < 0 || (N > 0 && (!F || !params || !s))) {
    lobpcg::set_thread_error("lobpcg_mlp_forward: NULL argument");
    return LOBPCG_EINVAL;
  }
  MLP_GUARD({
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    mlp::launch_forward(N, F, params, s, bf16 != 0, st);
    LB_CUDA(cudaStreamSynchronize(st));
  })
}

extern "C" lobpcg_status lobpcg_mlp_backward(int64_t N, const float* F, const float* params, const float* g,
                                             float* grad, int bf16, lobpcg_stream stream) {
  if (N < 0 || (N > 0 && (!F || !params || !g || !grad))) {
    lobpcg::set_thread_error("lobpcg_mlp_backward: NULL argument");
    return LOBPCG_EINVAL;
  }
  MLP_GUARD({
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    mlp::launch_backward(N, F, params, g, grad, bf16 != 0, st);
    LB_CUDA(cudaStreamSynchronize(st));
  })
}

extern "C" lobpcg_status lobpcg_mlp_loss(int64_t N, int ncol, const int32_t* col, const float* q, const float* e,
                                         const float* s, const double* far_we, const double* far_ww, const double* ee,
                                         double* work, float* dLds, double* loss, lobpcg_stream stream) {
  if (N < 0 || ncol < 1 || !col || !q || !e || !s || !far_we || !far_ww || !ee || !work || !dLds || !loss) {
    lobpcg::set_thread_error("lobpcg_mlp_loss: invalid argument");
    return LOBPCG_EINVAL;
  }
  MLP_GUARD({
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double* we = work;
    double* ww = work + ncol;
    LB_CUDA(cudaMemcpyAsync(we, far_we, ncol * sizeof(double), cudaMemcpyDeviceToDevice, st));
    LB_CUDA(cudaMemcpyAsync(ww, far_ww, ncol * sizeof(double), cudaMemcpyDeviceToDevice, st));
    mlp::col_sums_kernel<<<mlp::grid(N, 256), 256, 0, st>>>(N, col, q, e, s, we, ww);
    LB_LAUNCH_CHECK();
    mlp::loss_grad_kernel<<<mlp::grid(N, 256), 256, 0, st>>>(N, ncol, col, q, e, s, we, ww, ee, dLds, loss);
    LB_LAUNCH_CHECK();
    LB_CUDA(cudaStreamSynchronize(st));
  })
}

extern "C" lobpcg_status lobpcg_mlp_adam(int np, float* params, float* grad, float* m, float* v, int step, float lr,
                                         float beta1, float beta2, float eps, lobpcg_stream stream) {
  if (np != mlp::kNumParams || !params || !grad || !m || !v || step < 1) {
    lobpcg::set_thread_error("lobpcg_mlp_adam: invalid argument");
    return LOBPCG_EINVAL;
  }
  MLP_GUARD({
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    mlp::adam_kernel<<<mlp::grid(np, 256), 256, 0, st>>>(np, params, grad, m, v, lr, beta1, beta2, eps, c1, c2);
    LB_LAUNCH_CHECK();
    LB_CUDA(cudaStreamSynchronize(st));
  })
}

extern "C" lobpcg_status lobpcg_precond_features(int64_t n, int p, const double* X, const double* AX, int ld,
                                                 const double* lam, const double* diag, const float* rho, float cscale,
                                                 const double* colmax, const double* XS, const double* alpha, float* F,
                                                 float* q, float* e, int* near, double* sums, lobpcg_stream stream) {
  if (n < 1 || p < 1 || ld < p || !X || !AX || !lam || !diag || !rho || !colmax || !XS || !alpha || !F || !q ||
      !e || !near || !sums || !(cscale > 0.f)) {
    lobpcg::set_thread_error("lobpcg_precond_features: invalid argument");
    return LOBPCG_EINVAL;
  }
  MLP_GUARD({
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    LB_CUDA(cudaMemsetAsync(sums, 0, 3 * p * sizeof(double), st));
    mlp::features_kernel<<<mlp::grid(n * p, 256), 256, 0, st>>>(n, p, X, AX, ld, lam, diag, rho, cscale, colmax, XS,
                                                                 alpha, F, q, e, near, sums, sums + p, sums + 2 * p);
    LB_LAUNCH_CHECK();
    LB_CUDA(cudaStreamSynchronize(st));
  })
}

extern "C" lobpcg_status lobpcg_row_norms(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                                          const double* dense, int64_t lda, float* rho, double* mean_out,
                                          lobpcg_stream stream) {
  if (n < 1 || !rho || !mean_out || (!dense && (!row_ptr || !col_idx || !val))) {
    lobpcg::set_thread_error("lobpcg_row_norms: invalid argument");
    return LOBPCG_EINVAL;
  }
  MLP_GUARD({
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double* scratch = nullptr;
    LB_CUDA(cudaMallocAsync(&scratch, sizeof(double), st));
    *mean_out = mlp::row_norms(n, row_ptr, col_idx, val, dense, lda, rho, scratch, st);
    LB_CUDA(cudaFreeAsync(scratch, st));
    LB_CUDA(cudaStreamSynchronize(st));
  })
}
