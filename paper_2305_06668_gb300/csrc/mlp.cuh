// Learned preconditioner scale: shared declarations (see mlp.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace lobpcg {
namespace mlp {

constexpr int kHidden = 64;
constexpr int kNumParams = kHidden * 3 + kHidden + kHidden * kHidden + kHidden + kHidden + 1;  // 4481

// W_ij = s_ij r_ij / guard(d_i - theta_j) for the active columns c0 .. c0 + a - 1, with
// s = softplus(MLP(f)) where |d_i - theta_j| <= 64 cscale and s = 1 elsewhere.
template <class T>
void launch_precond_learned(int64_t n, const T* X, const T* AX, int ld, const double* lam, int c0, int a,
                            const double* diag, const float* rho, float cscale, const double* colmax, const float* P,
                            T* W, int ldw, cudaStream_t st);

// rho_i = off-diagonal 2-norm of row i (CSR when dense == nullptr); returns mean(rho).
// Synchronises the stream.  scratch: one device double.
double row_norms(int64_t n, const int64_t* rp, const int32_t* ci, const double* val, const double* dense,
                 int64_t lda, float* rho, double* scratch, cudaStream_t st);

}  // namespace mlp
}  // namespace lobpcg
