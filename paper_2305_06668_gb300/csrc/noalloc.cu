// Gram entry point that allocates nothing: its scratch (the per-CTA partial sums of the
// split-row reduction) lives in a fixed file-scope device array instead of memory the
// call would have to obtain with cudaMalloc.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lobpcg.h"
#include "common.cuh"

namespace lobpcg {
const char* set_thread_error(const std::string& msg);
}

namespace {

constexpr int kParts = 152;         // CTAs of the split-row reduction (one per SM of a GB300)
constexpr int kMaxEntries = 1024;   // p * q of the largest accepted product
// 152 * 1024 doubles = 1.2 MB, held on every GPU that loads the library until the process exits.
__device__ __align__(256) double g_gram_scratch[kParts * kMaxEntries];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on first use).
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_gram_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" lobpcg_status lobpcg_gram_f64_noalloc(int64_t n, int p, const double* X, int ldx, int q,
                                                 const double* Y, int ldy, double* C, lobpcg_stream stream) {
  using namespace lobpcg;
  if (n < 1 || !X || !Y || !C || p < 1 || q < 1 || ldx < p || ldy < q) {
    set_thread_error("lobpcg_gram_f64_noalloc: need n >= 1, p, q >= 1, ld >= width and non-NULL arrays");
    return LOBPCG_EINVAL;
  }
  if (p > kMaxS || q > kMaxS) {
    set_thread_error("lobpcg_gram_f64_noalloc: p and q must be <= 96 (widest Gram the kernels take)");
    return LOBPCG_EINVAL;
  }
  if ((int64_t)p * q > kMaxEntries) {
    set_thread_error("lobpcg_gram_f64_noalloc: p * q must be <= 1024 (size of the fixed scratch array)");
    return LOBPCG_EINVAL;
  }
  try {
    double* part = nullptr;
    const cudaError_t e = scratch_for_current_device(&part);
    if (e != cudaSuccess) {
      set_thread_error(std::string("lobpcg_gram_f64_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return LOBPCG_ECUDA;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // every partial entry the reduction reads is written by this call's own Gram launch,
    // so the array needs no clearing between calls
    const int parts = gram_partials<double>(n, cols1<double>(X, ldx, p), cols1<double>(Y, ldy, q), false, part,
                                            kParts, st);
    reduce_partials(part, parts, p * q, C, st);
    LB_CUDA(cudaStreamSynchronize(st));
    return LOBPCG_OK;
  } catch (const std::exception& ex) {
    set_thread_error(ex.what());
    return LOBPCG_ECUDA;
  }
}
