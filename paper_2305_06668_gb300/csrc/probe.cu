// Throughput probe of the FMA pipes (FP64 and FP32): the denominator of the "alu"
// rooflines the benchmark reports.  Not part of the method; it measures the part.
//
// Every thread runs 8 independent fused multiply-add chains (x <- x * b + c) for `iters`
// rounds of 16 steps; the grid fills every SM with 8 CTAs of 256 threads, enough
// independent work to keep either pipe issuing every cycle.  The chains' sums are stored
// so the compiler keeps the arithmetic.  Flops = 2 * threads * iters * 16 * 8.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/lobpcg.h"
#include "common.cuh"

namespace lobpcg {
const char* set_thread_error(const std::string& msg);
}

namespace {

template <class T>
__global__ void __launch_bounds__(256) fma_rate_kernel(int iters, T b, T c, T* __restrict__ out) {
  T x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fma(x[j], b, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
double run(int iters, int blocks, T* out, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  LB_CUDA(cudaEventRecord(e0, st));
  fma_rate_kernel<T><<<blocks, 256, 0, st>>>(iters, (T)0.9999999, (T)1e-7, out);
  LB_LAUNCH_CHECK();
  LB_CUDA(cudaEventRecord(e1, st));
  LB_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  LB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  return ms * 1e-3;
}

template <class T>
double probe(cudaStream_t st) {
  int dev = 0, sms = 0;
  LB_CUDA(cudaGetDevice(&dev));
  LB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 8 * sms;
  T* out = nullptr;
  LB_CUDA(cudaMalloc(&out, (size_t)blocks * 256 * sizeof(T)));
  cudaEvent_t e0, e1;
  LB_CUDA(cudaEventCreate(&e0));
  LB_CUDA(cudaEventCreate(&e1));
  double best = 0.0;
  try {
    // calibrate to about 50 ms per launch, then keep the best of 5
    int iters = 64;
    double t = run<T>(iters, blocks, out, st, e0, e1);
    while (t < 0.01 && iters < (1 << 24)) {
      iters *= 4;
      t = run<T>(iters, blocks, out, st, e0, e1);
    }
    iters = (int)std::fmin((double)(1 << 26), iters * std::fmax(1.0, 0.05 / t));
    for (int r = 0; r < 5; ++r) {
      t = run<T>(iters, blocks, out, st, e0, e1);
      const double flops = 2.0 * blocks * 256.0 * iters * 16.0 * 8.0;
      best = std::fmax(best, flops / t);
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  LB_CUDA(cudaFree(out));
  return best * 1e-12;
}

}  // namespace

extern "C" lobpcg_status lobpcg_probe_fma_rate(int fp64, double* tflops, lobpcg_stream stream) {
  using namespace lobpcg;
  if (!tflops) {
    set_thread_error("lobpcg_probe_fma_rate: tflops must not be NULL");
    return LOBPCG_EINVAL;
  }
  try {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    *tflops = fp64 ? probe<double>(st) : probe<float>(st);
    return LOBPCG_OK;
  } catch (const std::exception& ex) {
    set_thread_error(ex.what());
    return LOBPCG_ECUDA;
  }
}
