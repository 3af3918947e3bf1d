// Arithmetic peak of the FP32 and FP64 pipes (the ceiling of the FP64
// banded passes, which run at one multiply-add per 8-byte load and are
// bound by the FP64 pipe on this GPU, not by HBM).  A measurement utility
// of the library, not a step of the method.
#include <cuda_runtime.h>

#include <string>

#include "common.cuh"
#include "lcmg.h"

namespace lcmg {

void set_error_message(const std::string& s);

constexpr int kFmaChains = 8;     // independent accumulators per thread
constexpr int kFmaThreads = 256;

// every thread runs kFmaChains independent chains of iters multiply-adds;
// the result is written only when it equals a value it never takes, so the
// chains are live but nothing is stored
template <class T>
__global__ void __launch_bounds__(kFmaThreads) k_fma_peak(int iters, T a, T b, T* sink) {
  T acc[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) acc[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) acc[k] = acc[k] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += acc[k];
  if (s == (T)-12345.678) *sink = s;
}

template <class T>
static double measure(int device) {
  LCMG_CUDA(cudaSetDevice(device));
  int sms = 0, per = 0;
  LCMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  LCMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fma_peak<T>, kFmaThreads, 0));
  const int blocks = sms * (per > 0 ? per : 1);
  const int iters = sizeof(T) == 8 ? 4096 : 65536;
  T* sink = nullptr;
  LCMG_CUDA(cudaMalloc(&sink, sizeof(T)));
  cudaEvent_t e0, e1;
  LCMG_CUDA(cudaEventCreate(&e0));
  LCMG_CUDA(cudaEventCreate(&e1));
  // a = 1 - 2^-20, b = 2^-30: the values stay finite and normal
  const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1073741824.0);
  k_fma_peak<T><<<blocks, kFmaThreads>>>(iters, a, b, sink);  // warm-up
  LCMG_CUDA(cudaGetLastError());
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    LCMG_CUDA(cudaEventRecord(e0));
    k_fma_peak<T><<<blocks, kFmaThreads>>>(iters, a, b, sink);
    LCMG_CUDA(cudaEventRecord(e1));
    LCMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    LCMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  const double flops = 2.0 * (double)blocks * kFmaThreads * kFmaChains * (double)iters;
  return flops / (best * 1e-3) / 1e12;
}

}  // namespace lcmg

extern "C" int lcmg_fma_peak(int device, int32_t precision, double* tflops) {
  try {
    if (!tflops) throw lcmg::ArgError("null output pointer");
    if (precision != LCMG_PREC_FP64 && precision != LCMG_PREC_MIXED) throw lcmg::ArgError("invalid precision");
    *tflops = precision == LCMG_PREC_FP64 ? lcmg::measure<double>(device) : lcmg::measure<float>(device);
    return LCMG_OK;
  } catch (const lcmg::ArgError& e) {
    lcmg::set_error_message(e.what());
    return LCMG_ERR_INVALID_ARG;
  } catch (const std::exception& e) {
    lcmg::set_error_message(e.what());
    return LCMG_ERR_CUDA;
  }
}
