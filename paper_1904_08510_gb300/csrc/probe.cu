// FMA throughput probe: the measured denominator of the solver kernel's ALU
// roofline. The solve is bound by the FP64 pipe, whose peak neither an HBM copy
// nor a BF16 GEMM measures; this kernel runs independent FMA chains on every
// SM and reports the achieved FMA rate (2 flops per FMA).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/sdcef.h"

namespace sdcef_impl {
int report_error(int code, const char* msg);
}
using sdcef_impl::report_error;

namespace {

constexpr int kChains = 8;     // independent FMA chains per thread
constexpr int kUnroll = 16;    // FMAs per chain per loop trip
constexpr int kThreads = 256;

// a <- a x + y with |x| < 1: every chain converges to y / (1 - x), so no
// value leaves the normal range; the sum of the chains is stored so that
// nothing is dead code.
template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(T* out, int iters, T x, T y) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], x, y);
    }
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[(size_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

template <typename T>
int run_probe(int iters, cudaStream_t st, double* tflops) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<T>, kThreads, 0);
  if (e != cudaSuccess) return report_error(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  const int grid = sms * std::max(per_sm, 1);
  T* out = nullptr;
  e = cudaMalloc(&out, sizeof(T) * (size_t)grid * kThreads);
  if (e != cudaSuccess) return report_error(SDCEF_ERR_NOMEM, cudaGetErrorString(e));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T x = (T)0.999, y = (T)1e-4;
  fma_probe_kernel<T><<<grid, kThreads, 0, st>>>(out, iters, x, y);   // warm-up
  float best = 0.0f;
  for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
    cudaEventRecord(e0, st);
    fma_probe_kernel<T><<<grid, kThreads, 0, st>>>(out, iters, x, y);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (best == 0.0f || ms < best)) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return report_error(SDCEF_ERR_CUDA, cudaGetErrorString(e));
  const double flops = 2.0 * kChains * kUnroll * (double)iters * grid * kThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return SDCEF_SUCCESS;
}

}  // namespace

extern "C" int sdcef_fma_peak_probe(int precision, int iters, void* stream, double* tflops) {
  if (!tflops || iters < 1 || (precision != SDCEF_FP64 && precision != SDCEF_MIXED))
    return report_error(SDCEF_ERR_INVALID, "fma_peak_probe: precision must be FP64 or MIXED "
                                           "(FP32), iters >= 1, tflops non-NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return precision == SDCEF_FP64 ? run_probe<double>(iters, st, tflops)
                                 : run_probe<float>(iters, st, tflops);
}
