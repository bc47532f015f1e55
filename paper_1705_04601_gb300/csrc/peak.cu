// Measured fused multiply-add rates of the current device, the denominators
// of the roofline fractions of the FP64 and FP32 CUDA-core kernels: a kernel
// of independent FMA chains on every streaming multiprocessor, timed with
// CUDA events.  Not part of the method.
#include <cstdint>

#include "kernels.h"

namespace h2sp {
namespace {

constexpr int kChains = 8;      // independent chains per thread
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(T *__restrict__ out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = T(threadIdx.x + 1) * T(1e-3) + T(i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  // a store that depends on every chain keeps them all
  if (s == T(-1.2345)) out[blockIdx.x] = s;
}

template <typename T>
cudaError_t time_peak(int iters, double *tflops, cudaStream_t s) {
  const int nsm = device_sms();
  const int blocks = nsm * 8;
  T *out = nullptr;
  cudaError_t e = cudaMallocAsync(&out, sizeof(T) * size_t(blocks), s);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T a = T(0.999999), b = T(1e-7);
  k_fma_peak<T><<<blocks, kPeakThreads, 0, s>>>(out, iters / 8, a, b);  // warm-up
  cudaEventRecord(e0, s);
  k_fma_peak<T><<<blocks, kPeakThreads, 0, s>>>(out, iters, a, b);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess && ms > 0.f)
    *tflops = 2.0 * kChains * double(iters) * double(blocks) * kPeakThreads / (double(ms) * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  cudaStreamSynchronize(s);
  return e;
}

}  // namespace

cudaError_t measure_fma_peak(int kind, double *tflops, cudaStream_t s) {
  // about 50 ms each at the nominal rates (FP64 ~1.25, FP32 ~80 TFLOP/s)
  return kind == 0 ? time_peak<double>(12000, tflops, s) : time_peak<float>(800000, tflops, s);
}

}  // namespace h2sp
