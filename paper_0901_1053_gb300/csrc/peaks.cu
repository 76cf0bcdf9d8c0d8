// Arithmetic-rate microbenchmark (tetm_measure_fma_rate): the float64 and
// float32 fused multiply-add rates of the device, the denominators of the
// ALU roofline of the float64 update kernels. Each thread runs eight
// independent FMA chains (enough to cover the pipeline latency), the grid
// fills every SM several times, and the rate is flops (2 per FMA) over the
// kernel time measured with CUDA events on the given stream.
#include <cuda_runtime.h>

#include "tetm.h"

namespace {

template <typename T>
__global__ void fma_chains(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = T(threadIdx.x + q) * T(1e-7);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  if (s == T(-1.2345)) out[0] = s;  // keeps the chains live; never true for these inputs
}

template <typename T>
int rate(double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TETM_E_CUDA;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return TETM_E_NOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8, threads = 256;
  const int iters = sizeof(T) == 8 ? 4096 : 16384;
  fma_chains<T><<<blocks, threads, 0, st>>>(out, iters / 16, T(0.999999), T(1e-9));  // warm-up
  cudaEventRecord(e0, st);
  fma_chains<T><<<blocks, threads, 0, st>>>(out, iters, T(0.999999), T(1e-9));
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || ms <= 0.f) {
    cudaGetLastError();
    return TETM_E_CUDA;
  }
  const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return TETM_OK;
}

}  // namespace

extern "C" int tetm_measure_fma_rate(int32_t precision, double* tflops, void* stream) {
  if (!tflops || (precision != TETM_FP64 && precision != TETM_FP32)) return TETM_E_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return precision == TETM_FP64 ? rate<double>(tflops, st) : rate<float>(tflops, st);
}
