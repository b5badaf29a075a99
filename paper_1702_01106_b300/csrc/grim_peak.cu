// FMA-throughput microbenchmark: the float64 and float32 peaks that bound
// the ALU-limited Newton kernels (roofline denominators).
#include <cuda_runtime.h>
#include "../../include/grim.h"

namespace grim {

// Eight independent FMA chains per thread, no memory traffic in the loop.
template <typename T>
__global__ void fma_chains(T* out, int iters, T a, T b) {
  T x0 = T(threadIdx.x) * T(1e-3), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
  T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
#pragma unroll 4
  for (int i = 0; i < iters; i++) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
static double time_chains(int blocks, int threads, int iters, T* buf) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains<T><<<blocks, threads>>>(buf, iters / 8, T(0.999999), T(1e-6));  // warm-up
  cudaEventRecord(e0);
  fma_chains<T><<<blocks, threads>>>(buf, iters, T(0.999999), T(1e-6));
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  double flops = 2.0 * 8.0 * (double)blocks * threads * (double)iters;
  return flops / (ms * 1e-3) / 1e12;
}

}  // namespace grim

extern "C" int grim_peak_flops(double* fp64_tflops, double* fp32_tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GRIM_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 8;
  void* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * threads * blocks) != cudaSuccess) return GRIM_ENOMEM;
  double t64 = grim::time_chains<double>(blocks, threads, 4096, (double*)buf);
  double t32 = grim::time_chains<float>(blocks, threads, 65536, (float*)buf);
  cudaError_t e = cudaDeviceSynchronize();
  cudaFree(buf);
  if (e != cudaSuccess) return GRIM_ECUDA;
  if (fp64_tflops) *fp64_tflops = t64;
  if (fp32_tflops) *fp32_tflops = t32;
  return GRIM_OK;
}
