// FMA throughput probe: the ALU roofline denominator for the FP64 path.
// Eight independent FMA chains per thread keep the pipes full; 8 resident
// blocks of 256 threads per SM.
#include "common.h"

namespace aim {

template <typename T>
__global__ void k_fma_chain(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T> static int run(int iters, double* tflops) {
  int dev = 0, sms = 0;
  AIM_CUDA_TRY(cudaGetDevice(&dev));
  AIM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  AIM_CUDA_TRY(cudaMalloc(&out, sizeof(T) * blocks * threads));
  cudaEvent_t e0, e1;
  AIM_CUDA_TRY(cudaEventCreate(&e0));
  AIM_CUDA_TRY(cudaEventCreate(&e1));
  k_fma_chain<T><<<blocks, threads>>>(out, iters / 10, (T)0.999, (T)1e-3);  // warm-up
  AIM_CUDA_TRY(cudaEventRecord(e0));
  k_fma_chain<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)1e-3);
  AIM_CUDA_TRY(cudaEventRecord(e1));
  AIM_CUDA_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  AIM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return AIM_OK;
}

int probe_fma(int which, double* tflops) {
  return which == 64 ? run<double>(2000, tflops) : run<float>(20000, tflops);
}

}  // namespace aim
