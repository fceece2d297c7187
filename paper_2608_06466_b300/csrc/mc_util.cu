// mc_util.cu -- measurement utility: FP64 / FP32 fused multiply-add issue rate
// of the current device (the ceiling of this ALU-bound burn), with CUDA events.
#include "mc_internal.h"

namespace {

template <typename T>
__global__ void k_fma_rate(T *out, int iters, T a, T b) {
  T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
    x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
    x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
  }
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
mc_status rate(int iters, int blocks_per_sm, double *tflops) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 128, blocks = sms * blocks_per_sm;
  T *buf = nullptr;
  cudaError_t e = mc::dev_malloc((void **)&buf, sizeof(T) * (size_t)blocks * threads);
  if (e != cudaSuccess) return mc::cuda_error(e, "probe allocation");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_rate<T><<<blocks, threads>>>(buf, 16, (T)1.0000001, (T)1e-9);
  cudaEventRecord(e0);
  k_fma_rate<T><<<blocks, threads>>>(buf, iters, (T)1.0000001, (T)1e-9);
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  mc::count_launch(2);
  if (e != cudaSuccess) return mc::cuda_error(e, "probe");
  *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
  return MC_OK;
}

}  // namespace

extern "C" mc_status mc_probe_fma_rate(double *tflops_fp64, double *tflops_fp32) {
  mc_status s = MC_OK;
  if (tflops_fp64) s = rate<double>(4000, 8, tflops_fp64);
  if (s == MC_OK && tflops_fp32) s = rate<float>(40000, 8, tflops_fp32);
  return s;
}
