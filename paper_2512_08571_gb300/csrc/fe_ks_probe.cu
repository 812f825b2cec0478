// Diagnostics: a bounded FMA-throughput probe giving the live FP64 / FP32
// pipe peak that the roofline of the FP64 / FP32 operator is measured against.
#include "fe_ks_internal.h"

namespace feks {

template <typename T, int CH>
__global__ void fma_probe_kernel(T* out, int iters, T a, T b) {
  T acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = fma(acc[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace feks

using namespace feks;

extern "C" fe_ks_status fe_ks_measure_fma_peak(int precision, double* tflops) {
  if (!tflops) return fail(FE_KS_ERR_ARG, "tflops is NULL");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(FE_KS_ERR_CUDA, "no CUDA device");
  const int blocks = sms * 4, threads = 256;
  const int iters = (precision == FE_KS_F64) ? 4000 : 200000;
  void* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * blocks * threads) != cudaSuccess) return fail(FE_KS_ERR_OOM, "probe buffer");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  for (int rep = 0; rep < 2; ++rep) {   // first run warms up
    cudaEventRecord(e0);
    if (precision == FE_KS_F64)
      fma_probe_kernel<double, 8><<<blocks, threads>>>((double*)buf, iters, 0.999, 0.001);
    else
      fma_probe_kernel<float, 8><<<blocks, threads>>>((float*)buf, iters, 0.999f, 0.001f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, cudaGetErrorString(err));
  *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
  return FE_KS_OK;
}
