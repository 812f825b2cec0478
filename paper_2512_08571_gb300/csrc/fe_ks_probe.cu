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

// Warp-level tensor-core rate: CH independent m16n8k16 BF16 MMAs per step,
// operands held in registers (no memory traffic inside the loop).
template <int CH>
__global__ void mma_probe_kernel(float* out, int iters, unsigned a_bits, unsigned b_bits) {
  float c[CH][4];
#pragma unroll
  for (int k = 0; k < CH; ++k)
#pragma unroll
    for (int r = 0; r < 4; ++r) c[k][r] = 0.f;
  const unsigned a0 = a_bits ^ (threadIdx.x & 1u), a1 = a_bits, a2 = a_bits, a3 = a_bits ^ 2u;
  const unsigned b0 = b_bits, b1 = b_bits ^ (threadIdx.x & 2u);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CH; ++k)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+f"(c[k][0]), "+f"(c[k][1]), "+f"(c[k][2]), "+f"(c[k][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += c[k][0] + c[k][1] + c[k][2] + c[k][3];
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
  const bool tc = precision == FE_KS_BF16;
  const int iters = tc ? 20000 : (precision == FE_KS_F64) ? 4000 : 200000;
  void* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * blocks * threads) != cudaSuccess) return fail(FE_KS_ERR_OOM, "probe buffer");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  for (int rep = 0; rep < 2; ++rep) {   // first run warms up
    cudaEventRecord(e0);
    if (tc)   // bf16 pairs 0x3C00 = 2^-7 (products stay far from overflow)
      mma_probe_kernel<8><<<blocks, threads>>>((float*)buf, iters, 0x3C003C00u, 0x3C003C00u);
    else if (precision == FE_KS_F64)
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
  if (tc)   // 8 MMAs of 16 x 8 x 16 per warp per step
    *tflops = 2.0 * 16 * 8 * 16 * 8.0 * (double)iters * blocks * (threads / 32) / (ms * 1e-3) / 1e12;
  else
    *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
  return FE_KS_OK;
}
