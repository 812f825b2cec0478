// The batched persistent kernel for one block size (compiled once per size
// with -DFEKS_BNT=<threads>, so the sizes build in parallel).
#include "fe_ks_batched.cuh"

#ifndef FEKS_BNT
#error "FEKS_BNT must be defined"
#endif

namespace feks {

// Two resident CTAs per SM halve the register budget; at 672 threads that
// budget (48 registers) spills heavily, so that size is built for one CTA only.
constexpr bool kTwoPerSm = FEKS_BNT <= 512;

template <>
cudaError_t batched_prepare<FEKS_BNT>(size_t smem, int blocks_per_sm, int* per_sm) {
  cudaError_t err = cudaFuncSetAttribute(fe_batched_kernel<FEKS_BNT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  if constexpr (kTwoPerSm) {
    err = cudaFuncSetAttribute(fe_batched_kernel<FEKS_BNT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    if (blocks_per_sm == 2)
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fe_batched_kernel<FEKS_BNT, 2>, FEKS_BNT, smem);
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fe_batched_kernel<FEKS_BNT, 1>, FEKS_BNT, smem);
}

template <>
cudaError_t batched_launch<FEKS_BNT>(const BatchParams& P, int grid, size_t smem, int blocks_per_sm, cudaStream_t s) {
  if constexpr (kTwoPerSm) {
    if (blocks_per_sm == 2) {
      fe_batched_kernel<FEKS_BNT, 2><<<grid, FEKS_BNT, smem, s>>>(P);
      return cudaGetLastError();
    }
  }
  fe_batched_kernel<FEKS_BNT, 1><<<grid, FEKS_BNT, smem, s>>>(P);
  return cudaGetLastError();
}

// Class objects: their register budget is that of one class's routines, capped
// at half the register file (MINB = 2), so that one CTA of the FP64 object and
// one of the FP32 object can share an SM when the shared memory allows it.
template <>
cudaError_t batched_prepare_class<FEKS_BNT>(int cls, size_t smem, int* per_sm) {
  auto k = cls == kClassF64 ? fe_batched_kernel<FEKS_BNT, 2, kClassF64> : fe_batched_kernel<FEKS_BNT, 2, kClassF32>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, FEKS_BNT, smem);
}

template <>
cudaError_t batched_launch_class<FEKS_BNT>(int cls, const BatchParams& P, int grid, size_t smem, cudaStream_t s) {
  if (cls == kClassF64)
    fe_batched_kernel<FEKS_BNT, 2, kClassF64><<<grid, FEKS_BNT, smem, s>>>(P);
  else
    fe_batched_kernel<FEKS_BNT, 2, kClassF32><<<grid, FEKS_BNT, smem, s>>>(P);
  return cudaGetLastError();
}

}  // namespace feks
