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

}  // namespace feks
