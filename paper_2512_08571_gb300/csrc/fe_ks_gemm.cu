// Dense FP64 GEMM for the Rayleigh-Ritz step (Algorithm 3): a thin wrapper of
// cuBLAS, optionally with its FP64 emulation on integer tensor cores
// (fixed-point slices, CUBLAS_COMPUTE_64F_EMULATED_FIXEDPOINT).  The Gram
// matrices Y^H Y, Y^H (Hs Y) and the rotation Y E are plain library GEMMs.
#include <cublas_v2.h>

#include <mutex>

#include "fe_ks_internal.h"

namespace feks {

static std::mutex g_blas_mu;
static cublasHandle_t g_blas[64] = {};

static fe_ks_status blas_handle(cublasHandle_t* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(FE_KS_ERR_CUDA, "cudaGetDevice failed");
  std::lock_guard<std::mutex> lock(g_blas_mu);
  if (!g_blas[dev] && cublasCreate(&g_blas[dev]) != CUBLAS_STATUS_SUCCESS)
    return fail(FE_KS_ERR_CUDA, "cublasCreate failed");
  *out = g_blas[dev];
  return FE_KS_OK;
}

}  // namespace feks

using namespace feks;

extern "C" fe_ks_status fe_ks_gemm_f64(int trans_a, int trans_b, int64_t m, int64_t n, int64_t k, double alpha,
                                       const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                                       double* C, int64_t ldc, int emulated, void* cuda_stream) {
  set_error("");
  if (!A || !B || !C) return fail(FE_KS_ERR_ARG, "NULL matrix");
  if (m < 0 || n < 0 || k < 0 || m > INT32_MAX || n > INT32_MAX || k > INT32_MAX || lda > INT32_MAX ||
      ldb > INT32_MAX || ldc > INT32_MAX)
    return fail(FE_KS_ERR_ARG, "GEMM sizes out of range");
  cublasHandle_t h;
  fe_ks_status st = blas_handle(&h);
  if (st != FE_KS_OK) return st;
  cublasSetStream(h, static_cast<cudaStream_t>(cuda_stream));
  const cublasOperation_t ta = trans_a ? CUBLAS_OP_T : CUBLAS_OP_N;
  const cublasOperation_t tb = trans_b ? CUBLAS_OP_T : CUBLAS_OP_N;
  const cublasComputeType_t ct = emulated ? CUBLAS_COMPUTE_64F_EMULATED_FIXEDPOINT : CUBLAS_COMPUTE_64F;
  // emulation: always use it when asked (the default strategy keeps native FP64 where it estimates that to be faster)
  cublasSetMathMode(h, emulated ? CUBLAS_FP64_EMULATED_FIXEDPOINT_MATH : CUBLAS_DEFAULT_MATH);
  cublasSetEmulationStrategy(h, emulated ? CUBLAS_EMULATION_STRATEGY_EAGER : CUBLAS_EMULATION_STRATEGY_DEFAULT);
  cublasStatus_t s = cublasGemmEx(h, ta, tb, (int)m, (int)n, (int)k, &alpha, A, CUDA_R_64F, (int)lda, B, CUDA_R_64F,
                                  (int)ldb, &beta, C, CUDA_R_64F, (int)ldc, ct, CUBLAS_GEMM_DEFAULT);
  if (s != CUBLAS_STATUS_SUCCESS)
    return fail(emulated ? FE_KS_ERR_UNSUPPORTED : FE_KS_ERR_CUDA,
                std::string("cublasGemmEx failed with status ") + std::to_string((int)s));
  return FE_KS_OK;
}

