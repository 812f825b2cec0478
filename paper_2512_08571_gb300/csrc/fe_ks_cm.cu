// Cell-matrix (CM) baseline: the local part of H applied as dense per-cell
// matrices, as in the paper's cell-matrix method that the matrix-free
// algorithms are measured against (Sec. 3: H^(e) assembled by quadrature and
// applied cell by cell, then the assembly Q^T).
//
//   setup : H_loc^(e) [n_p^3][n_p^3] for every cell, FP64, obtained by running
//           the library's FP64 matrix-free cell kernel on identity blocks over a
//           disjoint per-cell DoF numbering (column j of H^(e) is H^(e) e_j), so
//           the cell matrices and the matrix-free operator agree by construction;
//           stored in the apply precision (FP64 or FP32).
//   apply : per colour, gather X^(e) into dense blocks, one batched library GEMM
//           Y^(e) = H_loc^(e) X^(e) over the colour's cells, and a colour-exclusive
//           scatter-add that also adds the nonlocal expansion F Delta P; the
//           projection P is the operator's own pair-form kernel.
// Real operators only.  The GEMMs are plain library GEMMs (cuBLAS) on purpose:
// this is the baseline, not the method.
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include <vector>

#include "fe_ks_internal.h"

namespace feks {

__global__ void k_cm_identity(double* X, int64_t rows, int np3) {
  const int64_t n = rows * np3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / np3;
    X[i] = ((r % np3) == (i % np3)) ? 1.0 : 0.0;
  }
}

// disjoint numbering: node n of cell e -> (e % chunk) n_p^3 + n
__global__ void k_cm_disjoint(int* dis, int64_t E, int chunk, int np3) {
  const int64_t n = E * np3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dis[i] = (int)(((i / np3) % chunk) * np3 + i % np3);
}

__global__ void k_cm_iota(int* v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (int)i;
}

__global__ void k_cm_to_float(float* dst, const double* src, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

__global__ void k_cm_to_bf16(__nv_bfloat16* dst, const double* src, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __double2bfloat16(src[i]);
}

// BF16 operand blocks from FP32 X (round to nearest even)
__global__ void k_cm_gather_bf16(__nv_bfloat16* __restrict__ Xg, const float* __restrict__ X, int64_t ld, int ncols,
                                 const int* __restrict__ cell_dofs, const int* __restrict__ cells, int n_cells,
                                 int np3) {
  const int64_t rows = (int64_t)n_cells * np3;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const int c = (int)(r / np3), n = (int)(r % np3);
    const int d = cell_dofs[(int64_t)cells[c] * np3 + n];
    for (int v = threadIdx.x; v < ncols; v += blockDim.x) Xg[r * ncols + v] = __float2bfloat16_rn(X[(int64_t)d * ld + v]);
  }
}

// Xg[c][n][v] = X[dofs(cell c, n)][v] for the cells of one colour
template <typename T>
__global__ void k_cm_gather(T* __restrict__ Xg, const T* __restrict__ X, int64_t ld, int ncols,
                            const int* __restrict__ cell_dofs, const int* __restrict__ cells, int n_cells, int np3) {
  const int64_t rows = (int64_t)n_cells * np3;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const int c = (int)(r / np3), n = (int)(r % np3);
    const int d = cell_dofs[(int64_t)cells[c] * np3 + n];
    for (int v = threadIdx.x; v < ncols; v += blockDim.x) Xg[r * ncols + v] = X[(int64_t)d * ld + v];
  }
}

// batched-GEMM operand pointers of one colour (TA: operand type, TC: result type)
template <typename TA, typename TC>
__global__ void k_cm_ptrs(const TA** A, const TA** B, TC** C, const TA* Xg, const TA* H, TC* Yg, const int* cells,
                          int n_cells, int np3, int ncols) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x) {
    A[c] = Xg + (int64_t)c * np3 * ncols;
    B[c] = H + (int64_t)cells[c] * np3 * np3;
    C[c] = Yg + (int64_t)c * np3 * ncols;
  }
}

// Y[dofs(cell c, n)][v] += Yg[c][n][v] + sum_pairs sum_b F[pair][b][n] Q[atom][b][v]
// (colour-exclusive: no other cell of the colour touches the same rows)
template <typename T>
__global__ void k_cm_scatter(T* __restrict__ Y, const T* __restrict__ Yg, int64_t ld, int ncols,
                             const int* __restrict__ cell_dofs, const int* __restrict__ cells, int n_cells, int np3,
                             const int* __restrict__ cell_pair_ptr, const int* __restrict__ cell_pairs,
                             const int* __restrict__ pair_atom, const T* __restrict__ F, const T* __restrict__ Q,
                             int n_proj) {
  const int64_t rows = (int64_t)n_cells * np3;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const int c = (int)(r / np3), n = (int)(r % np3);
    const int e = cells[c];
    const int d = cell_dofs[(int64_t)e * np3 + n];
    const int pb = cell_pair_ptr ? cell_pair_ptr[e] : 0, pe = cell_pair_ptr ? cell_pair_ptr[e + 1] : 0;
    for (int v = threadIdx.x; v < ncols; v += blockDim.x) {
      T y = Yg[r * ncols + v];
      for (int pi = pb; pi < pe; ++pi) {
        const int pr = cell_pairs[pi];
        const T* Qa = Q + (int64_t)pair_atom[pr] * n_proj * ld;
        for (int b = 0; b < n_proj; ++b) y = fma(F[((int64_t)pr * n_proj + b) * np3 + n], Qa[(int64_t)b * ld + v], y);
      }
      Y[(int64_t)d * ld + v] += y;
    }
  }
}

static int ew_grid(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 32); }

}  // namespace feks

using namespace feks;

struct fe_ks_cm {
  fe_ks_ctx* ctx = nullptr;
  int prec = FE_KS_F64;
  int64_t n_v_max = 0;
  void* H = nullptr;
  void* Xg = nullptr;
  void* Yg = nullptr;
  void** ptrs = nullptr;   // [3][max_cells]
  int max_cells = 0;
  cublasHandle_t blas = nullptr;
  double setup_ms = 0.0;
  size_t bytes = 0;
};

static void cm_free(fe_ks_cm* cm) {
  if (!cm) return;
  cudaFree(cm->H);
  cudaFree(cm->Xg);
  cudaFree(cm->Yg);
  cudaFree(cm->ptrs);
  if (cm->blas) cublasDestroy(cm->blas);
  delete cm;
}

extern "C" {

fe_ks_status fe_ks_cm_create(fe_ks_ctx* ctx, int precision, int64_t n_v_max, fe_ks_cm** out) {
  set_error("");
  if (!ctx || !out) return fail(FE_KS_ERR_ARG, "NULL argument");
  *out = nullptr;
  Ctx& c = ctx->c;
  if (c.cplx) return fail(FE_KS_ERR_UNSUPPORTED, "the cell-matrix baseline supports real operators");
  if (precision != FE_KS_F64 && precision != FE_KS_F32 && precision != FE_KS_BF16)
    return fail(FE_KS_ERR_UNSUPPORTED, "precision F64, F32 or BF16");
  if (n_v_max < 1 || n_v_max > c.n_v_max) return fail(FE_KS_ERR_ARG, "n_v_max must be in 1..the context's n_v_max");
  const int np3 = c.np3;
  const int64_t E = c.E;
  const size_t esz = precision == FE_KS_F64 ? 8 : precision == FE_KS_F32 ? 4 : 2;   // cell-matrix entries
  cudaStream_t s = c.stream;
  fe_ks_cm* cm = new fe_ks_cm;
  cm->ctx = ctx;
  cm->prec = precision;
  cm->n_v_max = n_v_max;
  for (size_t k = 0; k + 1 < c.colour_ptr.size(); ++k)
    cm->max_cells = std::max(cm->max_cells, c.colour_ptr[k + 1] - c.colour_ptr[k]);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  // cell matrices, computed in chunks of cells with the FP64 matrix-free kernel
  const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(E, (int64_t)(2.0e9 / ((double)np3 * np3 * 8))));
  double* Xid = nullptr;
  double* Ych = nullptr;
  int* dis = nullptr;
  int* iota = nullptr;
  auto bad = [&](const char* what, fe_ks_status code = FE_KS_ERR_OOM) {
    cudaFree(Xid);
    cudaFree(Ych);
    cudaFree(dis);
    cudaFree(iota);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cm_free(cm);
    cudaGetLastError();
    return fail(code, std::string("cell-matrix setup: ") + what);
  };
  const size_t hbytes = (size_t)E * np3 * np3 * esz;
  if (cudaMalloc(&cm->H, hbytes) != cudaSuccess) return bad("cell matrices");
  if (cudaMalloc(&Xid, (size_t)chunk * np3 * np3 * 8) != cudaSuccess) return bad("identity blocks");
  if (precision != FE_KS_F64 && cudaMalloc(&Ych, (size_t)chunk * np3 * np3 * 8) != cudaSuccess)
    return bad("chunk buffer");
  if (cudaMalloc(&dis, (size_t)E * np3 * sizeof(int)) != cudaSuccess) return bad("disjoint map");
  if (cudaMalloc(&iota, (size_t)E * sizeof(int)) != cudaSuccess) return bad("cell list");
  k_cm_identity<<<ew_grid((int64_t)chunk * np3 * np3), 256, 0, s>>>(Xid, (int64_t)chunk * np3, np3);
  k_cm_disjoint<<<ew_grid(E * np3), 256, 0, s>>>(dis, E, chunk, np3);
  k_cm_iota<<<ew_grid(E), 256, 0, s>>>(iota, E);
  LocalParams<double> lp{};
  lp.X = Xid;
  lp.ld = np3;
  lp.ncols = np3;
  lp.cell_dofs = dis;
  lp.coef = c.f64.coef;
  lp.ncoef = c.ncoef;
  lp.gga = c.gga;
  lp.alpha = 1.0;
  lp.tab = c.f64.tab;
  for (int64_t e0c = 0; e0c < E; e0c += chunk) {
    const int nc = (int)std::min<int64_t>(chunk, E - e0c);
    double* Y = precision == FE_KS_F64 ? static_cast<double*>(cm->H) + (size_t)e0c * np3 * np3 : Ych;
    cudaMemsetAsync(Y, 0, (size_t)nc * np3 * np3 * 8, s);
    lp.Y = Y;
    lp.cells = iota + e0c;
    lp.n_cells = nc;
    cudaError_t err = launch_local<double, double>(c, lp, s);
    if (err != cudaSuccess) return bad(cudaGetErrorString(err), FE_KS_ERR_CUDA);
    if (precision == FE_KS_F32)
      k_cm_to_float<<<ew_grid((int64_t)nc * np3 * np3), 256, 0, s>>>(
          static_cast<float*>(cm->H) + (size_t)e0c * np3 * np3, Y, (int64_t)nc * np3 * np3);
    else if (precision == FE_KS_BF16)
      k_cm_to_bf16<<<ew_grid((int64_t)nc * np3 * np3), 256, 0, s>>>(
          static_cast<__nv_bfloat16*>(cm->H) + (size_t)e0c * np3 * np3, Y, (int64_t)nc * np3 * np3);
  }
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cm->setup_ms = ms;
  cudaFree(Xid);
  cudaFree(Ych);
  cudaFree(dis);
  cudaFree(iota);
  Xid = Ych = nullptr;
  dis = iota = nullptr;
  // apply buffers
  // gathered X blocks and GEMM results (BF16: FP32 results, so both sized for 4 bytes)
  const size_t gbytes = (size_t)cm->max_cells * np3 * n_v_max * std::max<size_t>(esz, 4);
  if (cudaMalloc(&cm->Xg, gbytes) != cudaSuccess || cudaMalloc(&cm->Yg, gbytes) != cudaSuccess ||
      cudaMalloc(&cm->ptrs, (size_t)3 * cm->max_cells * sizeof(void*)) != cudaSuccess)
    return bad("apply buffers");
  if (cublasCreate(&cm->blas) != CUBLAS_STATUS_SUCCESS) return bad("cublasCreate", FE_KS_ERR_CUDA);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cm->bytes = hbytes + 2 * gbytes;
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    cm_free(cm);
    return fail(FE_KS_ERR_CUDA, std::string("cell-matrix setup: ") + cudaGetErrorString(err));
  }
  *out = cm;
  return FE_KS_OK;
}

fe_ks_status fe_ks_cm_apply(fe_ks_cm* cm, const void* Xv, void* Yv, int64_t n_v) {
  set_error("");
  if (!cm || !Xv || !Yv) return fail(FE_KS_ERR_ARG, "NULL argument");
  if (n_v < 1 || n_v > cm->n_v_max) return fail(FE_KS_ERR_ARG, "n_v must be in 1..n_v_max");
  Ctx& c = cm->ctx->c;
  cudaStream_t s = c.stream;
  const int np3 = c.np3, ncols = (int)n_v;
  const bool f64 = cm->prec == FE_KS_F64;
  const bool bf16 = cm->prec == FE_KS_BF16;
  const size_t esz = f64 ? 8 : 4;   // X and Y (BF16: FP32 storage)
  cudaMemsetAsync(Yv, 0, (size_t)c.m * ncols * esz, s);
  const bool nl = (c.terms & FE_KS_TERM_NL) && c.n_pairs > 0;
  if (nl) {   // P = Delta F^T X, the operator's own projection
    cudaError_t err;
    if (f64) {
      ProjParams<double> pp{};
      pp.X = static_cast<const double*>(Xv);
      pp.ld = ncols;
      pp.ncols = ncols;
      pp.cell_dofs = c.cell_dofs;
      pp.atom_pair_ptr = c.atom_pair_ptr;
      pp.pair_cell = c.pair_cell;
      pp.F = c.f64.F;
      pp.h = c.h64;
      pp.Q = c.f64.Q;
      pp.n_proj = c.n_proj;
      pp.np3 = np3;
      pp.part = c.f64.part;
      pp.n_pairs = c.n_pairs;
      err = launch_proj_pairs<double>(c, pp, c.n_atoms, s);
    } else {
      ProjParams<float> pp{};
      pp.X = static_cast<const float*>(Xv);
      pp.ld = ncols;
      pp.ncols = ncols;
      pp.cell_dofs = c.cell_dofs;
      pp.atom_pair_ptr = c.atom_pair_ptr;
      pp.pair_cell = c.pair_cell;
      pp.F = c.f32.F;
      pp.h = c.h32;
      pp.Q = c.f32.Q;
      pp.n_proj = c.n_proj;
      pp.np3 = np3;
      pp.part = c.f32.part;
      pp.n_pairs = c.n_pairs;
      err = launch_proj_pairs<float>(c, pp, c.n_atoms, s);
    }
    if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("projection: ") + cudaGetErrorString(err));
  }
  cublasSetStream(cm->blas, s);
  for (size_t col = 0; col + 1 < c.colour_ptr.size(); ++col) {
    const int* cells = c.colour_cells + c.colour_ptr[col];
    const int n = c.colour_ptr[col + 1] - c.colour_ptr[col];
    if (n == 0) continue;
    const int grid = (int)std::min<int64_t>((int64_t)n * np3, 152 * 64);
    cublasStatus_t bs;
    if (f64) {
      const double* X = static_cast<const double*>(Xv);
      double* Y = static_cast<double*>(Yv);
      double* Xg = static_cast<double*>(cm->Xg);
      double* Yg = static_cast<double*>(cm->Yg);
      // three pointer arrays of max_cells entries each: A, B, C operands
      const double** A = (const double**)(cm->ptrs);
      const double** B = (const double**)(cm->ptrs + cm->max_cells);
      double** C = (double**)(cm->ptrs + 2 * (size_t)cm->max_cells);
      k_cm_gather<double><<<grid, 128, 0, s>>>(Xg, X, ncols, ncols, c.cell_dofs, cells, n, np3);
      k_cm_ptrs<double, double><<<(n + 127) / 128, 128, 0, s>>>(A, B, C, Xg, static_cast<const double*>(cm->H), Yg, cells, n,
                                                       np3, ncols);
      const double one = 1.0, zero = 0.0;
      bs = cublasDgemmBatched(cm->blas, CUBLAS_OP_N, CUBLAS_OP_N, ncols, np3, np3, &one, A, ncols, B, np3, &zero, C,
                              ncols, n);
      k_cm_scatter<double><<<grid, 128, 0, s>>>(Y, Yg, ncols, ncols, c.cell_dofs, cells, n, np3,
                                                nl ? c.cell_pair_ptr : nullptr, c.cell_pairs, c.pair_atom, c.f64.F,
                                                c.f64.Q, c.n_proj);
    } else {
      const float* X = static_cast<const float*>(Xv);
      float* Y = static_cast<float*>(Yv);
      float* Yg = static_cast<float*>(cm->Yg);
      const float one = 1.f, zero = 0.f;
      if (bf16) {   // BF16 x BF16 -> FP32 on the tensor cores
        __nv_bfloat16* Xg = static_cast<__nv_bfloat16*>(cm->Xg);
        const __nv_bfloat16** A = (const __nv_bfloat16**)(cm->ptrs);
        const __nv_bfloat16** B = (const __nv_bfloat16**)(cm->ptrs + cm->max_cells);
        float** C = (float**)(cm->ptrs + 2 * (size_t)cm->max_cells);
        k_cm_gather_bf16<<<grid, 128, 0, s>>>(Xg, X, ncols, ncols, c.cell_dofs, cells, n, np3);
        k_cm_ptrs<__nv_bfloat16, float><<<(n + 127) / 128, 128, 0, s>>>(
            A, B, C, Xg, static_cast<const __nv_bfloat16*>(cm->H), Yg, cells, n, np3, ncols);
        bs = cublasGemmBatchedEx(cm->blas, CUBLAS_OP_N, CUBLAS_OP_N, ncols, np3, np3, &one, (const void* const*)A,
                                 CUDA_R_16BF, ncols, (const void* const*)B, CUDA_R_16BF, np3, &zero,
                                 (void* const*)C, CUDA_R_32F, ncols, n, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
      } else {
        float* Xg = static_cast<float*>(cm->Xg);
        // three pointer arrays of max_cells entries each: A, B, C operands
        const float** A = (const float**)(cm->ptrs);
        const float** B = (const float**)(cm->ptrs + cm->max_cells);
        float** C = (float**)(cm->ptrs + 2 * (size_t)cm->max_cells);
        k_cm_gather<float><<<grid, 128, 0, s>>>(Xg, X, ncols, ncols, c.cell_dofs, cells, n, np3);
        k_cm_ptrs<float, float><<<(n + 127) / 128, 128, 0, s>>>(A, B, C, Xg, static_cast<const float*>(cm->H), Yg, cells, n,
                                                        np3, ncols);
        bs = cublasSgemmBatched(cm->blas, CUBLAS_OP_N, CUBLAS_OP_N, ncols, np3, np3, &one, A, ncols, B, np3, &zero,
                                C, ncols, n);
      }
      k_cm_scatter<float><<<grid, 128, 0, s>>>(Y, Yg, ncols, ncols, c.cell_dofs, cells, n, np3,
                                               nl ? c.cell_pair_ptr : nullptr, c.cell_pairs, c.pair_atom, c.f32.F,
                                               c.f32.Q, c.n_proj);
    }
    if (bs != CUBLAS_STATUS_SUCCESS) return fail(FE_KS_ERR_CUDA, "cell-matrix batched GEMM failed");
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("cell-matrix apply: ") + cudaGetErrorString(err));
  return FE_KS_OK;
}

fe_ks_status fe_ks_cm_info(const fe_ks_cm* cm, double* setup_ms, size_t* bytes) {
  if (!cm) return fail(FE_KS_ERR_ARG, "NULL argument");
  if (setup_ms) *setup_ms = cm->setup_ms;
  if (bytes) *bytes = cm->bytes;
  return FE_KS_OK;
}

void fe_ks_cm_destroy(fe_ks_cm* cm) { cm_free(cm); }

}  // extern "C"
