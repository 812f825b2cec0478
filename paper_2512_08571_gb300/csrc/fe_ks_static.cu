// Allocation-free variant of the nonlocal pseudopotential term.
//
// Some callers cannot call cudaMalloc: their device memory is owned by
// another allocator (for example a framework's memory pool that must see
// every byte), or they run where a cudaMalloc would implicitly synchronise
// the device or break a fixed memory budget.  fe_ks_nonlocal_apply_static
// serves them: the caller passes every input and output as device pointers,
// and the only scratch the computation needs -- the per-atom projections
// P_a = diag(h_a) F_a^H X between the projection and the expansion -- lives in
// the file-scope array below, which every GPU that loads the library holds
// until the process exits.
#include <algorithm>
#include <mutex>

#include "fe_ks_internal.h"

namespace feks {

// Maximum scratch: n_atoms * n_proj * (real columns) doubles.
constexpr int64_t kStaticScratchDoubles = 524288;   // 4 MiB
static __device__ __align__(256) double g_nl_scratch[kStaticScratchDoubles];

// Y[dof] += sum_b F[pair][b][node] Q[atom][b][col] for every (pair, node);
// pairs of different cells share DoFs, so the update is an FP64 atomic add.
// The order of those adds is not fixed, so results can differ from run to run
// in the last bits (rounding only); every other apply path of the library is
// bitwise deterministic.
template <bool CPLX>
__global__ void fe_expand_atomic_kernel(double* __restrict__ Y, int64_t ld, int ncols, const int* __restrict__ cell_dofs,
                                        const int* __restrict__ pair_cell, const int* __restrict__ pair_atom_of,
                                        const double* __restrict__ F, const double* __restrict__ Q, int n_proj,
                                        int np3, int64_t n_pairs) {
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const bool act = col < ncols;
  const int64_t nrows = n_pairs * np3;
  for (int64_t r = blockIdx.y * (int64_t)nwarps + warp; r < nrows; r += (int64_t)gridDim.y * nwarps) {
    const int64_t pr = r / np3;
    const int node = (int)(r % np3);
    const int a = pair_atom_of[pr];
    const int d = cell_dofs[(int64_t)pair_cell[pr] * np3 + node];
    if (!act) continue;
    double acc = 0.0;
    for (int b = 0; b < n_proj; ++b) {
      const double* Qa = Q + ((int64_t)a * n_proj + b) * ld;
      if (!CPLX) {
        acc = fma(F[(pr * n_proj + b) * np3 + node], Qa[col], acc);
      } else {
        const double fr = F[((pr * n_proj + b) * np3 + node) * 2], fi = F[((pr * n_proj + b) * np3 + node) * 2 + 1];
        const int cb = col & ~1;
        const double qr = Qa[cb], qi = Qa[cb + 1];
        acc += (col & 1) ? fma(fr, qi, fi * qr) : fma(fr, qr, -fi * qi);
      }
    }
    atomicAdd(Y + (int64_t)d * ld + col, acc);
  }
}

// Scratch address per device, looked up once with that device current.
static std::mutex g_scratch_mu;
static double* g_scratch_ptr[64] = {};

static fe_ks_status scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t gerr = cudaGetDevice(&dev);
  if (gerr != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(gerr));
  if (dev < 0 || dev >= 64)
    return fail(FE_KS_ERR_UNSUPPORTED, "device index " + std::to_string(dev) + " is beyond the 64 devices this entry point tracks");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_nl_scratch);
    if (err != cudaSuccess || !p) return fail(FE_KS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(err));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return FE_KS_OK;
}

}  // namespace feks

using namespace feks;

extern "C" fe_ks_status fe_ks_nonlocal_apply_static(const double* X, double* Y, int64_t n_v, int32_t is_complex,
                                                    int32_t degree, int64_t n_dofs, const int32_t* cell_dofs,
                                                    int32_t n_atoms, int32_t n_proj, const int32_t* atom_pair_ptr,
                                                    const int32_t* pair_cell, const int32_t* pair_atom, int64_t n_pairs,
                                                    const double* F, const double* h_coef, void* cuda_stream) {
  set_error("");
  if (!X || !Y || !cell_dofs || !atom_pair_ptr || !pair_cell || !pair_atom || !F || !h_coef)
    return fail(FE_KS_ERR_ARG, "NULL argument");
  if (degree < 1 || degree > 8) return fail(FE_KS_ERR_UNSUPPORTED, "degree must be in 1..8");
  if (n_v < 1 || n_dofs < 1 || n_atoms < 1 || n_pairs < 1) return fail(FE_KS_ERR_ARG, "sizes must be positive");
  if (n_proj < 1 || n_proj > 16) return fail(FE_KS_ERR_UNSUPPORTED, "n_proj must be in 1..16");
  const int64_t ncols = n_v * (is_complex ? 2 : 1);
  if (ncols > INT32_MAX) return fail(FE_KS_ERR_ARG, "n_v too large");
  if ((int64_t)n_atoms * n_proj * ncols > kStaticScratchDoubles)
    return fail(FE_KS_ERR_ARG, "n_atoms * n_proj * columns exceeds the static scratch of 524288 doubles (4 MiB)");
  const size_t bytes = (size_t)n_dofs * ncols * sizeof(double);
  const char* xb = reinterpret_cast<const char*>(X);
  const char* yb = reinterpret_cast<const char*>(Y);
  if (xb < yb + bytes && yb < xb + bytes) return fail(FE_KS_ERR_ARG, "X and Y overlap");
  double* Q = nullptr;
  fe_ks_status st = scratch_for_current_device(&Q);
  if (st != FE_KS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int np = degree + 1, np3 = np * np * np;
  Ctx c;
  c.cplx = is_complex ? 1 : 0;
  ProjParams<double> pp{};
  pp.X = X;
  pp.ld = ncols;
  pp.ncols = (int)ncols;
  pp.cell_dofs = cell_dofs;
  pp.atom_pair_ptr = atom_pair_ptr;
  pp.pair_cell = pair_cell;
  pp.F = F;
  pp.h = h_coef;
  pp.dscale = nullptr;
  pp.Q = Q;
  pp.n_proj = n_proj;
  pp.np3 = np3;
  cudaError_t err = launch_proj<double>(c, pp, n_atoms, s);
  if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("projection kernel: ") + cudaGetErrorString(err));
  const int64_t nrows = n_pairs * np3;
  const int gy = (int)std::min<int64_t>((nrows + 7) / 8, 65535);
  dim3 grid((unsigned)((ncols + 31) / 32), (unsigned)gy);
  if (is_complex)
    fe_expand_atomic_kernel<true><<<grid, 256, 0, s>>>(Y, ncols, (int)ncols, cell_dofs, pair_cell, pair_atom, F, Q,
                                                       n_proj, np3, n_pairs);
  else
    fe_expand_atomic_kernel<false><<<grid, 256, 0, s>>>(Y, ncols, (int)ncols, cell_dofs, pair_cell, pair_atom, F, Q,
                                                        n_proj, np3, n_pairs);
  err = cudaGetLastError();
  if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("expansion kernel: ") + cudaGetErrorString(err));
  return FE_KS_OK;
}
