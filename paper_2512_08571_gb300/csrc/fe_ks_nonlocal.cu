// Nonlocal projection Q_a = Delta^a sum_{e in E(a)} F^(a,e)^H X^(e)
// (eq. AXmatrixfreenonloc, first factor; Algorithm 1 T1 -> T2 -> T3).
// One CTA per (atom, 32-column tile); each warp strides over the atom's
// (cell, node) rows, lanes own columns, the n_proj partial sums stay in
// registers and are reduced across warps in shared memory (deterministic).
#include "fe_ks_internal.h"

namespace feks {

constexpr int kProjWarps = 8;
constexpr int kMaxProj = 16;

template <typename T, bool CPLX>
__global__ void __launch_bounds__(32 * kProjWarps) fe_proj_kernel(const __grid_constant__ ProjParams<T> p) {
  __shared__ T red[kProjWarps][kMaxProj][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  const int a = blockIdx.y;
  const bool act = col < p.ncols;
  T acc[kMaxProj];
#pragma unroll
  for (int b = 0; b < kMaxProj; ++b) acc[b] = T(0);
  const int pb = p.atom_pair_ptr[a], pe = p.atom_pair_ptr[a + 1];
  const int64_t nrows = (int64_t)(pe - pb) * p.np3;
  for (int64_t r = warp; r < nrows; r += kProjWarps) {
    const int pr = pb + (int)(r / p.np3);
    const int node = (int)(r % p.np3);
    const int cell = p.pair_cell[pr];
    const int d = p.cell_dofs[(int64_t)cell * p.np3 + node];
    T x = act ? p.X[(int64_t)d * p.ld + col] : T(0);
    if (p.dscale) x *= p.dscale[d];
    if (!CPLX) {
      const T* Fr = p.F + (int64_t)pr * p.n_proj * p.np3 + node;
#pragma unroll
      for (int b = 0; b < kMaxProj; ++b)
        if (b < p.n_proj) acc[b] = fma(Fr[(int64_t)b * p.np3], x, acc[b]);
    } else {
      const T xp = __shfl_xor_sync(0xffffffffu, x, 1);
      const T* Fr = p.F + ((int64_t)pr * p.n_proj * p.np3 + node) * 2;
#pragma unroll
      for (int b = 0; b < kMaxProj; ++b) {
        if (b < p.n_proj) {
          const T fr = Fr[2 * (int64_t)b * p.np3], fi = Fr[2 * (int64_t)b * p.np3 + 1];
          // conj(F) x : re = fr xr + fi xi ; im = fr xi - fi xr
          acc[b] = (lane & 1) ? fma(fr, x, fma(-fi, xp, acc[b])) : fma(fr, x, fma(fi, xp, acc[b]));
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < kMaxProj; ++b)
    if (b < p.n_proj) red[warp][b][lane] = acc[b];
  __syncthreads();
  for (int idx = threadIdx.x; idx < p.n_proj * 32; idx += 32 * kProjWarps) {
    const int b = idx / 32, l = idx % 32;
    const int c = blockIdx.x * 32 + l;
    T s = T(0);
#pragma unroll
    for (int w = 0; w < kProjWarps; ++w) s += red[w][b][l];
    if (c < p.ncols) p.Q[((int64_t)a * p.n_proj + b) * p.ld + c] = s * p.h[a * p.n_proj + b];
  }
}

template <typename T>
cudaError_t launch_proj(const Ctx& c, const ProjParams<T>& prm, int n_atoms, cudaStream_t s) {
  if (n_atoms == 0) return cudaSuccess;
  dim3 grid((prm.ncols + 31) / 32, n_atoms);
  if (c.cplx)
    fe_proj_kernel<T, true><<<grid, 32 * kProjWarps, 0, s>>>(prm);
  else
    fe_proj_kernel<T, false><<<grid, 32 * kProjWarps, 0, s>>>(prm);
  return cudaGetLastError();
}

template cudaError_t launch_proj<double>(const Ctx&, const ProjParams<double>&, int, cudaStream_t);
template cudaError_t launch_proj<float>(const Ctx&, const ProjParams<float>&, int, cudaStream_t);

}  // namespace feks
