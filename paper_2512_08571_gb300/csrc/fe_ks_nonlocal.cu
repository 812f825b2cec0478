// Nonlocal projection Q_a = Delta^a sum_{e in E(a)} F^(a,e)^H X^(e)
// (eq. AXmatrixfreenonloc, first factor; Algorithm 1 T1 -> T2 -> T3).
// One CTA per (atom, 32-column tile); each warp strides over the atom's
// (cell, node) rows, lanes own columns, the n_proj partial sums stay in
// registers and are reduced across warps in shared memory (deterministic).
#include "fe_ks_internal.h"

namespace feks {

// Conversion helpers between the storage type TS and the arithmetic type T.
template <typename T>
struct ProjNum {
  static __device__ __forceinline__ T zero() { return T(0); }
  template <typename TS>
  static __device__ __forceinline__ T in(TS x) { return (T)x; }
  template <typename TS>
  static __device__ __forceinline__ TS out(T x) { return (TS)x; }
  static __device__ __forceinline__ T shfl1(T v) { return __shfl_xor_sync(0xffffffffu, v, 1); }
};
template <>
struct ProjNum<ff2> {
  static __device__ __forceinline__ ff2 zero() { return ff_make(0.f, 0.f); }
  static __device__ __forceinline__ ff2 in(double x) { return ff_split_bits(x); }
  static __device__ __forceinline__ ff2 in(ff2 x) { return x; }
  template <typename TS>
  static __device__ __forceinline__ TS out(ff2 x) { return ff_to_double(x); }
  static __device__ __forceinline__ ff2 shfl1(ff2 v) {
    return ff_make(__shfl_xor_sync(0xffffffffu, v.hi, 1), __shfl_xor_sync(0xffffffffu, v.lo, 1));
  }
};

constexpr int kProjWarps = 8;
constexpr int kMaxProj = 16;

// T: arithmetic type; TS: storage type of X, h and Q; TF: storage type of F.
template <typename T, typename TS, typename TF, bool CPLX>
__global__ void __launch_bounds__(32 * kProjWarps)
fe_proj_kernel(const TS* __restrict__ Xg, int64_t ld, int ncols, const int* __restrict__ cell_dofs,
               const int* __restrict__ atom_pair_ptr, const int* __restrict__ pair_cell, const TF* __restrict__ Fg,
               const TS* __restrict__ h, const TS* __restrict__ dscale, TS* __restrict__ Q, int n_proj, int np3) {
  __shared__ T red[kProjWarps][kMaxProj][32];
  using N = ProjNum<T>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  const int a = blockIdx.y;
  const bool act = col < ncols;
  T acc[kMaxProj];
#pragma unroll
  for (int b = 0; b < kMaxProj; ++b) acc[b] = N::zero();
  const int pb = atom_pair_ptr[a], pe = atom_pair_ptr[a + 1];
  const int64_t nrows = (int64_t)(pe - pb) * np3;
  for (int64_t r = warp; r < nrows; r += kProjWarps) {
    const int pr = pb + (int)(r / np3);
    const int node = (int)(r % np3);
    const int cell = pair_cell[pr];
    const int d = cell_dofs[(int64_t)cell * np3 + node];
    TS xs = act ? Xg[(int64_t)d * ld + col] : TS(0);
    if (dscale) xs *= dscale[d];
    const T x = N::in(xs);
    if (!CPLX) {
      const TF* Fr = Fg + (int64_t)pr * n_proj * np3 + node;
#pragma unroll
      for (int b = 0; b < kMaxProj; ++b)
        if (b < n_proj) acc[b] = fma(N::in(Fr[(int64_t)b * np3]), x, acc[b]);
    } else {
      const T xp = N::shfl1(x);
      const TF* Fr = Fg + ((int64_t)pr * n_proj * np3 + node) * 2;
#pragma unroll
      for (int b = 0; b < kMaxProj; ++b) {
        if (b < n_proj) {
          const T fr = N::in(Fr[2 * (int64_t)b * np3]), fi = N::in(Fr[2 * (int64_t)b * np3 + 1]);
          // conj(F) x : re = fr xr + fi xi ; im = fr xi - fi xr
          acc[b] = (lane & 1) ? fma(fr, x, fma(-fi, xp, acc[b])) : fma(fr, x, fma(fi, xp, acc[b]));
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < kMaxProj; ++b)
    if (b < n_proj) red[warp][b][lane] = acc[b];
  __syncthreads();
  for (int idx = threadIdx.x; idx < n_proj * 32; idx += 32 * kProjWarps) {
    const int b = idx / 32, l = idx % 32;
    const int c = blockIdx.x * 32 + l;
    T s = red[0][b][l];
#pragma unroll
    for (int w = 1; w < kProjWarps; ++w) s = s + red[w][b][l];
    if (c < ncols) Q[((int64_t)a * n_proj + b) * ld + c] = N::template out<TS>(s * N::in(h[a * n_proj + b]));
  }
}

template <typename T>
cudaError_t launch_proj(const Ctx& c, const ProjParams<T>& prm, int n_atoms, cudaStream_t s) {
  if (n_atoms == 0) return cudaSuccess;
  dim3 grid((prm.ncols + 31) / 32, n_atoms);
  if (c.cplx)
    fe_proj_kernel<T, T, T, true><<<grid, 32 * kProjWarps, 0, s>>>(prm.X, prm.ld, prm.ncols, prm.cell_dofs,
                                                                   prm.atom_pair_ptr, prm.pair_cell, prm.F, prm.h,
                                                                   prm.dscale, prm.Q, prm.n_proj, prm.np3);
  else
    fe_proj_kernel<T, T, T, false><<<grid, 32 * kProjWarps, 0, s>>>(prm.X, prm.ld, prm.ncols, prm.cell_dofs,
                                                                    prm.atom_pair_ptr, prm.pair_cell, prm.F, prm.h,
                                                                    prm.dscale, prm.Q, prm.n_proj, prm.np3);
  return cudaGetLastError();
}

// FP64 projections computed in pairs of floats (F given as float pairs).
cudaError_t launch_proj_emu(const Ctx& c, const ProjParams<double>& prm, const ff2* F, int n_atoms, cudaStream_t s) {
  if (n_atoms == 0) return cudaSuccess;
  dim3 grid((prm.ncols + 31) / 32, n_atoms);
  if (c.cplx)
    fe_proj_kernel<ff2, double, ff2, true><<<grid, 32 * kProjWarps, 0, s>>>(
        prm.X, prm.ld, prm.ncols, prm.cell_dofs, prm.atom_pair_ptr, prm.pair_cell, F, prm.h, prm.dscale, prm.Q,
        prm.n_proj, prm.np3);
  else
    fe_proj_kernel<ff2, double, ff2, false><<<grid, 32 * kProjWarps, 0, s>>>(
        prm.X, prm.ld, prm.ncols, prm.cell_dofs, prm.atom_pair_ptr, prm.pair_cell, F, prm.h, prm.dscale, prm.Q,
        prm.n_proj, prm.np3);
  return cudaGetLastError();
}

template cudaError_t launch_proj<double>(const Ctx&, const ProjParams<double>&, int, cudaStream_t);
template cudaError_t launch_proj<float>(const Ctx&, const ProjParams<float>&, int, cudaStream_t);

}  // namespace feks
