// Nonlocal projection Q_a = Delta^a sum_{e in E(a)} F^(a,e)^H X^(e)
// (eq. AXmatrixfreenonloc, first factor; Algorithm 1 T1 -> T2 -> T3).
//
// Two forms, both deterministic:
//  - pair form (the operator's path): one CTA per (atom, cell) pair and column
//    chunk stages the pair's F block and the cell's DoF list in shared memory
//    and forms P_pair = F^(a,e)^H X^(e) with one column per thread (rows of X
//    read coalesced, four rows in flight); a second kernel sums the pairs of
//    each atom in pair order and scales by Delta.  Needs a partial buffer
//    [pair][n_proj][columns].
//  - atom form (the allocation-free entry point): one CTA per (atom, 32-column
//    tile); warps stride over the atom's (cell, node) rows, lanes own columns,
//    partial sums are reduced across warps in shared memory.
#include <algorithm>

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

// ---- pair form

constexpr int kPairThreads = 256;

// P[pr][b][col] = sum_node conj(F[pr][b][node]) x(d(node), col), x scaled by
// D^{-1/2} when dscale is given.  cw (32, 64, 128 or 256) columns per CTA, the
// 256 / cw row slices of a CTA reduced in shared memory in slice order.
template <typename T, typename TS, typename TF, bool CPLX>
__global__ void __launch_bounds__(kPairThreads)
fe_proj_pair_kernel(const TS* __restrict__ Xg, int64_t ld, int ncols, const int* __restrict__ cell_dofs,
                    const int* __restrict__ pair_cell, const TF* __restrict__ Fg, const TS* __restrict__ dscale,
                    TS* __restrict__ part, int n_proj, int np3, int cw) {
  using N = ProjNum<T>;
  constexpr int CW = CPLX ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smp[];
  TF* Fs = reinterpret_cast<TF*>(smp);
  const int nf = n_proj * np3 * CW;
  int* ds = reinterpret_cast<int*>(smp + (size_t)nf * sizeof(TF));
  T* red = reinterpret_cast<T*>(smp + (((size_t)nf * sizeof(TF) + (size_t)np3 * sizeof(int) + 15) & ~(size_t)15));
  const int pr = blockIdx.x;
  const int rs = kPairThreads / cw;
  const int lc = threadIdx.x % cw, sl = threadIdx.x / cw;
  const int col = blockIdx.y * cw + lc;
  const bool act = col < ncols;
  const TF* Fp = Fg + (int64_t)pr * nf;
  for (int i = threadIdx.x; i < nf; i += kPairThreads) Fs[i] = Fp[i];
  const int cell = pair_cell[pr];
  for (int i = threadIdx.x; i < np3; i += kPairThreads) ds[i] = cell_dofs[(int64_t)cell * np3 + i];
  __syncthreads();
  T acc[kMaxProj];
#pragma unroll
  for (int b = 0; b < kMaxProj; ++b) acc[b] = N::zero();
  // rows sl, sl + rs, ... in groups of four (warp-uniform: cw is a multiple of 32)
  for (int n0 = sl; n0 < np3; n0 += 4 * rs) {
    TS xs[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int node = n0 + u * rs;
      xs[u] = TS(0);
      if (node < np3) {
        const int d = ds[node];
        if (act) xs[u] = Xg[(int64_t)d * ld + col];
        if (dscale) xs[u] *= dscale[d];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int node = n0 + u * rs;
      if (node >= np3) break;
      const T x = N::in(xs[u]);
      if constexpr (!CPLX) {
#pragma unroll
        for (int b = 0; b < kMaxProj; ++b)
          if (b < n_proj) acc[b] = fma(N::in(Fs[b * np3 + node]), x, acc[b]);
      } else {
        const T xp = N::shfl1(x);
#pragma unroll
        for (int b = 0; b < kMaxProj; ++b) {
          if (b < n_proj) {
            const T fr = N::in(Fs[2 * (b * np3 + node)]), fi = N::in(Fs[2 * (b * np3 + node) + 1]);
            // conj(F) x : re = fr xr + fi xi ; im = fr xi - fi xr
            acc[b] = (lc & 1) ? fma(fr, x, fma(-fi, xp, acc[b])) : fma(fr, x, fma(fi, xp, acc[b]));
          }
        }
      }
    }
  }
  if (rs == 1) {
    if (act)
#pragma unroll
      for (int b = 0; b < kMaxProj; ++b)
        if (b < n_proj) part[((int64_t)pr * n_proj + b) * ld + col] = N::template out<TS>(acc[b]);
    return;
  }
#pragma unroll
  for (int b = 0; b < kMaxProj; ++b)
    if (b < n_proj) red[((size_t)sl * n_proj + b) * cw + lc] = acc[b];
  __syncthreads();
  for (int idx = threadIdx.x; idx < n_proj * cw; idx += kPairThreads) {
    const int b = idx / cw, c = idx % cw;
    T v = red[(size_t)b * cw + c];
    for (int k = 1; k < rs; ++k) v = v + red[((size_t)k * n_proj + b) * cw + c];
    const int cc = blockIdx.y * cw + c;
    if (cc < ncols) part[((int64_t)pr * n_proj + b) * ld + cc] = N::template out<TS>(v);
  }
}

// Q[a][b][col] = h[a][b] * sum over the pairs of atom a, in pair order, of P[pr][b][col]
template <typename TS>
__global__ void fe_proj_sum_kernel(const TS* __restrict__ part, const TS* __restrict__ h,
                                   const int* __restrict__ atom_pair_ptr, TS* __restrict__ Q, int n_atoms, int n_proj,
                                   int64_t ld, int ncols) {
  const int64_t total = (int64_t)n_atoms * n_proj * ncols;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(idx % ncols);
    const int64_t ab = idx / ncols;
    const int a = (int)(ab / n_proj), b = (int)(ab % n_proj);
    TS s = TS(0);
    for (int pr = atom_pair_ptr[a]; pr < atom_pair_ptr[a + 1]; ++pr) s += part[((int64_t)pr * n_proj + b) * ld + col];
    Q[ab * ld + col] = s * h[ab];
  }
}

// Column chunk of the pair kernel: the smallest multiple of 32 covering the
// columns, at most 256.
static int pair_chunk(int ncols) {
  int cw = 32;
  while (cw < 256 && cw < ncols) cw *= 2;
  return cw;
}

template <typename T, typename TS, typename TF, bool CPLX>
static cudaError_t launch_pair(const ProjParams<TS>& prm, const TF* F, int n_atoms, cudaStream_t s) {
  const int cw = pair_chunk(prm.ncols);
  const int rs = kPairThreads / cw;
  const size_t nf = (size_t)prm.n_proj * prm.np3 * (CPLX ? 2 : 1);
  const size_t head = (nf * sizeof(TF) + (size_t)prm.np3 * sizeof(int) + 15) & ~(size_t)15;
  const size_t smem = head + (rs > 1 ? (size_t)rs * prm.n_proj * cw * sizeof(T) : 0);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t err = cudaFuncSetAttribute(fe_proj_pair_kernel<T, TS, TF, CPLX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  dim3 grid((unsigned)prm.n_pairs, (unsigned)((prm.ncols + cw - 1) / cw));
  fe_proj_pair_kernel<T, TS, TF, CPLX><<<grid, kPairThreads, smem, s>>>(
      prm.X, prm.ld, prm.ncols, prm.cell_dofs, prm.pair_cell, F, prm.dscale, prm.part, prm.n_proj, prm.np3, cw);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int64_t total = (int64_t)n_atoms * prm.n_proj * prm.ncols;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  fe_proj_sum_kernel<TS><<<blocks, 256, 0, s>>>(prm.part, prm.h, prm.atom_pair_ptr, prm.Q, n_atoms, prm.n_proj,
                                                prm.ld, prm.ncols);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_proj_pairs(const Ctx& c, const ProjParams<T>& prm, int n_atoms, cudaStream_t s) {
  if (n_atoms == 0 || prm.n_pairs == 0) return cudaSuccess;
  if (!prm.part) return cudaErrorInvalidValue;
  return c.cplx ? launch_pair<T, T, T, true>(prm, prm.F, n_atoms, s) : launch_pair<T, T, T, false>(prm, prm.F, n_atoms, s);
}

cudaError_t launch_proj_pairs_emu(const Ctx& c, const ProjParams<double>& prm, const ff2* F, int n_atoms,
                                  cudaStream_t s) {
  if (n_atoms == 0 || prm.n_pairs == 0) return cudaSuccess;
  if (!prm.part) return cudaErrorInvalidValue;
  return c.cplx ? launch_pair<ff2, double, ff2, true>(prm, F, n_atoms, s)
                : launch_pair<ff2, double, ff2, false>(prm, F, n_atoms, s);
}

template cudaError_t launch_proj<double>(const Ctx&, const ProjParams<double>&, int, cudaStream_t);
template cudaError_t launch_proj<float>(const Ctx&, const ProjParams<float>&, int, cudaStream_t);
template cudaError_t launch_proj_pairs<double>(const Ctx&, const ProjParams<double>&, int, cudaStream_t);
template cudaError_t launch_proj_pairs<float>(const Ctx&, const ProjParams<float>&, int, cudaStream_t);

}  // namespace feks
