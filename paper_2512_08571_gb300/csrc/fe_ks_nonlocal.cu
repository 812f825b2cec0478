// Nonlocal projection Q_a = Delta^a sum_{e in E(a)} F^(a,e)^H X^(e)
// (eq. AXmatrixfreenonloc, first factor; Algorithm 1 T1 -> T2 -> T3).
//
// Two forms, both deterministic:
//  - pair form (the operator's path): one CTA per (atom, cell) pair and column
//    chunk stages the pair's F block and the cell's DoF list in shared memory
//    and forms P_pair = F^(a,e)^H X^(e) with one column per thread (rows of X
//    read coalesced, four to eight rows in flight); a second kernel sums the pairs of
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

// 16 bytes of shared memory into 16 / sizeof(TF) values (one vector load)
__device__ __forceinline__ void ld16(const float* p, float* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w;
}
__device__ __forceinline__ void ld16(const double* p, double* o) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  o[0] = v.x, o[1] = v.y;
}
__device__ __forceinline__ void ld16(const ff2* p, ff2* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = ff_make(v.x, v.y), o[1] = ff_make(v.z, v.w);
}

// Elements per node of the transposed F block: MAXP projectors (x2 complex),
// rounded up to a whole number of 16-byte chunks.
template <typename TF, bool CPLX, int MAXP>
__host__ __device__ constexpr int pair_fstride() {
  return ((MAXP * (CPLX ? 2 : 1) * (int)sizeof(TF) + 15) / 16) * 16 / (int)sizeof(TF);
}

// P[pr][b][col] = sum_node conj(F[pr][b][node]) x(d(node), col), x scaled by
// D^{-1/2} when dscale is given.  Each thread owns V = 16 / sizeof(TS)
// adjacent columns (one 16-byte load per row; for complex data the re/im
// partner is in the same thread); cg column groups per CTA, the 256 / cg row
// slices of a CTA reduced in shared memory in slice order.  MAXP >= n_proj.
template <typename T, typename TS, typename TF, bool CPLX, int MAXP>
__global__ void __launch_bounds__(kPairThreads)
fe_proj_pair_kernel(const TS* __restrict__ Xg, int64_t ld, int ncols, const int* __restrict__ cell_dofs,
                    const int* __restrict__ pair_cell, const TF* __restrict__ Fg, const TS* __restrict__ dscale,
                    TS* __restrict__ part, int n_proj, int np3, int cg) {
  using N = ProjNum<T>;
  constexpr int V = 16 / (int)sizeof(TS);
  constexpr int CW = CPLX ? 2 : 1;
  constexpr int PB = pair_fstride<TF, CPLX, MAXP>();   // F row of one node: [b][re, im], padded to 16 B
  extern __shared__ __align__(16) unsigned char smp[];
  TF* Fs = reinterpret_cast<TF*>(smp);   // [node][PB]
  const int nf = n_proj * np3 * CW;
  int* ds = reinterpret_cast<int*>(smp + (size_t)np3 * PB * sizeof(TF));
  T* red = reinterpret_cast<T*>(smp + (((size_t)np3 * PB * sizeof(TF) + (size_t)np3 * sizeof(int) + 15) & ~(size_t)15));
  const int pr = blockIdx.x;
  const int rs = kPairThreads / cg;
  const int lc = threadIdx.x % cg, sl = threadIdx.x / cg;
  const int c0 = (blockIdx.y * cg + lc) * V;
  const bool vec = (ld % V == 0) && (((uintptr_t)Xg & 15) == 0) && c0 + V <= ncols;
  const TF* Fp = Fg + (int64_t)pr * nf;
  // transpose F[b][node][re,im] -> Fs[node][b][re,im] (global reads coalesced over node)
  for (int i = threadIdx.x; i < nf; i += kPairThreads) {
    const int b = i / (np3 * CW), rem = i - b * np3 * CW;
    const int node = rem / CW, ri = rem - node * CW;
    Fs[node * PB + b * CW + ri] = Fp[i];
  }
  const int cell = pair_cell[pr];
  for (int i = threadIdx.x; i < np3; i += kPairThreads) ds[i] = cell_dofs[(int64_t)cell * np3 + i];
  __syncthreads();
  T acc[MAXP][V];
#pragma unroll
  for (int b = 0; b < MAXP; ++b)
#pragma unroll
    for (int v = 0; v < V; ++v) acc[b][v] = N::zero();
  constexpr int RU = 4;   // rows in flight per thread
  for (int n0 = sl; n0 < np3; n0 += RU * rs) {
    TS xs[RU][V];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int node = n0 + u * rs;
#pragma unroll
      for (int v = 0; v < V; ++v) xs[u][v] = TS(0);
      if (node < np3) {
        const int d = ds[node];
        const TS* xr = Xg + (int64_t)d * ld + c0;
        if (vec) {
          const uint4 w = *reinterpret_cast<const uint4*>(xr);
          const TS* wv = reinterpret_cast<const TS*>(&w);
#pragma unroll
          for (int v = 0; v < V; ++v) xs[u][v] = wv[v];
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v)
            if (c0 + v < ncols) xs[u][v] = xr[v];
        }
        if (dscale) {
          const TS sc = dscale[d];
#pragma unroll
          for (int v = 0; v < V; ++v) xs[u][v] *= sc;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int node = n0 + u * rs;
      if (node >= np3) break;
      T x[V];
#pragma unroll
      for (int v = 0; v < V; ++v) x[v] = N::in(xs[u][v]);
      // the node's F row with 16-byte shared loads (all lanes read the same row)
      TF frow[PB];
#pragma unroll
      for (int q = 0; q < PB; q += 16 / (int)sizeof(TF)) ld16(Fs + node * PB + q, frow + q);
#pragma unroll
      for (int b = 0; b < MAXP; ++b) {
        if (b < n_proj) {
          if constexpr (!CPLX) {
            const T f = N::in(frow[b]);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[b][v] = fma(f, x[v], acc[b][v]);
          } else {
            // conj(F) x : re = fr xr + fi xi ; im = fr xi - fi xr  (re, im adjacent in the thread)
            const T fr = N::in(frow[2 * b]), fi = N::in(frow[2 * b + 1]);
#pragma unroll
            for (int v = 0; v < V; v += 2) {
              acc[b][v] = fma(fr, x[v], fma(fi, x[v + 1], acc[b][v]));
              acc[b][v + 1] = fma(fr, x[v + 1], fma(-fi, x[v], acc[b][v + 1]));
            }
          }
        }
      }
    }
  }
  if (rs == 1) {
#pragma unroll
    for (int b = 0; b < MAXP; ++b)
      if (b < n_proj)
#pragma unroll
        for (int v = 0; v < V; ++v)
          if (c0 + v < ncols) part[((int64_t)pr * n_proj + b) * ld + c0 + v] = N::template out<TS>(acc[b][v]);
    return;
  }
  const int cols = cg * V;   // columns of this CTA
#pragma unroll
  for (int b = 0; b < MAXP; ++b)
    if (b < n_proj)
#pragma unroll
      for (int v = 0; v < V; ++v) red[((size_t)sl * n_proj + b) * cols + lc * V + v] = acc[b][v];
  __syncthreads();
  for (int idx = threadIdx.x; idx < n_proj * cols; idx += kPairThreads) {
    const int b = idx / cols, c = idx % cols;
    T v = red[(size_t)b * cols + c];
    for (int k = 1; k < rs; ++k) v = v + red[((size_t)k * n_proj + b) * cols + c];
    const int cc = blockIdx.y * cols + c;
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

// Column groups (of 16 / sizeof(TS) columns) per CTA of the pair kernel: the
// smallest multiple of 32 covering the columns, at most 256.
template <typename TS>
static int pair_groups(int ncols) {
  const int groups = (ncols + (16 / (int)sizeof(TS)) - 1) / (16 / (int)sizeof(TS));
  int cg = 32;
  while (cg < 256 && cg < groups) cg *= 2;
  return cg;
}

template <typename T, typename TS, typename TF, bool CPLX, int MAXP>
static cudaError_t launch_pair_p(const ProjParams<TS>& prm, const TF* F, int n_atoms, cudaStream_t s) {
  constexpr int V = 16 / (int)sizeof(TS);
  const int cg = pair_groups<TS>(prm.ncols);
  const int rs = kPairThreads / cg;
  constexpr int PB = pair_fstride<TF, CPLX, MAXP>();
  const size_t head = ((size_t)prm.np3 * PB * sizeof(TF) + (size_t)prm.np3 * sizeof(int) + 15) & ~(size_t)15;
  const size_t smem = head + (rs > 1 ? (size_t)rs * prm.n_proj * cg * V * sizeof(T) : 0);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t err = cudaFuncSetAttribute(fe_proj_pair_kernel<T, TS, TF, CPLX, MAXP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  dim3 grid((unsigned)prm.n_pairs, (unsigned)((prm.ncols + cg * V - 1) / (cg * V)));
  fe_proj_pair_kernel<T, TS, TF, CPLX, MAXP><<<grid, kPairThreads, smem, s>>>(
      prm.X, prm.ld, prm.ncols, prm.cell_dofs, prm.pair_cell, F, prm.dscale, prm.part, prm.n_proj, prm.np3, cg);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int64_t total = (int64_t)n_atoms * prm.n_proj * prm.ncols;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  fe_proj_sum_kernel<TS><<<blocks, 256, 0, s>>>(prm.part, prm.h, prm.atom_pair_ptr, prm.Q, n_atoms, prm.n_proj,
                                                prm.ld, prm.ncols);
  return cudaGetLastError();
}

template <typename T, typename TS, typename TF, bool CPLX>
static cudaError_t launch_pair(const ProjParams<TS>& prm, const TF* F, int n_atoms, cudaStream_t s) {
  if (prm.n_proj <= 9) return launch_pair_p<T, TS, TF, CPLX, 9>(prm, F, n_atoms, s);
  return launch_pair_p<T, TS, TF, CPLX, kMaxProj>(prm, F, n_atoms, s);
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
