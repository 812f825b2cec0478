// Matrix-free cell tile: gather -> N, D~ contractions -> quadrature-point
// coefficients -> D~^T, N^T contractions -> nonlocal expansion -> scatter-add,
// for one cell and one tile of VT vector columns.
//
// Paper: Algorithm 2 (cell-level evaluation; eq. ggaReal / eq. ggaCmplx),
// called from Algorithm 1 (extraction Q C P X, assembly Q^T, F Delta T3).
// The paper's level-2 batch b^(2) (SIMD width) becomes the VT-column tile held
// in shared memory with the vector index fastest; each 1D contraction uses the
// even-odd decomposition (Sec. 5.4).
//
// Every phase is a loop over (line or column) x (vector column) work items
// with a compile-time thread count NT, so the same routine serves the
// one-cell-per-CTA kernel (NT = VT n_q^2) and the persistent batched kernel
// (fixed NT).  No register state survives a barrier: the pointwise phase
// writes its partial sum back into tile A, which is free at that point.
#pragma once
#include "fe_ks_internal.h"

namespace feks {

// y = M x for an NO x NI matrix with M[NO-1-o][NI-1-i] = S M[o][i], given its
// even-odd split (see EOMat).  All indices are compile-time constants, so the
// table entries are read straight from the kernel parameter bank.
template <int NI, int NO, int S, typename T>
__device__ __forceinline__ void eo_apply(const T* x, T* y, const EOMat<T>& m) {
  constexpr int HI = NI / 2, HO = NO / 2;
  T xe[HI], xo[HI];
#pragma unroll
  for (int i = 0; i < HI; ++i) {
    xe[i] = x[i] + x[NI - 1 - i];
    xo[i] = x[i] - x[NI - 1 - i];
  }
#pragma unroll
  for (int o = 0; o < HO; ++o) {
    T ye = m.E[o][0] * xe[0];
#pragma unroll
    for (int i = 1; i < HI; ++i) ye = fma(m.E[o][i], xe[i], ye);
    if (NI % 2) ye = fma(m.E[o][HI], x[HI], ye);
    T yo = m.O[o][0] * xo[0];
#pragma unroll
    for (int i = 1; i < HI; ++i) yo = fma(m.O[o][i], xo[i], yo);
    y[o] = ye + yo;
    y[NO - 1 - o] = (S > 0) ? (ye - yo) : (yo - ye);
  }
  if (NO % 2) {
    T ym;
    if (S > 0) {
      ym = m.MID[0] * xe[0];
#pragma unroll
      for (int i = 1; i < HI; ++i) ym = fma(m.MID[i], xe[i], ym);
      if (NI % 2) ym = fma(m.MID[HI], x[HI], ym);
    } else {
      ym = m.MID[0] * xo[0];
#pragma unroll
      for (int i = 1; i < HI; ++i) ym = fma(m.MID[i], xo[i], ym);
    }
    y[HO] = ym;
  }
}

// Shared-memory layout of one cell tile: tiles A, B, C of [n_q^3][VT] values
// (y pitch padded for even n_q), the cell's coefficients [ncoef][n_q^3] and its
// DoF list [n_p^3].
template <typename T, int NP, int NQ, int VT, bool CPLX>
struct CellShape {
  static constexpr int PY = (NQ % 2 == 0) ? NQ + 1 : NQ;
  static constexpr int SX = VT, SY = PY * VT, SZ = NQ * SY, BUF = NQ * SZ;
  static constexpr int NQ3 = NQ * NQ * NQ, NP3 = NP * NP * NP;
  static constexpr int NCOEF = CPLX ? kCoefCplx : kCoefReal;
  // FP32 stages the cell's coefficients in shared memory (its loads are latency
  // bound); FP64 is bound by the FP64 pipe and keeps the occupancy instead.
  static constexpr bool STAGE_COEF = sizeof(T) == 4;
  static constexpr size_t bytes =
      (size_t)(3 * BUF + (STAGE_COEF ? NCOEF * NQ3 : 0)) * sizeof(T) + (size_t)NP3 * sizeof(int);
  static constexpr bool fits = bytes <= 227 * 1024;
};

__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

// One cell e, columns [col0, col0 + VT).  All NT threads of the block call it.
// Prm is any struct with the operand fields of LocalParams (X, Y, ld, ncols,
// cell_dofs, coef, ncoef, gga, dscale, cell_pair_ptr, cell_pairs, pair_atom,
// F, Q, n_proj, alpha); the 1D tables come separately so that they stay in
// the kernel parameter bank.
template <typename T, int NP, int NQ, int VT, bool CPLX, int NT, class Prm>
__device__ __forceinline__ void cell_tile(const Prm& p, const EOTables<T>& tb, int e, int col0, unsigned char* smem) {
  using S = CellShape<T, NP, NQ, VT, CPLX>;
  constexpr int SX = S::SX, SY = S::SY, SZ = S::SZ, BUF = S::BUF, NQ3 = S::NQ3, NP3 = S::NP3;
  constexpr int NCOEF = S::NCOEF;
  T* A = reinterpret_cast<T*>(smem);
  T* B = A + BUF;
  T* C = B + BUF;
  T* CF = C + BUF;
  int* sd = reinterpret_cast<int*>(CF + (S::STAGE_COEF ? NCOEF * NQ3 : 0));
  const int tid = threadIdx.x;

  __syncthreads();   // the previous tile's readers of the shared tiles are done
  // cell coefficients: asynchronous copy, overlapped with phases (1)-(4)
  if (S::STAGE_COEF) {
    const T* g = p.coef + (int64_t)e * p.ncoef * NQ3;
    const int n = p.ncoef * NQ3;
    for (int i = tid; i < n; i += NT) {
      if (sizeof(T) == 8)
        cp_async_8(CF + i, g + i);
      else
        cp_async_4(CF + i, g + i);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int i = tid; i < NP3; i += NT) sd[i] = p.cell_dofs[(int64_t)e * NP3 + i];
  __syncthreads();

  // (1) extraction T0 = Q X (Algorithm 1) fused with N^1D along z
#pragma unroll 1
  for (int w = tid; w < NP * NP * VT; w += NT) {
    const int v = w % VT, ln = w / VT;
    const int i = ln % NP, j = ln / NP;
    const int col = col0 + v;
    const bool act = col < p.ncols;
    T x[NP], t[NQ];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int d = sd[i + NP * (j + NP * k)];
      T val = act ? p.X[(int64_t)d * p.ld + col] : T(0);
      if (p.dscale) val *= p.dscale[d];
      x[k] = val;
    }
    eo_apply<NP, NQ, 1>(x, t, tb.N);
    T* Av = A + v;
#pragma unroll
    for (int q = 0; q < NQ; ++q) Av[i * SX + j * SY + q * SZ] = t[q];
  }
  __syncthreads();
  // (2) N^1D along y
#pragma unroll 1
  for (int w = tid; w < NP * NQ * VT; w += NT) {
    const int v = w % VT, ln = w / VT;
    const int i = ln % NP, qz = ln / NP;
    T* Av = A + v;
    T x[NP], t[NQ];
#pragma unroll
    for (int j = 0; j < NP; ++j) x[j] = Av[i * SX + j * SY + qz * SZ];
    eo_apply<NP, NQ, 1>(x, t, tb.N);
#pragma unroll
    for (int q = 0; q < NQ; ++q) Av[i * SX + q * SY + qz * SZ] = t[q];
  }
  __syncthreads();
  // (3) N^1D along x  ->  A = Y~0 (values at quadrature points)
#pragma unroll 1
  for (int w = tid; w < NQ * NQ * VT; w += NT) {
    const int v = w % VT, ln = w / VT;
    const int qy = ln % NQ, qz = ln / NQ;
    T* Av = A + v;
    T x[NP], t[NQ];
#pragma unroll
    for (int i = 0; i < NP; ++i) x[i] = Av[i * SX + qy * SY + qz * SZ];
    eo_apply<NP, NQ, 1>(x, t, tb.N);
#pragma unroll
    for (int q = 0; q < NQ; ++q) Av[q * SX + qy * SY + qz * SZ] = t[q];
  }
  __syncthreads();
  // (4) Y~1: D~ along x (A -> B) and along y (A -> C)
#pragma unroll 1
  for (int w = tid; w < NQ * NQ * VT; w += NT) {
    const int v = w % VT, ln = w / VT;
    const int a0 = ln % NQ, qz = ln / NQ;
    const T* Av = A + v;
    T* Bv = B + v;
    T* Cv = C + v;
    T x[NQ], t[NQ];
#pragma unroll
    for (int r = 0; r < NQ; ++r) x[r] = Av[r * SX + a0 * SY + qz * SZ];
    eo_apply<NQ, NQ, -1>(x, t, tb.D);
#pragma unroll
    for (int q = 0; q < NQ; ++q) Bv[q * SX + a0 * SY + qz * SZ] = t[q];
#pragma unroll
    for (int r = 0; r < NQ; ++r) x[r] = Av[a0 * SX + r * SY + qz * SZ];
    eo_apply<NQ, NQ, -1>(x, t, tb.D);
#pragma unroll
    for (int q = 0; q < NQ; ++q) Cv[a0 * SX + q * SY + qz * SZ] = t[q];
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  // (5) D~ along z in registers, then the quadrature-point step of
  //     Algorithm 2:  Z = V^L Y0 + V^G.Y1 - i V^K.Y1,
  //                   W_s = sum_d G_sd Y1_d + V^G_s Y0;
  //     W_x -> B, W_y -> C, Z + D~z^T W_z -> A (in place, this column only).
  //     All lanes run every iteration so the re/im partner shuffle is uniform.
#pragma unroll 1
  for (int w0 = 0; w0 < NQ * NQ * VT; w0 += NT) {
    const int w = w0 + tid;
    const bool ok = w < NQ * NQ * VT;
    const int ww = ok ? w : 0;
    const int v = ww % VT, ln = ww / VT;
    const int qx = ln % NQ, qy = ln / NQ;
    T* Av = A + v;
    T* Bv = B + v;
    T* Cv = C + v;
    T u[NQ], g[NQ], zc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) u[q] = Av[qx * SX + qy * SY + q * SZ];
    eo_apply<NQ, NQ, -1>(u, g, tb.D);
    const T* cf = (S::STAGE_COEF ? CF : p.coef + (int64_t)e * p.ncoef * NQ3) + qx + NQ * qy;
#pragma unroll
    for (int qz = 0; qz < NQ; ++qz) {
      const int o = qz * NQ * NQ;
      const int s = qx * SX + qy * SY + qz * SZ;
      const T gx = Bv[s], gy = Cv[s], gz = g[qz], uu = u[qz];
      const T G00 = cf[0 * NQ3 + o], G01 = cf[1 * NQ3 + o], G02 = cf[2 * NQ3 + o];
      const T G11 = cf[3 * NQ3 + o], G12 = cf[4 * NQ3 + o], G22 = cf[5 * NQ3 + o];
      const T VL = cf[6 * NQ3 + o];
      T z = VL * uu;
      T w0v = fma(G00, gx, fma(G01, gy, G02 * gz));
      T w1v = fma(G01, gx, fma(G11, gy, G12 * gz));
      T w2v = fma(G02, gx, fma(G12, gy, G22 * gz));
      if (p.gga) {
        const T V0 = cf[7 * NQ3 + o], V1 = cf[8 * NQ3 + o], V2 = cf[9 * NQ3 + o];
        z = fma(V0, gx, fma(V1, gy, fma(V2, gz, z)));
        w0v = fma(V0, uu, w0v);
        w1v = fma(V1, uu, w1v);
        w2v = fma(V2, uu, w2v);
      }
      if (CPLX) {
        const T K0 = cf[10 * NQ3 + o], K1 = cf[11 * NQ3 + o], K2 = cf[12 * NQ3 + o];
        const T kk = fma(K0, gx, fma(K1, gy, K2 * gz));
        const T kp = __shfl_xor_sync(0xffffffffu, kk, 1);
        // -i (a + i b) = b - i a : real column adds Im, imaginary column subtracts Re
        z += (v & 1) ? -kp : kp;
      }
      if (ok) {
        Bv[s] = w0v;
        Cv[s] = w1v;
      }
      u[qz] = w2v;
      zc[qz] = z;
    }
    T t[NQ];
    eo_apply<NQ, NQ, -1>(u, t, tb.Dt);
    if (ok) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) Av[qx * SX + qy * SY + q * SZ] = zc[q] + t[q];
    }
  }
  __syncthreads();
  // (6) D~^T along x on B and along y on C (in place)
#pragma unroll 1
  for (int w = tid; w < NQ * NQ * VT; w += NT) {
    const int v = w % VT, ln = w / VT;
    const int a0 = ln % NQ, qz = ln / NQ;
    T* Bv = B + v;
    T* Cv = C + v;
    T x[NQ], t[NQ];
#pragma unroll
    for (int r = 0; r < NQ; ++r) x[r] = Bv[r * SX + a0 * SY + qz * SZ];
    eo_apply<NQ, NQ, -1>(x, t, tb.Dt);
#pragma unroll
    for (int q = 0; q < NQ; ++q) Bv[q * SX + a0 * SY + qz * SZ] = t[q];
#pragma unroll
    for (int r = 0; r < NQ; ++r) x[r] = Cv[a0 * SX + r * SY + qz * SZ];
    eo_apply<NQ, NQ, -1>(x, t, tb.Dt);
#pragma unroll
    for (int q = 0; q < NQ; ++q) Cv[a0 * SX + q * SY + qz * SZ] = t[q];
  }
  __syncthreads();
  // (7) Z += D~x^T W_x + D~y^T W_y, then N^T along z -> A
#pragma unroll 1
  for (int w = tid; w < NQ * NQ * VT; w += NT) {
    const int v = w % VT, ln = w / VT;
    const int qx = ln % NQ, qy = ln / NQ;
    T* Av = A + v;
    const T* Bv = B + v;
    const T* Cv = C + v;
    T zc[NQ], t[NP];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int s = qx * SX + qy * SY + q * SZ;
      zc[q] = Av[s] + (Bv[s] + Cv[s]);
    }
    eo_apply<NQ, NP, 1>(zc, t, tb.Nt);
#pragma unroll
    for (int k = 0; k < NP; ++k) Av[qx * SX + qy * SY + k * SZ] = t[k];
  }
  __syncthreads();
  // (8) N^T along y
#pragma unroll 1
  for (int w = tid; w < NQ * NP * VT; w += NT) {
    const int v = w % VT, ln = w / VT;
    const int qx = ln % NQ, k = ln / NQ;
    T* Av = A + v;
    T x[NQ], t[NP];
#pragma unroll
    for (int q = 0; q < NQ; ++q) x[q] = Av[qx * SX + q * SY + k * SZ];
    eo_apply<NQ, NP, 1>(x, t, tb.Nt);
#pragma unroll
    for (int j = 0; j < NP; ++j) Av[qx * SX + j * SY + k * SZ] = t[j];
  }
  __syncthreads();
  // (9) N^T along x, + sum_a F Delta P (nonlocal), assembly Y += alpha Q^T T0
#pragma unroll 1
  for (int w = tid; w < NP * NP * VT; w += NT) {
    const int v = w % VT, ln = w / VT;
    const int j = ln % NP, k = ln / NP;
    const int col = col0 + v;
    if (col >= p.ncols) continue;
    const T* Av = A + v;
    T x[NQ], y[NP];
#pragma unroll
    for (int q = 0; q < NQ; ++q) x[q] = Av[q * SX + j * SY + k * SZ];
    eo_apply<NQ, NP, 1>(x, y, tb.Nt);
    if (p.cell_pair_ptr) {
      const int pb = p.cell_pair_ptr[e], pe = p.cell_pair_ptr[e + 1];
      for (int pi = pb; pi < pe; ++pi) {
        const int pr = p.cell_pairs[pi];
        const int a = p.pair_atom[pr];
        for (int b = 0; b < p.n_proj; ++b) {
          const T* Qa = p.Q + ((int64_t)a * p.n_proj + b) * p.ld;
          if (!CPLX) {
            const T* Fr = p.F + ((int64_t)pr * p.n_proj + b) * NP3 + NP * (j + NP * k);
            const T q = Qa[col];
#pragma unroll
            for (int i = 0; i < NP; ++i) y[i] = fma(Fr[i], q, y[i]);
          } else {
            const T* Fr = p.F + (((int64_t)pr * p.n_proj + b) * NP3 + NP * (j + NP * k)) * 2;
            const int cb = col & ~1;
            const T qr = Qa[cb], qi = Qa[cb + 1];
#pragma unroll
            for (int i = 0; i < NP; ++i) {
              const T fr = Fr[2 * i], fi = Fr[2 * i + 1];
              y[i] += (v & 1) ? fma(fr, qi, fi * qr) : fma(fr, qr, -fi * qi);
            }
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const int d = sd[i + NP * (j + NP * k)];
      T val = y[i] * p.alpha;
      if (p.dscale) val *= p.dscale[d];
      T* yp = p.Y + (int64_t)d * p.ld + col;
      *yp += val;
    }
  }
}

// One CTA per (cell of the colour, VT-column tile); loops over cells when the
// colour has more cells than gridDim.y.
template <typename T, int NP, int NQ, int VT, bool CPLX, int NT>
__global__ void __launch_bounds__(NT) fe_local_kernel(const __grid_constant__ LocalParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int ci = blockIdx.y; ci < p.n_cells; ci += gridDim.y)
    cell_tile<T, NP, NQ, VT, CPLX, NT>(p, p.tab, p.cells[ci], blockIdx.x * VT, smem_raw);
}

// Tile configurations the launcher may pick from (chosen per context by
// fe_ks_tune; index 0 is the default): columns per tile VT and block size NT.
template <int NQ>
__host__ __device__ constexpr int cfg_vt(int cfg) {
  return cfg == 0 ? (NQ >= 7 ? 4 : 8) : cfg == 1 ? (NQ >= 7 ? 8 : 16) : (NQ >= 7 ? 16 : 32);
}
__host__ __device__ constexpr int cfg_nt(int vt, int nq) {
  return vt * nq * nq > 1024 ? 512 : ((vt * nq * nq + 31) / 32) * 32;
}

template <typename T, int NP, int NQ, int VT, int NT>
cudaError_t launch_local_cfg(const Ctx& c, const LocalParams<T>& prm, cudaStream_t s) {
  const int tiles = (prm.ncols + VT - 1) / VT;
  const int gy = prm.n_cells < 65535 ? prm.n_cells : 65535;
  if (prm.n_cells == 0) return cudaSuccess;
  dim3 grid(tiles, gy);
  // the shared-memory opt-in is a per-device function attribute: set it once per device
  static bool attr_done[2][64] = {};
  const int dev = c.device & 63;
  if (c.cplx) {
    using S = CellShape<T, NP, NQ, VT, true>;
    if constexpr (!S::fits) {
      return cudaErrorInvalidConfiguration;
    } else {
      auto k = fe_local_kernel<T, NP, NQ, VT, true, NT>;
      if (!attr_done[1][dev]) {
        cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
        if (err != cudaSuccess) return err;
        attr_done[1][dev] = true;
      }
      k<<<grid, NT, S::bytes, s>>>(prm);
    }
  } else {
    using S = CellShape<T, NP, NQ, VT, false>;
    if constexpr (!S::fits) {
      return cudaErrorInvalidConfiguration;
    } else {
      auto k = fe_local_kernel<T, NP, NQ, VT, false, NT>;
      if (!attr_done[0][dev]) {
        cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
        if (err != cudaSuccess) return err;
        attr_done[0][dev] = true;
      }
      k<<<grid, NT, S::bytes, s>>>(prm);
    }
  }
  return cudaGetLastError();
}

template <typename T, int P>
cudaError_t launch_local_deg(const Ctx& c, const LocalParams<T>& prm, cudaStream_t s) {
  constexpr int NP = P + 1, NQ = P + 1;
  constexpr int V0 = cfg_vt<NQ>(0), V1 = cfg_vt<NQ>(1), V2 = cfg_vt<NQ>(2);
  const int cfg = sizeof(T) == 8 ? c.cfg64 : c.cfg32;
  switch (cfg) {
    case 1: return launch_local_cfg<T, NP, NQ, V1, cfg_nt(V1, NQ)>(c, prm, s);
    case 2: return launch_local_cfg<T, NP, NQ, V2, cfg_nt(V2, NQ)>(c, prm, s);
    default: return launch_local_cfg<T, NP, NQ, V0, cfg_nt(V0, NQ)>(c, prm, s);
  }
}

}  // namespace feks
