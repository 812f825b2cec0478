// Fused matrix-free cell kernel: gather -> N, D~ contractions -> quadrature
// point coefficients -> D~^T, N^T contractions -> nonlocal expansion ->
// scatter-add, for one colour of cells and one tile of VT vector columns.
//
// Paper: Algorithm 2 (cell-level evaluation; eq. ggaReal / eq. ggaCmplx),
// called from Algorithm 1 (extraction Q C P X, assembly Q^T, F Delta T3).
// The paper's level-2 batch b^(2) (SIMD width) becomes the VT-column tile held
// in shared memory with the vector index fastest; each 1D contraction uses the
// even-odd decomposition (Sec. 5.4).
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

template <typename T, int NQ>
struct LocalShape {
  static constexpr int PY = (NQ % 2 == 0) ? NQ + 1 : NQ;   // pad even pitches (bank spread)
};

template <typename T, int NP, int NQ, int VT>
constexpr size_t local_smem_bytes() {
  return 3 * sizeof(T) * (size_t)(NQ * LocalShape<T, NQ>::PY * NQ * VT) + sizeof(int) * NP * NP * NP;
}

template <typename T, int NP, int NQ, int VT, bool CPLX>
__global__ void __launch_bounds__(VT * NQ * NQ)
fe_local_kernel(const __grid_constant__ LocalParams<T> p) {
  constexpr int NT = VT * NQ * NQ;
  constexpr int SX = VT;
  constexpr int SY = LocalShape<T, NQ>::PY * VT;
  constexpr int SZ = NQ * SY;
  constexpr int BUF = NQ * SZ;
  constexpr int NP3 = NP * NP * NP;
  constexpr int NQ3 = NQ * NQ * NQ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* B = A + BUF;
  T* C = B + BUF;
  int* sd = reinterpret_cast<int*>(C + BUF);

  const int tid = threadIdx.x;
  const int v = tid % VT;
  const int ln = tid / VT;
  const int col = blockIdx.x * VT + v;
  const bool act = col < p.ncols;
  const EOTables<T>& tb = p.tab;
  // this thread's column inside the [point][VT] tiles
  T* Av = A + v;
  T* Bv = B + v;
  T* Cv = C + v;

  for (int ci = blockIdx.y; ci < p.n_cells; ci += gridDim.y) {
    const int e = p.cells[ci];
    __syncthreads();
    for (int i = tid; i < NP3; i += NT) sd[i] = p.cell_dofs[(int64_t)e * NP3 + i];
    __syncthreads();

    // (1) extraction T0 = Q X (Algorithm 1) fused with N^1D along z
    if (ln < NP * NP) {
      const int i = ln % NP, j = ln / NP;
      T x[NP], t[NQ];
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int d = sd[i + NP * (j + NP * k)];
        T val = act ? p.X[(int64_t)d * p.ld + col] : T(0);
        if (p.dscale) val *= p.dscale[d];
        x[k] = val;
      }
      eo_apply<NP, NQ, 1>(x, t, tb.N);
#pragma unroll
      for (int q = 0; q < NQ; ++q) Av[i * SX + j * SY + q * SZ] = t[q];
    }
    __syncthreads();
    // (2) N^1D along y
    if (ln < NP * NQ) {
      const int i = ln % NP, qz = ln / NP;
      T x[NP], t[NQ];
#pragma unroll
      for (int j = 0; j < NP; ++j) x[j] = Av[i * SX + j * SY + qz * SZ];
      eo_apply<NP, NQ, 1>(x, t, tb.N);
#pragma unroll
      for (int q = 0; q < NQ; ++q) Av[i * SX + q * SY + qz * SZ] = t[q];
    }
    __syncthreads();
    // (3) N^1D along x  ->  A = Y~0 (values at quadrature points)
    {
      const int qy = ln % NQ, qz = ln / NQ;
      T x[NP], t[NQ];
#pragma unroll
      for (int i = 0; i < NP; ++i) x[i] = Av[i * SX + qy * SY + qz * SZ];
      eo_apply<NP, NQ, 1>(x, t, tb.N);
#pragma unroll
      for (int q = 0; q < NQ; ++q) Av[q * SX + qy * SY + qz * SZ] = t[q];
    }
    __syncthreads();
    // (4) Y~1: D~ along x (A -> B) and along y (A -> C)
    {
      const int a0 = ln % NQ, qz = ln / NQ;
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
    __syncthreads();
    // (5) D~ along z in registers, then the quadrature-point step of
    //     Algorithm 2:  Z = V^L Y0 + V^G.Y1 - i V^K.Y1,
    //                   W_s = sum_d G_sd Y1_d + V^G_s Y0;
    //     W_x -> B, W_y -> C, and D~^T along z of W_z accumulated into Z.
    T zc[NQ];
    {
      const int qx = ln % NQ, qy = ln / NQ;
      T u[NQ], g[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) u[q] = Av[qx * SX + qy * SY + q * SZ];
      eo_apply<NQ, NQ, -1>(u, g, tb.D);
      const T* cf = p.coef + (int64_t)e * p.ncoef * NQ3 + qx + NQ * qy;
#pragma unroll
      for (int qz = 0; qz < NQ; ++qz) {
        const int o = qz * NQ * NQ;
        const int s = qx * SX + qy * SY + qz * SZ;
        const T gx = Bv[s], gy = Cv[s], gz = g[qz], uu = u[qz];
        const T G00 = cf[0 * NQ3 + o], G01 = cf[1 * NQ3 + o], G02 = cf[2 * NQ3 + o];
        const T G11 = cf[3 * NQ3 + o], G12 = cf[4 * NQ3 + o], G22 = cf[5 * NQ3 + o];
        const T VL = cf[6 * NQ3 + o];
        T z = VL * uu;
        T w0 = fma(G00, gx, fma(G01, gy, G02 * gz));
        T w1 = fma(G01, gx, fma(G11, gy, G12 * gz));
        T w2 = fma(G02, gx, fma(G12, gy, G22 * gz));
        if (p.gga) {
          const T V0 = cf[7 * NQ3 + o], V1 = cf[8 * NQ3 + o], V2 = cf[9 * NQ3 + o];
          z = fma(V0, gx, fma(V1, gy, fma(V2, gz, z)));
          w0 = fma(V0, uu, w0);
          w1 = fma(V1, uu, w1);
          w2 = fma(V2, uu, w2);
        }
        if (CPLX) {
          const T K0 = cf[10 * NQ3 + o], K1 = cf[11 * NQ3 + o], K2 = cf[12 * NQ3 + o];
          const T kk = fma(K0, gx, fma(K1, gy, K2 * gz));
          const T kp = __shfl_xor_sync(0xffffffffu, kk, 1);
          // -i (a + i b) = b - i a : real column adds Im, imaginary column subtracts Re
          z += (v & 1) ? -kp : kp;
        }
        Bv[s] = w0;
        Cv[s] = w1;
        u[qz] = w2;
        zc[qz] = z;
      }
      T t[NQ];
      eo_apply<NQ, NQ, -1>(u, t, tb.Dt);
#pragma unroll
      for (int q = 0; q < NQ; ++q) zc[q] += t[q];
    }
    __syncthreads();
    // (6) D~^T along x on B and along y on C (in place)
    {
      const int a0 = ln % NQ, qz = ln / NQ;
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
    {
      const int qx = ln % NQ, qy = ln / NQ;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int s = qx * SX + qy * SY + q * SZ;
        zc[q] += Bv[s] + Cv[s];
      }
      T t[NP];
      eo_apply<NQ, NP, 1>(zc, t, tb.Nt);
#pragma unroll
      for (int k = 0; k < NP; ++k) Av[qx * SX + qy * SY + k * SZ] = t[k];
    }
    __syncthreads();
    // (8) N^T along y
    if (ln < NQ * NP) {
      const int qx = ln % NQ, k = ln / NQ;
      T x[NQ], t[NP];
#pragma unroll
      for (int q = 0; q < NQ; ++q) x[q] = Av[qx * SX + q * SY + k * SZ];
      eo_apply<NQ, NP, 1>(x, t, tb.Nt);
#pragma unroll
      for (int j = 0; j < NP; ++j) Av[qx * SX + j * SY + k * SZ] = t[j];
    }
    __syncthreads();
    // (9) N^T along x, + sum_a F Delta P (nonlocal), assembly Y += Q^T T0
    if (ln < NP * NP) {
      const int j = ln % NP, k = ln / NP;
      T x[NQ], y[NP];
#pragma unroll
      for (int q = 0; q < NQ; ++q) x[q] = Av[q * SX + j * SY + k * SZ];
      eo_apply<NQ, NP, 1>(x, y, tb.Nt);
      if (act) {
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
  }
}

// Columns per CTA: the shared-memory tile is 3 buffers of n_q^3 x VT values.
template <typename T, int NQ>
constexpr int local_vt() {
  return (NQ >= 7) ? 4 : 8;
}

template <typename T, int P>
cudaError_t launch_local_deg(const Ctx& c, const LocalParams<T>& prm, cudaStream_t s) {
  constexpr int NP = P + 1, NQ = P + 1;
  constexpr int VT = local_vt<T, NQ>();
  constexpr size_t smem = local_smem_bytes<T, NP, NQ, VT>();
  const int tiles = (prm.ncols + VT - 1) / VT;
  const int gy = prm.n_cells < 65535 ? prm.n_cells : 65535;
  if (prm.n_cells == 0) return cudaSuccess;
  dim3 grid(tiles, gy);
  // the shared-memory opt-in is a per-device function attribute: set it once per device
  static bool attr_done[2][64] = {};
  const int dev = c.device & 63;
  if (c.cplx) {
    auto k = fe_local_kernel<T, NP, NQ, VT, true>;
    if (!attr_done[1][dev]) {
      cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      attr_done[1][dev] = true;
    }
    k<<<grid, VT * NQ * NQ, smem, s>>>(prm);
  } else {
    auto k = fe_local_kernel<T, NP, NQ, VT, false>;
    if (!attr_done[0][dev]) {
      cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      attr_done[0][dev] = true;
    }
    k<<<grid, VT * NQ * NQ, smem, s>>>(prm);
  }
  return cudaGetLastError();
}

}  // namespace feks
