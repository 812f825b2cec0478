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
#include <type_traits>

#include "fe_ks_internal.h"

namespace feks {

// Arithmetic-type traits: zero, conversion from the storage type, the
// scatter-add into the storage type, and the re/im partner shuffle.
template <typename T>
struct Num {
  static __device__ __forceinline__ T zero() { return T(0); }
  static __device__ __forceinline__ T one() { return T(1); }
  template <typename TS>
  static __device__ __forceinline__ T in(TS x) { return (T)x; }
  template <typename TS>
  static __device__ __forceinline__ void add_to(TS* y, T v) { *y += v; }
  static __device__ __forceinline__ T shfl1(T v) { return __shfl_xor_sync(0xffffffffu, v, 1); }
};
template <>
struct Num<ff2> {
  static __device__ __forceinline__ ff2 zero() { return ff_make(0.f, 0.f); }
  static __device__ __forceinline__ ff2 one() { return ff_make(1.f, 0.f); }
  static __device__ __forceinline__ ff2 in(double x) { return ff_split_bits(x); }
  // Two fire-and-forget reductions (performed in the L2, in issue order for the
  // one address) instead of a load, two FP64 adds and a store: on this part the
  // FP64 adds cost as much issue time as the whole pair-of-floats tile work.
  // The scatter is colour-exclusive, so the result stays deterministic.
  static __device__ __forceinline__ void add_to(double* y, ff2 v) {
    atomicAdd(y, f2d_bits(v.hi));
    atomicAdd(y, f2d_bits(v.lo));
  }
  static __device__ __forceinline__ ff2 shfl1(ff2 v) {
    return ff_make(__shfl_xor_sync(0xffffffffu, v.hi, 1), __shfl_xor_sync(0xffffffffu, v.lo, 1));
  }
};

// Two FP32 columns in one 64-bit register: the packed FP32x2 instructions of
// this architecture (add / sub / mul / fma .f32x2) do the two columns' work in
// one issue slot, each half rounded exactly as its scalar instruction.
struct f2v {
  unsigned long long v;
};
__device__ __forceinline__ f2v f2v_make(float lo, float hi) {
  f2v r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 f2v_split(f2v x) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x.v));
  return make_float2(lo, hi);
}
__device__ __forceinline__ f2v operator+(f2v a, f2v b) {
  f2v r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2v operator-(f2v a, f2v b) {
  f2v r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2v operator*(float a, f2v b) {
  f2v r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(f2v_make(a, a).v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2v fma(float a, f2v b, f2v c) {
  f2v r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(f2v_make(a, a).v), "l"(b.v), "l"(c.v));
  return r;
}

// y = M x for an NO x NI matrix with M[NO-1-o][NI-1-i] = S M[o][i], given its
// even-odd split (see EOMat).  All indices are compile-time constants, so the
// table entries are read straight from the kernel parameter bank.  T is the
// data type (also f2v: two FP32 columns at once), TM the matrix entries' type.
template <int NI, int NO, int S, typename T, typename TM>
__device__ __forceinline__ void eo_apply(const T* x, T* y, const EOMat<TM>& m) {
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

// eo_apply for each of a thread's VPT columns: x[VPT][NI] -> o[NO][VPT]
// (O_COL_MAJOR false) or o[VPT][NO] (true).  FP32 columns go two at a time
// through the packed FP32x2 instructions; the results are bit for bit those
// of the per-column scalar form.
template <int NI, int NO, int S, bool O_COL_MAJOR = false, typename T, int VPT, typename TO>
__device__ __forceinline__ void eo_apply_cols(const T (&x)[VPT][NI], TO& o, const EOMat<T>& m) {
  if constexpr (std::is_same<T, float>::value && VPT % 2 == 0) {
#pragma unroll
    for (int u = 0; u < VPT; u += 2) {
      f2v xx[NI], tt[NO];
#pragma unroll
      for (int k = 0; k < NI; ++k) xx[k] = f2v_make(x[u][k], x[u + 1][k]);
      eo_apply<NI, NO, S>(xx, tt, m);
#pragma unroll
      for (int q = 0; q < NO; ++q) {
        const float2 r = f2v_split(tt[q]);
        if constexpr (O_COL_MAJOR) {
          o[u][q] = r.x;
          o[u + 1][q] = r.y;
        } else {
          o[q][u] = r.x;
          o[q][u + 1] = r.y;
        }
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < VPT; ++u) {
      T t[NO];
      eo_apply<NI, NO, S>(x[u], t, m);
#pragma unroll
      for (int q = 0; q < NO; ++q) {
        if constexpr (O_COL_MAJOR)
          o[u][q] = t[q];
        else
          o[q][u] = t[q];
      }
    }
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
  // coefficient block padded to a multiple of 16 bytes, so that what follows
  // it stays 16-byte aligned (cp.async of 16 bytes needs aligned targets)
  static constexpr int CF_ELEMS = ((NCOEF * NQ3 * (int)sizeof(T) + 15) / 16) * 16 / (int)sizeof(T);
  // FP32 stages the cell's coefficients in shared memory (its loads are latency
  // bound); FP64 is bound by the FP64 pipe and keeps the occupancy instead.
  static constexpr bool STAGE_COEF = sizeof(T) == 4;
  static constexpr size_t bytes =
      (size_t)(3 * BUF + (STAGE_COEF ? CF_ELEMS : 0)) * sizeof(T) + (size_t)NP3 * sizeof(int);
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

// Phases (1)-(9) of one cell tile.  xs: staged gather [n_p^3][VT] in shared
// memory, or nullptr to gather from global memory; cfs: the cell's
// coefficients (shared or global); ATOMIC: scatter with fire-and-forget
// reductions instead of read-modify-write.
template <typename T, int NP, int NQ, int VT, bool CPLX, int NT, bool ATOMIC, class Prm>
__device__ __forceinline__ void tile_body(const Prm& p, const EOTables<T>& tb, int e, int col0, T* A, T* B, T* C,
                                          const T* cfs, const int* sd, const T* xs, bool wait_coef) {
  using S = CellShape<T, NP, NQ, VT, CPLX>;
  constexpr int SX = S::SX, SY = S::SY, SZ = S::SZ, NQ3 = S::NQ3, NP3 = S::NP3;
  const int tid = threadIdx.x;
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
      const int node = i + NP * (j + NP * k);
      const int d = sd[node];
      T val = xs ? xs[node * VT + v] : (act ? Num<T>::in(p.X[(int64_t)d * p.ld + col]) : Num<T>::zero());
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
  if (wait_coef) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
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
    const T* cf = cfs + qx + NQ * qy;
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
        const T kp = Num<T>::shfl1(kk);
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
          const auto* Qa = p.Q + ((int64_t)a * p.n_proj + b) * p.ld;
          if (!CPLX) {
            const T* Fr = p.F + ((int64_t)pr * p.n_proj + b) * NP3 + NP * (j + NP * k);
            const T q = Num<T>::in(Qa[col]);
#pragma unroll
            for (int i = 0; i < NP; ++i) y[i] = fma(Fr[i], q, y[i]);
          } else {
            const T* Fr = p.F + (((int64_t)pr * p.n_proj + b) * NP3 + NP * (j + NP * k)) * 2;
            const int cb = col & ~1;
            const T qr = Num<T>::in(Qa[cb]), qi = Num<T>::in(Qa[cb + 1]);
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
      auto* yp = p.Y + (int64_t)d * p.ld + col;
      if constexpr (ATOMIC)
        atomicAdd(yp, val);   // fire-and-forget reduction; the colouring keeps it race-free anyway
      else
        Num<T>::add_to(yp, val);
    }
  }
}

// One cell e, columns [col0, col0 + VT).  All NT threads of the block call it.
// Prm is any struct with the operand fields of LocalParams (X, Y, ld, ncols,
// cell_dofs, coef, ncoef, gga, dscale, cell_pair_ptr, cell_pairs, pair_atom,
// F, Q, n_proj, alpha); the 1D tables come separately so that they stay in
// the kernel parameter bank.
template <typename T, int NP, int NQ, int VT, bool CPLX, int NT, class Prm>
__device__ __forceinline__ void cell_tile(const Prm& p, const EOTables<T>& tb, int e, int col0, unsigned char* smem) {
  using S = CellShape<T, NP, NQ, VT, CPLX>;
  constexpr int BUF = S::BUF, NQ3 = S::NQ3, NP3 = S::NP3;
  T* A = reinterpret_cast<T*>(smem);
  T* B = A + BUF;
  T* C = B + BUF;
  T* CF = C + BUF;
  int* sd = reinterpret_cast<int*>(CF + (S::STAGE_COEF ? S::CF_ELEMS : 0));
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
  tile_body<T, NP, NQ, VT, CPLX, NT, false>(p, tb, e, col0, A, B, C,
                                           S::STAGE_COEF ? CF : p.coef + (int64_t)e * p.ncoef * NQ3, sd, nullptr,
                                           S::STAGE_COEF);
}

// One CTA per (cell of the colour, VT-column tile); loops over cells when the
// colour has more cells than gridDim.y.
template <typename T, typename TS, int NP, int NQ, int VT, bool CPLX, int NT>
__global__ void __launch_bounds__(NT) fe_local_kernel(const __grid_constant__ LocalParams<T, TS> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int ci = blockIdx.y; ci < p.n_cells; ci += gridDim.y)
    cell_tile<T, NP, NQ, VT, CPLX, NT>(p, p.tab, p.cells[ci], blockIdx.x * VT, smem_raw);
}

// Column-group loads / stores: VPT consecutive columns of one point, as one
// shared-memory access when VPT * sizeof(T) is 8 or 16 bytes.
template <typename T, int VPT>
__device__ __forceinline__ void ld_cols(const T* p, T* out) {
  if constexpr (VPT * sizeof(T) == 16) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    const T* t = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int u = 0; u < VPT; ++u) out[u] = t[u];
  } else if constexpr (VPT * sizeof(T) == 8) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    const T* t = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int u = 0; u < VPT; ++u) out[u] = t[u];
  } else {
#pragma unroll
    for (int u = 0; u < VPT; ++u) out[u] = p[u];
  }
}
template <typename T, int VPT>
__device__ __forceinline__ void st_cols(T* p, const T* in) {
  if constexpr (VPT * sizeof(T) == 16) {
    float4 v;
    T* t = reinterpret_cast<T*>(&v);
#pragma unroll
    for (int u = 0; u < VPT; ++u) t[u] = in[u];
    *reinterpret_cast<float4*>(p) = v;
  } else if constexpr (VPT * sizeof(T) == 8) {
    float2 v;
    T* t = reinterpret_cast<T*>(&v);
#pragma unroll
    for (int u = 0; u < VPT; ++u) t[u] = in[u];
    *reinterpret_cast<float2*>(p) = v;
  } else {
#pragma unroll
    for (int u = 0; u < VPT; ++u) p[u] = in[u];
  }
}

// Phases (1)-(9) of one cell tile with VPT consecutive columns per thread
// (vector shared-memory accesses; the coefficients of a point are read once
// for its VPT columns; for complex operators the re/im partner column sits in
// the same thread).  Gathers from the staged buffer xs only; scatters with
// reductions.  Same arithmetic, in the same order per column, as tile_body.
struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// Coefficient read: from shared memory (staged) or from global memory through
// the read-only L1 path (GLOBAL_CF).
template <bool GLOBAL_CF, typename T>
__device__ __forceinline__ T ld_coef(const T* p) {
  if constexpr (GLOBAL_CF)
    return __ldg(p);
  else
    return *p;
}

// after1: called by every thread right after phase (1) has finished reading xs
// (after its barrier), so a single staging buffer can be refilled while
// phases (2)-(9) run.
template <typename T, int NP, int NQ, int VT, int VPT, bool CPLX, int NT, class Prm, bool GLOBAL_CF = false,
          class Hook = NoHook>
__device__ __forceinline__ void tile_body_v(const Prm& p, const EOTables<T>& tb, int e, int col0, T* A, T* B, T* C,
                                            const T* cfs, const int* sd, const T* xs, Hook after1 = Hook()) {
  using S = CellShape<T, NP, NQ, VT, CPLX>;
  constexpr int SX = S::SX, SY = S::SY, SZ = S::SZ, NQ3 = S::NQ3, NP3 = S::NP3;
  constexpr int VG = VT / VPT;
  static_assert(VT % VPT == 0 && (!CPLX || VPT % 2 == 0), "column groups must hold whole complex pairs");
  const int tid = threadIdx.x;

  // (1) N^1D along z from the staged gather
#pragma unroll 1
  for (int w = tid; w < NP * NP * VG; w += NT) {
    const int v0 = (w % VG) * VPT, ln = w / VG;
    const int i = ln % NP, j = ln / NP;
    T x[VPT][NP], t[NQ];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int node = i + NP * (j + NP * k);
      T c[VPT];
      ld_cols<T, VPT>(xs + node * VT + v0, c);
      if (p.dscale) {
        const T ds = p.dscale[sd[node]];
#pragma unroll
        for (int u = 0; u < VPT; ++u) c[u] *= ds;
      }
#pragma unroll
      for (int u = 0; u < VPT; ++u) x[u][k] = c[u];
    }
    T o[NQ][VPT];
    eo_apply_cols<NP, NQ, 1>(x, o, tb.N);
#pragma unroll
    for (int q = 0; q < NQ; ++q) st_cols<T, VPT>(A + i * SX + j * SY + q * SZ + v0, o[q]);
  }
  __syncthreads();
  after1();
  // (2) N^1D along y
#pragma unroll 1
  for (int w = tid; w < NP * NQ * VG; w += NT) {
    const int v0 = (w % VG) * VPT, ln = w / VG;
    const int i = ln % NP, qz = ln / NP;
    T x[VPT][NP], t[NQ], o[NQ][VPT];
#pragma unroll
    for (int jj = 0; jj < NP; ++jj) {
      T c[VPT];
      ld_cols<T, VPT>(A + i * SX + jj * SY + qz * SZ + v0, c);
#pragma unroll
      for (int u = 0; u < VPT; ++u) x[u][jj] = c[u];
    }
    eo_apply_cols<NP, NQ, 1>(x, o, tb.N);
#pragma unroll
    for (int q = 0; q < NQ; ++q) st_cols<T, VPT>(A + i * SX + q * SY + qz * SZ + v0, o[q]);
  }
  __syncthreads();
  // (3) N^1D along x
#pragma unroll 1
  for (int w = tid; w < NQ * NQ * VG; w += NT) {
    const int v0 = (w % VG) * VPT, ln = w / VG;
    const int qy = ln % NQ, qz = ln / NQ;
    T x[VPT][NP], t[NQ], o[NQ][VPT];
#pragma unroll
    for (int ii = 0; ii < NP; ++ii) {
      T c[VPT];
      ld_cols<T, VPT>(A + ii * SX + qy * SY + qz * SZ + v0, c);
#pragma unroll
      for (int u = 0; u < VPT; ++u) x[u][ii] = c[u];
    }
    eo_apply_cols<NP, NQ, 1>(x, o, tb.N);
#pragma unroll
    for (int q = 0; q < NQ; ++q) st_cols<T, VPT>(A + q * SX + qy * SY + qz * SZ + v0, o[q]);
  }
  __syncthreads();
  // (4) D~ along x (A -> B) and along y (A -> C)
#pragma unroll 1
  for (int w = tid; w < NQ * NQ * VG; w += NT) {
    const int v0 = (w % VG) * VPT, ln = w / VG;
    const int a0 = ln % NQ, qz = ln / NQ;
    T x[VPT][NQ], t[NQ], o[NQ][VPT];
#pragma unroll
    for (int r = 0; r < NQ; ++r) {
      T c[VPT];
      ld_cols<T, VPT>(A + r * SX + a0 * SY + qz * SZ + v0, c);
#pragma unroll
      for (int u = 0; u < VPT; ++u) x[u][r] = c[u];
    }
    eo_apply_cols<NQ, NQ, -1>(x, o, tb.D);
#pragma unroll
    for (int q = 0; q < NQ; ++q) st_cols<T, VPT>(B + q * SX + a0 * SY + qz * SZ + v0, o[q]);
#pragma unroll
    for (int r = 0; r < NQ; ++r) {
      T c[VPT];
      ld_cols<T, VPT>(A + a0 * SX + r * SY + qz * SZ + v0, c);
#pragma unroll
      for (int u = 0; u < VPT; ++u) x[u][r] = c[u];
    }
    eo_apply_cols<NQ, NQ, -1>(x, o, tb.D);
#pragma unroll
    for (int q = 0; q < NQ; ++q) st_cols<T, VPT>(C + a0 * SX + q * SY + qz * SZ + v0, o[q]);
  }
  __syncthreads();
  // (5) D~ along z, quadrature-point step, D~z^T; W_x -> B, W_y -> C, Z -> A
#pragma unroll 1
  for (int w = tid; w < NQ * NQ * VG; w += NT) {
    const int v0 = (w % VG) * VPT, ln = w / VG;
    const int qx = ln % NQ, qy = ln / NQ;
    T u_[VPT][NQ], g_[VPT][NQ], z_[VPT][NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T c[VPT];
      ld_cols<T, VPT>(A + qx * SX + qy * SY + q * SZ + v0, c);
#pragma unroll
      for (int u = 0; u < VPT; ++u) u_[u][q] = c[u];
    }
    eo_apply_cols<NQ, NQ, -1, true>(u_, g_, tb.D);
    const T* cf = cfs + qx + NQ * qy;
#pragma unroll
    for (int qz = 0; qz < NQ; ++qz) {
      const int o = qz * NQ * NQ;
      const int s = qx * SX + qy * SY + qz * SZ + v0;
      T gx[VPT], gy[VPT], w0[VPT], w1[VPT], kk[VPT];
      ld_cols<T, VPT>(B + s, gx);
      ld_cols<T, VPT>(C + s, gy);
      const T G00 = ld_coef<GLOBAL_CF>(cf + 0 * NQ3 + o), G01 = ld_coef<GLOBAL_CF>(cf + 1 * NQ3 + o);
      const T G02 = ld_coef<GLOBAL_CF>(cf + 2 * NQ3 + o), G11 = ld_coef<GLOBAL_CF>(cf + 3 * NQ3 + o);
      const T G12 = ld_coef<GLOBAL_CF>(cf + 4 * NQ3 + o), G22 = ld_coef<GLOBAL_CF>(cf + 5 * NQ3 + o);
      const T VL = ld_coef<GLOBAL_CF>(cf + 6 * NQ3 + o);
      T V0 = Num<T>::zero(), V1 = V0, V2 = V0;
      if (p.gga) {
        V0 = ld_coef<GLOBAL_CF>(cf + 7 * NQ3 + o);
        V1 = ld_coef<GLOBAL_CF>(cf + 8 * NQ3 + o);
        V2 = ld_coef<GLOBAL_CF>(cf + 9 * NQ3 + o);
      }
#pragma unroll
      for (int u = 0; u < VPT; ++u) {
        const T gz = g_[u][qz], uu = u_[u][qz];
        T z = VL * uu;
        T a0v = fma(G00, gx[u], fma(G01, gy[u], G02 * gz));
        T a1v = fma(G01, gx[u], fma(G11, gy[u], G12 * gz));
        T a2v = fma(G02, gx[u], fma(G12, gy[u], G22 * gz));
        if (p.gga) {
          z = fma(V0, gx[u], fma(V1, gy[u], fma(V2, gz, z)));
          a0v = fma(V0, uu, a0v);
          a1v = fma(V1, uu, a1v);
          a2v = fma(V2, uu, a2v);
        }
        if (CPLX) {
          const T K0 = ld_coef<GLOBAL_CF>(cf + 10 * NQ3 + o), K1 = ld_coef<GLOBAL_CF>(cf + 11 * NQ3 + o);
          const T K2 = ld_coef<GLOBAL_CF>(cf + 12 * NQ3 + o);
          kk[u] = fma(K0, gx[u], fma(K1, gy[u], K2 * gz));
        }
        w0[u] = a0v;
        w1[u] = a1v;
        u_[u][qz] = a2v;
        z_[u][qz] = z;
      }
      if (CPLX) {
        // -i (a + i b) = b - i a : the partner column of u is u ^ 1 in this thread
#pragma unroll
        for (int u = 0; u < VPT; ++u) z_[u][qz] += (u & 1) ? -kk[u ^ 1] : kk[u ^ 1];
      }
      st_cols<T, VPT>(B + s, w0);
      st_cols<T, VPT>(C + s, w1);
    }
    T o[NQ][VPT];
    eo_apply_cols<NQ, NQ, -1>(u_, o, tb.Dt);
#pragma unroll
    for (int u = 0; u < VPT; ++u)
#pragma unroll
      for (int q = 0; q < NQ; ++q) o[q][u] = z_[u][q] + o[q][u];
#pragma unroll
    for (int q = 0; q < NQ; ++q) st_cols<T, VPT>(A + qx * SX + qy * SY + q * SZ + v0, o[q]);
  }
  __syncthreads();
  // (6) D~^T along x on B and along y on C (in place)
#pragma unroll 1
  for (int w = tid; w < NQ * NQ * VG; w += NT) {
    const int v0 = (w % VG) * VPT, ln = w / VG;
    const int a0 = ln % NQ, qz = ln / NQ;
    T x[VPT][NQ], t[NQ], o[NQ][VPT];
#pragma unroll
    for (int r = 0; r < NQ; ++r) {
      T c[VPT];
      ld_cols<T, VPT>(B + r * SX + a0 * SY + qz * SZ + v0, c);
#pragma unroll
      for (int u = 0; u < VPT; ++u) x[u][r] = c[u];
    }
    eo_apply_cols<NQ, NQ, -1>(x, o, tb.Dt);
#pragma unroll
    for (int q = 0; q < NQ; ++q) st_cols<T, VPT>(B + q * SX + a0 * SY + qz * SZ + v0, o[q]);
#pragma unroll
    for (int r = 0; r < NQ; ++r) {
      T c[VPT];
      ld_cols<T, VPT>(C + a0 * SX + r * SY + qz * SZ + v0, c);
#pragma unroll
      for (int u = 0; u < VPT; ++u) x[u][r] = c[u];
    }
    eo_apply_cols<NQ, NQ, -1>(x, o, tb.Dt);
#pragma unroll
    for (int q = 0; q < NQ; ++q) st_cols<T, VPT>(C + a0 * SX + q * SY + qz * SZ + v0, o[q]);
  }
  __syncthreads();
  // (7) Z += D~x^T W_x + D~y^T W_y, then N^T along z -> A
#pragma unroll 1
  for (int w = tid; w < NQ * NQ * VG; w += NT) {
    const int v0 = (w % VG) * VPT, ln = w / VG;
    const int qx = ln % NQ, qy = ln / NQ;
    T zc[VPT][NQ], t[NP], o[NP][VPT];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int s = qx * SX + qy * SY + q * SZ + v0;
      T a[VPT], b[VPT], c[VPT];
      ld_cols<T, VPT>(A + s, a);
      ld_cols<T, VPT>(B + s, b);
      ld_cols<T, VPT>(C + s, c);
#pragma unroll
      for (int u = 0; u < VPT; ++u) zc[u][q] = a[u] + (b[u] + c[u]);
    }
    eo_apply_cols<NQ, NP, 1>(zc, o, tb.Nt);
#pragma unroll
    for (int k = 0; k < NP; ++k) st_cols<T, VPT>(A + qx * SX + qy * SY + k * SZ + v0, o[k]);
  }
  __syncthreads();
  // (8) N^T along y
#pragma unroll 1
  for (int w = tid; w < NQ * NP * VG; w += NT) {
    const int v0 = (w % VG) * VPT, ln = w / VG;
    const int qx = ln % NQ, k = ln / NQ;
    T x[VPT][NQ], t[NP], o[NP][VPT];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T c[VPT];
      ld_cols<T, VPT>(A + qx * SX + q * SY + k * SZ + v0, c);
#pragma unroll
      for (int u = 0; u < VPT; ++u) x[u][q] = c[u];
    }
    eo_apply_cols<NQ, NP, 1>(x, o, tb.Nt);
#pragma unroll
    for (int jj = 0; jj < NP; ++jj) st_cols<T, VPT>(A + qx * SX + jj * SY + k * SZ + v0, o[jj]);
  }
  __syncthreads();
  // (9) N^T along x, + sum_a F Delta P, assembly by reductions
#pragma unroll 1
  for (int w = tid; w < NP * NP * VG; w += NT) {
    const int v0 = (w % VG) * VPT, ln = w / VG;
    const int j = ln % NP, k = ln / NP;
    T x[VPT][NQ], y[VPT][NP];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T c[VPT];
      ld_cols<T, VPT>(A + q * SX + j * SY + k * SZ + v0, c);
#pragma unroll
      for (int u = 0; u < VPT; ++u) x[u][q] = c[u];
    }
    eo_apply_cols<NQ, NP, 1, true>(x, y, tb.Nt);
    if (p.cell_pair_ptr) {
      const int pb = p.cell_pair_ptr[e], pe = p.cell_pair_ptr[e + 1];
      for (int pi = pb; pi < pe; ++pi) {
        const int pr = p.cell_pairs[pi];
        const int a = p.pair_atom[pr];
        for (int b = 0; b < p.n_proj; ++b) {
          const auto* Qa = p.Q + ((int64_t)a * p.n_proj + b) * p.ld + col0 + v0;
          T q[VPT];
#pragma unroll
          for (int u = 0; u < VPT; ++u) q[u] = (col0 + v0 + u < p.ncols) ? Num<T>::in(Qa[u]) : Num<T>::zero();
          if (!CPLX) {
            const T* Fr = p.F + ((int64_t)pr * p.n_proj + b) * NP3 + NP * (j + NP * k);
#pragma unroll
            for (int i = 0; i < NP; ++i) {
              const T f = Fr[i];
#pragma unroll
              for (int u = 0; u < VPT; ++u) y[u][i] = fma(f, q[u], y[u][i]);
            }
          } else {
            const T* Fr = p.F + (((int64_t)pr * p.n_proj + b) * NP3 + NP * (j + NP * k)) * 2;
#pragma unroll
            for (int i = 0; i < NP; ++i) {
              const T fr = Fr[2 * i], fi = Fr[2 * i + 1];
#pragma unroll
              for (int u = 0; u < VPT; u += 2) {
                const T qr = q[u], qi = q[u + 1];
                y[u][i] += fma(fr, qr, -fi * qi);
                y[u + 1][i] += fma(fr, qi, fi * qr);
              }
            }
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const int d = sd[i + NP * (j + NP * k)];
      const T ds = p.dscale ? p.dscale[d] : Num<T>::one();
      auto* yp = p.Y + (int64_t)d * p.ld + col0 + v0;
#pragma unroll
      for (int u = 0; u < VPT; ++u)
        if (col0 + v0 + u < p.ncols) atomicAdd(yp + u, y[u][i] * p.alpha * ds);
    }
  }
}

// Cell-major variant: one CTA per cell of the colour.  It stages the cell's
// coefficients and DoF list once, then walks all column tiles of the cell,
// gathering the next tile's rows of X into a second shared buffer with
// cp.async while the current tile is computed; the scatter uses
// fire-and-forget reductions, so no thread waits on a read of Y.
template <typename T, int NP, int NQ, int VT, bool CPLX>
struct StagedShape {
  using S = CellShape<T, NP, NQ, VT, CPLX>;
  static constexpr size_t xs_elems = (size_t)S::NP3 * VT;
  static constexpr size_t bytes = (size_t)(3 * S::BUF + S::CF_ELEMS + 2 * xs_elems) * sizeof(T) +
                                  (size_t)S::NP3 * sizeof(int);
  static_assert((3 * S::BUF * sizeof(T)) % 16 == 0 && (S::CF_ELEMS * sizeof(T)) % 16 == 0 &&
                    (xs_elems * sizeof(T)) % 16 == 0,
                "staged gather buffers must start on 16-byte boundaries");
  static constexpr bool fits = bytes <= 227 * 1024;
};

__device__ __forceinline__ void cp_async_16z(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_4z(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_8z(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}

// Issue the gather of columns [col0, col0 + VT) of the cell's rows into xs.
template <typename T, int NP3, int VT, int NT>
__device__ __forceinline__ void stage_rows(const T* __restrict__ X, int64_t ld, int ncols, const int* sd, int col0,
                                           T* xs, bool vec_ok) {
  constexpr int EPC = 16 / sizeof(T);   // elements per 16-byte chunk
  if (vec_ok) {
    constexpr int CH = VT / EPC;
    for (int idx = threadIdx.x; idx < NP3 * CH; idx += NT) {
      const int node = idx / CH, ch = idx % CH;
      const int col = col0 + ch * EPC;
      int nb = (ncols - col) * (int)sizeof(T);
      nb = nb < 0 ? 0 : (nb > 16 ? 16 : nb);
      const T* src = nb > 0 ? X + (int64_t)sd[node] * ld + col : X;
      cp_async_16z(xs + node * VT + ch * EPC, src, nb);
    }
  } else {
    for (int idx = threadIdx.x; idx < NP3 * VT; idx += NT) {
      const int node = idx / VT, v = idx % VT;
      const int col = col0 + v;
      const bool in = col < ncols;
      const T* src = in ? X + (int64_t)sd[node] * ld + col : X;
      if (sizeof(T) == 8)
        cp_async_8z(xs + idx, src, in ? 8 : 0);
      else
        cp_async_4z(xs + idx, src, in ? 4 : 0);
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <typename T, int NP, int NQ, int VT, bool CPLX, int NT, int VPT>
__global__ void __launch_bounds__(NT) fe_local_staged_kernel(const __grid_constant__ LocalParams<T, T> p) {
  using S = CellShape<T, NP, NQ, VT, CPLX>;
  using SS = StagedShape<T, NP, NQ, VT, CPLX>;
  constexpr int BUF = S::BUF, NQ3 = S::NQ3, NP3 = S::NP3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* B = A + BUF;
  T* C = B + BUF;
  T* CF = C + BUF;
  T* XS0 = CF + S::CF_ELEMS;
  T* XS1 = XS0 + SS::xs_elems;
  int* sd = reinterpret_cast<int*>(XS1 + SS::xs_elems);
  const int ntiles = (p.ncols + VT - 1) / VT;
  const bool vec_ok = (VT * sizeof(T)) % 16 == 0 && ((uintptr_t)p.X % 16) == 0 && ((p.ld * sizeof(T)) % 16) == 0;
  for (int ci = blockIdx.x; ci < p.n_cells; ci += gridDim.x) {
    const int e = p.cells[ci];
    __syncthreads();   // previous cell's readers are done with the shared buffers
    {
      const T* g = p.coef + (int64_t)e * p.ncoef * NQ3;
      const int n = p.ncoef * NQ3;
      for (int i = threadIdx.x; i < n; i += NT) {
        if (sizeof(T) == 8)
          cp_async_8(CF + i, g + i);
        else
          cp_async_4(CF + i, g + i);
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    for (int i = threadIdx.x; i < NP3; i += NT) sd[i] = p.cell_dofs[(int64_t)e * NP3 + i];
    __syncthreads();
    stage_rows<T, NP3, VT, NT>(p.X, p.ld, p.ncols, sd, 0, XS0, vec_ok);
    for (int t = 0; t < ntiles; ++t) {
      T* cur = (t & 1) ? XS1 : XS0;
      T* nxt = (t & 1) ? XS0 : XS1;
      if (t + 1 < ntiles) {
        stage_rows<T, NP3, VT, NT>(p.X, p.ld, p.ncols, sd, (t + 1) * VT, nxt, vec_ok);
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      }
      __syncthreads();
      if constexpr (VPT == 1)
        tile_body<T, NP, NQ, VT, CPLX, NT, true>(p, p.tab, e, t * VT, A, B, C, CF, sd, cur, false);
      else
        tile_body_v<T, NP, NQ, VT, VPT, CPLX, NT>(p, p.tab, e, t * VT, A, B, C, CF, sd, cur);
      __syncthreads();
    }
  }
}

// Lean cell-major variant: the same walk over a cell's column tiles with ONE
// staging buffer, refilled with the next tile's rows of X (cp.async) as soon
// as phase (1) has consumed it, and the cell's coefficients read from global
// memory through the read-only L1 path instead of being staged.  That halves
// the shared memory of the staged variant (96 KB at p = 8, VT = 8, FP32), so
// MINB CTAs share an SM and there are about twice the warps to hide the
// latency of the sweeps' shared-memory round trips.
template <typename T, int NP, int NQ, int VT, bool CPLX>
struct LeanShape {
  using S = CellShape<T, NP, NQ, VT, CPLX>;
  static constexpr size_t xs_elems = (size_t)S::NP3 * VT;
  static constexpr size_t bytes = (size_t)(3 * S::BUF + xs_elems) * sizeof(T) + (size_t)S::NP3 * sizeof(int);
  static_assert((3 * S::BUF * sizeof(T)) % 16 == 0 && (xs_elems * sizeof(T)) % 16 == 0,
                "the staging buffer must start on a 16-byte boundary");
  static constexpr bool fits = bytes <= 227 * 1024;
};

template <typename T, int NP, int NQ, int VT, bool CPLX, int NT, int VPT, int MINB>
__global__ void __launch_bounds__(NT, MINB) fe_local_lean_kernel(const __grid_constant__ LocalParams<T, T> p) {
  using S = CellShape<T, NP, NQ, VT, CPLX>;
  using LS = LeanShape<T, NP, NQ, VT, CPLX>;
  constexpr int BUF = S::BUF, NQ3 = S::NQ3, NP3 = S::NP3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* B = A + BUF;
  T* C = B + BUF;
  T* XS = C + BUF;
  int* sd = reinterpret_cast<int*>(XS + LS::xs_elems);
  const int ntiles = (p.ncols + VT - 1) / VT;
  const bool vec_ok = (VT * sizeof(T)) % 16 == 0 && ((uintptr_t)p.X % 16) == 0 && ((p.ld * sizeof(T)) % 16) == 0;
  for (int ci = blockIdx.x; ci < p.n_cells; ci += gridDim.x) {
    const int e = p.cells[ci];
    __syncthreads();   // the previous cell's readers are done with sd and XS
    for (int i = threadIdx.x; i < NP3; i += NT) sd[i] = p.cell_dofs[(int64_t)e * NP3 + i];
    __syncthreads();
    stage_rows<T, NP3, VT, NT>(p.X, p.ld, p.ncols, sd, 0, XS, vec_ok);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const T* cfg = p.coef + (int64_t)e * p.ncoef * NQ3;
    for (int t = 0; t < ntiles; ++t) {
      auto refill = [&]() {
        if (t + 1 < ntiles) stage_rows<T, NP3, VT, NT>(p.X, p.ld, p.ncols, sd, (t + 1) * VT, XS, vec_ok);
      };
      tile_body_v<T, NP, NQ, VT, VPT, CPLX, NT, LocalParams<T, T>, true>(p, p.tab, e, t * VT, A, B, C, cfg, sd, XS,
                                                                          refill);
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      __syncthreads();
    }
  }
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

template <typename T, typename TS, int NP, int NQ, int VT, int NT>
cudaError_t launch_local_cfg(const Ctx& c, const LocalParams<T, TS>& prm, cudaStream_t s) {
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
      auto k = fe_local_kernel<T, TS, NP, NQ, VT, true, NT>;
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
      auto k = fe_local_kernel<T, TS, NP, NQ, VT, false, NT>;
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

template <typename T, typename TS, int NP, int NQ, int VT, int NT, int VPT = 1>
cudaError_t launch_staged_cfg(const Ctx& c, const LocalParams<T, TS>& prm, cudaStream_t s) {
  if constexpr (!std::is_same<T, TS>::value) {
    return cudaErrorInvalidConfiguration;   // the reduction scatter needs T == storage type
  } else {
    if (prm.n_cells == 0) return cudaSuccess;
    const int gx = prm.n_cells < (1 << 30) ? prm.n_cells : (1 << 30);
    static bool attr_done[2][64] = {};
    const int dev = c.device & 63;
    if (c.cplx) {
      using SS = StagedShape<T, NP, NQ, VT, true>;
      if constexpr (!SS::fits) {
        return cudaErrorInvalidConfiguration;
      } else {
        auto k = fe_local_staged_kernel<T, NP, NQ, VT, true, NT, VPT>;
        if (!attr_done[1][dev]) {
          cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SS::bytes);
          if (err != cudaSuccess) return err;
          attr_done[1][dev] = true;
        }
        k<<<gx, NT, SS::bytes, s>>>(prm);
      }
    } else {
      using SS = StagedShape<T, NP, NQ, VT, false>;
      if constexpr (!SS::fits) {
        return cudaErrorInvalidConfiguration;
      } else {
        auto k = fe_local_staged_kernel<T, NP, NQ, VT, false, NT, VPT>;
        if (!attr_done[0][dev]) {
          cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SS::bytes);
          if (err != cudaSuccess) return err;
          attr_done[0][dev] = true;
        }
        k<<<gx, NT, SS::bytes, s>>>(prm);
      }
    }
    return cudaGetLastError();
  }
}

template <typename T, typename TS, int NP, int NQ, int VT, int NT, int VPT, int MINB>
cudaError_t launch_lean_cfg(const Ctx& c, const LocalParams<T, TS>& prm, cudaStream_t s) {
  if constexpr (!std::is_same<T, TS>::value) {
    return cudaErrorInvalidConfiguration;   // the reduction scatter needs T == storage type
  } else {
    if (prm.n_cells == 0) return cudaSuccess;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device);
    static bool attr_done[2][64] = {};
    const int dev = c.device & 63;
    if (c.cplx) {
      using LS = LeanShape<T, NP, NQ, VT, true>;
      if constexpr (!LS::fits) {
        return cudaErrorInvalidConfiguration;
      } else {
        auto k = fe_local_lean_kernel<T, NP, NQ, VT, true, NT, VPT, MINB>;
        if (!attr_done[1][dev]) {
          cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LS::bytes);
          if (err != cudaSuccess) return err;
          attr_done[1][dev] = true;
        }
        const int gx = prm.n_cells < MINB * (sms > 0 ? sms : 152) * 8 ? prm.n_cells : MINB * (sms > 0 ? sms : 152) * 8;
        k<<<gx, NT, LS::bytes, s>>>(prm);
      }
    } else {
      using LS = LeanShape<T, NP, NQ, VT, false>;
      if constexpr (!LS::fits) {
        return cudaErrorInvalidConfiguration;
      } else {
        auto k = fe_local_lean_kernel<T, NP, NQ, VT, false, NT, VPT, MINB>;
        if (!attr_done[0][dev]) {
          cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LS::bytes);
          if (err != cudaSuccess) return err;
          attr_done[0][dev] = true;
        }
        const int gx = prm.n_cells < MINB * (sms > 0 ? sms : 152) * 8 ? prm.n_cells : MINB * (sms > 0 ? sms : 152) * 8;
        k<<<gx, NT, LS::bytes, s>>>(prm);
      }
    }
    return cudaGetLastError();
  }
}

template <typename T, typename TS>
__host__ __forceinline__ int cfg_for(const Ctx& c) {
  if (std::is_same<T, double>::value) return c.cfg64;
  if (std::is_same<T, float>::value) return c.cfg32;
  return c.cfgE;
}

template <typename T, typename TS, int P, int NQX>
cudaError_t launch_local_deg(const Ctx& c, const LocalParams<T, TS>& prm, cudaStream_t s) {
  constexpr int NP = P + 1, NQ = P + 1 + NQX;
  constexpr int V0 = cfg_vt<NQ>(0), V1 = cfg_vt<NQ>(1), V2 = cfg_vt<NQ>(2);
  switch (cfg_for<T, TS>(c)) {
    case 1: return launch_local_cfg<T, TS, NP, NQ, V1, cfg_nt(V1, NQ)>(c, prm, s);
    case 2: return launch_local_cfg<T, TS, NP, NQ, V2, cfg_nt(V2, NQ)>(c, prm, s);
    case 3: return launch_staged_cfg<T, TS, NP, NQ, V0, cfg_nt(V0, NQ)>(c, prm, s);
    case 4: return launch_staged_cfg<T, TS, NP, NQ, V1, cfg_nt(V1, NQ)>(c, prm, s);
    case 5: return launch_staged_cfg<T, TS, NP, NQ, V1, cfg_nt(V1 / 2, NQ), 2>(c, prm, s);
    case 6: return launch_staged_cfg<T, TS, NP, NQ, V1, cfg_nt(V1 / 4, NQ), 4>(c, prm, s);
    case 7: return launch_lean_cfg<T, TS, NP, NQ, V1, cfg_nt(V1 / 2, NQ), 2, 2>(c, prm, s);
    case 8: return launch_lean_cfg<T, TS, NP, NQ, V1, cfg_nt(V1 / 4, NQ), 4, 2>(c, prm, s);
    case 9: return launch_lean_cfg<T, TS, NP, NQ, V0, cfg_nt(V0 / 2, NQ), 2, 3>(c, prm, s);
    default: return launch_local_cfg<T, TS, NP, NQ, V0, cfg_nt(V0, NQ)>(c, prm, s);
  }
}

}  // namespace feks
