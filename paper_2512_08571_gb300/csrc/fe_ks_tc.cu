// Tensor-core cell kernel (FE_KS_BF16, FE_KS_F16): the 1D contractions of
// Algorithm 2 as warp-level BF16 or FP16 MMAs with FP32 accumulation, the
// quadrature-point step, nonlocal expansion and scatter in FP32.  FP16 has 8x
// the precision of BF16 but a narrow range, so every column of a gathered cell
// tile is scaled by its own power of two (its largest entry to below 1/16;
// the re/im columns of a complex vector share one) and the result unscaled at
// the scatter: each column is an independent right-hand side of a linear
// chain, and the scaling is exact.  One scale per tile would not do: columns
// of very different size (converged and unconverged vectors inside the
// eigensolver) would push the small ones into FP16's subnormals.
//
// Paper: Algorithm 2 (cell-level evaluation, eq. ggaReal / eq. ggaCmplx) called
// from Algorithm 1 (extraction Q C P X, F Delta T3, assembly Q^T).  The
// sum-factorised chain is regrouped so that every tensor-product factor is a
// contraction of ONE index with a small dense 1D matrix:
//   Y0  = N_z N_y N_x X,  Y1_x = N_z N_y D_x X,  Y1_y = N_z D_y N_x X,
//   Y1_z = D_z N_y N_x X  with D = D~ N (the Gauss-point derivative of the
//   nodal basis; D~ N = D exactly for n_q = n_p, Sec. 3.2),
//   Y = N_x^T [N_y^T (N_z^T Z + D_z^T W_z) + D_y^T N_z^T W_y]
//     + D_x^T N_y^T N_z^T W_x.
// One sweep contracts a line of n values for 16 lines at a time (8 vector
// columns x 2 lines): A = data (16 lines x K), B = the 1D matrix (K x n_q),
// K = 16 (n = 9) or 8 (n <= 8), FP32 accumulators.  Between sweeps the lines
// are re-formed through shared memory with ldmatrix / stmatrix (.trans), so
// every array stays [point][8 columns] with the column index fastest; the last
// forward sweep, the quadrature-point step and the first transposed sweep are
// chained in registers (an accumulator fragment of one MMA is the A fragment
// of the next along the same index).
//
// The 1D sweeps are tiny (9 x 9 matrices): the legacy warp-level MMA keeps
// the chain in registers without a tensor-memory round trip per sweep, and
// the kernel's time goes to shared-memory transposes and the FP32 pointwise
// work, not to tensor issue.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fe_ks_internal.h"

namespace feks {

// Kernel operands (one colour of cells; FP32 storage).
struct TcParams {
  const float* X;
  float* Y;
  int64_t ld;
  int ncols;
  const int* cell_dofs;
  const int* cells;
  int n_cells;
  const float* coef;       // [E][ncoef][n^3]
  int ncoef;
  int gga;
  const float* dscale;     // D^{-1/2} or nullptr
  const int* cell_pair_ptr;
  const int* cell_pairs;
  const int* pair_atom;
  const float* F;          // [pair][n_proj][n^3] (complex: x2 interleaved)
  const float* Q;          // [atom][n_proj][ld], scaled by Delta
  int n_proj;
  float alpha;
  const uint32_t* frag;    // B fragments [4 ops][2 tiles][32 lanes][2]
  const uint2* fpack;      // F as BF16 / FP16 B fragments [pair][row tile][half][tile][K step][32 lanes]
  const uint32_t* frag_lo; // split precision: BF16 remainders of frag
  const uint2* fpack_lo;   // split precision: BF16 remainders of fpack
};

namespace tc {

// Shared-memory geometry for n = n_p = n_q points per direction.  Point
// (a, b, c) of any stage sits at a + SY b + SZ c with odd SY and SZ, so that
// the 8 rows (16 bytes each) of every ldmatrix / stmatrix phase fall in 8
// different 16-byte bank groups for all three sweep directions.
template <int N, bool CPLX, bool SPLIT = false>
struct Geom {
  static constexpr int SY = (N & 1) ? N : N + 1;
  static constexpr int SZ = (N & 1) ? N * N : N * (N + 1) + 1;
  static constexpr int NPTS = (N - 1) * (1 + SY + SZ) + 1;
  static constexpr int N3 = N * N * N;
  static constexpr bool K16 = N > 8;
  static constexpr int NTL = K16 ? 2 : 1;        // 8-column output tiles per sweep
  static constexpr int G = N * N;                 // lines per column per sweep
  static constexpr int NMT = (G + 1) / 2;         // MMA row tiles (2 lines x 8 columns)
  static constexpr int NW = N == 9 ? 7 : N == 8 ? 8 : N == 7 ? 7 : N == 6 ? 6 : N == 5 ? 7 : 4;
  static constexpr int NT = 32 * NW;
  static constexpr int NC = CPLX ? 14 : 12;       // coefficient floats per point (padded)
  // byte offsets: arrays 0-2 (BF16 / FP16 data), and for the split precision
  // their low parts 3-5 (array k's twin at + LO)
  static constexpr int ARR = NPTS * 16;
  static constexpr int NARR = SPLIT ? 6 : 3;
  static constexpr int LO = 3 * ARR;
  static constexpr int OFF_ZERO = NARR * ARR;
  static constexpr int OFF_TRASH = OFF_ZERO + 16;
  static constexpr int OFF_COEF = OFF_TRASH + 32 * 16;
  static constexpr int OFF_DOFS = OFF_COEF + NPTS * NC * 4;
  // FP32 cell result [node][SST] (8 columns, padded to 12 floats so the
  // fragment-order writes and the row reads are both conflict-free)
  static constexpr int SST = 12;
  static constexpr int OFF_STAGE = (OFF_DOFS + N3 * 4 + 15) / 16 * 16;
  // FP16 column scaling: per-warp column maxima [NW][8] and the unscale factors [8]
  static constexpr int OFF_RED = OFF_STAGE + N3 * SST * 4;
  static constexpr int OFF_UNSCALE = OFF_RED + 8 * 8 * 4;
  static constexpr int BYTES = OFF_UNSCALE + 8 * 4;
  // Two resident CTAs per SM.  (Three fit the shared memory at n = 9, but the
  // register cap that lets 21 warps share the SM's four 16K-register files
  // (80 per thread) made the kernel spill and measured no faster.)
  // The split precision doubles the data arrays and the live fragments: one CTA.
  static constexpr int MINB = SPLIT ? 1 : 2;
  static_assert(ARR % 16 == 0 && OFF_COEF % 16 == 0 && OFF_DOFS % 4 == 0 && OFF_STAGE % 16 == 0, "alignment");
  static_assert(MINB * (BYTES + 1024) <= 233472, "MINB CTAs per SM must fit");
  static_assert((NC * 4) % 16 == 0 || (NC * 4) % 8 == 0, "coefficient loads need 8-byte point stride");

  // point index of line `grp` (the two untouched coordinates) at position k
  // along the swept direction DIM (0 = x, 1 = y, 2 = z)
  template <int DIM>
  __device__ static __forceinline__ int pt(int grp, int k) {
    const int o1 = grp % N, o2 = grp / N;
    if constexpr (DIM == 0) return k + SY * o1 + SZ * o2;
    if constexpr (DIM == 1) return o1 + SY * k + SZ * o2;
    return o1 + SY * o2 + SZ * k;
  }
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ uint32_t pack_f16(float lo, float hi) {
  __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// two values rounded to the kernel's 16-bit type, packed (lower index low)
template <bool F16>
__device__ __forceinline__ uint32_t pack16(float lo, float hi) {
  if constexpr (F16)
    return pack_f16(lo, hi);
  else
    return pack_bf16(lo, hi);
}

template <bool K16>
__device__ __forceinline__ void ldsm(uint32_t addr, uint32_t (&r)[4]) {
  if constexpr (K16) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr)
                 : "memory");
  } else {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(addr)
                 : "memory");
    r[2] = r[3] = 0u;
  }
}

template <int NTL>
__device__ __forceinline__ void stsm(uint32_t addr, const uint32_t (&r)[4]) {
  if constexpr (NTL == 2)
    asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1,%2,%3,%4};\n" ::"r"(addr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3])
                 : "memory");
  else
    asm volatile("stmatrix.sync.aligned.m8n8.x2.trans.shared.b16 [%0], {%1,%2};\n" ::"r"(addr), "r"(r[0]), "r"(r[1])
                 : "memory");
}

// d += a * b for one 16 x 8 output tile (BF16 or FP16 operands, FP32 accumulators)
template <bool K16, bool F16 = false>
__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  if constexpr (K16 && F16)
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  else if constexpr (K16)
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  else if constexpr (F16)
    asm("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(b[0]));
  else
    asm("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(b[0]));
}

// d = a * b (zero accumulator input)
template <bool K16, bool F16 = false>
__device__ __forceinline__ void mma0(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  const float z = 0.f;
  if constexpr (K16 && F16)
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%10,%10,%10};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "f"(z));
  else if constexpr (K16)
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%10,%10,%10};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "f"(z));
  else if constexpr (F16)
    asm("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%7,%7,%7,%7};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(b[0]), "f"(z));
  else
    asm("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%7,%7,%7,%7};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(b[0]), "f"(z));
}

// Accumulator tiles -> 16-bit fragment: the A operand of an MMA contracting
// the same index, and the register order stmatrix expects.
template <int NTL, bool F16 = false>
__device__ __forceinline__ void to_frag(const float (&d)[NTL][4], uint32_t (&a)[4]) {
  a[0] = pack16<F16>(d[0][0], d[0][1]);
  a[1] = pack16<F16>(d[0][2], d[0][3]);
  if constexpr (NTL == 2) {
    a[2] = pack16<F16>(d[1][0], d[1][1]);
    a[3] = pack16<F16>(d[1][2], d[1][3]);
  } else {
    a[2] = a[3] = 0u;
  }
}

template <int NTL>
__device__ __forceinline__ void zero(float (&d)[NTL][4]) {
#pragma unroll
  for (int j = 0; j < NTL; ++j) d[j][0] = d[j][1] = d[j][2] = d[j][3] = 0.f;
}

// Split precision (FE_KS_BF16X2): an operand x is held as hi = bf16(x) and
// lo = bf16(x - hi); a product a b becomes a_hi b_hi + a_hi b_lo + a_lo b_hi on
// the tensor cores (the a_lo b_lo term, about 2^-18 of the product, is
// dropped), all into the same FP32 accumulator.  With SPLIT = false these
// reduce to the single 16-bit product and the lo arguments are not read.
template <bool K16, bool F16, bool SPLIT>
__device__ __forceinline__ void mmaZ(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&al)[4],
                                     const uint32_t (&b)[2], const uint32_t (&bl)[2]) {
  mma0<K16, F16>(d, a, b);
  if constexpr (SPLIT) {
    mma<K16, F16>(d, a, bl);
    mma<K16, F16>(d, al, b);
  }
}

template <bool K16, bool F16, bool SPLIT>
__device__ __forceinline__ void mmaA(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&al)[4],
                                     const uint32_t (&b)[2], const uint32_t (&bl)[2]) {
  mma<K16, F16>(d, a, b);
  if constexpr (SPLIT) {
    mma<K16, F16>(d, a, bl);
    mma<K16, F16>(d, al, b);
  }
}

// accumulator tiles -> hi fragment (and, split, the lo fragment of the remainders)
template <int NTL, bool F16, bool SPLIT>
__device__ __forceinline__ void to_frag2(const float (&d)[NTL][4], uint32_t (&a)[4], uint32_t (&al)[4]) {
  to_frag<NTL, F16>(d, a);
  if constexpr (SPLIT) {
    float r[NTL][4];
#pragma unroll
    for (int j = 0; j < NTL; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) r[j][q] = d[j][q] - __bfloat162float(__float2bfloat16_rn(d[j][q]));
    to_frag<NTL, false>(r, al);
  }
}

// two values -> packed hi pair and (split) packed lo pair
template <bool F16, bool SPLIT>
__device__ __forceinline__ void pack2(float x, float y, uint32_t& h, uint32_t& l) {
  h = pack16<F16>(x, y);
  if constexpr (SPLIT)
    l = pack_bf16(x - __bfloat162float(__float2bfloat16_rn(x)), y - __bfloat162float(__float2bfloat16_rn(y)));
  else
    l = 0u;
}

// Byte offset of this lane's row for ldmatrix / stmatrix on row tile
// (g0, g0 + 1) along direction DIM, or -1 past the line's end: lane l serves
// matrix l / 8 (bit 0: line g0 or g0 + 1; bit 1: k + 8) and row l % 8 of it.
template <int N, bool CPLX, int DIM>
__device__ __forceinline__ int row_off(int g0, int lane) {
  using Gm = Geom<N, CPLX>;
  const int grp = g0 + ((lane >> 3) & 1);
  const int k = (lane & 7) + ((lane & 16) ? 8 : 0);
  if (grp >= Gm::G || k >= N) return -1;
  return 16 * Gm::template pt<DIM>(grp, k);
}

__device__ __forceinline__ uint32_t at(uint32_t arr, int off, uint32_t spare) {
  return off >= 0 ? arr + (uint32_t)off : spare;
}

// ldmatrix / stmatrix of a row tile of array `arr` and, split, of its low twin at arr + lo
template <bool K16, bool SPLIT>
__device__ __forceinline__ void ldsm2(uint32_t arr, uint32_t lo, int off, uint32_t zrow, uint32_t (&a)[4],
                                      uint32_t (&al)[4]) {
  ldsm<K16>(at(arr, off, zrow), a);
  if constexpr (SPLIT) ldsm<K16>(at(arr + lo, off, zrow), al);
}

template <int NTL, bool SPLIT>
__device__ __forceinline__ void stsm2(uint32_t arr, uint32_t lo, int off, uint32_t trash, const uint32_t (&o)[4],
                                      const uint32_t (&ol)[4]) {
  stsm<NTL>(at(arr, off, trash), o);
  if constexpr (SPLIT) stsm<NTL>(at(arr + lo, off, trash), ol);
}

// Power of two s with s * mx < 1/16 (s = 1 for mx = 0), from the exponent bits
// of mx: mx < 2^(E - 126) for biased exponent E, so s = 2^(122 - E).
__device__ __forceinline__ float tile_scale(float mx) {
  if (!(mx > 0.f)) return 1.f;
  int e = (int)((__float_as_uint(mx) >> 23) & 0xFFu);
  e = e < 1 ? 1 : (e > 248 ? 248 : e);
  return __uint_as_float((uint32_t)(249 - e) << 23);
}

// Assembly Y += alpha D^{-1/2} Q^T Y^(e) of the staged FP32 cell result for
// columns [c0, c0 + 8): one node per thread, two 16-byte reductions per node
// when the rows are 16-byte aligned.  Colour-exclusive launches: no other
// cell of the launch touches the same DoF rows.
template <int N, bool CPLX, bool F16>
__device__ __forceinline__ void scatter_stage(const TcParams& p, const float* stage, const int* sd, int c0, bool vecy,
                                              const float* unscale) {
  using Gm = Geom<N, CPLX>;
  const bool fullv = vecy && c0 + 8 <= p.ncols;
  float4 ua = make_float4(1.f, 1.f, 1.f, 1.f), ub = ua;   // per-column unscale (FP16)
  if constexpr (F16) {
    ua = *reinterpret_cast<const float4*>(unscale);
    ub = *reinterpret_cast<const float4*>(unscale + 4);
  }
  for (int node = threadIdx.x; node < Gm::N3; node += Gm::NT) {
    const float* sp = stage + node * Gm::SST;
    float4 a = *reinterpret_cast<const float4*>(sp);
    float4 b = *reinterpret_cast<const float4*>(sp + 4);
    const int d = sd[node];
    const float sc = p.dscale ? p.alpha * __ldg(p.dscale + d) : p.alpha;
    a.x *= sc * ua.x, a.y *= sc * ua.y, a.z *= sc * ua.z, a.w *= sc * ua.w;
    b.x *= sc * ub.x, b.y *= sc * ub.y, b.z *= sc * ub.z, b.w *= sc * ub.w;
    float* yp = p.Y + (int64_t)d * p.ld + c0;
    if (fullv) {
      atomicAdd(reinterpret_cast<float4*>(yp), a);
      atomicAdd(reinterpret_cast<float4*>(yp) + 1, b);
    } else {
      const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (c0 + c < p.ncols) atomicAdd(yp + c, v[c]);
    }
  }
}

template <int N, bool CPLX, bool F16, bool SPLIT>
__global__ void __launch_bounds__(Geom<N, CPLX, SPLIT>::NT, Geom<N, CPLX, SPLIT>::MINB)
    fe_tc_kernel(const __grid_constant__ TcParams p) {
  using Gm = Geom<N, CPLX, SPLIT>;
  constexpr bool K16 = Gm::K16;
  constexpr int NTL = Gm::NTL, NT = Gm::NT, NW = Gm::NW, N3 = Gm::N3, NC = Gm::NC, NMT = Gm::NMT;
  constexpr int SY = Gm::SY, SZ = Gm::SZ;
  constexpr int S = CPLX ? 2 : 1;   // K steps of the expansion (F real part, F imaginary part)
  extern __shared__ __align__(16) unsigned char smem[];
  float* cf = reinterpret_cast<float*>(smem + Gm::OFF_COEF);
  int* sd = reinterpret_cast<int*>(smem + Gm::OFF_DOFS);
  float* stage = reinterpret_cast<float*>(smem + Gm::OFF_STAGE);
  const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t A0 = s0, A1 = s0 + Gm::ARR, A2 = s0 + 2 * Gm::ARR;
  constexpr uint32_t LO = Gm::LO;   // byte distance from an array to its low twin (split precision)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2, tig = lane & 3;   // accumulator row (column v) and column-pair index
  const uint32_t zero_row = s0 + Gm::OFF_ZERO;
  const uint32_t trash = s0 + Gm::OFF_TRASH + 16u * lane;
  if (tid < 4) reinterpret_cast<float*>(smem + Gm::OFF_ZERO)[tid] = 0.f;

  // B fragments of N^T-as-B (forward N), D (forward), N and D (transposed sweeps)
  uint32_t bN[NTL][2], bD[NTL][2], bNt[NTL][2], bDt[NTL][2];
  uint32_t bNl[NTL][2], bDl[NTL][2], bNtl[NTL][2], bDtl[NTL][2];   // split: their BF16 remainders
#pragma unroll
  for (int j = 0; j < NTL; ++j)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      bN[j][r] = p.frag[((0 * 2 + j) * 32 + lane) * 2 + r];
      bD[j][r] = p.frag[((1 * 2 + j) * 32 + lane) * 2 + r];
      bNt[j][r] = p.frag[((2 * 2 + j) * 32 + lane) * 2 + r];
      bDt[j][r] = p.frag[((3 * 2 + j) * 32 + lane) * 2 + r];
      if constexpr (SPLIT) {
        bNl[j][r] = p.frag_lo[((0 * 2 + j) * 32 + lane) * 2 + r];
        bDl[j][r] = p.frag_lo[((1 * 2 + j) * 32 + lane) * 2 + r];
        bNtl[j][r] = p.frag_lo[((2 * 2 + j) * 32 + lane) * 2 + r];
        bDtl[j][r] = p.frag_lo[((3 * 2 + j) * 32 + lane) * 2 + r];
      } else {
        bNl[j][r] = bDl[j][r] = bNtl[j][r] = bDtl[j][r] = 0u;
      }
    }
  const int ntiles = (p.ncols + 7) / 8;
  const bool vec = (p.ld % 4 == 0) && (((uintptr_t)p.X & 15) == 0);
  const bool vecy = (p.ld % 4 == 0) && (((uintptr_t)p.Y & 15) == 0);

  for (int ci = blockIdx.x; ci < p.n_cells; ci += gridDim.x) {
    const int e = p.cells[ci];
    __syncthreads();   // the previous cell's scatter has finished with sd
    // stage the DoF list and the coefficients, point-major [pt][NC]
    for (int w = tid; w < N3; w += NT) sd[w] = p.cell_dofs[(int64_t)e * N3 + w];
    {
      const float* gc = p.coef + (int64_t)e * p.ncoef * N3;
      const int total = p.ncoef * N3;
#pragma unroll 4
      for (int w = tid; w < total; w += NT) {
        const int c = w / N3, q = w - c * N3;
        const int qx = q % N, qy = (q / N) % N, qz = q / (N * N);
        cf[(qx + SY * qy + SZ * qz) * NC + c] = gc[w];
      }
    }
    const int pb = p.cell_pair_ptr ? p.cell_pair_ptr[e] : 0;
    const int pe = p.cell_pair_ptr ? p.cell_pair_ptr[e + 1] : 0;
    __syncthreads();
    int prev0 = -1;          // columns of the staged result still to be assembled
    float* unscale = reinterpret_cast<float*>(smem + Gm::OFF_UNSCALE);   // of the staged tile
    for (int t = blockIdx.y; t < ntiles; t += gridDim.y) {
      const int col0 = 8 * t;
      const int col = col0 + gq;
      const bool full = vec && col0 + 8 <= p.ncols;
      float tscale = 1.f;   // power-of-two scale of this thread's column gq (FP16 only)
      // (1) extraction Q C P X (Algorithm 1): rows of X -> 16-bit array 2 [node][8]
      //     (array 2 is not read by the previous tile's last sweep); the loads
      //     are in flight while the previous tile's staged result is assembled
      {
        constexpr int GPT = (N3 + NT - 1) / NT;
        float4 xa[GPT], xb[GPT];
        float sc[GPT];
#pragma unroll
        for (int r = 0; r < GPT; ++r) {
          const int node = tid + r * NT;
          xa[r] = xb[r] = make_float4(0.f, 0.f, 0.f, 0.f);
          sc[r] = 1.f;
          if (node < N3) {
            const int d = sd[node];
            const float* xr = p.X + (int64_t)d * p.ld + col0;
            if (full) {
              xa[r] = __ldg(reinterpret_cast<const float4*>(xr));
              xb[r] = __ldg(reinterpret_cast<const float4*>(xr) + 1);
            } else {
              float v[8];
#pragma unroll
              for (int c = 0; c < 8; ++c) v[c] = (col0 + c < p.ncols) ? __ldg(xr + c) : 0.f;
              xa[r] = make_float4(v[0], v[1], v[2], v[3]);
              xb[r] = make_float4(v[4], v[5], v[6], v[7]);
            }
            if (p.dscale) sc[r] = __ldg(p.dscale + d);
          }
        }
        if (prev0 >= 0) scatter_stage<N, CPLX, F16>(p, stage, sd, prev0, vecy, unscale);
        // FP16: scale every column of the tile by a power of two so that its
        // largest entry is below 1/16 (exact; undone at the scatter)
        float cs[8] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f};
        if constexpr (F16) {
          float cm[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int r = 0; r < GPT; ++r) {
            const float s = fabsf(sc[r]);
            cm[0] = fmaxf(cm[0], fabsf(xa[r].x) * s), cm[1] = fmaxf(cm[1], fabsf(xa[r].y) * s);
            cm[2] = fmaxf(cm[2], fabsf(xa[r].z) * s), cm[3] = fmaxf(cm[3], fabsf(xa[r].w) * s);
            cm[4] = fmaxf(cm[4], fabsf(xb[r].x) * s), cm[5] = fmaxf(cm[5], fabsf(xb[r].y) * s);
            cm[6] = fmaxf(cm[6], fabsf(xb[r].z) * s), cm[7] = fmaxf(cm[7], fabsf(xb[r].w) * s);
          }
#pragma unroll
          for (int c = 0; c < 8; ++c)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cm[c] = fmaxf(cm[c], __shfl_xor_sync(0xffffffffu, cm[c], o));
          float* wmax = reinterpret_cast<float*>(smem + Gm::OFF_RED);   // [NW][8]
          if (lane < 8) {
            float v = cm[0];
#pragma unroll
            for (int c = 1; c < 8; ++c) v = lane == c ? cm[c] : v;
            wmax[warp * 8 + lane] = v;
          }
          __syncthreads();
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            float m = 0.f;
            for (int w = 0; w < NW; ++w) m = fmaxf(m, wmax[w * 8 + c]);
            cm[c] = m;
          }
          // a complex vector's re/im columns share one scale (the -iK term mixes them)
          if constexpr (CPLX)
#pragma unroll
            for (int c = 0; c < 8; c += 2) cm[c] = cm[c + 1] = fmaxf(cm[c], cm[c + 1]);
#pragma unroll
          for (int c = 0; c < 8; ++c) cs[c] = tile_scale(cm[c]);
          float m = cm[0];
#pragma unroll
          for (int c = 1; c < 8; ++c) m = gq == c ? cm[c] : m;
          tscale = tile_scale(m);
          if (tid < 8) {   // the scatter of this tile undoes the scale (read after later barriers)
            float v = cs[0];
#pragma unroll
            for (int c = 1; c < 8; ++c) v = tid == c ? cs[c] : v;
            unscale[tid] = 1.f / v;   // exact: a power of two
          }
        }
#pragma unroll
        for (int r = 0; r < GPT; ++r) {
          const int node = tid + r * NT;
          if (node < N3) {
            const int i = node % N, j = (node / N) % N, k = node / (N * N);
            const float s = sc[r];
            uint4 u, ul;
            pack2<F16, SPLIT>(xa[r].x * s * cs[0], xa[r].y * s * cs[1], u.x, ul.x);
            pack2<F16, SPLIT>(xa[r].z * s * cs[2], xa[r].w * s * cs[3], u.y, ul.y);
            pack2<F16, SPLIT>(xb[r].x * s * cs[4], xb[r].y * s * cs[5], u.z, ul.z);
            pack2<F16, SPLIT>(xb[r].z * s * cs[6], xb[r].w * s * cs[7], u.w, ul.w);
            *reinterpret_cast<uint4*>(smem + 2 * Gm::ARR + 16 * (i + SY * j + SZ * k)) = u;
            if constexpr (SPLIT) *reinterpret_cast<uint4*>(smem + 2 * Gm::ARR + LO + 16 * (i + SY * j + SZ * k)) = ul;
          }
        }
      }
      __syncthreads();
      // Every sweep below reads and writes the same points (the two lines of its
      // row tile, all positions along the swept direction), so the arrays are
      // updated in place; ldmatrix results are in registers before the stores.
      // (2) x sweep: U = N_x X -> 0, U' = D_x X -> 1.  Each warp takes BX row
      //     tiles at a time so that 4 BX independent MMAs are in flight (the
      //     warp-level MMA has a latency of ~100 cycles on this part).
      {
        constexpr int BX = SPLIT ? 2 : 3;
#pragma unroll 1
        for (int mt0 = warp; mt0 < NMT; mt0 += NW * BX) {
          int off[BX];
          uint32_t a[BX][4], al[BX][4];
          float u[BX][NTL][4], ud[BX][NTL][4];
#pragma unroll
          for (int b = 0; b < BX; ++b) {
            const int mt = mt0 + b * NW;
            off[b] = mt < NMT ? row_off<N, CPLX, 0>(2 * mt, lane) : -1;
            ldsm2<K16, SPLIT>(A2, LO, off[b], zero_row, a[b], al[b]);
          }
#pragma unroll
          for (int b = 0; b < BX; ++b)
#pragma unroll
            for (int j = 0; j < NTL; ++j) {
              mmaZ<K16, F16, SPLIT>(u[b][j], a[b], al[b], bN[j], bNl[j]);
              mmaZ<K16, F16, SPLIT>(ud[b][j], a[b], al[b], bD[j], bDl[j]);
            }
#pragma unroll
          for (int b = 0; b < BX; ++b) {
            uint32_t o[4], ol[4];
            to_frag2<NTL, F16, SPLIT>(u[b], o, ol);
            stsm2<NTL, SPLIT>(A0, LO, off[b], trash, o, ol);
            to_frag2<NTL, F16, SPLIT>(ud[b], o, ol);
            stsm2<NTL, SPLIT>(A1, LO, off[b], trash, o, ol);
          }
        }
      }
      __syncthreads();
      // (3) y sweep: N_y U -> 0, D_y U -> 1, N_y U' -> 2 (BY row tiles per warp at a time)
      {
        constexpr int BY = SPLIT ? 1 : 2;
#pragma unroll 1
        for (int mt0 = warp; mt0 < NMT; mt0 += NW * BY) {
          int off[BY];
          uint32_t a[BY][4], b2[BY][4], al[BY][4], b2l[BY][4];
          float t0[BY][NTL][4], t1[BY][NTL][4], t2[BY][NTL][4];
#pragma unroll
          for (int b = 0; b < BY; ++b) {
            const int mt = mt0 + b * NW;
            off[b] = mt < NMT ? row_off<N, CPLX, 1>(2 * mt, lane) : -1;
            ldsm2<K16, SPLIT>(A0, LO, off[b], zero_row, a[b], al[b]);
            ldsm2<K16, SPLIT>(A1, LO, off[b], zero_row, b2[b], b2l[b]);
          }
#pragma unroll
          for (int b = 0; b < BY; ++b)
#pragma unroll
            for (int j = 0; j < NTL; ++j) {
              mmaZ<K16, F16, SPLIT>(t0[b][j], a[b], al[b], bN[j], bNl[j]);
              mmaZ<K16, F16, SPLIT>(t1[b][j], a[b], al[b], bD[j], bDl[j]);
              mmaZ<K16, F16, SPLIT>(t2[b][j], b2[b], b2l[b], bN[j], bNl[j]);
            }
#pragma unroll
          for (int b = 0; b < BY; ++b) {
            uint32_t o[4], ol[4];
            to_frag2<NTL, F16, SPLIT>(t0[b], o, ol);
            stsm2<NTL, SPLIT>(A0, LO, off[b], trash, o, ol);
            to_frag2<NTL, F16, SPLIT>(t1[b], o, ol);
            stsm2<NTL, SPLIT>(A1, LO, off[b], trash, o, ol);
            to_frag2<NTL, F16, SPLIT>(t2[b], o, ol);
            stsm2<NTL, SPLIT>(A2, LO, off[b], trash, o, ol);
          }
        }
      }
      __syncthreads();
      // (4) z sweep -> Y0, Y1 at the quadrature points (registers), the
      //     quadrature-point step of Algorithm 2, and the transposed z sweep:
      //     N_z^T Z + D_z^T W_z -> 0, N_z^T W_y -> 1, N_z^T W_x -> 2
#pragma unroll 1
      for (int mt = warp; mt < NMT; mt += NW) {
        const int g0 = 2 * mt;
        const int off = row_off<N, CPLX, 2>(g0, lane);
        uint32_t a[4], b[4], c[4], al[4], bl[4], cl[4];
        ldsm2<K16, SPLIT>(A0, LO, off, zero_row, a, al);
        ldsm2<K16, SPLIT>(A1, LO, off, zero_row, b, bl);
        ldsm2<K16, SPLIT>(A2, LO, off, zero_row, c, cl);
        float u[NTL][4], gx[NTL][4], gy[NTL][4], gz[NTL][4];
#pragma unroll
        for (int j = 0; j < NTL; ++j) {
          mmaZ<K16, F16, SPLIT>(u[j], a, al, bN[j], bNl[j]);
          mmaZ<K16, F16, SPLIT>(gz[j], a, al, bD[j], bDl[j]);
          mmaZ<K16, F16, SPLIT>(gy[j], b, bl, bN[j], bNl[j]);
          mmaZ<K16, F16, SPLIT>(gx[j], c, cl, bN[j], bNl[j]);
        }
        // element (j, r): line g0 + (r >> 1), column v = gq, qz = 8 j + 2 tig + (r & 1);
        // the coefficients of a line start at cbase[r >> 1], qz adds SZ NC per step
        const float* cbase[2];
        bool lok[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int grp = g0 + h;
          lok[h] = grp < Gm::G;
          const int gc = lok[h] ? grp : 0;
          cbase[h] = cf + ((gc % N) + SY * (gc / N) + SZ * 2 * tig) * NC;
        }
#pragma unroll
        for (int j = 0; j < NTL; ++j)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int qz = 8 * j + 2 * tig + (r & 1);
            const bool ok = lok[r >> 1] && qz < N;
            float z = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f, kk = 0.f;
            const float uu = u[j][r], x = gx[j][r], y = gy[j][r], zz = gz[j][r];
            if (ok) {
              // slots: G00 G01 G02 G11 G12 G22 VL V0 V1 V2 (K0 K1 K2); the point
              // stride is 48 B (real, 16-byte loads) or 56 B (complex, 8-byte loads)
              const float* c0 = cbase[r >> 1] + (8 * j + (r & 1)) * SZ * NC;
              float G00, G01, G02, G11, G12, G22, VL, V0, V1, V2;
              if constexpr (NC % 4 == 0) {
                const float4 ga = *reinterpret_cast<const float4*>(c0);
                const float4 gb = *reinterpret_cast<const float4*>(c0 + 4);
                const float2 gc = *reinterpret_cast<const float2*>(c0 + 8);
                G00 = ga.x, G01 = ga.y, G02 = ga.z, G11 = ga.w;
                G12 = gb.x, G22 = gb.y, VL = gb.z, V0 = gb.w, V1 = gc.x, V2 = gc.y;
              } else {
                const float2 ga = *reinterpret_cast<const float2*>(c0);
                const float2 gb = *reinterpret_cast<const float2*>(c0 + 2);
                const float2 gc = *reinterpret_cast<const float2*>(c0 + 4);
                const float2 gd = *reinterpret_cast<const float2*>(c0 + 6);
                const float2 ge = *reinterpret_cast<const float2*>(c0 + 8);
                G00 = ga.x, G01 = ga.y, G02 = gb.x, G11 = gb.y;
                G12 = gc.x, G22 = gc.y, VL = gd.x, V0 = gd.y, V1 = ge.x, V2 = ge.y;
              }
              z = VL * uu;
              w0 = fmaf(G00, x, fmaf(G01, y, G02 * zz));
              w1 = fmaf(G01, x, fmaf(G11, y, G12 * zz));
              w2 = fmaf(G02, x, fmaf(G12, y, G22 * zz));
              if (p.gga) {
                z = fmaf(V0, x, fmaf(V1, y, fmaf(V2, zz, z)));
                w0 = fmaf(V0, uu, w0);
                w1 = fmaf(V1, uu, w1);
                w2 = fmaf(V2, uu, w2);
              }
              if constexpr (CPLX) {
                const float2 ka = *reinterpret_cast<const float2*>(c0 + 10);   // K0 K1
                const float k2 = c0[12];
                kk = fmaf(ka.x, x, fmaf(ka.y, y, k2 * zz));
              }
            }
            if constexpr (CPLX) {
              // -i (a + i b) = b - i a: the real column adds Im, the imaginary one subtracts Re
              const float kp = __shfl_xor_sync(0xffffffffu, kk, 4);
              if (ok) z += (gq & 1) ? -kp : kp;
            }
            u[j][r] = z;
            gx[j][r] = w0;
            gy[j][r] = w1;
            gz[j][r] = w2;
          }
        uint32_t fz[4], fx[4], fy[4], fw[4], o[4], fzl[4], fxl[4], fyl[4], fwl[4], ol[4];
        to_frag2<NTL, F16, SPLIT>(u, fz, fzl);
        to_frag2<NTL, F16, SPLIT>(gx, fx, fxl);
        to_frag2<NTL, F16, SPLIT>(gy, fy, fyl);
        to_frag2<NTL, F16, SPLIT>(gz, fw, fwl);
        float va[NTL][4], va2[NTL][4], vb[NTL][4], vc[NTL][4];
#pragma unroll
        for (int j = 0; j < NTL; ++j) {   // four independent accumulators
          mmaZ<K16, F16, SPLIT>(va[j], fz, fzl, bNt[j], bNtl[j]);
          mmaZ<K16, F16, SPLIT>(va2[j], fw, fwl, bDt[j], bDtl[j]);
          mmaZ<K16, F16, SPLIT>(vb[j], fy, fyl, bNt[j], bNtl[j]);
          mmaZ<K16, F16, SPLIT>(vc[j], fx, fxl, bNt[j], bNtl[j]);
        }
#pragma unroll
        for (int j = 0; j < NTL; ++j)
#pragma unroll
          for (int r = 0; r < 4; ++r) va[j][r] += va2[j][r];
        to_frag2<NTL, F16, SPLIT>(va, o, ol);
        stsm2<NTL, SPLIT>(A0, LO, off, trash, o, ol);
        to_frag2<NTL, F16, SPLIT>(vb, o, ol);
        stsm2<NTL, SPLIT>(A1, LO, off, trash, o, ol);
        to_frag2<NTL, F16, SPLIT>(vc, o, ol);
        stsm2<NTL, SPLIT>(A2, LO, off, trash, o, ol);
      }
      __syncthreads();
      // (5) transposed y sweep: N_y^T V_a + D_y^T V_b -> 0, N_y^T V_c -> 1
      //     (BR row tiles per warp at a time, independent accumulators)
      {
        constexpr int BR = SPLIT ? 1 : 2;
#pragma unroll 1
        for (int mt0 = warp; mt0 < NMT; mt0 += NW * BR) {
          int off[BR];
          uint32_t a[BR][4], b2[BR][4], c2[BR][4], al[BR][4], b2l[BR][4], c2l[BR][4];
          float sa[BR][NTL][4], sa2[BR][NTL][4], sb[BR][NTL][4];
#pragma unroll
          for (int b = 0; b < BR; ++b) {
            const int mt = mt0 + b * NW;
            off[b] = mt < NMT ? row_off<N, CPLX, 1>(2 * mt, lane) : -1;
            ldsm2<K16, SPLIT>(A0, LO, off[b], zero_row, a[b], al[b]);
            ldsm2<K16, SPLIT>(A1, LO, off[b], zero_row, b2[b], b2l[b]);
            ldsm2<K16, SPLIT>(A2, LO, off[b], zero_row, c2[b], c2l[b]);
          }
#pragma unroll
          for (int b = 0; b < BR; ++b)
#pragma unroll
            for (int j = 0; j < NTL; ++j) {
              mmaZ<K16, F16, SPLIT>(sa[b][j], a[b], al[b], bNt[j], bNtl[j]);
              mmaZ<K16, F16, SPLIT>(sa2[b][j], b2[b], b2l[b], bDt[j], bDtl[j]);
              mmaZ<K16, F16, SPLIT>(sb[b][j], c2[b], c2l[b], bNt[j], bNtl[j]);
            }
#pragma unroll
          for (int b = 0; b < BR; ++b) {
#pragma unroll
            for (int j = 0; j < NTL; ++j)
#pragma unroll
              for (int r = 0; r < 4; ++r) sa[b][j][r] += sa2[b][j][r];
            uint32_t o[4], ol[4];
            to_frag2<NTL, F16, SPLIT>(sa[b], o, ol);
            stsm2<NTL, SPLIT>(A0, LO, off[b], trash, o, ol);
            to_frag2<NTL, F16, SPLIT>(sb[b], o, ol);
            stsm2<NTL, SPLIT>(A1, LO, off[b], trash, o, ol);
          }
        }
      }
      __syncthreads();
      // (6) transposed x sweep, + F Delta P (nonlocal, as MMAs with the pair's
      //     pre-packed F fragments), assembly Y += alpha Q^T Y^(e)
#pragma unroll 1
      for (int mt = warp; mt < NMT; mt += NW) {
        const int g0 = 2 * mt;
        const int off = row_off<N, CPLX, 0>(g0, lane);
        uint32_t a[4], b[4], al[4], bl[4];
        ldsm2<K16, SPLIT>(A0, LO, off, zero_row, a, al);
        ldsm2<K16, SPLIT>(A1, LO, off, zero_row, b, bl);
        float y[NTL][4], y2[NTL][4], ye[2][NTL][4];
        zero(ye[0]);
        zero(ye[1]);
#pragma unroll
        for (int j = 0; j < NTL; ++j) {
          mmaZ<K16, F16, SPLIT>(y[j], a, al, bNt[j], bNtl[j]);
          mmaZ<K16, F16, SPLIT>(y2[j], b, bl, bDt[j], bDtl[j]);
        }
        // Y^(e)[(line, v)][i] += sum_b Q[a][b][v] F[pair][b][i + N line]: A = Q^T
        // (rows of one line only, the other half zero), B = the packed F block
        for (int pi = pb; pi < pe; ++pi) {   // uniform over the block
          const int pr = p.cell_pairs[pi];
          const float* Qa = p.Q + (int64_t)p.pair_atom[pr] * p.n_proj * p.ld;
          const bool act = col < p.ncols;
          uint32_t aq[S][2], aql[S][2];
#pragma unroll
          for (int kh = 0; kh < 2; ++kh) {
            const int b0 = 2 * tig + 8 * kh;
            float q[2][2];   // [beta offset][re, im]
#pragma unroll
            for (int o2 = 0; o2 < 2; ++o2) {
              const bool okb = act && b0 + o2 < p.n_proj;
              if constexpr (CPLX) {
                const float* qr = Qa + (int64_t)(b0 + o2) * p.ld + (col & ~1);
                q[o2][0] = okb ? __ldg(qr) * tscale : 0.f;
                q[o2][1] = okb ? __ldg(qr + 1) * tscale : 0.f;
              } else {
                q[o2][0] = okb ? __ldg(Qa + (int64_t)(b0 + o2) * p.ld + col) * tscale : 0.f;
                q[o2][1] = 0.f;
              }
            }
            if constexpr (CPLX) {
              // real column: Fr Qr - Fi Qi; imaginary column: Fr Qi + Fi Qr
              const bool im = gq & 1;
              pack2<F16, SPLIT>(im ? q[0][1] : q[0][0], im ? q[1][1] : q[1][0], aq[0][kh], aql[0][kh]);
              pack2<F16, SPLIT>(im ? q[0][0] : -q[0][1], im ? q[1][0] : -q[1][1], aq[S - 1][kh], aql[S - 1][kh]);
            } else {
              pack2<F16, SPLIT>(q[0][0], q[1][0], aq[0][kh], aql[0][kh]);
            }
          }
          const size_t fofs = ((size_t)pr * NMT + mt) * (2 * NTL * S * 32) + lane;
          const uint2* fp = p.fpack + fofs;
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < NTL; ++j)
#pragma unroll
              for (int st = 0; st < S; ++st) {
                const uint2 fb = __ldg(fp + ((h * NTL + j) * S + st) * 32);
                const uint32_t bb[2] = {fb.x, fb.y};
                uint32_t bbl[2] = {0u, 0u};
                if constexpr (SPLIT) {
                  const uint2 fl = __ldg(p.fpack_lo + fofs + ((h * NTL + j) * S + st) * 32);
                  bbl[0] = fl.x;
                  bbl[1] = fl.y;
                }
                uint32_t af[4], afl[4];
                af[0] = h == 0 ? aq[st][0] : 0u;
                af[1] = h == 1 ? aq[st][0] : 0u;
                af[2] = h == 0 ? aq[st][1] : 0u;
                af[3] = h == 1 ? aq[st][1] : 0u;
                afl[0] = h == 0 ? aql[st][0] : 0u;
                afl[1] = h == 1 ? aql[st][0] : 0u;
                afl[2] = h == 0 ? aql[st][1] : 0u;
                afl[3] = h == 1 ? aql[st][1] : 0u;
                mmaA<true, F16, SPLIT>(ye[h][j], af, afl, bb, bbl);
              }
        }
#pragma unroll
        for (int j = 0; j < NTL; ++j)
#pragma unroll
          for (int r = 0; r < 4; ++r) y[j][r] += y2[j][r] + (ye[0][j][r] + ye[1][j][r]);
        // the cell result, FP32, to the stage [node][column]
#pragma unroll
        for (int j = 0; j < NTL; ++j)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int grp = g0 + (r >> 1);
            const int i = 8 * j + 2 * tig + (r & 1);
            if (grp < Gm::G && i < N) stage[(i + N * grp) * Gm::SST + gq] = y[j][r];
          }
        __syncwarp();   // reconverge before the next row tile's ldmatrix
      }
      __syncthreads();   // the stage is complete; array 2 is free for the next extraction
      prev0 = col0;
    }
    if (prev0 >= 0) scatter_stage<N, CPLX, F16>(p, stage, sd, prev0, vecy, unscale);
  }
}

template <int N, bool CPLX, bool F16, bool SPLIT = false>
cudaError_t launch_tc_n(const TcParams& p, cudaStream_t s) {
  using Gm = Geom<N, CPLX, SPLIT>;
  if (p.n_cells == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t err = cudaFuncSetAttribute(fe_tc_kernel<N, CPLX, F16, SPLIT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, Gm::BYTES);
  if (err != cudaSuccess) return err;
  // ask for the largest shared-memory carveout so that MINB CTAs fit on an SM with room to spare
  err = cudaFuncSetAttribute(fe_tc_kernel<N, CPLX, F16, SPLIT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (err != cudaSuccess) return err;
  const int ntiles = (p.ncols + 7) / 8;
  // about eight resident waves of CTAs: split the column tiles of a cell over
  // gridDim.y CTAs when the colour has few cells
  const int want = 8 * Gm::MINB * (sms > 0 ? sms : 152);
  int gy = (want + p.n_cells - 1) / p.n_cells;
  gy = gy < 1 ? 1 : (gy > ntiles ? ntiles : gy);
  if (gy > 65535) gy = 65535;
  const int gx = p.n_cells < (1 << 30) ? p.n_cells : (1 << 30);
  fe_tc_kernel<N, CPLX, F16, SPLIT><<<dim3(gx, gy), Gm::NT, Gm::BYTES, s>>>(p);
  return cudaGetLastError();
}

}  // namespace tc

void build_tc_fpack(int n, bool cplx, int n_proj, int64_t n_pairs, const double* F, int kind, std::vector<uint2>& out) {
  const int G = n * n, NMT = (G + 1) / 2, NTL = n > 8 ? 2 : 1, S = cplx ? 2 : 1, np3 = n * n * n;
  out.assign((size_t)n_pairs * NMT * 2 * NTL * S * 32, make_uint2(0u, 0u));
  size_t w = 0;
  for (int64_t pr = 0; pr < n_pairs; ++pr)
    for (int mt = 0; mt < NMT; ++mt)
      for (int h = 0; h < 2; ++h)
        for (int j = 0; j < NTL; ++j)
          for (int st = 0; st < S; ++st)
            for (int lane = 0; lane < 32; ++lane, ++w) {
              const int g = 2 * mt + h, i = 8 * j + lane / 4, tig = lane % 4;
              auto B = [&](int k) -> double {   // B[k][i] = F_st[beta = k][node = i + n g]
                if (k >= n_proj || i >= n || g >= G) return 0.0;
                const size_t idx = ((size_t)pr * n_proj + k) * np3 + i + (size_t)n * g;
                return cplx ? F[2 * idx + st] : F[idx];
              };
              auto h = [&](double x) -> uint32_t {
                return kind == 1 ? f16_bits(x) : kind == 2 ? bf16_lo_bits(x) : bf16_bits(x);
              };
              out[w].x = h(B(2 * tig)) | (h(B(2 * tig + 1)) << 16);
              out[w].y = h(B(2 * tig + 8)) | (h(B(2 * tig + 9)) << 16);
            }
}

// Shared-memory bytes of the BF16 cell kernel for n points per direction
// (0 when n is unsupported).
size_t tc_smem_bytes(int n, bool cplx) {
  switch (n) {
#define FEKS_TC_CASE(NN) \
  case NN: return cplx ? tc::Geom<NN, true>::BYTES : tc::Geom<NN, false>::BYTES;
    FEKS_TC_CASE(2)
    FEKS_TC_CASE(3)
    FEKS_TC_CASE(4)
    FEKS_TC_CASE(5)
    FEKS_TC_CASE(6)
    FEKS_TC_CASE(7)
    FEKS_TC_CASE(8)
    FEKS_TC_CASE(9)
#undef FEKS_TC_CASE
    default: return 0;
  }
}

cudaError_t launch_tc(const Ctx& c, const LocalParams<float>& lp, cudaStream_t s, int tc) {
  const bool f16 = tc == 2, split = tc == 3;
  TcParams p{};
  p.X = lp.X;
  p.Y = lp.Y;
  p.ld = lp.ld;
  p.ncols = lp.ncols;
  p.cell_dofs = lp.cell_dofs;
  p.cells = lp.cells;
  p.n_cells = lp.n_cells;
  p.coef = lp.coef;
  p.ncoef = lp.ncoef;
  p.gga = lp.gga;
  p.dscale = lp.dscale;
  p.cell_pair_ptr = lp.cell_pair_ptr;
  p.cell_pairs = lp.cell_pairs;
  p.pair_atom = lp.pair_atom;
  p.F = lp.F;
  p.Q = lp.Q;
  p.n_proj = lp.n_proj;
  p.alpha = lp.alpha;
  p.frag = f16 ? c.tc_frag16 : c.tc_frag;
  p.fpack = f16 ? c.tc_fpack16 : c.tc_fpack;
  p.frag_lo = c.tc_frag_lo;
  p.fpack_lo = c.tc_fpack_lo;
  if (p.cell_pair_ptr && (!p.fpack || (split && !p.fpack_lo))) return cudaErrorInvalidValue;
  switch (c.np) {
#define FEKS_TC_LAUNCH(NN)                                                                                    \
  case NN:                                                                                                    \
    if (f16) return c.cplx ? tc::launch_tc_n<NN, true, true>(p, s) : tc::launch_tc_n<NN, false, true>(p, s);  \
    if (split)                                                                                                \
      return c.cplx ? tc::launch_tc_n<NN, true, false, true>(p, s) : tc::launch_tc_n<NN, false, false, true>(p, s); \
    return c.cplx ? tc::launch_tc_n<NN, true, false>(p, s) : tc::launch_tc_n<NN, false, false>(p, s);
    FEKS_TC_LAUNCH(2)
    FEKS_TC_LAUNCH(3)
    FEKS_TC_LAUNCH(4)
    FEKS_TC_LAUNCH(5)
    FEKS_TC_LAUNCH(6)
    FEKS_TC_LAUNCH(7)
    FEKS_TC_LAUNCH(8)
    FEKS_TC_LAUNCH(9)
#undef FEKS_TC_LAUNCH
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace feks
