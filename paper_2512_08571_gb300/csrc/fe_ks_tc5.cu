// Cell kernel on the 5th-generation tensor cores (tcgen05) for FE_KS_BF16 and
// FE_KS_F16, real operators, n_q = n_p = N.
//
// Paper: Algorithm 2 (cell-level evaluation, eq. ggaReal) called from
// Algorithm 1 (extraction Q C P X, expansion F Delta T3, assembly Q^T).  The
// sum-factorised chain is regrouped into four dense contractions per cell and
// tile of VT = 4 vectors, each a tcgen05.mma chain with FP32 accumulators in
// tensor memory and 16-bit operands in shared memory:
//   GEMM1 (plane, forward):   P_t[(v,c)][p'] = sum_p K_t[p][p'] X[(p,c)][v],
//         K_0 = N (x) N, K_1 = D (x) N, K_2 = N (x) D  over the in-plane node
//         index p = a + N b (the x and y sweeps of Algorithm 2 in one product;
//         D = D~ N is the Gauss-point derivative of the nodal basis);
//   GEMM2 (z sweep):  Y0 = N_z P_0, Y_x = N_z P_1, Y_y = N_z P_2, Y_z = D_z P_0;
//   FP32 quadrature-point step in registers (eq. ggaReal: G = J^-1 J^-T det J w,
//         V^L, V^G): Z = V^L Y0 + V^G.grad Y, W = G grad Y + V^G Y0;
//   GEMM3 (transposed z sweep):  T_0 = N_z^T Z + D_z^T W_z, T_1 = N_z^T W_x,
//         T_2 = N_z^T W_y;
//   GEMM4 (plane, transposed):   Y^(e)[(p,c)][v] = sum_t sum_p' K_t[p][p'] T_t[(v,p')][c].
// The plane products cost more multiplications than two 1D sweeps (81 x 81
// against 2 x 9 x 81 per line pair) but the tensor cores have that to spare;
// what they save is the relayouts between sweeps, which bound the warp-level
// kernel.  Every relayout here is a thread-per-row tensor-memory read
// (tcgen05.ld.32x32b, thread = accumulator row) followed by 16-byte shared
// stores: each operand is laid out K-major or MN-major (canonical no-swizzle
// core matrices of 8 rows x 16 bytes) so that the 8 values one thread holds
// are 16 contiguous bytes of the next operand.
//
// A CTA (512 threads, one per SM) runs two independent pipelines of 8 warps,
// each with its own X tile, operand buffer, mbarrier, named barrier, MMA-
// issuing thread and half of the tensor memory; they take alternate column
// tiles of the same cell, whose operators, coefficients, DoF list and
// projector pairs they share, so one pipeline's CUDA-core steps can run
// while the other waits on its products.
//
// Layouts (N = 9: NN = 81 in-plane nodes, 729 cell nodes, row r = t NN + p'):
//   KM   plane operators, rows r (256), 16-byte row per 8 p: r*16 + (p%8)*2 +
//        (p/8)*PGS; GEMM1 reads it K-major as A [(t,p')][p]; GEMM4 reads the same
//        bytes MN-major as A [p][(t,p')] (its transpose).
//   XS   the gathered X tile, B of GEMM1, MN-major [p][v + 4 c].
//   AB   A of GEMM2 [(v,p')][(t,c)] and of GEMM3 [(v,p')][(c',q)] (K-major, row
//        r2 = v + 4 p', 8-row groups 144 bytes apart), then B of GEMM4
//        [(t,p')][c + 16 v] (MN-major).
//   B2, B3  the 1D operators of the z sweeps, K-major.
// Tensor memory (from the pipeline's base column 256 g): GEMM1 tiles at 0 and
// 64, GEMM2/3 tiles at 64 T, GEMM4 at 192 (each read out before the next
// product that writes there is issued).
//
// One thread per pipeline issues each product's MMAs and commits them to one
// of the pipeline's two mbarriers; it sits in the lane quarter whose in-plane
// nodes (96..127) have no expansion or scatter work.  A tile's X tile is
// gathered while the previous tile's GEMM4 runs, and its GEMM1 is issued once
// that GEMM4 is done (the two do not share tensor-memory columns), beside the
// previous tile's scatter: a tile starts with its plane product done.  Every
// wait is bounded (on expiry the pipeline stops, the CTA sets the error word
// after the unit, lets the MMAs in flight drain with a last bounded wait, frees
// its tensor memory and returns).  The nonlocal
// expansion F Delta P (FP32: the pair's F rows and the tile's Delta-scaled
// projections Q, staged in shared memory) is computed while GEMM4 runs and
// added to the accumulators in registers before the scatter; colour-exclusive
// launches make the assembly reductions deterministic.  FP16: every column of
// a gathered tile is scaled by a power of two (its largest entry below 1/16),
// undone before the expansion and scatter.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "fe_ks_internal.h"

namespace feks {
namespace tc5 {

template <int N>
struct G5 {
  static constexpr int NN = N * N, N3 = N * NN, VT = 4, NT = 512, GT = 256, NC = 10;
  static constexpr int KP = (NN + 15) / 16 * 16;      // GEMM1 K: in-plane node p (padded)
  static constexpr int R1 = 3 * NN;                    // rows (t, p') of the plane operators
  static constexpr int MT1 = (R1 + 127) / 128;         // GEMM1 M tiles
  static constexpr int R1P = MT1 * 128;
  static constexpr int K4 = (R1 + 15) / 16 * 16;       // GEMM4 K
  static constexpr int N1 = (VT * N + 15) / 16 * 16;   // GEMM1 N: v + 4 c (padded)
  static constexpr int R2 = VT * NN;                   // GEMM2/3 rows v + 4 p' (a node's vectors adjacent)
  static constexpr int MT2 = (R2 + 127) / 128;
  static constexpr int N2 = (4 * N + 15) / 16 * 16;    // GEMM2 N: 4 c' + q
  static constexpr int K2 = 48;                        // GEMM2 K: 16 t + c
  static constexpr int K3 = N2;                        // GEMM3 K: 4 c' + q
  static constexpr int N3C = 48;                       // GEMM3 N: 16 t + c
  static constexpr int N4 = 16 * VT;                   // GEMM4 N: c + 16 v
  static constexpr int CH0 = 2 * ((N + 2) / 4);        // c' of the first half of a quadrature-point row
  static constexpr int CSL = K3 / 4;                   // c' slots of a row (with padding)
  static constexpr int NC3 = 3 * (N > 8 ? 2 : 1);      // 16-byte chunks of a GEMM4 operand row group
  static constexpr int MAXC = (N + 1) / 2;             // z planes per warp half in the final step
  static constexpr int PWC = (CH0 > (CSL < N ? CSL : N) - CH0 ? CH0 : (CSL < N ? CSL : N) - CH0);
                                                       // planes c' < N in a half of the quadrature-point step
  static constexpr int R3C = NC3 - NC3 / 2;            // chunks in a half of the GEMM3 readout (the larger)
  static constexpr int PG = 16;                        // p groups of KM (GEMM4 M = 128)
  static constexpr int PGS = R1P * 16;                 // byte stride of a p group in KM
  static constexpr int QCAP = 64, PCAP = 16;           // staged (pair, projector) rows; staged pairs
  static constexpr int CFS = 12;                       // floats per point of the staged coefficients
  // shared by the two pipelines: operators, and the current cell's data
  static constexpr int OFF_KM = 0;
  static constexpr int OFF_B2 = OFF_KM + PG * PGS;
  static constexpr int OFF_B3 = OFF_B2 + N2 * K2 * 2;
  static constexpr int SZ_CST = OFF_B3 + N3C * K3 * 2;   // constant block, copied verbatim
  static constexpr int OFF_CF = SZ_CST;                  // coefficients [point][CFS], FP32
  static constexpr int OFF_SD = OFF_CF + CFS * N3 * 4;   // DoF of each node
  static constexpr int OFF_DS = OFF_SD + (N3 * 4 + 15) / 16 * 16;   // D^{-1/2} of each node
  static constexpr int OFF_SP = OFF_DS + (N3 * 4 + 15) / 16 * 16;   // [PCAP] pairs, [PCAP] their atoms
  static constexpr int OFF_PIPE = OFF_SP + 2 * PCAP * 4;
  // per pipeline, at OFF_PIPE + g * PIPE
  static constexpr int XSB = KP * 16;                  // n-group stride of the X tile
  static constexpr int SZ_XS = (N1 / 8) * XSB;
  static constexpr int SBO2 = 144;                     // 8-row group stride of the GEMM2/3 A operands (padded:
                                                       // the 16-byte row stores of a warp spread over all banks)
  static constexpr int LBO2 = MT2 * 16 * SBO2;         // k-chunk stride of the GEMM2/3 A operands
  static constexpr int SBO4 = K4 * 16 + 16;            // n-group stride of the GEMM4 B operand (padded likewise)
  static constexpr int SZ_AB0 = LBO2 * (K2 > K3 ? K2 : K3) / 8;
  static constexpr int SZ_AB = SZ_AB0 > (N4 / 8) * SBO4 ? SZ_AB0 : (N4 / 8) * SBO4;
  static constexpr int P_XS = 0;
  static constexpr int P_AB = P_XS + SZ_XS;
  static constexpr int P_QS = P_AB + SZ_AB;            // [QCAP][VT] Delta-scaled projections of the tile
  static constexpr int P_RED = P_QS + QCAP * VT * 4;   // FP16: [8 warps][VT] column maxima, [VT] scales
  static constexpr int P_USC = P_RED + 9 * VT * 4;     // [2][VT] unscale factors (two tiles in flight)
  static constexpr int P_MBAR = (P_USC + 2 * VT * 4 + 7) / 8 * 8;   // two mbarriers: GEMM2-4, GEMM1
  static constexpr int PIPE = (P_MBAR + 16 + 15) / 16 * 16;
  static constexpr int OFF_TMEM = OFF_PIPE + 2 * PIPE;
  static constexpr int BYTES = OFF_TMEM + 8;
  // tensor-memory columns, from the pipeline's base (256 g): GEMM1 tiles at 64 T, GEMM2/3 tiles at 64 T
  // (T <= 2: columns 0..175), GEMM4 at 192 (so the next tile's GEMM1 can run while GEMM4's
  // accumulators are read out)
  static constexpr uint32_t TM_D1S = 64, TM_D23S = 64, TM_D4 = 192;
  static_assert(N >= 2 && N <= 9, "N");
  static_assert(NN <= 128 && MT1 <= 2 && N1 <= 64 && N2 <= 64 && MT2 <= 3 && N4 <= 64, "tile shapes");
  static_assert((MT2 - 1) * TM_D23S + N2 <= TM_D4 && (MT1 - 1) * TM_D1S + N1 <= TM_D4 && TM_D4 + N4 <= 256,
                "tensor-memory columns");
  static_assert(SZ_CST % 16 == 0 && OFF_PIPE % 16 == 0 && PIPE % 16 == 0 && P_AB % 16 == 0 && P_QS % 16 == 0,
                "alignment");
  static_assert(BYTES <= 232448, "shared memory");
};

constexpr int kWaitIters = 1 << 22;           // bound of an mbarrier wait (try_wait polls)
constexpr int kWaitItersInjected = 1 << 12;   // the same under host-side fault injection

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of the 5th-generation tensor core; no swizzle
  return d;
}

// kind::f16 instruction descriptor: FP32 accumulator; A and B BF16 (or FP16);
// a_mn / b_mn: operand MN-major (else K-major); M = 128.
template <bool F16>
__host__ __device__ constexpr uint32_t idesc(int n, int a_mn, int b_mn) {
  return (1u << 4) | (F16 ? 0u : (1u << 7) | (1u << 10)) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t dt, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dt),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void ld16(uint32_t ta, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 8 (4) consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void ld8(uint32_t ta, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(ta));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void ld4(uint32_t ta, float* v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(ta));
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// bounded wait for phase `parity` of the mbarrier; false on expiry
__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity, int iters = kWaitIters) {
  uint32_t done = 0;
  for (int it = 0; it < iters && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mb), "r"(parity)
        : "memory");
  }
  return done != 0;
}

// two FP32 values in one 64-bit register, and the packed FMA acc += a * b (each half
// rounded as fmaf)
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 up2(uint64_t x) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x));
  return make_float2(lo, hi);
}
__device__ __forceinline__ void fma2(uint64_t& acc, uint64_t a, uint64_t b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

template <bool F16>
__device__ __forceinline__ uint32_t pack(float lo, float hi) {
  if constexpr (F16) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  } else {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
}

__device__ __forceinline__ void st16(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// power of two s with s * mx < 1/16 (1 for a zero or non-finite maximum)
__device__ __forceinline__ float col_scale(float mx) {
  if (!(mx > 0.f) || !(mx < 3.0e38f)) return 1.f;
  int e = (int)((__float_as_uint(mx) >> 23) & 0xFFu);
  e = e < 1 ? 1 : (e > 248 ? 248 : e);
  return __uint_as_float((uint32_t)(249 - e) << 23);
}

struct Params {
  const float* X;
  float* Y;
  int64_t ld;
  int ncols;
  const int* cell_dofs;
  const int* cells;
  int n_cells;
  const float* coef;     // [E][ncoef][N^3]
  int ncoef;
  int gga;
  const float* dscale;   // D^{-1/2} or nullptr
  const int* cell_pair_ptr;
  const int* cell_pairs;
  const int* pair_atom;
  const float* F;        // [pair][n_proj][N^3]
  const float* Q;        // [atom][n_proj][ld], scaled by Delta
  int n_proj;
  float alpha;
  const uint4* cst;      // the constant block (KM, B2, B3) in shared-memory layout
  int units_per_cell;    // a cell's column tiles are split into this many work units
  int tiles_per_unit;
  int stagger;           // pipeline 1 starts a unit once pipeline 0 has passed: 0 no point,
                         // 1 its first GEMM1, 2 its first quadrature-point step
  int inject;            // host-side fault injection: each pipeline's first GEMM1 is neither
                         // issued nor committed, so its waits (short limit) expire
  int* err;              // set to 1 when a bounded wait expires
};

// named barrier of one pipeline (256 threads); and its OR-reduction of a predicate
__device__ __forceinline__ void gsync(int g) { asm volatile("bar.sync %0, 256;\n" ::"r"(g + 1) : "memory"); }
__device__ __forceinline__ bool gsync_or(int g, bool c) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, 256, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)c), "r"(g + 1)
      : "memory");
  return r != 0;
}

// bound of the kernel's mbarrier waits (short under host-side fault injection)
__device__ __forceinline__ int wait_limit(const Params& p) { return p.inject ? kWaitItersInjected : kWaitIters; }

// barrier 3: pipeline 0 arrives (256 threads), pipeline 1 waits (256 threads)
__device__ __forceinline__ void stagger_arrive() { asm volatile("bar.arrive 3, 512;\n" ::: "memory"); }
__device__ __forceinline__ void stagger_wait() { asm volatile("bar.sync 3, 512;\n" ::: "memory"); }

template <int N, bool F16>
__global__ void __launch_bounds__(512, 1) fe_tc5_kernel(const __grid_constant__ Params p) {
  using G = G5<N>;
  constexpr int NT = G::NT, GT = G::GT, NN = G::NN, N3 = G::N3, VT = G::VT;
  constexpr int GPT = (N3 + GT - 1) / GT;   // gathered nodes per thread
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = tid / GT, gt = tid % GT;               // pipeline and thread within it
  const int quarter = warp & 3, sub = (warp >> 2) & 1; // tensor-memory lane quarter; warp half of the pipeline
  const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem);
  unsigned char* pb_ = smem + G::OFF_PIPE + g * G::PIPE;   // this pipeline's buffers
  const uint32_t sP = s0 + G::OFF_PIPE + g * G::PIPE;
  const uint32_t sXS = sP + G::P_XS, sAB = sP + G::P_AB, mbar = sP + G::P_MBAR, mbar1 = mbar + 8;
  // the MMA-issuing thread: lane 0 of the pipeline's last warp (lane quarter 3: its in-plane
  // nodes 96..127 have no expansion or scatter work, so issuing delays no other step)
  constexpr int ISS = GT - 32;
  float* cf = reinterpret_cast<float*>(smem + G::OFF_CF);
  int* sd = reinterpret_cast<int*>(smem + G::OFF_SD);
  float* sds = reinterpret_cast<float*>(smem + G::OFF_DS);
  int* spr = reinterpret_cast<int*>(smem + G::OFF_SP);
  int* spa = spr + G::PCAP;
  float* qs = reinterpret_cast<float*>(pb_ + G::P_QS);
  float* red = reinterpret_cast<float*>(pb_ + G::P_RED);
  float* usc = reinterpret_cast<float*>(pb_ + G::P_USC);

  // (0) constants; both pipelines' X tiles and operand buffers start zeroed
  //     (their padding is read by the tensor cores, multiplied by zero operator
  //     entries, and must be finite)
  for (int i = tid; i < G::SZ_CST / 16; i += NT) reinterpret_cast<uint4*>(smem)[i] = __ldg(p.cst + i);
  for (int i = tid; i < 2 * G::PIPE / 16; i += NT)
    reinterpret_cast<uint4*>(smem + G::OFF_PIPE)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  if (gt < 2 * VT) usc[gt] = 1.f;
  if (gt == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar1));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(s0 + G::OFF_TMEM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *reinterpret_cast<const uint32_t*>(smem + G::OFF_TMEM) + 256u * (uint32_t)g;
  const uint32_t tlane = tbase + ((uint32_t)(32 * quarter) << 16);   // this warp's lane quarter

  constexpr uint32_t ID1 = idesc<F16>(G::N1, 0, 1), ID2 = idesc<F16>(G::N2, 0, 0);
  constexpr uint32_t ID3 = idesc<F16>(G::N3C, 0, 0), ID4 = idesc<F16>(G::N4, 1, 1);
  // descriptors of the operands' first core matrices (later ones: + byte offset / 16)
  const uint64_t dKM1 = sdesc(s0 + G::OFF_KM, G::PGS, 128), dXS = sdesc(sXS, 128, G::XSB);
  const uint64_t dA2 = sdesc(sAB, G::LBO2, G::SBO2), dB2 = sdesc(s0 + G::OFF_B2, G::N2 * 16, 128);
  const uint64_t dB3 = sdesc(s0 + G::OFF_B3, G::N3C * 16, 128);
  const uint64_t dKM4 = sdesc(s0 + G::OFF_KM, 128, G::PGS), dB4 = sdesc(sAB, 128, G::SBO4);

  const int ntiles = (p.ncols + VT - 1) / VT;
  const bool vec = (p.ld % 4 == 0) && (((uintptr_t)p.X & 15) == 0) && (((uintptr_t)p.Q & 15) == 0);
  const bool vecy = (p.ld % 4 == 0) && (((uintptr_t)p.Y & 15) == 0);
  const int units = p.n_cells * p.units_per_cell;
  // this warp half's z planes in the final step
  const int cbeg = sub ? (N + 1) / 2 : 0, ccnt = sub ? N / 2 : (N + 1) / 2;
  // mbarrier phases: `mbar` tracks GEMM2-4, `mbar1` GEMM1 (issued one tile ahead)
  uint32_t phase = 0, phase1 = 0, failed_phase = 0, failed_bar = 0;
  bool failed = false, pend1 = false;   // pend1: a committed GEMM1 not yet waited for
  int staged = -1;

  // the pipeline's threads: bounded wait for the products just committed; uniform result
  // (the barrier also hands the generic-proxy shared stores before it to the tensor cores)
  auto wait_products = [&]() -> bool {
    const bool ok = mbar_wait(mbar, phase, wait_limit(p));
    fence_async_smem();
    if (gsync_or(g, !ok)) {
      failed = true;
      failed_bar = mbar;
      failed_phase = phase;
      return false;
    }
    phase ^= 1u;
    fence_after();
    return true;
  };
  auto pipe_sync = [&]() {   // generic-proxy shared stores -> tensor cores; tensor-memory reads done
    fence_async_smem();
    fence_before();
    gsync(g);
  };
  // a bounded wait whose outcome is combined at the next pipe_sync_or instead of its own
  // barrier: a thread whose wait expired only moves stale tensor-memory values into shared
  // buffers that the failed tile never uses (the wait before the scatter keeps its own check)
  bool expired = false;
  auto wait_local = [&](uint32_t bar, uint32_t& ph) {
    if (!mbar_wait(bar, ph, wait_limit(p))) expired = true;
    ph ^= 1u;
    fence_after();
  };
  // pipe_sync, and whether any thread's wait expired; bar / ph: the barrier of the last
  // wait and its phase after that wait
  auto pipe_sync_or = [&](uint32_t bar, uint32_t ph) -> bool {
    fence_async_smem();
    fence_before();
    if (gsync_or(g, expired)) {
      failed = true;
      failed_bar = bar;
      failed_phase = ph ^ 1u;
      return false;
    }
    return true;
  };
  auto issue_gemm1 = [&]() {   // (2) GEMM1: P_t = K_t^T X per plane
#pragma unroll
    for (int T = 0; T < G::MT1; ++T)
#pragma unroll
      for (int ks = 0; ks < G::KP / 16; ++ks)
        mma(tbase + T * G::TM_D1S, dKM1 + (uint64_t)((T * 2048 + ks * 2 * G::PGS) >> 4),
            dXS + (uint64_t)((ks * 256) >> 4), ID1, ks > 0);
  };
  // this thread's gathered nodes of column tile [cx, cx + 4) and their D^{-1/2}
  // (registers; nothing waits on the loads until the tile's gather)
  float xn[GPT][VT], xs[GPT];
  auto load_x = [&](int cx) {
    const bool fullx = vec && cx + VT <= p.ncols;
#pragma unroll
    for (int r = 0; r < GPT; ++r) {
      const int node = gt + r * GT;
#pragma unroll
      for (int c = 0; c < VT; ++c) xn[r][c] = 0.f;
      xs[r] = 1.f;
      if (node < N3) {
        const int d = sd[node];
        const float* xr = p.X + (int64_t)d * p.ld + cx;
        if (fullx) {
          const float4 a = __ldg(reinterpret_cast<const float4*>(xr));
          xn[r][0] = a.x, xn[r][1] = a.y, xn[r][2] = a.z, xn[r][3] = a.w;
        } else {
#pragma unroll
          for (int c = 0; c < VT; ++c) xn[r][c] = cx + c < p.ncols ? __ldg(xr + c) : 0.f;
        }
        xs[r] = sds[node];
      }
    }
  };

  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int ci = u / p.units_per_cell;
    const int t_begin = (u % p.units_per_cell) * p.tiles_per_unit;
    const int t_end = min(ntiles, t_begin + p.tiles_per_unit);
    if (t_begin >= t_end) continue;
    const int e = p.cells[ci];
    __syncthreads();   // both pipelines have finished the previous unit
    if (ci != staged) {
      for (int w = tid; w < N3; w += NT) {
        const int d = p.cell_dofs[(int64_t)e * N3 + w];
        sd[w] = d;
        sds[w] = p.dscale ? __ldg(p.dscale + d) : 1.f;
      }
      const float* gc = p.coef + (int64_t)e * p.ncoef * N3;
      for (int w = tid; w < G::NC * N3; w += NT) {
        const int slot = w / N3, q = w - slot * N3;
        cf[q * G::CFS + slot] = __ldg(gc + w);
      }
      if (p.cell_pair_ptr) {
        const int b0 = p.cell_pair_ptr[e], n = min(p.cell_pair_ptr[e + 1] - b0, G::PCAP);
        if (tid < n) {
          const int pr = p.cell_pairs[b0 + tid];
          spr[tid] = pr;
          spa[tid] = p.pair_atom[pr];
        }
      }
      staged = ci;
    }
    __syncthreads();
    const int pb = p.cell_pair_ptr ? p.cell_pair_ptr[e] : 0;
    const int pe = p.cell_pair_ptr ? p.cell_pair_ptr[e + 1] : 0;
    const int nqrows = (pe - pb) * p.n_proj;
    const bool qstaged = nqrows <= G::QCAP && pe - pb <= G::PCAP;
    // (1) extraction Q C P X (Algorithm 1) of column tile [cx, cx + 4): the prefetched rows
    //     of X (xn) -> the MN-major X tile; FP16 scales -> unscale set ubn; the tile's rows of
    //     Q -> q (stored to shared memory once the previous tile's expansion is done)
    auto gather = [&](int cx, int ubn, float4& q) {
#pragma unroll
      for (int r = 0; r < GPT; ++r)
#pragma unroll
        for (int c = 0; c < VT; ++c) xn[r][c] *= xs[r];
      if constexpr (F16) {
        float cm[VT];
#pragma unroll
        for (int c = 0; c < VT; ++c) {
          float m = 0.f;
#pragma unroll
          for (int r = 0; r < GPT; ++r) m = fmaxf(m, fabsf(xn[r][c]));
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
          cm[c] = m;
        }
        if (lane < VT) {
          float v = cm[0];
#pragma unroll
          for (int c = 1; c < VT; ++c) v = lane == c ? cm[c] : v;
          red[(gt >> 5) * VT + lane] = v;
        }
        gsync(g);
        if (gt < VT) {
          float m = 0.f;
#pragma unroll
          for (int w = 0; w < 8; ++w) m = fmaxf(m, red[w * VT + gt]);
          const float sc = col_scale(m);
          red[8 * VT + gt] = sc;
          usc[ubn * VT + gt] = 1.f / sc;   // exact: a power of two
        }
        gsync(g);
#pragma unroll
        for (int c = 0; c < VT; ++c) {
          const float sc = red[8 * VT + c];
#pragma unroll
          for (int r = 0; r < GPT; ++r) xn[r][c] *= sc;
        }
      }
#pragma unroll
      for (int r = 0; r < GPT; ++r) {
        const int node = gt + r * GT;
        if (node < N3) {
          const int pn = node % NN, c = node / NN;
          const uint32_t a = sXS + pn * 16 + (c & 1) * 8 + (c >> 1) * G::XSB;
          asm volatile("st.shared.v2.b32 [%0], {%1,%2};\n" ::"r"(a), "r"(pack<F16>(xn[r][0], xn[r][1])),
                       "r"(pack<F16>(xn[r][2], xn[r][3]))
                       : "memory");
        }
      }
      // the tile's rows of Q (one row per thread)
      q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (qstaged && gt < nqrows) {
        const int b = gt % p.n_proj;
        const float* qr = p.Q + ((int64_t)spa[gt / p.n_proj] * p.n_proj + b) * p.ld + cx;
        if (vec && cx + 4 <= p.ncols) {
          q = __ldg(reinterpret_cast<const float4*>(qr));
        } else {
          if (cx < p.ncols) q.x = __ldg(qr);
          if (cx + 1 < p.ncols) q.y = __ldg(qr + 1);
          if (cx + 2 < p.ncols) q.z = __ldg(qr + 2);
          if (cx + 3 < p.ncols) q.w = __ldg(qr + 3);
        }
      }
    };
    // offset the two pipelines within the unit: pipeline 1 waits until pipeline 0 has passed
    // the stagger point of its first tile (pipeline 0 always has one; it arrives exactly once,
    // also when its wait fails, so the barrier always completes)
    bool arrived = p.stagger == 0 || g == 1;
    if (p.stagger != 0 && g == 1) stagger_wait();
    // this pipeline's column tiles of the unit: every other one.  A tile's GEMM1 is issued
    // during the previous tile (once its GEMM4 is done), or here for the first.
    int ub = 0;   // the unscale set of the current tile
    float4 qreg = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t_begin + g < t_end) {
      load_x(VT * (t_begin + g));
      gather(VT * (t_begin + g), 0, qreg);
      pipe_sync();
      // fault injection (host side): the CTA's first GEMM1 of each pipeline is not issued
      if (gt == ISS && !(p.inject && u == (int)blockIdx.x)) {
        fence_after();
        issue_gemm1();
        commit(mbar1);
      }
      pend1 = true;
    }
    for (int t = t_begin + g; t < t_end; t += 2) {
      const int col0 = VT * t;
      const bool nxt = t + 2 < t_end;   // this pipeline has another tile in the unit
      wait_local(mbar1, phase1);
      pend1 = false;
      if (!arrived && p.stagger == 1) {
        stagger_arrive();
        arrived = true;
      }
      if (qstaged && gt < nqrows) reinterpret_cast<float4*>(qs)[gt] = qreg;
      // (3) GEMM1 rows (t, p') -> A2 rows v + 4 p', k = 16 t + c; one GEMM1 tile per warp half
      if (sub < G::MT1) {
        const int T = sub;
        float a[G::N1];
#pragma unroll
        for (int j = 0; j < G::N1 / 16; ++j) ld16(tlane + T * G::TM_D1S + 16 * j, a + 16 * j);
        ld_wait();
        const int r1 = 128 * T + 32 * quarter + lane;
        if (r1 < G::R1) {
          const int tt = r1 / NN, pp = r1 - tt * NN;
#pragma unroll
          for (int v = 0; v < VT; ++v) {
            const int r2 = v + 4 * pp;
            const uint32_t row = sAB + (r2 & 7) * 16 + (r2 >> 3) * G::SBO2;
            float c8[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) c8[c] = c < N ? a[v + VT * c] : 0.f;
            st16(row + (2 * tt) * G::LBO2, pack<F16>(c8[0], c8[1]), pack<F16>(c8[2], c8[3]), pack<F16>(c8[4], c8[5]),
                 pack<F16>(c8[6], c8[7]));
            // second chunk (c = 8..15): the plane c = 8, or zeros (the buffer is shared with the
            // other products; a NaN left there would survive the zero operator entries)
            st16(row + (2 * tt + 1) * G::LBO2, N > 8 ? pack<F16>(a[v + VT * (N > 8 ? 8 : 0)], 0.f) : 0u, 0u, 0u, 0u);
          }
        }
      }
      if (!pipe_sync_or(mbar1, phase1)) break;
      // (4) GEMM2: the z sweep
      if (gt == ISS) {
        fence_after();
#pragma unroll
        for (int T = 0; T < G::MT2; ++T)
#pragma unroll
          for (int ks = 0; ks < G::K2 / 16; ++ks)
            mma(tbase + T * G::TM_D23S, dA2 + (uint64_t)((T * 16 * G::SBO2 + ks * 2 * G::LBO2) >> 4),
                dB2 + (uint64_t)((ks * 2 * G::N2 * 16) >> 4), ID2, ks > 0);
        commit(mbar);
      }
      wait_local(mbar, phase);
      // (5) quadrature-point step: (Y0, Y_x, Y_y, Y_z)[c'] -> (Z, W_x, W_y, W_z)[c'] (A3, k = 4 c' + q).
      //     Items (tile T, half H of the c' range): a warp half takes (0, H), (1, !H), (2, H) (the
      //     upper half holds more planes).  It loads the accumulator columns (4 per plane) of the
      //     first two, waits once, and loads the third's while it computes the first.
      auto pw_load = [&](int T, auto H, float* y) {
        constexpr int LO = decltype(H)::value ? G::CH0 : 0, HI = decltype(H)::value ? G::CSL : G::CH0;
        constexpr int NV = (HI < N ? HI : N) - LO;   // planes c' < N of the half
#pragma unroll
        for (int k = 0; k < NV; ++k) ld4(tlane + T * G::TM_D23S + 4 * (LO + k), y + 4 * k);
      };
      auto pw_compute = [&](int T, auto H, const float* y) {
        constexpr int LO = decltype(H)::value ? G::CH0 : 0, HI = decltype(H)::value ? G::CSL : G::CH0;
        const int r2 = 128 * T + 32 * quarter + lane;
        if (r2 < G::R2) {
          const int pp = r2 >> 2;
          float o[4 * (HI - LO) + 1];
#pragma unroll
          for (int c = LO; c < HI; ++c) {
            float z = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f;
            if (c < N) {
              const float* cp = cf + (pp + NN * c) * G::CFS;   // the vectors of a node share the address
              const float4 ca = *reinterpret_cast<const float4*>(cp);
              const float4 cb = *reinterpret_cast<const float4*>(cp + 4);
              const float G00 = ca.x, G01 = ca.y, G02 = ca.z, G11 = ca.w, G12 = cb.x, G22 = cb.y, VL = cb.z;
              const float* yc = y + 4 * (c - LO);
              const float u = yc[0], gx = yc[1], gy = yc[2], gz = yc[3];
              z = VL * u;
              w0 = fmaf(G00, gx, fmaf(G01, gy, G02 * gz));
              w1 = fmaf(G01, gx, fmaf(G11, gy, G12 * gz));
              w2 = fmaf(G02, gx, fmaf(G12, gy, G22 * gz));
              if (p.gga) {
                const float2 cc = *reinterpret_cast<const float2*>(cp + 8);
                const float V0 = cb.w, V1 = cc.x, V2 = cc.y;
                z = fmaf(V0, gx, fmaf(V1, gy, fmaf(V2, gz, z)));
                w0 = fmaf(V0, u, w0);
                w1 = fmaf(V1, u, w1);
                w2 = fmaf(V2, u, w2);
              }
            }
            o[4 * (c - LO)] = z;
            o[4 * (c - LO) + 1] = w0;
            o[4 * (c - LO) + 2] = w1;
            o[4 * (c - LO) + 3] = w2;
          }
          const uint32_t row = sAB + (r2 & 7) * 16 + (r2 >> 3) * G::SBO2;
#pragma unroll
          for (int kc = 0; kc < (HI - LO) / 2; ++kc)
            st16(row + (LO / 2 + kc) * G::LBO2, pack<F16>(o[8 * kc], o[8 * kc + 1]),
                 pack<F16>(o[8 * kc + 2], o[8 * kc + 3]), pack<F16>(o[8 * kc + 4], o[8 * kc + 5]),
                 pack<F16>(o[8 * kc + 6], o[8 * kc + 7]));
        }
      };
      auto pw_items = [&](auto H) {
        using HA = std::integral_constant<int, decltype(H)::value>;
        using HB = std::integral_constant<int, 1 - decltype(H)::value>;
        float y0[4 * G::PWC], y1[4 * G::PWC], y2[4 * G::PWC];
        pw_load(0, HA{}, y0);
        if constexpr (G::MT2 > 1) pw_load(1, HB{}, y1);
        ld_wait();
        pw_compute(0, HA{}, y0);
        if constexpr (G::MT2 > 2) pw_load(2, HA{}, y2);
        if constexpr (G::MT2 > 1) pw_compute(1, HB{}, y1);
        if constexpr (G::MT2 > 2) {
          ld_wait();
          pw_compute(2, HA{}, y2);
        }
      };
      if (sub)
        pw_items(std::integral_constant<int, 1>{});
      else
        pw_items(std::integral_constant<int, 0>{});
      if (!arrived) {   // stagger point 2: after the first quadrature-point step
        stagger_arrive();
        arrived = true;
      }
      if (!pipe_sync_or(mbar, phase)) break;
      // (6) GEMM3: the transposed z sweep
      if (gt == ISS) {
        fence_after();
#pragma unroll
        for (int T = 0; T < G::MT2; ++T)
#pragma unroll
          for (int ks = 0; ks < G::K3 / 16; ++ks)
            mma(tbase + T * G::TM_D23S, dA2 + (uint64_t)((T * 16 * G::SBO2 + ks * 2 * G::LBO2) >> 4),
                dB3 + (uint64_t)((ks * 2 * G::N3C * 16) >> 4), ID3, ks > 0);
        commit(mbar);
      }
      // the next tile's rows of X, in flight until its gather during GEMM4
      if (nxt) load_x(col0 + 2 * VT);
      wait_local(mbar, phase);
      // (7) GEMM3 rows v + 4 p', columns 16 t + c -> B4 [(t, p')][c + 16 v] (MN-major);
      //     items (tile T, half H = the warp half of the 16-byte chunks (t, 8-column half)): the
      //     chunks of all three tiles are loaded (8 columns each), then stored after one wait
      constexpr int HCN = N > 8 ? 2 : 1;   // 8-column chunks of a 16-column group
      auto r3_load = [&](int T, auto H, float* d) {
        constexpr int C0 = decltype(H)::value ? G::NC3 / 2 : 0, C1 = decltype(H)::value ? G::NC3 : G::NC3 / 2;
#pragma unroll
        for (int ch = C0; ch < C1; ++ch)
          ld8(tlane + T * G::TM_D23S + 16 * (ch / HCN) + 8 * (ch % HCN), d + 8 * (ch - C0));
      };
      auto r3_store = [&](int T, auto H, const float* d) {
        constexpr int C0 = decltype(H)::value ? G::NC3 / 2 : 0, C1 = decltype(H)::value ? G::NC3 : G::NC3 / 2;
        const int r2 = 128 * T + 32 * quarter + lane;
        if (r2 < G::R2) {
          const int v = r2 & 3, pp = r2 >> 2;
#pragma unroll
          for (int ch = C0; ch < C1; ++ch) {
            const int tt = ch / HCN, hc = ch % HCN;
            const float* sv = d + 8 * (ch - C0);
            st16(sAB + (tt * NN + pp) * 16 + (hc + 2 * v) * G::SBO4, pack<F16>(sv[0], sv[1]), pack<F16>(sv[2], sv[3]),
                 pack<F16>(sv[4], sv[5]), pack<F16>(sv[6], sv[7]));
          }
        }
      };
      auto r3_items = [&](auto H) {
        float d0[8 * G::R3C], d1[8 * G::R3C], d2[8 * G::R3C];
        r3_load(0, H, d0);
        if constexpr (G::MT2 > 1) r3_load(1, H, d1);
        if constexpr (G::MT2 > 2) r3_load(2, H, d2);
        ld_wait();
        r3_store(0, H, d0);
        if constexpr (G::MT2 > 1) r3_store(1, H, d1);
        if constexpr (G::MT2 > 2) r3_store(2, H, d2);
      };
      if (sub)
        r3_items(std::integral_constant<int, 1>{});
      else
        r3_items(std::integral_constant<int, 0>{});
      // the K padding of GEMM4 (rows R1..K4 of B4, multiplied by zero rows of KM) must be
      // finite: zero it, as the buffer held other products' data
      for (int i = gt; i < (G::K4 - G::R1) * (G::N4 / 8); i += GT)
        st16(sAB + (G::R1 + i / (G::N4 / 8)) * 16 + (i % (G::N4 / 8)) * G::SBO4, 0u, 0u, 0u, 0u);
      if (!pipe_sync_or(mbar, phase)) break;
      // (8) GEMM4: the transposed plane product
      if (gt == ISS) {
        fence_after();
#pragma unroll
        for (int ks = 0; ks < G::K4 / 16; ++ks)
          mma(tbase + G::TM_D4, dKM4 + (uint64_t)((ks * 256) >> 4), dB4 + (uint64_t)((ks * 256) >> 4), ID4, ks > 0);
        commit(mbar);
      }
      // (9) F Delta P (nonlocal expansion) for this thread's nodes, computed while
      //     GEMM4 runs; then Y += alpha D^{-1/2} Q^T (Y^(e) + F Delta P)
      const int pp = 32 * quarter + lane;   // in-plane node of this lane
      float ex[G::MAXC][VT];
#pragma unroll
      for (int j = 0; j < G::MAXC; ++j)
#pragma unroll
        for (int v = 0; v < VT; ++v) ex[j][v] = 0.f;
      if (pp < NN && pb < pe && qstaged) {
        // every F load of a pair issued before the arithmetic; Q from shared memory (broadcast)
        constexpr int BCH = 9;
        for (int pi = pb; pi < pe; ++pi) {
          const float* Fp = p.F + (int64_t)spr[pi - pb] * p.n_proj * N3 + pp + NN * cbeg;
          const float* qp = qs + (pi - pb) * p.n_proj * VT;
#pragma unroll 1
          for (int b0 = 0; b0 < p.n_proj; b0 += BCH) {
            float f[BCH][G::MAXC];
#pragma unroll
            for (int bb = 0; bb < BCH; ++bb)
#pragma unroll
              for (int j = 0; j < G::MAXC; ++j)
                f[bb][j] = b0 + bb < p.n_proj && j < ccnt ? __ldg(Fp + (int64_t)(b0 + bb) * N3 + NN * j) : 0.f;
            uint64_t ex2[G::MAXC][2];   // packed accumulators, vectors (2 w, 2 w + 1)
#pragma unroll
            for (int j = 0; j < G::MAXC; ++j)
#pragma unroll
              for (int w = 0; w < 2; ++w) ex2[j][w] = pk2(ex[j][2 * w], ex[j][2 * w + 1]);
#pragma unroll
            for (int bb = 0; bb < BCH; ++bb) {
              if (b0 + bb >= p.n_proj) break;
              const float4 q0 = *reinterpret_cast<const float4*>(qp + (b0 + bb) * VT);
              const uint64_t q2[2] = {pk2(q0.x, q0.y), pk2(q0.z, q0.w)};
#pragma unroll
              for (int j = 0; j < G::MAXC; ++j) {
                const uint64_t ff = pk2(f[bb][j], f[bb][j]);
                fma2(ex2[j][0], ff, q2[0]);
                fma2(ex2[j][1], ff, q2[1]);
              }
            }
#pragma unroll
            for (int j = 0; j < G::MAXC; ++j)
#pragma unroll
              for (int w = 0; w < 2; ++w) {
                const float2 e2 = up2(ex2[j][w]);
                ex[j][2 * w] = e2.x;
                ex[j][2 * w + 1] = e2.y;
              }
          }
        }
      } else if (pp < NN && pb < pe) {
        for (int pi = pb; pi < pe; ++pi) {
          const int pr = p.cell_pairs[pi];
          const float* Fp = p.F + (int64_t)pr * p.n_proj * N3 + pp + NN * cbeg;
          const float* Qa = p.Q + (int64_t)p.pair_atom[pr] * p.n_proj * p.ld + col0;
#pragma unroll 1
          for (int b = 0; b < p.n_proj; ++b) {
            float q[VT];
#pragma unroll
            for (int v = 0; v < VT; ++v) q[v] = col0 + v < p.ncols ? __ldg(Qa + (int64_t)b * p.ld + v) : 0.f;
#pragma unroll
            for (int j = 0; j < G::MAXC; ++j) {
              const float f = j < ccnt ? __ldg(Fp + (int64_t)b * N3 + NN * j) : 0.f;
#pragma unroll
              for (int v = 0; v < VT; ++v) ex[j][v] = fmaf(f, q[v], ex[j][v]);
            }
          }
        }
      }
      // the next tile's X tile (free: this tile's GEMM1 is done), while GEMM4 runs
      if (nxt) gather(col0 + 2 * VT, ub ^ 1, qreg);
      if (!wait_products()) break;
      // the next tile's GEMM1 (its accumulators do not overlap GEMM4's), beside this tile's scatter
      if (gt == ISS && nxt) {
        issue_gemm1();
        commit(mbar1);
      }
      pend1 = nxt;
      {
        float o[G::MAXC][VT];
#pragma unroll
        for (int j = 0; j < G::MAXC; ++j)
#pragma unroll
          for (int v = 0; v < VT; ++v) {
            uint32_t r;
            const int c = cbeg + (j < ccnt ? j : 0);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n"
                         : "=r"(r)
                         : "r"(tlane + G::TM_D4 + (uint32_t)(c + 16 * v)));
            o[j][v] = __uint_as_float(r);
          }
        ld_wait();
        fence_before();
        if (pp < NN) {
#pragma unroll
          for (int j = 0; j < G::MAXC; ++j) {
            if (j >= ccnt) break;
            const int c = cbeg + j;
            const int d = sd[pp + NN * c];
            const float s = p.alpha * sds[pp + NN * c];
            float w[VT];
#pragma unroll
            for (int v = 0; v < VT; ++v) w[v] = s * fmaf(o[j][v], usc[ub * VT + v], ex[j][v]);
            float* yp = p.Y + (int64_t)d * p.ld + col0;
            if (vecy && col0 + VT <= p.ncols) {
              atomicAdd(reinterpret_cast<float4*>(yp), make_float4(w[0], w[1], w[2], w[3]));
            } else {
#pragma unroll
              for (int v = 0; v < VT; ++v)
                if (col0 + v < p.ncols) atomicAdd(yp + v, w[v]);
            }
          }
        }
      }
      ub ^= 1;
    }
    if (!arrived) stagger_arrive();   // pipeline 0 left the unit before its stagger point
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
  }
  __syncthreads();
  if (failed && gt == 0) {
    atomicExch(p.err, 1);
    // a last bounded chance for the MMAs in flight to drain: the products of the wait that
    // expired, and a GEMM1 committed ahead (a pipeline stopped only by the other one has none)
    if (failed_bar) (void)mbar_wait(failed_bar, failed_phase, wait_limit(p));
    if (pend1 && failed_bar != mbar1) (void)mbar_wait(mbar1, phase1, wait_limit(p));
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tbase - 256u * (uint32_t)g));
}

// The constant block of one degree: the plane operators KM and the z-sweep
// operators B2, B3, as 16-bit values in their shared-memory layout (host).
template <int N>
void build_const(const double (*Nm)[kMaxN], const double (*Dm)[kMaxN], bool f16, std::vector<uint4>& out) {
  using G = G5<N>;
  std::vector<uint16_t> h(G::SZ_CST / 2, 0);
  auto put = [&](int byte_off, double x) { h[byte_off / 2] = f16 ? f16_bits(x) : bf16_bits(x); };
  for (int r = 0; r < G::R1; ++r) {
    const int t = r / G::NN, pq = r % G::NN, aq = pq % N, bq = pq / N;
    for (int pn = 0; pn < G::NN; ++pn) {
      const int an = pn % N, bn = pn / N;
      const double v = t == 0 ? Nm[aq][an] * Nm[bq][bn] : t == 1 ? Dm[aq][an] * Nm[bq][bn] : Nm[aq][an] * Dm[bq][bn];
      put(G::OFF_KM + r * 16 + (pn % 8) * 2 + (pn / 8) * G::PGS, v);
    }
  }
  // B2 [n = 4 c' + q][k = 16 t + c]: Y0 = N P_0, Y_x = N P_1, Y_y = N P_2, Y_z = D P_0
  for (int q = 0; q < 4; ++q)
    for (int cq = 0; cq < N; ++cq)
      for (int cn = 0; cn < N; ++cn) {
        const int n = 4 * cq + q, t = q == 3 ? 0 : q, k = 16 * t + cn;
        put(G::OFF_B2 + n * 16 + (k % 8) * 2 + (k / 8) * (G::N2 * 16), q == 3 ? Dm[cq][cn] : Nm[cq][cn]);
      }
  // B3 [n = 16 t + c][k = 4 c' + q]: T_0 = N^T Z + D^T W_z, T_1 = N^T W_x, T_2 = N^T W_y
  for (int q = 0; q < 4; ++q)
    for (int cq = 0; cq < N; ++cq)
      for (int cn = 0; cn < N; ++cn) {
        const int t = q == 3 ? 0 : q, n = 16 * t + cn, k = 4 * cq + q;
        put(G::OFF_B3 + n * 16 + (k % 8) * 2 + (k / 8) * (G::N3C * 16), q == 3 ? Dm[cq][cn] : Nm[cq][cn]);
      }
  out.resize(G::SZ_CST / 16);
  std::memcpy(out.data(), h.data(), G::SZ_CST);
}

template <int N, bool F16>
cudaError_t launch_n(Params p, cudaStream_t s) {
  using G = G5<N>;
  if (p.n_cells == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 152;
  cudaError_t err = cudaFuncSetAttribute(fe_tc5_kernel<N, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::BYTES);
  if (err != cudaSuccess) return err;
  const int ntiles = (p.ncols + G::VT - 1) / G::VT;
  // split a cell's column tiles into units so that every SM gets about 16 or more;
  // a unit's tiles alternate between the CTA's two pipelines, so keep the count even
  int upc = 1;
  while (2 * upc < ntiles && (int64_t)p.n_cells * upc < 16LL * sms) upc *= 2;
  p.tiles_per_unit = (ntiles + upc - 1) / upc;
  p.tiles_per_unit += p.tiles_per_unit & 1;
  p.units_per_cell = (ntiles + p.tiles_per_unit - 1) / p.tiles_per_unit;
  const int64_t units = (int64_t)p.n_cells * p.units_per_cell;
  const int grid = (int)std::min<int64_t>(units, sms);
  fe_tc5_kernel<N, F16><<<grid, G::NT, G::BYTES, s>>>(p);
  return cudaGetLastError();
}

}  // namespace tc5

size_t tc5_const_words(int n) {
  switch (n) {
#define FEKS_TC5_CASE(NN) \
  case NN: return tc5::G5<NN>::SZ_CST / 16;
    FEKS_TC5_CASE(2)
    FEKS_TC5_CASE(3)
    FEKS_TC5_CASE(4)
    FEKS_TC5_CASE(5)
    FEKS_TC5_CASE(6)
    FEKS_TC5_CASE(7)
    FEKS_TC5_CASE(8)
    FEKS_TC5_CASE(9)
#undef FEKS_TC5_CASE
    default: return 0;
  }
}

void build_tc5_const(int p, bool f16, std::vector<uint4>& out) {
  const int n = p + 1;
  double xg[kMaxN], wg[kMaxN], xq[kMaxN], wq[kMaxN], val[kMaxN], der[kMaxN];
  gauss_lobatto(n, xg, wg);
  gauss_legendre(n, xq, wq);
  double Nm[kMaxN][kMaxN] = {}, Dm[kMaxN][kMaxN] = {};   // [Gauss point][node]
  for (int q = 0; q < n; ++q) {
    lagrange_eval(n, xg, xq[q], val, der);
    for (int i = 0; i < n; ++i) {
      Nm[q][i] = val[i];
      Dm[q][i] = der[i];
    }
  }
  switch (n) {
#define FEKS_TC5_BUILD(NN) \
  case NN: tc5::build_const<NN>(Nm, Dm, f16, out); return;
    FEKS_TC5_BUILD(2)
    FEKS_TC5_BUILD(3)
    FEKS_TC5_BUILD(4)
    FEKS_TC5_BUILD(5)
    FEKS_TC5_BUILD(6)
    FEKS_TC5_BUILD(7)
    FEKS_TC5_BUILD(8)
    FEKS_TC5_BUILD(9)
#undef FEKS_TC5_BUILD
    default: out.clear();
  }
}

cudaError_t launch_tc5(const Ctx& c, const LocalParams<float>& lp, cudaStream_t s, bool f16, int stagger) {
  tc5::Params p{};
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
  p.cst = f16 ? c.tc5_cst16 : c.tc5_cst;
  p.stagger = stagger;
  p.inject = c.inject_fault;
  p.err = c.dev_status;
  if (!p.cst || !p.err || c.cplx || c.nq != c.np) return cudaErrorInvalidValue;
  switch (c.np) {
#define FEKS_TC5_LAUNCH(NN) \
  case NN: return f16 ? tc5::launch_n<NN, true>(p, s) : tc5::launch_n<NN, false>(p, s);
    FEKS_TC5_LAUNCH(2)
    FEKS_TC5_LAUNCH(3)
    FEKS_TC5_LAUNCH(4)
    FEKS_TC5_LAUNCH(5)
    FEKS_TC5_LAUNCH(6)
    FEKS_TC5_LAUNCH(7)
    FEKS_TC5_LAUNCH(8)
    FEKS_TC5_LAUNCH(9)
#undef FEKS_TC5_LAUNCH
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace feks
