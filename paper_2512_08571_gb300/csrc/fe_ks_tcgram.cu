// FP64-accurate Gram product C = Y^T Z of the Rayleigh-Ritz step (Algorithm 3)
// on the tensor cores, by exact integer slices (in the manner of Ozaki's
// error-free splitting of a matrix product into low-precision products).
//
// The product has a long contraction (the m DoF rows) and a small output
// (n x n, n = N_v): a dense contraction, but one that must be FP64-accurate.
// Rows are taken in chunks of R = 32.  For each chunk and each column of Y
// (and of Z), every value is written in fixed point relative to the column's
// largest exponent in the chunk (integer operations on its bit pattern) and
// cut into eight unsigned 7-bit slices c_0..c_7 (bits 63..8 of the aligned
// 64-bit significand; the sign goes with each slice):
//     y = 2^E sum_s (+-c_s) 2^(-7 s),  E = (largest biased exponent) - 1029.
// Each scaled slice (+-c_s) 2^(-7 s) is a BF16 number exactly, and a product
// of a Y slice and a Z slice is exact in FP32 (|c_s d_t| < 2^14).  The tensor
// cores add the products of a group of slice pairs in an FP32 accumulator.
// That accumulation was measured to behave like a truncating adder of about
// 21-22 significant bits (a first version's error matched such a model to
// within 10 %), so the grouping keeps every group whose loss could matter
// exact within 21 bits: the pairs with s + t = d for d = 0..4 each get an
// accumulator of their own (at most (d+1) x 32 x 127^2 < 2^21.3 in units of
// 2^(-7d); the d = 4 group may lose one bit, 2^(-49) of the result), and the
// pairs with s + t = 5..7 (at most 2^(-35) of the result) share a sixth.
// Pairs with s + t > 7 are dropped (below 2^(-56)).  The six accumulators of a
// 128 x 64 output tile take 384 of the 512 tensor-memory columns.
//
// After each chunk the tile is read back (tcgen05.ld), the six accumulators
// are combined in pairs of floats, scaled by 2^(E_i + E_j) and added to a
// running pair-of-floats sum per output in registers.  A CTA covers one
// 128 x 64 output tile and 8192 rows (256 chunks); its FP64 partial goes to the same
// [chunk][n][n] workspace as the pair-of-floats Gram kernel, whose
// compensated, fixed-order reduction finishes the product.  Deterministic.
//
// Operand staging: thread t slices column t of the tile (Y for t < 128, Z for
// 128 <= t < 192), so the column's maximum exponent needs no reduction; its 32
// row values per slice are four 16-byte rows of the canonical K-major,
// no-swizzle layout (8 rows x 16 bytes per core matrix; core matrices 128
// bytes apart along K, 512 bytes apart along M / N).  One thread issues the 72 MMAs of a
// chunk (36 slice pairs x 2 K-steps of 16), tcgen05.commit signals an
// mbarrier, all threads wait on it (bounded).
#include <cuda_bf16.h>

#include "fe_ks_internal.h"

namespace feks {
namespace tg {

constexpr int R = 32;                        // rows per chunk
constexpr int NS = 8;                        // 7-bit slices
constexpr int TILE = 128;                    // output tile rows (operand A rows, MMA M)
constexpr int TN = 64;                       // output tile columns (operand B rows, MMA N)
constexpr int NACC = 6;                      // accumulators: s + t = 0..4, and 5..7
constexpr int NT = 256;
constexpr uint32_t LBO = 128;                // K-direction core-matrix stride (bytes)
constexpr uint32_t SBO = 512;                // M/N-direction core-matrix stride (bytes)
constexpr int SLICE = TILE * R * 2;          // bytes of one A slice operand (8 KB)
constexpr int SLICE_B = TN * R * 2;          // bytes of one B slice operand (4 KB)
constexpr int OFF_A = 0;
constexpr int OFF_B = NS * SLICE;
constexpr int OFF_E = OFF_B + NS * SLICE_B;  // [256] int: chunk exponent of each operand row
constexpr int OFF_MBAR = OFF_E + NT * 4;
constexpr int OFF_TMEM = OFF_MBAR + 8;
constexpr int OFF_FLAG = OFF_TMEM + 4;
constexpr int BYTES = OFF_FLAG + 12;
constexpr uint32_t TMEM_COLS = 512;          // six 64-column FP32 accumulators (384 used)
constexpr long long kWaitIters = 1LL << 22;  // bound of an mbarrier wait (try_wait polls)

static_assert(TILE * R * 2 == SLICE && R % 16 == 0 && NACC * TN <= (int)TMEM_COLS, "chunk shape");

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((LBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((SBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of the 5th-generation tensor core; no swizzle
  return d;
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M = 128, N = 64
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TILE >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t dt, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dt),
      "l"(a), "l"(b), "r"(idesc()), "r"(acc));
}

// 8 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void ld8(uint32_t ta, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(ta));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// bounded wait for phase `parity` of the mbarrier; returns false on expiry
__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < kWaitIters && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mb), "r"(parity)
        : "memory");
  }
  return done != 0;
}

// hi + lo = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Slice the 32 values src[r * stride] (r < count; zero beyond) of operand row m
// (0..127) into the eight slice buffers at opbase (K-major, no swizzle);
// returns the chunk exponent E of that row.  Pass 1 finds the largest biased
// exponent, pass 2 reloads (L1) and cuts the aligned significands.
__device__ __forceinline__ int slice_row(const double* __restrict__ src, int64_t stride, int count, int m,
                                         uint32_t opbase, int slice_bytes) {
  int emax = 0;
#pragma unroll 8
  for (int r = 0; r < R; ++r) {
    const double v = r < count ? src[(int64_t)r * stride] : 0.0;
    const int eb = (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FFu);
    emax = eb > emax ? eb : emax;
  }
  const int m8 = m & 7, mg = m >> 3;
#pragma unroll 1
  for (int g = 0; g < R / 8; ++g) {
    uint32_t w[NS][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float f[2][NS];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = 8 * g + 2 * q + h;
        const double v = r < count ? src[(int64_t)r * stride] : 0.0;
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        const int eb = (int)((b >> 52) & 0x7FFu);
        const int sh = emax - eb;
        unsigned long long al = 0ull;
        if (eb != 0 && sh < 64) al = (((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull) << 11) >> sh;
        const float sg = (b >> 63) ? -1.f : 1.f;
#pragma unroll
        for (int s = 0; s < NS; ++s)
          f[h][s] = sg * (float)(unsigned)((al >> (57 - 7 * s)) & 0x7Full) * __uint_as_float((uint32_t)(127 - 7 * s) << 23);
      }
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        __nv_bfloat162 p2 = __floats2bfloat162_rn(f[0][s], f[1][s]);   // exact: <= 7 significant bits
        w[s][q] = *reinterpret_cast<uint32_t*>(&p2);
      }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const uint32_t a = opbase + s * slice_bytes + m8 * 16 + mg * SBO + g * LBO;
      asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(a), "r"(w[s][0]), "r"(w[s][1]), "r"(w[s][2]),
                   "r"(w[s][3])
                   : "memory");
    }
  }
  return emax - 1029;
}

// One thread: the chunk's 72 MMAs (pair (s, t) -> accumulator min(s + t, 5)), then commit.
__device__ __forceinline__ void issue_chunk(uint32_t s0, uint32_t tmem, uint32_t mbar) {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  uint32_t started = 0;   // bit g: accumulator g has received its first product of the chunk
#pragma unroll 1
  for (int d = 0; d < NS; ++d)
#pragma unroll 1
    for (int s = 0; s <= d; ++s) {
      const int t = d - s, g = d < NACC - 1 ? d : NACC - 1;
#pragma unroll
      for (int ks = 0; ks < R / 16; ++ks) {
        const uint64_t da = sdesc(s0 + OFF_A + s * SLICE + ks * 2 * LBO);
        const uint64_t db = sdesc(s0 + OFF_B + t * SLICE_B + ks * 2 * LBO);
        mma(tmem + (uint32_t)(g * TN), da, db, (started >> g) & 1u);
        started |= 1u << g;
      }
    }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

// Read this thread's 32 outputs of the chunk (row orow of the tile, columns
// ocol0..ocol0+31), combine the six accumulators in pairs of floats (every
// addition error-free), scale by 2^(E_row + E_col) and add to the running pairs.
__device__ __forceinline__ void accumulate_chunk(uint32_t tmem, int warp, int orow, int ocol0, const int* Es,
                                                 float (&acc_hi)[32], float (&acc_lo)[32], int* sflag) {
  const int Ei = Es[orow];
#pragma unroll
  for (int cb = 0; cb < 4; ++cb) {
    float a[NACC][8];
    const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(ocol0 + 8 * cb);
#pragma unroll
    for (int g = 0; g < NACC; ++g) ld8(ta + (uint32_t)(g * TN), a[g]);
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int jj = 8 * cb + j;
      const int E = Ei + Es[TILE + ocol0 + jj];
      float h = a[0][j], l = 0.f;
#pragma unroll
      for (int g = 1; g < NACC; ++g) {
        float e;
        two_sum(h, a[g][j], h, e);
        l += e;
      }
      if (E < -126 || E > 127) {
        if (h != 0.f || l != 0.f) *sflag = 1;
        continue;
      }
      const float sc = __uint_as_float((uint32_t)(E + 127) << 23);
      h *= sc;
      l *= sc;
      float s, e;   // running pair += (h, l)
      two_sum(acc_hi[jj], h, s, e);
      e += acc_lo[jj] + l;
      acc_hi[jj] = s + e;
      acc_lo[jj] = e - (acc_hi[jj] - s);
    }
  }
}

// MODE 0 (symmetric Gram C = Y^T Z): tile rows [128 blockIdx.y, +128), columns [64 blockIdx.x, +64),
//   skipped when every row index exceeds every column index; rows [8192 blockIdx.z, +8192) of Y
//   and Z, chunks of 32 rows; partial -> part[blockIdx.z][n][n].
// MODE 1 (rotation X = Y E, Y [m][n], E [n][k]): column tile blockIdx.x of X, row tiles
//   blockIdx.y, blockIdx.y + gridDim.y, ... (persistent); chunks of 32 of the n contraction
//   indices; each row tile's result -> X.
// err[0]: a wait expired; err[1]: a chunk's scale 2^(E_i + E_j) left the FP32 range.
template <int MODE>
__global__ void __launch_bounds__(NT, 1) tc_slice_kernel(const double* __restrict__ Y, const double* __restrict__ Z,
                                                         double* __restrict__ out, int64_t m, int n, int k, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (MODE == 0 && ti * TILE > tj * TN + TN - 1) return;   // symmetric: a tile wholly below the diagonal
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem);
  int* Es = reinterpret_cast<int*>(smem + OFF_E);
  const uint32_t mbar = s0 + OFF_MBAR;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + OFF_TMEM);
  int* sflag = reinterpret_cast<int*>(smem + OFF_FLAG);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *sflag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(s0 + OFF_TMEM),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;

  const int side = tid >> 7, cl = tid & 127;   // operand A (t < 128) or B (128 <= t < 192), its row cl
  const bool slicer = side == 0 || cl < TN;
  const uint32_t opbase = s0 + (side ? OFF_B : OFF_A);
  const int slice_bytes = side ? SLICE_B : SLICE;
  const int orow = 32 * (warp & 3) + lane;     // readout: TMEM lane quarter, column half
  const int ocol0 = 32 * (warp >> 2);
  float acc_hi[32], acc_lo[32];
  bool failed = false;
  uint32_t phase = 0, failed_phase = 0;

  const int64_t ntile_r = MODE == 0 ? 1 : (m + TILE - 1) / TILE;
  for (int64_t tr = (MODE == 0 ? 0 : ti); tr < ntile_r && !failed; tr += (MODE == 0 ? 1 : gridDim.y)) {
#pragma unroll
    for (int j = 0; j < 32; ++j) acc_hi[j] = acc_lo[j] = 0.f;
    int64_t c_begin, c_end;   // contraction range of this tile
    if (MODE == 0) {
      c_begin = (int64_t)blockIdx.z * kGramChunkRows;
      c_end = c_begin + kGramChunkRows < m ? c_begin + kGramChunkRows : m;
    } else {
      c_begin = 0;
      c_end = n;
    }
    const int nch = (int)((c_end - c_begin + R - 1) / R);
    for (int ch = 0; ch < nch; ++ch) {
      const int64_t c0 = c_begin + (int64_t)ch * R;
      const int cnt = (int)(c_end - c0 < R ? c_end - c0 : R);
      // (1) this thread's operand row over the chunk
      if (!slicer) {
      } else if (MODE == 0) {
        const int col = side ? tj * TN + cl : ti * TILE + cl;
        const double* src = (side ? Z : Y) + c0 * n + col;
        Es[tid] = slice_row(src, n, col < n ? cnt : 0, cl, opbase, slice_bytes);
      } else if (side == 0) {
        const int64_t row = tr * TILE + cl;
        Es[tid] = slice_row(Y + row * n + c0, 1, row < m ? cnt : 0, cl, opbase, slice_bytes);
      } else {
        const int col = tj * TN + cl;
        Es[tid] = slice_row(Z + c0 * k + col, k, col < k ? cnt : 0, cl, opbase, slice_bytes);
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncthreads();
      // (2) MMAs, (3) bounded wait and readout
      if (tid == 0) issue_chunk(s0, tmem, mbar);
      const bool ok = mbar_wait(mbar, phase);
      if (__syncthreads_or(!ok)) {
        failed = true;
        failed_phase = phase;
        break;
      }
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      accumulate_chunk(tmem, warp, orow, ocol0, Es, acc_hi, acc_lo, sflag);
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncthreads();   // the next chunk overwrites the operands and the accumulators
    }
    if (failed) break;
    if (MODE == 0) {
      double* o = out + (int64_t)blockIdx.z * n * n;
      const int i = ti * TILE + orow;
      if (i < n)
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const int j = tj * TN + ocol0 + jj;
          if (j < n) o[(int64_t)i * n + j] = (double)acc_hi[jj] + (double)acc_lo[jj];
        }
    } else {
      const int64_t row = tr * TILE + orow;
      if (row < m)
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const int j = tj * TN + ocol0 + jj;
          if (j < k) out[row * k + j] = (double)acc_hi[jj] + (double)acc_lo[jj];
        }
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (failed) atomicExch(err, 1);
    if (*sflag) atomicExch(err + 1, 1);
  }
  if (failed && tid == 0) {
    // give MMAs still in flight a last bounded chance to drain before the tensor memory is released
    (void)mbar_wait(mbar, failed_phase);
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
}

// shared-memory opt-in of a kernel mode, once per device
template <int MODE>
fe_ks_status prepare() {
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!done[dev & 63]) {
    cudaError_t e = cudaFuncSetAttribute(tc_slice_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, BYTES);
    if (e != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("tensor-core slice kernel attribute: ") + cudaGetErrorString(e));
    done[dev & 63] = true;
  }
  return FE_KS_OK;
}

}  // namespace tg
}  // namespace feks

using namespace feks;

extern "C" {

fe_ks_status fe_ks_gram_tc_workspace(int64_t m, int n, size_t* bytes) {
  set_error("");
  if (!bytes || m < 1 || n < 1) return fail(FE_KS_ERR_ARG, "bad sizes");
  size_t b = 0;
  fe_ks_status st = fe_ks_gram_ff_workspace(m, n, n, &b);
  if (st != FE_KS_OK) return st;
  *bytes = b + 256;   // two status words (first 256 bytes), then the partials
  return FE_KS_OK;
}

fe_ks_status fe_ks_gram_tc_sym(const double* Y, const double* Z, double* C, int64_t m, int n, void* work,
                               size_t work_bytes, void* cuda_stream) {
  set_error("");
  if (!Y || !Z || !C || !work) return fail(FE_KS_ERR_ARG, "NULL argument");
  size_t need = 0;
  fe_ks_status st = fe_ks_gram_tc_workspace(m, n, &need);
  if (st != FE_KS_OK) return st;
  if (work_bytes < need) return fail(FE_KS_ERR_ARG, "workspace too small");
  if (((uintptr_t)work & 255) || ((uintptr_t)Y & 7) || ((uintptr_t)Z & 7)) return fail(FE_KS_ERR_ARG, "misaligned argument");
  const int64_t nch = (m + kGramChunkRows - 1) / kGramChunkRows;
  if (nch > 65535 || n > 4096) return fail(FE_KS_ERR_ARG, "sizes too large for the tensor-core Gram kernel");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int* flags = static_cast<int*>(work);
  double* part = reinterpret_cast<double*>(static_cast<char*>(work) + 256);
  fe_ks_status ast = tg::prepare<0>();
  if (ast != FE_KS_OK) return ast;
  if (cudaMemsetAsync(flags, 0, 2 * sizeof(int), s) != cudaSuccess) return fail(FE_KS_ERR_CUDA, "cudaMemsetAsync");
  dim3 grid((unsigned)((n + tg::TN - 1) / tg::TN), (unsigned)((n + tg::TILE - 1) / tg::TILE), (unsigned)nch);
  tg::tc_slice_kernel<0><<<grid, tg::NT, tg::BYTES, s>>>(Y, Z, part, m, n, n, flags);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_gram_reduce(part, C, (int)nch, n, n, 1, s);
  if (e != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("tensor-core Gram kernels: ") + cudaGetErrorString(e));
  return FE_KS_OK;
}

fe_ks_status fe_ks_rotate_tc(const double* Y, const double* E, double* X, int64_t m, int n, int k, int* flags,
                             void* cuda_stream) {
  set_error("");
  if (!Y || !E || !X || !flags) return fail(FE_KS_ERR_ARG, "NULL argument");
  if (m < 1 || n < 1 || k < 1 || n > 4096 || k > 4096) return fail(FE_KS_ERR_ARG, "bad sizes");
  if (((uintptr_t)Y & 7) || ((uintptr_t)E & 7) || ((uintptr_t)X & 7) || ((uintptr_t)flags & 3))
    return fail(FE_KS_ERR_ARG, "misaligned argument");
  fe_ks_status ast = tg::prepare<1>();
  if (ast != FE_KS_OK) return ast;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (cudaMemsetAsync(flags, 0, 2 * sizeof(int), s) != cudaSuccess) return fail(FE_KS_ERR_CUDA, "cudaMemsetAsync");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int kt = (k + tg::TN - 1) / tg::TN;
  const int64_t rt = (m + tg::TILE - 1) / tg::TILE;
  const int64_t want = ((int64_t)(sms > 0 ? sms : 152) + kt - 1) / kt;   // about one CTA per SM, persistent
  const unsigned gy = (unsigned)(rt < want ? rt : want);
  tg::tc_slice_kernel<1><<<dim3((unsigned)kt, gy), tg::NT, tg::BYTES, s>>>(Y, E, X, m, n, k, flags);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("tensor-core rotation kernel: ") + cudaGetErrorString(e));
  return FE_KS_OK;
}

fe_ks_status fe_ks_gram_tc_status(const void* work, int* status) {
  set_error("");
  if (!work || !status) return fail(FE_KS_ERR_ARG, "bad arguments");
  int f[2] = {0, 0};
  const int* flags = static_cast<const int*>(work);
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(f, flags, sizeof(f), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(FE_KS_ERR_CUDA, "reading the Gram status failed");
  *status = (f[0] ? 1 : 0) | (f[1] ? 2 : 0);
  return FE_KS_OK;
}

}  // extern "C"
