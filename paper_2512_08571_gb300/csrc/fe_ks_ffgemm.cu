// FP64-accurate dense products for the Rayleigh-Ritz step of Algorithm 3,
// computed in pairs of floats on the FP32 pipe (GB300 runs FP64 at about 1/61
// of its FP32 rate, and its integer tensor cores are too slow for the
// fixed-point FP64 emulation to win):
//   Gram:     C = Y^T Z        (Y [m][n1], Z [m][n2] row-major FP64, m large)
//   rotation: X = Y E          (Y [m][n], E [n][k] row-major FP64)
// Inputs are split into hi + lo floats as they are staged in shared memory;
// every product is formed exactly with an FMA (TwoProduct) and accumulated as
// a float pair (TwoSum).  The Gram kernel splits the long dimension m into
// chunks whose FP64 partial sums are added by a second kernel in a fixed
// order (deterministic).
#include "fe_ks_internal.h"

namespace feks {

constexpr int kGB = 64;    // tile of C (or X) per CTA: 64 x 64
constexpr int kGK = 32;    // staged depth along the contracted dimension
constexpr int kGT = 256;   // threads: 16 x 16, each owning 4 x 4 outputs
constexpr int kGramChunk = kGramChunkRows;

// Compensated dot-product step (Ogita, Rump & Oishi's Dot2, with pair
// operands): acc.hi is the running float sum, acc.lo the accumulated error
// terms: acc += a * b.  The caller renormalises (ff_renorm) every few steps so
// that acc.lo stays within a few ulps of acc.hi: left to grow over thousands
// of terms, its own float rounding would cost about sqrt(n) u^2 of the sum.
__device__ __forceinline__ void ff_mac(ff2& acc, ff2 a, ff2 b) {
  const float ph = a.hi * b.hi;
  const float pl = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -ph)));
  const float t = acc.hi + ph;
  const float bb = t - acc.hi;
  const float e = (acc.hi - (t - bb)) + (ph - bb);
  acc.hi = t;
  acc.lo += e + pl;
}

__device__ __forceinline__ void ff_renorm(ff2& acc) { acc = ff_fast_two_sum(acc.hi, acc.lo); }

// partial[chunk][i][j] = sum over the chunk's rows r of Y[r][i] Z[r][j].
// upper: the result is known to be symmetric; only tiles on or above the
// diagonal are computed (the reduction mirrors them).
__global__ void __launch_bounds__(kGT) ff_gram_partial_kernel(const double* __restrict__ Y, const double* __restrict__ Z,
                                                              double* __restrict__ part, int64_t m, int n1, int n2,
                                                              int upper) {
  __shared__ ff2 Ys[kGK][kGB];
  __shared__ ff2 Zs[kGK][kGB];
  if (upper && blockIdx.y > blockIdx.x) return;   // whole CTA: below the diagonal
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int j0 = blockIdx.x * kGB, i0 = blockIdx.y * kGB;
  const int64_t r_begin = (int64_t)blockIdx.z * kGramChunk;
  const int64_t r_end = r_begin + kGramChunk < m ? r_begin + kGramChunk : m;
  ff2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = ff_make(0.f, 0.f);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kGK) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kGK * kGB; idx += kGT) {
      const int kk = idx / kGB, c = idx % kGB;
      const int64_t r = r0 + kk;
      const bool in = r < r_end;
      Ys[kk][c] = ff_split_bits(in && i0 + c < n1 ? Y[r * n1 + i0 + c] : 0.0);
      Zs[kk][c] = ff_split_bits(in && j0 + c < n2 ? Z[r * n2 + j0 + c] : 0.0);
    }
    __syncthreads();
#pragma unroll 1
    for (int k0 = 0; k0 < kGK; k0 += 4) {
#pragma unroll
      for (int kk = k0; kk < k0 + 4; ++kk) {
        ff2 a[4], b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a[q] = Ys[kk][ty * 4 + q];
          b[q] = Zs[kk][tx * 4 + q];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) ff_mac(acc[p][q], a[p], b[q]);
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) ff_renorm(acc[p][q]);
    }
  }
  double* out = part + (int64_t)blockIdx.z * n1 * n2;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + ty * 4 + p, j = j0 + tx * 4 + q;
      if (i < n1 && j < n2) out[(int64_t)i * n2 + j] = (double)acc[p][q].hi + (double)acc[p][q].lo;
    }
}

// C[i][j] = sum over chunks of partial[chunk][i][j], in chunk order (upper:
// C[i][j] = C[j][i] = the sum at (min(i, j), max(i, j)), an entry of a tile on
// or above the diagonal)
__global__ void ff_gram_reduce_kernel(const double* __restrict__ part, double* __restrict__ C, int nchunks, int n1n2,
                                      int n2, int upper) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n1n2; idx += gridDim.x * blockDim.x) {
    int src = idx;
    if (upper) {
      const int i = idx / n2, j = idx % n2;
      src = i <= j ? idx : j * n2 + i;
    }
    double s = 0.0, c = 0.0;   // compensated (Kahan-Babuska) summation of the chunk partials
    for (int ch = 0; ch < nchunks; ++ch) {
      const double v = part[(int64_t)ch * n1n2 + src];
      const double t = s + v;
      c += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
      s = t;
    }
    C[idx] = s + c;
  }
}

// X[r][j] = sum_l Y[r][l] E[l][j] for a 64 x 64 tile of X
__global__ void __launch_bounds__(kGT) ff_rotate_kernel(const double* __restrict__ Y, const double* __restrict__ E,
                                                        double* __restrict__ X, int64_t m, int n, int k) {
  __shared__ ff2 Ys[kGB][kGK + 1];
  __shared__ ff2 Es[kGK][kGB];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int j0 = blockIdx.y * kGB;
  const int64_t r0 = (int64_t)blockIdx.x * kGB;
  ff2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = ff_make(0.f, 0.f);
  for (int l0 = 0; l0 < n; l0 += kGK) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kGB * kGK; idx += kGT) {
      const int rr = idx / kGK, ll = idx % kGK;
      const int64_t r = r0 + rr;
      Ys[rr][ll] = ff_split_bits(r < m && l0 + ll < n ? Y[r * n + l0 + ll] : 0.0);
      const int le = idx / kGB, c = idx % kGB;
      Es[le][c] = ff_split_bits(l0 + le < n && j0 + c < k ? E[(int64_t)(l0 + le) * k + j0 + c] : 0.0);
    }
    __syncthreads();
#pragma unroll 1
    for (int l1 = 0; l1 < kGK; l1 += 4) {
#pragma unroll
      for (int ll = l1; ll < l1 + 4; ++ll) {
        ff2 a[4], b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a[q] = Ys[ty * 4 + q][ll];
          b[q] = Es[ll][tx * 4 + q];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) ff_mac(acc[p][q], a[p], b[q]);
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) ff_renorm(acc[p][q]);
    }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t r = r0 + ty * 4 + p;
      const int j = j0 + tx * 4 + q;
      if (r < m && j < k) X[r * k + j] = (double)acc[p][q].hi + (double)acc[p][q].lo;
    }
}

cudaError_t launch_gram_reduce(const double* part, double* C, int nchunks, int n1, int n2, int upper, cudaStream_t s) {
  const int nn = n1 * n2;
  ff_gram_reduce_kernel<<<(nn + 255) / 256, 256, 0, s>>>(part, C, nchunks, nn, n2, upper);
  return cudaGetLastError();
}

}  // namespace feks

using namespace feks;

extern "C" {

fe_ks_status fe_ks_gram_ff_workspace(int64_t m, int n1, int n2, size_t* bytes) {
  if (!bytes || m < 1 || n1 < 1 || n2 < 1) return fail(FE_KS_ERR_ARG, "bad sizes");
  const int64_t nch = (m + kGramChunk - 1) / kGramChunk;
  *bytes = (size_t)nch * n1 * n2 * sizeof(double);
  return FE_KS_OK;
}

static fe_ks_status gram_ff(const double* Y, const double* Z, double* C, int64_t m, int n1, int n2, void* work,
                            size_t work_bytes, void* cuda_stream, int upper) {
  set_error("");
  if (!Y || !Z || !C || !work) return fail(FE_KS_ERR_ARG, "NULL argument");
  if (upper && n1 != n2) return fail(FE_KS_ERR_ARG, "a symmetric Gram matrix is square");
  size_t need = 0;
  fe_ks_status st = fe_ks_gram_ff_workspace(m, n1, n2, &need);
  if (st != FE_KS_OK) return st;
  if (work_bytes < need) return fail(FE_KS_ERR_ARG, "workspace too small");
  const int64_t nch = (m + kGramChunk - 1) / kGramChunk;
  if (nch > 65535) return fail(FE_KS_ERR_ARG, "m too large for the chunked Gram kernel");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  dim3 grid((n2 + kGB - 1) / kGB, (n1 + kGB - 1) / kGB, (unsigned)nch);
  double* part = static_cast<double*>(work);
  ff_gram_partial_kernel<<<grid, kGT, 0, s>>>(Y, Z, part, m, n1, n2, upper);
  const int nn = n1 * n2;
  ff_gram_reduce_kernel<<<(nn + 255) / 256, 256, 0, s>>>(part, C, (int)nch, nn, n2, upper);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("Gram kernels: ") + cudaGetErrorString(err));
  return FE_KS_OK;
}

fe_ks_status fe_ks_gram_ff(const double* Y, const double* Z, double* C, int64_t m, int n1, int n2, void* work,
                           size_t work_bytes, void* cuda_stream) {
  return gram_ff(Y, Z, C, m, n1, n2, work, work_bytes, cuda_stream, 0);
}

fe_ks_status fe_ks_gram_ff_sym(const double* Y, const double* Z, double* C, int64_t m, int n, void* work,
                               size_t work_bytes, void* cuda_stream) {
  return gram_ff(Y, Z, C, m, n, n, work, work_bytes, cuda_stream, 1);
}

fe_ks_status fe_ks_rotate_ff(const double* Y, const double* E, double* X, int64_t m, int n, int k, void* cuda_stream) {
  set_error("");
  if (!Y || !E || !X) return fail(FE_KS_ERR_ARG, "NULL argument");
  if (m < 1 || n < 1 || k < 1) return fail(FE_KS_ERR_ARG, "bad sizes");
  const int64_t gx = (m + kGB - 1) / kGB;
  if (gx > INT32_MAX || (k + kGB - 1) / kGB > 65535) return fail(FE_KS_ERR_ARG, "sizes too large");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  dim3 grid((unsigned)gx, (k + kGB - 1) / kGB);
  ff_rotate_kernel<<<grid, kGT, 0, s>>>(Y, E, X, m, n, k);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("rotation kernel: ") + cudaGetErrorString(err));
  return FE_KS_OK;
}

}  // extern "C"
