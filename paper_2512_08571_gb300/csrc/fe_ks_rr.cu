// Rayleigh-Ritz step (Algorithm 3) and the Lanczos spectral upper bound used
// for the filter's bounds (Algorithm 4's lam_max), behind the C interface.
//
// Rayleigh-Ritz on span(X), standard form (Op = Hs, metric I) or generalised
// (Op = H, metric M with a mass context):
//   S = X^T M X                       Gram product (tall: m rows)
//   d_i = S_ii^{-1/2}, S' = d S d     column equilibration
//   S' = L L^T                        Cholesky (one CTA)
//   A = X^T Op X                      one application + Gram product
//   B = L^{-1} (d A d) L^{-T}         two triangular solves with n right-hand sides
//   B W = W Lam                       symmetric eigensolve (cuSOLVER syevd)
//   E = d L^{-T} W,  X <- X E         back-substitution, tall rotation
// which solves (X^T Op X) E = (X^T M X) E Lam with E^T (X^T M X) E = I.  The
// tall Gram products and the rotation are the only O(m n^2) work: with
// precision FE_KS_F64E they run in the library's pair-of-floats kernels
// (FP64-accurate on the FP32 pipe), with FE_KS_F64 in cuBLAS's native FP64
// GEMM (the plain-FP64 comparator).  Everything n x n is hand-written here,
// except the symmetric eigensolve.
//
// If a Cholesky pivot of S' falls below kCholTol (X is numerically close to
// rank-deficient, as a strongly filtered block can be) the step first
// orthonormalises X by shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa,
// Yamamoto & Yanagisawa, SIAM J. Sci. Comput. 2020: one Cholesky QR pass of
// S + s I with s = 11 (m n + n(n+1)) u ||X||^2, then two plain passes) and
// then does Rayleigh-Ritz on the orthonormal block with one application.
//
// Lanczos: k steps of the symmetric Lanczos recurrence on Hs from a given
// start vector, entirely on the device (the coefficients stay in device
// memory; the dot products are fixed-order two-stage reductions), then the
// host forms the k x k tridiagonal T_k and returns theta_max(T_k) + |beta_k|,
// theta_max by Sturm-sequence bisection.
#include <cusolverDn.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "fe_ks_internal.h"

namespace feks {

constexpr double kCholTol = 1e-10;   // smallest pivot of the equilibrated Gram matrix
constexpr int kRedBlocks = 1024;     // blocks of the fixed-order reductions
constexpr int kRedThreads = 256;
constexpr int kRrMaxN = 4096;

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// ---------------------------------------------------------------- n x n kernels

// Sp[i][j] = S[i][j] / sqrt(S[i][i] S[j][j]) (+ shift on the diagonal); d[i] = S[i][i]^{-1/2}.
// flag <- 1 if a diagonal entry is not positive and finite.
__global__ void k_rr_equilibrate(const double* __restrict__ S, double* __restrict__ Sp, double* __restrict__ d, int n,
                                 double shift, int* __restrict__ flag) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nn; idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    const double si = S[(int64_t)i * n + i], sj = S[(int64_t)j * n + j];
    if (!(si > 0.0) || !(sj > 0.0) || !isfinite(si) || !isfinite(sj)) {
      *flag = 1;
      Sp[idx] = 0.0;
      continue;
    }
    const double di = 1.0 / sqrt(si), dj = 1.0 / sqrt(sj);
    Sp[idx] = (S[idx] * di) * dj + (i == j ? shift : 0.0);
    if (j == 0) d[i] = di;
  }
}

// In-place lower Cholesky factor of the symmetric positive definite A (row-major
// n x n; the lower triangle is read and overwritten, the strict upper triangle
// is zeroed).  One CTA, right-looking: column j is scaled by the pivot's root,
// then the trailing lower triangle takes the rank-1 update.  A pivot <= tol (or
// not finite) sets *flag = 1 + j and stops; every thread reads the same pivot,
// so the exit is uniform.
__global__ void k_rr_cholesky(double* __restrict__ A, int n, double tol, int* __restrict__ flag) {
  for (int j = 0; j < n; ++j) {
    __syncthreads();
    const double piv = A[(int64_t)j * n + j];
    if (!(piv > tol) || !isfinite(piv)) {
      if (threadIdx.x == 0) *flag = 1 + j;
      return;
    }
    const double r = sqrt(piv);
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(int64_t)i * n + j] /= r;
    __syncthreads();
    if (threadIdx.x == 0) A[(int64_t)j * n + j] = r;
    const int w = n - j - 1;
    const int64_t tot = (int64_t)w * w;
    for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) {
      const int i = j + 1 + (int)(t / w), k = j + 1 + (int)(t % w);
      if (k <= i) A[(int64_t)i * n + k] -= A[(int64_t)i * n + j] * A[(int64_t)k * n + j];
    }
  }
  __syncthreads();
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
    const int i = (int)(t / n), k = (int)(t % n);
    if (k > i) A[t] = 0.0;
  }
}

// Solve L Z = B in place (L lower triangular n x n, B row-major [n][nr]); one thread per column of B.
__global__ void k_rr_trsm_lower(const double* __restrict__ L, double* __restrict__ B, int n, int nr) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= nr) return;
  for (int i = 0; i < n; ++i) {
    double s = B[(int64_t)i * nr + col];
    const double* Li = L + (int64_t)i * n;
    for (int k = 0; k < i; ++k) s = fma(-Li[k], B[(int64_t)k * nr + col], s);
    B[(int64_t)i * nr + col] = s / Li[i];
  }
}

// Solve L^T Z = B in place (L lower triangular, so L^T is upper); one thread per column of B.
__global__ void k_rr_trsm_lower_t(const double* __restrict__ L, double* __restrict__ B, int n, int nr) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= nr) return;
  for (int i = n - 1; i >= 0; --i) {
    double s = B[(int64_t)i * nr + col];
    for (int k = i + 1; k < n; ++k) s = fma(-L[(int64_t)k * n + i], B[(int64_t)k * nr + col], s);
    B[(int64_t)i * nr + col] = s / L[(int64_t)i * n + i];
  }
}

// Out[i][j] = rs[i] In[j][i] cs[j] (rs, cs may be nullptr = 1): transposed copy with row / column scaling
__global__ void k_rr_transpose_scale(const double* __restrict__ In, double* __restrict__ Out, int n,
                                     const double* __restrict__ rs, const double* __restrict__ cs) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nn; idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    double v = In[(int64_t)j * n + i];
    if (rs) v *= rs[i];
    if (cs) v *= cs[j];
    Out[idx] = v;
  }
}

// A <- (A + A^T)/2 on the upper triangle mirrored (exactly symmetric result)
__global__ void k_rr_symmetrize(double* __restrict__ A, int n) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nn; idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    if (i < j) {
      const double v = 0.5 * (A[idx] + A[(int64_t)j * n + i]);
      A[idx] = v;
      A[(int64_t)j * n + i] = v;
    }
  }
}

// Out = identity (n x n) scaled row-wise by d (d may be nullptr)
__global__ void k_rr_diag(double* __restrict__ Out, int n, const double* __restrict__ d) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nn; idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    Out[idx] = i == j ? (d ? d[i] : 1.0) : 0.0;
  }
}

// A[i][j] *= d[i]
__global__ void k_rr_row_scale(double* __restrict__ A, int n, const double* __restrict__ d) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nn; idx += (int64_t)gridDim.x * blockDim.x)
    A[idx] *= d[idx / n];
}

// ---------------------------------------------------------------- Lanczos kernels

// part[block] = sum over the block's fixed stride of a[i] b[i]
__global__ void __launch_bounds__(kRedThreads) k_dot_partial(const double* __restrict__ a, const double* __restrict__ b,
                                                             int64_t n, double* __restrict__ part) {
  __shared__ double sh[kRedThreads / 32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < n; i += (int64_t)kRedBlocks * kRedThreads)
    s = fma(a[i], b[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// out = sum of part (sqrt if root); one warp, fixed order
__global__ void k_dot_final(const double* __restrict__ part, double* __restrict__ out, int root) {
  double s = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += 32) s += part[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) *out = root ? sqrt(s) : s;
}

// v = x / *nrm
__global__ void k_scale_by_inv(double* __restrict__ v, const double* __restrict__ x, const double* __restrict__ nrm,
                               int64_t n) {
  const double r = 1.0 / *nrm;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = x[i] * r;
}

// w <- w - alpha v - beta v_prev  (beta == nullptr: no v_prev term)
__global__ void k_lanczos_orth(double* __restrict__ w, const double* __restrict__ v, const double* __restrict__ vp,
                               const double* __restrict__ alpha, const double* __restrict__ beta, int64_t n) {
  const double a = *alpha, b = beta ? *beta : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double x = fma(-a, v[i], w[i]);
    if (beta) x = fma(-b, vp[i], x);
    w[i] = x;
  }
}

static void dot_device(const double* a, const double* b, int64_t n, double* part, double* out, bool root,
                       cudaStream_t s) {
  k_dot_partial<<<kRedBlocks, kRedThreads, 0, s>>>(a, b, n, part);
  k_dot_final<<<1, 32, 0, s>>>(part, out, root ? 1 : 0);
}

// Largest eigenvalue of the symmetric tridiagonal matrix (diag a[0..k-1], off-diagonal b[0..k-2])
// by bisection on the Sturm count (number of eigenvalues below x).
static double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int k = (int)a.size();
  double lo = a[0], hi = a[0];
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(b[i]) : 0.0);
    lo = std::fmin(lo, a[i] - r);
    hi = std::fmax(hi, a[i] + r);
  }
  auto count_below = [&](double x) {
    int c = 0;
    double q = a[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < k; ++i) {
      const double qq = q != 0.0 ? q : 1e-300;
      q = (a[i] - x) - b[i - 1] * b[i - 1] / qq;
      if (q < 0) ++c;
    }
    return c;
  };
  // largest eigenvalue: the point where the count reaches k
  for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (count_below(mid) >= k) hi = mid; else lo = mid;
  }
  return hi;
}

// ---------------------------------------------------------------- cuSOLVER handle per device

static std::mutex g_solver_mu;
static cusolverDnHandle_t g_solver[64] = {};

static fe_ks_status solver_handle(cusolverDnHandle_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return fail(FE_KS_ERR_UNSUPPORTED, "device index beyond 64");
  std::lock_guard<std::mutex> lock(g_solver_mu);
  if (!g_solver[dev] && cusolverDnCreate(&g_solver[dev]) != CUSOLVER_STATUS_SUCCESS)
    return fail(FE_KS_ERR_CUDA, "cusolverDnCreate failed");
  *out = g_solver[dev];
  return FE_KS_OK;
}

// ---------------------------------------------------------------- workspace layout

struct RrWork {
  double* T;       // [m][ncols] application / rotation buffer
  double* part;    // Gram partials (pair-of-floats kernels)
  size_t part_bytes;
  double *S, *Sp, *A, *B, *W, *E, *d, *syev;
  int* flag;
  int* info;
  int lwork;
};

static fe_ks_status rr_layout(const Ctx& c, int64_t n_v, int precision, char* base, size_t* total, RrWork* w) {
  const int64_t ncols = n_v;
  const size_t nn = (size_t)n_v * n_v * 8;
  size_t part = 0;
  if (precision == FE_KS_F64E) {
    fe_ks_status st = fe_ks_gram_tc_workspace(c.m, (int)n_v, &part);   // >= the pair-of-floats kernel's
    if (st != FE_KS_OK) return st;
  }
  cusolverDnHandle_t h;
  fe_ks_status st = solver_handle(&h);
  if (st != FE_KS_OK) return st;
  int lwork = 0;
  if (cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, (int)n_v, nullptr, (int)n_v,
                                  nullptr, &lwork) != CUSOLVER_STATUS_SUCCESS)
    return fail(FE_KS_ERR_CUDA, "cusolverDnDsyevd_bufferSize failed");
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += al256(bytes);
    return p;
  };
  RrWork r{};
  r.T = reinterpret_cast<double*>(take((size_t)c.m * ncols * 8));
  r.part = reinterpret_cast<double*>(take(part > 0 ? part : 8));
  r.part_bytes = part;
  r.S = reinterpret_cast<double*>(take(nn));
  r.Sp = reinterpret_cast<double*>(take(nn));
  r.A = reinterpret_cast<double*>(take(nn));
  r.B = reinterpret_cast<double*>(take(nn));
  r.W = reinterpret_cast<double*>(take(nn));
  r.E = reinterpret_cast<double*>(take(nn));
  r.d = reinterpret_cast<double*>(take((size_t)n_v * 8));
  r.syev = reinterpret_cast<double*>(take((size_t)(lwork > 0 ? lwork : 1) * 8));
  r.flag = reinterpret_cast<int*>(take(256));
  r.info = reinterpret_cast<int*>(take(256));
  r.lwork = lwork;
  *total = off;
  if (w) *w = r;
  return FE_KS_OK;
}

// ---------------------------------------------------------------- tall products

// C[n][n] = Y^T Z (symmetric: one-triangle product).  Pairs plan: the tensor-core Gram,
// checked (one synchronisation) and redone in pairs of floats if its status is not clean.
static fe_ks_status rr_gram(const Ctx& c, int precision, const double* Y, const double* Z, double* C, int n,
                            const RrWork& w) {
  if (precision == FE_KS_F64E) {
    if (c.rr_gram_tc) {
      fe_ks_status st = fe_ks_gram_tc_sym(Y, Z, C, c.m, n, w.part, w.part_bytes, c.stream);
      if (st != FE_KS_OK) return st;
      int status = 0;
      if (cudaStreamSynchronize(c.stream) != cudaSuccess) return fail(FE_KS_ERR_CUDA, "Gram synchronisation");
      st = fe_ks_gram_tc_status(w.part, &status);
      if (st != FE_KS_OK) return st;
      if (status == 0) return FE_KS_OK;
    }
    return fe_ks_gram_ff_sym(Y, Z, C, c.m, n, w.part, w.part_bytes, c.stream);
  }
  // row-major [m][n] is column-major n x m: C = Yc Zc^T
  return fe_ks_gemm_f64(0, 1, n, n, c.m, 1.0, Y, n, Z, n, 0.0, C, n, 0, c.stream);
}

// X[m][n] = Y[m][n] E[n][n]; pairs plan: on the tensor cores (flags in the first bytes of the
// Gram workspace, free at this point), checked and redone in pairs of floats if not clean
static fe_ks_status rr_rotate(const Ctx& c, int precision, const double* Y, const double* E, double* X, int n,
                              const RrWork& w) {
  if (precision == FE_KS_F64E) {
    if (c.rr_gram_tc) {
      int* flags = reinterpret_cast<int*>(w.part);
      fe_ks_status st = fe_ks_rotate_tc(Y, E, X, c.m, n, n, flags, c.stream);
      if (st != FE_KS_OK) return st;
      int f[2] = {0, 0};
      if (cudaMemcpyAsync(f, flags, sizeof(f), cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
          cudaStreamSynchronize(c.stream) != cudaSuccess)
        return fail(FE_KS_ERR_CUDA, "rotation status");
      if (!f[0] && !f[1]) return FE_KS_OK;
    }
    return fe_ks_rotate_ff(Y, E, X, c.m, n, n, c.stream);
  }
  // column-major: Xc (n x m) = Ec (n x n) Yc (n x m), Ec = E^T in memory terms
  return fe_ks_gemm_f64(0, 0, n, c.m, n, 1.0, E, n, Y, n, 0.0, X, n, 0, c.stream);
}

static int small_blocks(int n) {
  const int64_t nn = (int64_t)n * n;
  return (int)std::min<int64_t>((nn + 255) / 256, 152 * 8);
}

static fe_ks_status last_cuda(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return FE_KS_OK;
}

// One Cholesky QR pass in the metric M (mass == nullptr: the identity): Out = Y d L^{-T}
// with d S d + shift I = L L^T, S = Y^T M Y, d = diag(S)^{-1/2}.  M Y is formed in Out
// itself (the Gram product reads it before the rotation overwrites it, in stream order).
// Sets *broke when the factorisation fails.
static fe_ks_status cholqr_pass(Ctx& c, fe_ks_ctx* mass, int precision, const double* Y, double* Out, int n,
                                double shift_rel, const RrWork& w, bool* broke) {
  cudaStream_t s = c.stream;
  const int nb = small_blocks(n);
  const double* MY = Y;
  if (mass) {
    cudaStream_t ms = mass->c.stream;
    mass->c.stream = s;
    fe_ks_status st = fe_ks_apply(mass, Y, Out, n, precision);
    mass->c.stream = ms;
    if (st != FE_KS_OK) return st;
    MY = Out;
  }
  fe_ks_status st = rr_gram(c, precision, Y, MY, w.S, n, w);
  if (st != FE_KS_OK) return st;
  cudaMemsetAsync(w.flag, 0, sizeof(int), s);
  k_rr_equilibrate<<<nb, 256, 0, s>>>(w.S, w.Sp, w.d, n, shift_rel, w.flag);
  k_rr_cholesky<<<1, 1024, 0, s>>>(w.Sp, n, 0.0, w.flag);
  if ((st = last_cuda("Cholesky QR kernels")) != FE_KS_OK) return st;
  int flag = 0;
  cudaMemcpyAsync(&flag, w.flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return last_cuda("Cholesky QR");
  *broke = flag != 0;
  if (*broke) return FE_KS_OK;
  // E = d L^{-T}: L^{-T} by solving with the identity, then its rows scaled by d
  k_rr_diag<<<nb, 256, 0, s>>>(w.E, n, nullptr);
  k_rr_trsm_lower_t<<<(n + 127) / 128, 128, 0, s>>>(w.Sp, w.E, n, n);
  k_rr_row_scale<<<nb, 256, 0, s>>>(w.E, n, w.d);
  if ((st = last_cuda("Cholesky QR triangular solve")) != FE_KS_OK) return st;
  return rr_rotate(c, precision, Y, w.E, Out, n, w);
}

}  // namespace feks

using namespace feks;

extern "C" {

fe_ks_status fe_ks_rayleigh_ritz_workspace(const fe_ks_ctx* ctx, int64_t n_v, int precision, size_t* bytes) {
  set_error("");
  if (!ctx || !bytes) return fail(FE_KS_ERR_ARG, "NULL argument");
  if (precision != FE_KS_F64 && precision != FE_KS_F64E)
    return fail(FE_KS_ERR_ARG, "precision must be FE_KS_F64 or FE_KS_F64E");
  if (ctx->c.cplx) return fail(FE_KS_ERR_UNSUPPORTED, "Rayleigh-Ritz is implemented for real operators");
  if (n_v < 1 || n_v > ctx->c.n_v_max || n_v > kRrMaxN) return fail(FE_KS_ERR_ARG, "n_v out of range");
  return rr_layout(ctx->c, n_v, precision, nullptr, bytes, nullptr);
}

fe_ks_status fe_ks_rayleigh_ritz(fe_ks_ctx* ctx, fe_ks_ctx* mass, double* X, double* ritz, int64_t n_v, int precision,
                                 void* work, size_t work_bytes, int* path) {
  set_error("");
  if (!ctx || !X || !ritz || !work) return fail(FE_KS_ERR_ARG, "NULL argument");
  Ctx& c = ctx->c;
  if (precision != FE_KS_F64 && precision != FE_KS_F64E)
    return fail(FE_KS_ERR_ARG, "precision must be FE_KS_F64 or FE_KS_F64E");
  if (c.cplx) return fail(FE_KS_ERR_UNSUPPORTED, "Rayleigh-Ritz is implemented for real operators");
  if (n_v < 1 || n_v > c.n_v_max || n_v > kRrMaxN) return fail(FE_KS_ERR_ARG, "n_v out of range");
  if (mass && (mass->c.m != c.m || mass->c.cplx || mass->c.n_v_max < n_v || mass->c.device != c.device))
    return fail(FE_KS_ERR_ARG, "the mass context must share the operator's DoFs, type, device and n_v range");
  if (((uintptr_t)work & 255) || ((uintptr_t)X & 7) || ((uintptr_t)ritz & 7))
    return fail(FE_KS_ERR_ARG, "misaligned X, ritz or workspace");
  size_t need = 0;
  RrWork w{};
  fe_ks_status st = rr_layout(c, n_v, precision, static_cast<char*>(work), &need, &w);
  if (st != FE_KS_OK) return st;
  if (work_bytes < need) return fail(FE_KS_ERR_ARG, "workspace too small");
  const size_t xbytes = (size_t)c.m * n_v * 8;
  {
    const char* xb = reinterpret_cast<const char*>(X);
    const char* wb = static_cast<const char*>(work);
    if (xb < wb + work_bytes && wb < xb + xbytes) return fail(FE_KS_ERR_ARG, "X overlaps the workspace");
  }
  NvtxRange range("fe_ks_rayleigh_ritz");
  cudaStream_t s = c.stream;
  const int n = (int)n_v;
  const int nb = small_blocks(n);
  auto apply_op = [&](const double* V, double* Out) -> fe_ks_status {
    return mass ? fe_ks_apply(ctx, V, Out, n_v, precision) : fe_ks_apply_scaled(ctx, V, Out, n_v, precision);
  };
  int used = 0;
  // ---- Cholesky path: S = X^T M X, equilibrate, factor
  bool broke = false;
  {
    const double* MX = X;
    if (mass) {
      cudaStream_t ms = mass->c.stream;
      mass->c.stream = s;
      st = fe_ks_apply(mass, X, w.T, n_v, precision);
      mass->c.stream = ms;
      if (st != FE_KS_OK) return st;
      MX = w.T;
    }
    if ((st = rr_gram(c, precision, X, MX, w.S, n, w)) != FE_KS_OK) return st;
    cudaMemsetAsync(w.flag, 0, sizeof(int), s);
    k_rr_equilibrate<<<nb, 256, 0, s>>>(w.S, w.Sp, w.d, n, 0.0, w.flag);
    k_rr_cholesky<<<1, 1024, 0, s>>>(w.Sp, n, kCholTol, w.flag);
    if ((st = last_cuda("Rayleigh-Ritz Cholesky")) != FE_KS_OK) return st;
    int flag = 0;
    cudaMemcpyAsync(&flag, w.flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return last_cuda("Rayleigh-Ritz");
    broke = flag != 0;
  }
  const double* basis = X;    // the block the projection uses
  if (!broke) {
    // A = X^T Op X, B = L^{-1} (d A d) L^{-T}
    if ((st = apply_op(X, w.T)) != FE_KS_OK) return st;
    if ((st = rr_gram(c, precision, X, w.T, w.A, n, w)) != FE_KS_OK) return st;
    k_rr_transpose_scale<<<nb, 256, 0, s>>>(w.A, w.B, n, w.d, w.d);      // d A^T d = d A d
    k_rr_trsm_lower<<<(n + 127) / 128, 128, 0, s>>>(w.Sp, w.B, n, n);    // Z = L^{-1} d A d
    k_rr_transpose_scale<<<nb, 256, 0, s>>>(w.B, w.W, n, nullptr, nullptr);
    k_rr_trsm_lower<<<(n + 127) / 128, 128, 0, s>>>(w.Sp, w.W, n, n);    // B = L^{-1} Z^T
    k_rr_symmetrize<<<nb, 256, 0, s>>>(w.W, n);
  } else {
    // ---- shifted CholeskyQR3: Q = X R^{-1} orthonormal in the metric, in X's own buffer
    used = 1;
    const double u = 0.5 * 2.220446049250313e-16;
    const double shift = 11.0 * ((double)c.m * n + (double)n * (n + 1)) * u * n;   // ||X d||_F^2 = n
    // pass 1 (shifted): X -> T;  pass 2: T -> X;  pass 3: X -> T; then copy T -> X
    bool b1 = false, b2 = false, b3 = false;
    if ((st = cholqr_pass(c, mass, precision, X, w.T, n, shift, w, &b1)) != FE_KS_OK) return st;
    if (b1) return fail(FE_KS_ERR_ARG, "X is numerically rank-deficient (shifted Cholesky QR failed)");
    if ((st = cholqr_pass(c, mass, precision, w.T, X, n, 0.0, w, &b2)) != FE_KS_OK) return st;
    if (b2) return fail(FE_KS_ERR_ARG, "X is numerically rank-deficient (Cholesky QR, second pass)");
    if ((st = cholqr_pass(c, mass, precision, X, w.T, n, 0.0, w, &b3)) != FE_KS_OK) return st;
    if (b3) return fail(FE_KS_ERR_ARG, "X is numerically rank-deficient (Cholesky QR, third pass)");
    cudaMemcpyAsync(X, w.T, xbytes, cudaMemcpyDeviceToDevice, s);
    // B = Q^T Op Q directly (Q orthonormal in the metric: Q^T M Q = I)
    if ((st = apply_op(X, w.T)) != FE_KS_OK) return st;
    if ((st = rr_gram(c, precision, X, w.T, w.W, n, w)) != FE_KS_OK) return st;
    k_rr_symmetrize<<<nb, 256, 0, s>>>(w.W, n);
    basis = X;
  }
  if ((st = last_cuda("Rayleigh-Ritz projection")) != FE_KS_OK) return st;
  // B W = W Lam (cuSOLVER, in place: eigenvectors as columns of the column-major result)
  cusolverDnHandle_t h;
  if ((st = solver_handle(&h)) != FE_KS_OK) return st;
  cusolverDnSetStream(h, s);
  if (cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, w.W, n, ritz, w.syev, w.lwork,
                       w.info) != CUSOLVER_STATUS_SUCCESS)
    return fail(FE_KS_ERR_CUDA, "cusolverDnDsyevd failed");
  // row-major eigenvector matrix E[i][j] = component i of vector j = transpose of the column-major result
  k_rr_transpose_scale<<<nb, 256, 0, s>>>(w.W, w.E, n, nullptr, nullptr);
  if (!broke) {
    k_rr_trsm_lower_t<<<(n + 127) / 128, 128, 0, s>>>(w.Sp, w.E, n, n);   // L^{-T} W
    k_rr_row_scale<<<nb, 256, 0, s>>>(w.E, n, w.d);                        // d L^{-T} W
  }
  if ((st = last_cuda("Rayleigh-Ritz back-substitution")) != FE_KS_OK) return st;
  if ((st = rr_rotate(c, precision, basis, w.E, w.T, n, w)) != FE_KS_OK) return st;
  cudaMemcpyAsync(X, w.T, xbytes, cudaMemcpyDeviceToDevice, s);
  int info = 0;
  cudaMemcpyAsync(&info, w.info, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return last_cuda("Rayleigh-Ritz");
  if (info != 0) return fail(FE_KS_ERR_CUDA, "the projected eigensolve did not converge (syevd info " +
                                                 std::to_string(info) + ")");
  if (path) *path = used;
  return FE_KS_OK;
}

fe_ks_status fe_ks_set_rr_gram(fe_ks_ctx* ctx, int tensor_cores) {
  set_error("");
  if (!ctx) return fail(FE_KS_ERR_ARG, "ctx is NULL");
  ctx->c.rr_gram_tc = tensor_cores ? 1 : 0;
  return FE_KS_OK;
}

fe_ks_status fe_ks_lanczos_bound_workspace(const fe_ks_ctx* ctx, int steps, size_t* bytes) {
  set_error("");
  if (!ctx || !bytes) return fail(FE_KS_ERR_ARG, "NULL argument");
  if (steps < 1 || steps > 1000) return fail(FE_KS_ERR_ARG, "steps must be in 1..1000");
  const size_t vb = al256((size_t)ctx->c.m * (ctx->c.cplx ? 2 : 1) * 8);
  *bytes = 3 * vb + al256((size_t)kRedBlocks * 8) + 2 * al256((size_t)(steps + 1) * 8);
  return FE_KS_OK;
}

fe_ks_status fe_ks_lanczos_bound(fe_ks_ctx* ctx, const double* v0, int steps, int precision, void* work,
                                 size_t work_bytes, double* lam_max, double* alpha, double* beta, int* steps_done) {
  set_error("");
  if (!ctx || !v0 || !work || !lam_max) return fail(FE_KS_ERR_ARG, "NULL argument");
  if (precision != FE_KS_F64 && precision != FE_KS_F64E)
    return fail(FE_KS_ERR_ARG, "precision must be FE_KS_F64 or FE_KS_F64E");
  size_t need = 0;
  fe_ks_status st = fe_ks_lanczos_bound_workspace(ctx, steps, &need);
  if (st != FE_KS_OK) return st;
  if (work_bytes < need) return fail(FE_KS_ERR_ARG, "workspace too small");
  if (((uintptr_t)work & 255) || ((uintptr_t)v0 & 7)) return fail(FE_KS_ERR_ARG, "misaligned v0 or workspace");
  Ctx& c = ctx->c;
  NvtxRange range("fe_ks_lanczos_bound");
  cudaStream_t s = c.stream;
  const int64_t n = c.m * (c.cplx ? 2 : 1);   // complex: Re(v^H w) is the real dot product of the interleaved arrays
  const size_t vb = al256((size_t)n * 8);
  char* base = static_cast<char*>(work);
  double* v = reinterpret_cast<double*>(base);
  double* vp = reinterpret_cast<double*>(base + vb);
  double* wv = reinterpret_cast<double*>(base + 2 * vb);
  double* part = reinterpret_cast<double*>(base + 3 * vb);
  double* dal = reinterpret_cast<double*>(base + 3 * vb + al256((size_t)kRedBlocks * 8));
  double* dbe = reinterpret_cast<double*>(base + 3 * vb + al256((size_t)kRedBlocks * 8) + al256((size_t)(steps + 1) * 8));
  {
    const char* vb0 = reinterpret_cast<const char*>(v0);
    if (vb0 < base + need && base < vb0 + n * 8) return fail(FE_KS_ERR_ARG, "v0 overlaps the workspace");
  }
  const int ew = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  // v = v0 / |v0|  (the norm goes to beta[steps] as scratch)
  dot_device(v0, v0, n, part, dbe + steps, true, s);
  k_scale_by_inv<<<ew, 256, 0, s>>>(v, v0, dbe + steps, n);
  for (int i = 0; i < steps; ++i) {
    st = fe_ks_apply_scaled(ctx, v, wv, 1, precision);
    if (st != FE_KS_OK) return st;
    dot_device(v, wv, n, part, dal + i, false, s);
    k_lanczos_orth<<<ew, 256, 0, s>>>(wv, v, vp, dal + i, i > 0 ? dbe + i - 1 : nullptr, n);
    dot_device(wv, wv, n, part, dbe + i, true, s);
    std::swap(v, vp);                                        // vp <- v (old)
    k_scale_by_inv<<<ew, 256, 0, s>>>(v, wv, dbe + i, n);    // v <- w / beta
  }
  if ((st = last_cuda("Lanczos kernels")) != FE_KS_OK) return st;
  std::vector<double> a(steps), b(steps);
  cudaMemcpyAsync(a.data(), dal, steps * 8, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(b.data(), dbe, steps * 8, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return last_cuda("Lanczos");
  // stop at the first exactly vanishing beta (an invariant subspace), as the recurrence would
  int k = steps;
  for (int i = 0; i < steps; ++i)
    if (b[i] == 0.0) {
      k = i + 1;
      break;
    }
  for (int i = 0; i < k; ++i)
    if (!std::isfinite(a[i]) || !std::isfinite(b[i])) return fail(FE_KS_ERR_ARG, "Lanczos produced a non-finite coefficient");
  std::vector<double> aa(a.begin(), a.begin() + k), bb(b.begin(), b.begin() + (k > 1 ? k - 1 : 0));
  *lam_max = tridiag_max_eig(aa, bb) + std::fabs(b[k - 1]);
  if (alpha) for (int i = 0; i < k; ++i) alpha[i] = a[i];
  if (beta) for (int i = 0; i < k; ++i) beta[i] = b[i];
  if (steps_done) *steps_done = k;
  return FE_KS_OK;
}

}  // extern "C"
