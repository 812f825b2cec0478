// Residual-based Chebyshev filter (R-ChFSI, Algorithm 4) on the standard form
// Hs = D^{-1/2} H D^{-1/2} (D = GLL-lumped mass, so D -> I and M -> I):
//
//   Y   = Hs X - X Lam                          (FP64: residual)
//   R_X = 0, R_Y = (s1/e) Y, Lam_X = 1, Lam_Y = (s1/e)(Lam - c)
//   k = 2..m: s2 = 1/(gamma - s)
//       R_X   <- (2 s2/e) [ (Hs - c) R_Y + Y Lam_Y ] - s s2 R_X   (precision of the call)
//       Lam_X <- (2 s2/e) Lam_Y (Lam - c) - s s2 Lam_X
//       swap(R_X, R_Y), swap(Lam_X, Lam_Y), s = s2
//   X   <- R_Y + X Lam_Y                        (FP64)
//
// The recurrence term (Hs - c) R_Y + Y Lam_Y is formed by first writing
// a(-c R_Y + Y Lam_Y) - b R_X in place into R_X (elementwise kernel) and then
// letting the fused cell kernel scatter-add a * Hs R_Y on top (alpha = a).
//
// Generalised form (H X = M X Lam with the consistent mass M, Algorithm 4 as
// printed): with R~ = D^{-1/2} R the recurrence (H D^{-1} - c) R_Y + Y Lam_Y
// is the standard-form one above on R~, so only the two ends change:
//   Y~  = D^{-1/2} (H X - M X Lam)              (FP64: residual with M)
//   X   <- D^{-1/2} R~_Y + X Lam_Y               (D^{-1} R_Y + X Lam_Y)
#include <cmath>
#include <type_traits>

#include "fe_ks_internal.h"

namespace feks {

constexpr int kEwThreads = 256;

static int ew_blocks(int64_t n) {
  int64_t b = (n + kEwThreads - 1) / kEwThreads;
  return (int)(b < 152 * 16 ? b : 152 * 16);
}

// Y = -X * lam[col / cw]   (so that a later accumulate-apply gives Hs X - X Lam)
__global__ void k_residual_init(double* __restrict__ Y, const double* __restrict__ X, const double* __restrict__ lam,
                                int64_t n, int64_t ncols, int cw) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = i % ncols;
    Y[i] = -X[i] * lam[col / cw];
  }
}

// Y <- -Y * lam[col / cw]
__global__ void k_scale_neg_lam(double* __restrict__ Y, const double* __restrict__ lam, int64_t n, int64_t ncols,
                                int cw) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Y[i] = -Y[i] * lam[(i % ncols) / cw];
}

// Y <- D^{-1/2} Y (row scaling)
__global__ void k_row_scale(double* __restrict__ Y, const double* __restrict__ ds, int64_t n, int64_t ncols) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Y[i] *= ds[i / ncols];
}

// Ylow = Y, R_Y = s1e * Y (in the precision of the recurrence)
template <typename T>
__global__ void k_residual_split(const double* __restrict__ Y, T* __restrict__ Yl, T* __restrict__ RY, double s1e,
                                 int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double y = Y[i];
    if (Yl != nullptr) Yl[i] = (T)y;
    RY[i] = (T)(s1e * y);
  }
}

// R_X <- a (-c R_Y + Y Lam_Y) - b R_X   (b == 0: R_X is not read)
template <typename T>
__global__ void k_cheb_prologue(T* __restrict__ RX, const T* __restrict__ RY, const T* __restrict__ Yl,
                                const double* __restrict__ LY, T a, T c, T b, int64_t n, int64_t ncols, int cw) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = i % ncols;
    const T ly = (T)LY[col / cw];
    T v = a * fma(Yl[i], ly, -c * RY[i]);
    if (b != T(0)) v = fma(-b, RX[i], v);
    RX[i] = v;
  }
}

// Lam_X <- a Lam_Y (lam - c) - b Lam_X ; init: Lam_X = 1, Lam_Y = s1e (lam - c)
__global__ void k_lambda(double* LX, double* LY, const double* lam, double a, double c, double b, int init, int n_v) {
  for (int j = threadIdx.x + blockIdx.x * blockDim.x; j < n_v; j += blockDim.x * gridDim.x) {
    if (init) {
      LX[j] = 1.0;
      LY[j] = a * (lam[j] - c);
    } else {
      LX[j] = a * LY[j] * (lam[j] - c) - b * LX[j];
    }
  }
}

// X <- D^{-1/2} R_Y + X Lam_Y (ds == nullptr: X <- R_Y + X Lam_Y)
template <typename T>
__global__ void k_cheb_final(double* __restrict__ X, const T* __restrict__ RY, const double* __restrict__ LY,
                             const double* __restrict__ ds, int64_t n, int64_t ncols, int cw) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = i % ncols;
    const double r = ds ? (double)RY[i] * ds[i / ncols] : (double)RY[i];
    X[i] = r + X[i] * LY[col / cw];
  }
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static size_t filter_bytes(const Ctx& c, int64_t n_v, int precision) {
  const size_t n = (size_t)c.m * n_v * (c.cplx ? 2 : 1);
  const bool low = precision == FE_KS_F32;
  const size_t lo = low ? 4 : 8;
  size_t b = align256(n * 8);                    // Y (FP64 residual)
  if (low) b += align256(n * lo);                // Y in the recurrence precision
  b += 2 * align256(n * lo);                     // R_X, R_Y
  b += 2 * align256((size_t)n_v * 8);            // Lam_X, Lam_Y
  return b;
}

// Recurrence application a * Hs R_Y accumulated into R_X, in the recurrence's arithmetic.
// emu: pair-of-floats kernel (T = double); tc: tensor-core kernel (T = float; 1 BF16, 2 FP16).
template <typename T>
static fe_ks_status recurrence_apply(Ctx& c, const T* RY, T* RX, int64_t ncols, double a, bool emu, int tc) {
  if constexpr (std::is_same<T, double>::value) {
    if (emu) return apply_core_emu(c, RY, RX, ncols, true, a, false);
  }
  return apply_core<T>(c, RY, RX, ncols, true, (T)a, false, tc);
}

template <typename T>
static fe_ks_status cheb_impl(Ctx& c, double* X, const double* lam, int64_t n_v, int degree, double lmin, double lT,
                              double lmax, char* work, bool rec_emu, bool res_emu, int rec_tc = 0,
                              Ctx* mass = nullptr) {
  NvtxRange range(mass ? "fe_ks_cheb_filter_ghep" : "fe_ks_cheb_filter");
  cudaStream_t s = c.stream;
  const int cw = c.cplx ? 2 : 1;
  const int64_t ncols = n_v * cw;
  const int64_t n = c.m * ncols;
  const bool low = sizeof(T) != 8;
  size_t off = 0;
  double* Y = reinterpret_cast<double*>(work + off);
  off += align256(n * 8);
  T* Yl = low ? reinterpret_cast<T*>(work + off) : reinterpret_cast<T*>(Y);
  if (low) off += align256(n * sizeof(T));
  T* RX = reinterpret_cast<T*>(work + off);
  off += align256(n * sizeof(T));
  T* RY = reinterpret_cast<T*>(work + off);
  off += align256(n * sizeof(T));
  double* LX = reinterpret_cast<double*>(work + off);
  off += align256(n_v * 8);
  double* LY = reinterpret_cast<double*>(work + off);

  const double e = 0.5 * (lmax - lT), cc = 0.5 * (lmax + lT);
  double sigma = e / (lmin - cc);
  const double sigma1 = sigma, gamma = 2.0 / sigma1;
  const int nb = ew_blocks(n);

  fe_ks_status st = FE_KS_OK;
  if (!mass) {
    // Y = Hs X - X Lam (FP64)
    k_residual_init<<<nb, kEwThreads, 0, s>>>(Y, X, lam, n, ncols, cw);
    st = res_emu ? apply_core_emu(c, X, Y, ncols, true, 1.0, false)
                 : apply_core<double>(c, X, Y, ncols, true, 1.0, false);
    if (st != FE_KS_OK) return st;
  } else {
    // Y~ = D^{-1/2} (H X - M X Lam) (FP64): M X on the mass context's stream
    // order (same stream), then -Lam, then + H X, then the row scaling
    cudaStream_t ms = mass->stream;
    mass->stream = s;
    st = res_emu ? apply_core_emu(*mass, X, Y, ncols, false, 1.0, true)
                 : apply_core<double>(*mass, X, Y, ncols, false, 1.0, true);
    mass->stream = ms;
    if (st != FE_KS_OK) return st;
    k_scale_neg_lam<<<nb, kEwThreads, 0, s>>>(Y, lam, n, ncols, cw);
    st = res_emu ? apply_core_emu(c, X, Y, ncols, false, 1.0, false)
                 : apply_core<double>(c, X, Y, ncols, false, 1.0, false);
    if (st != FE_KS_OK) return st;
    k_row_scale<<<nb, kEwThreads, 0, s>>>(Y, c.f64.dscale, n, ncols);
  }
  k_residual_split<T><<<nb, kEwThreads, 0, s>>>(Y, low ? Yl : nullptr, RY, sigma1 / e, n);
  k_lambda<<<(int)((n_v + 255) / 256), 256, 0, s>>>(LX, LY, lam, sigma1 / e, cc, 0.0, 1, (int)n_v);
  for (int k = 2; k <= degree; ++k) {
    const double sigma2 = 1.0 / (gamma - sigma);
    const double a = 2.0 * sigma2 / e, b = (k == 2) ? 0.0 : sigma * sigma2;
    k_cheb_prologue<T><<<nb, kEwThreads, 0, s>>>(RX, RY, Yl, LY, (T)a, (T)cc, (T)b, n, ncols, cw);
    st = recurrence_apply<T>(c, RY, RX, ncols, a, rec_emu, rec_tc);
    if (st != FE_KS_OK) return st;
    k_lambda<<<(int)((n_v + 255) / 256), 256, 0, s>>>(LX, LY, lam, a, cc, sigma * sigma2, 0, (int)n_v);
    std::swap(RX, RY);
    std::swap(LX, LY);
    sigma = sigma2;
  }
  k_cheb_final<T><<<nb, kEwThreads, 0, s>>>(X, RY, LY, mass ? c.f64.dscale : nullptr, n, ncols, cw);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("filter kernels: ") + cudaGetErrorString(err));
  return FE_KS_OK;
}

}  // namespace feks

using namespace feks;

extern "C" {

fe_ks_status fe_ks_cheb_filter_workspace(const fe_ks_ctx* ctx, int64_t n_v, int precision, size_t* bytes) {
  if (!ctx || !bytes) return fail(FE_KS_ERR_ARG, "NULL argument");
  if (precision != FE_KS_F64 && precision != FE_KS_F32 && precision != FE_KS_F64E && precision != FE_KS_BF16 &&
      precision != FE_KS_F16 && precision != FE_KS_BF16X2)
    return fail(FE_KS_ERR_UNSUPPORTED, "unknown precision");
  *bytes = filter_bytes(ctx->c, n_v, (precision == FE_KS_BF16 || precision == FE_KS_F16 || precision == FE_KS_BF16X2) ? FE_KS_F32 : precision);
  return FE_KS_OK;
}

static fe_ks_status filter_entry(fe_ks_ctx* ctx, fe_ks_ctx* mass, double* X, const double* ritz, int64_t n_v,
                                 int degree, double lam_min, double lam_T, double lam_max, int precision,
                                 int residual_precision, void* work, size_t work_bytes) {
  set_error("");
  if (!ctx || !X || !ritz || !work) return fail(FE_KS_ERR_ARG, "NULL argument");
  Ctx& c = ctx->c;
  if (n_v < 1 || n_v > c.n_v_max) return fail(FE_KS_ERR_ARG, "n_v must be in 1..n_v_max");
  if (mass && (mass->c.m != c.m || mass->c.cplx != c.cplx || mass->c.n_v_max < n_v || mass->c.device != c.device))
    return fail(FE_KS_ERR_ARG, "the mass context must share the operator's DoFs, type, device and n_v range");
  if (degree < 1) return fail(FE_KS_ERR_ARG, "degree must be >= 1");
  if (!(lam_min < lam_T && lam_T < lam_max)) return fail(FE_KS_ERR_ARG, "need lam_min < lam_T < lam_max");
  if (precision != FE_KS_F64 && precision != FE_KS_F32 && precision != FE_KS_F64E && precision != FE_KS_BF16 &&
      precision != FE_KS_F16 && precision != FE_KS_BF16X2)
    return fail(FE_KS_ERR_UNSUPPORTED, "unknown precision");
  if (residual_precision != FE_KS_F64 && residual_precision != FE_KS_F64E)
    return fail(FE_KS_ERR_ARG, "residual_precision must be FE_KS_F64 or FE_KS_F64E");
  if (work_bytes < filter_bytes(c, n_v, (precision == FE_KS_BF16 || precision == FE_KS_F16 || precision == FE_KS_BF16X2) ? FE_KS_F32 : precision))
    return fail(FE_KS_ERR_ARG, "workspace too small");
  if (((uintptr_t)work & 255) || ((uintptr_t)X & 7)) return fail(FE_KS_ERR_ARG, "misaligned X or workspace");
  char* w = static_cast<char*>(work);
  const bool res_emu = residual_precision == FE_KS_F64E;
  Ctx* mc = mass ? &mass->c : nullptr;
  if (precision == FE_KS_F32 || precision == FE_KS_BF16 || precision == FE_KS_F16 || precision == FE_KS_BF16X2)
    return cheb_impl<float>(c, X, ritz, n_v, degree, lam_min, lam_T, lam_max, w, false, res_emu,
                            precision == FE_KS_BF16    ? 1
                            : precision == FE_KS_F16   ? 2
                            : precision == FE_KS_BF16X2 ? 3
                                                        : 0,
                            mc);
  return cheb_impl<double>(c, X, ritz, n_v, degree, lam_min, lam_T, lam_max, w, precision == FE_KS_F64E, res_emu, 0,
                           mc);
}

fe_ks_status fe_ks_cheb_filter(fe_ks_ctx* ctx, double* X, const double* ritz, int64_t n_v, int degree, double lam_min,
                               double lam_T, double lam_max, int precision, int residual_precision, void* work,
                               size_t work_bytes) {
  return filter_entry(ctx, nullptr, X, ritz, n_v, degree, lam_min, lam_T, lam_max, precision, residual_precision,
                      work, work_bytes);
}

fe_ks_status fe_ks_cheb_filter_ghep(fe_ks_ctx* ctx, fe_ks_ctx* mass, double* X, const double* ritz, int64_t n_v,
                                    int degree, double lam_min, double lam_T, double lam_max, int precision,
                                    int residual_precision, void* work, size_t work_bytes) {
  if (!mass) return fail(FE_KS_ERR_ARG, "mass context is NULL");
  return filter_entry(ctx, mass, X, ritz, n_v, degree, lam_min, lam_T, lam_max, precision, residual_precision, work,
                      work_bytes);
}

}  // extern "C"
