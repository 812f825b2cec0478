// C-ABI of libfe_ks: setup (tables, geometry, projector matrices, colouring,
// workspace) and the stream-ordered application Y = H X (eq. HX).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>
#include <functional>
#include <thread>
#include <type_traits>

#include <map>
#include <mutex>
#include <tuple>

#include <nvtx3/nvToolsExt.h>

#include "fe_ks_internal.h"

namespace feks {

template <typename T, typename TS, int P, int NQX>
cudaError_t launch_local_deg(const Ctx&, const LocalParams<T, TS>&, cudaStream_t);

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

fe_ks_status fail(fe_ks_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

// n_q - n_p = NQX: 0 (the square rule) or 2 (the paper's default for accurate
// V_loc and V^G integrals, Sec. 6)
template <typename T, typename TS, int NQX>
static cudaError_t launch_local_nq(const Ctx& c, const LocalParams<T, TS>& prm, cudaStream_t s) {
  switch (c.p) {
    case 1: return launch_local_deg<T, TS, 1, NQX>(c, prm, s);
    case 2: return launch_local_deg<T, TS, 2, NQX>(c, prm, s);
    case 3: return launch_local_deg<T, TS, 3, NQX>(c, prm, s);
    case 4: return launch_local_deg<T, TS, 4, NQX>(c, prm, s);
    case 5: return launch_local_deg<T, TS, 5, NQX>(c, prm, s);
    case 6: return launch_local_deg<T, TS, 6, NQX>(c, prm, s);
    case 7: return launch_local_deg<T, TS, 7, NQX>(c, prm, s);
    case 8: return launch_local_deg<T, TS, 8, NQX>(c, prm, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, typename TS>
cudaError_t launch_local(const Ctx& c, const LocalParams<T, TS>& prm, cudaStream_t s) {
  if (c.nq == c.np) return launch_local_nq<T, TS, 0>(c, prm, s);
  if (c.nq == c.np + 2) return launch_local_nq<T, TS, 2>(c, prm, s);
  return cudaErrorInvalidValue;
}

// used from other translation units (the cell-matrix baseline's setup)
template cudaError_t launch_local<double, double>(const Ctx&, const LocalParams<double, double>&, cudaStream_t);
template cudaError_t launch_local<float, float>(const Ctx&, const LocalParams<float, float>&, cudaStream_t);

// Run body(i) for i in [0, n) on all host cores.
static void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& body) {
  unsigned nt = std::max(1u, std::thread::hardware_concurrency());
  if (n < 64 || nt == 1) {
    body(0, n);
    return;
  }
  nt = (unsigned)std::min<int64_t>(nt, n);
  std::vector<std::thread> th;
  const int64_t chunk = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    const int64_t b = t * chunk, e = std::min(n, b + chunk);
    if (b < e) th.emplace_back(body, b, e);
  }
  for (auto& x : th) x.join();
}

// Trilinear cell map: position x(xi) and Jacobian J[c][d] = dx_c / dxi_d.
static void trilinear(const double* V, const double xi[3], double x[3], double J[3][3]) {
  for (int c = 0; c < 3; ++c) {
    x[c] = 0.0;
    for (int d = 0; d < 3; ++d) J[c][d] = 0.0;
  }
  for (int v = 0; v < 8; ++v) {
    const double s[3] = {double(2 * (v & 1) - 1), double(2 * ((v >> 1) & 1) - 1), double(2 * ((v >> 2) & 1) - 1)};
    const double f[3] = {0.5 * (1.0 + s[0] * xi[0]), 0.5 * (1.0 + s[1] * xi[1]), 0.5 * (1.0 + s[2] * xi[2])};
    const double phi = f[0] * f[1] * f[2];
    const double dphi[3] = {0.5 * s[0] * f[1] * f[2], 0.5 * s[1] * f[0] * f[2], 0.5 * s[2] * f[0] * f[1]};
    for (int c = 0; c < 3; ++c) {
      x[c] += phi * V[3 * v + c];
      for (int d = 0; d < 3; ++d) J[c][d] += V[3 * v + c] * dphi[d];
    }
  }
}

static double inverse3(const double J[3][3], double Ji[3][3]) {
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  const double r = 1.0 / det;
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * r;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * r;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * r;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * r;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * r;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * r;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * r;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * r;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * r;
  return det;
}

template <typename T>
static fe_ks_status upload(Ctx* c, T** dst, const T* src, size_t count) {
  if (count == 0) {
    *dst = nullptr;
    return FE_KS_OK;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(FE_KS_ERR_OOM, "cudaMalloc failed during setup");
  }
  c->allocations.push_back(p);
  *dst = static_cast<T*>(p);
  if (src && cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(FE_KS_ERR_CUDA, "cudaMemcpy failed during setup");
  return FE_KS_OK;
}

// Greedy colouring of the cells so that no two cells of a colour share a DoF
// (their scatter-adds then never touch the same row of Y).  Cells are taken
// in index order; each gets the smallest colour not used by a cell sharing
// one of its DoFs.  Returns the number of colours, or -1 if more than 64 are
// needed.  cell_dofs entries must lie in [0, m).
int greedy_colouring(int64_t E, int np3, int64_t m, const int* cell_dofs, int* colour) {
  for (int64_t e = 0; e < E; ++e) colour[e] = -1;
  std::vector<int> cnt(m + 1, 0);
  for (int64_t i = 0; i < E * np3; ++i) cnt[cell_dofs[i] + 1]++;
  for (int64_t i = 0; i < m; ++i) cnt[i + 1] += cnt[i];
  std::vector<int> d2c(cnt[m]);
  std::vector<int> fillp(cnt.begin(), cnt.end() - 1);
  for (int64_t e = 0; e < E; ++e)
    for (int n = 0; n < np3; ++n) d2c[fillp[cell_dofs[e * np3 + n]]++] = (int)e;
  int n_colours = 0;
  for (int64_t e = 0; e < E; ++e) {
    uint64_t used = 0;
    for (int n = 0; n < np3; ++n) {
      const int d = cell_dofs[e * np3 + n];
      for (int t = cnt[d]; t < cnt[d + 1]; ++t) {
        const int o = colour[d2c[t]];
        if (o >= 0 && o < 64) used |= (1ull << o);
      }
    }
    int col = 0;
    while (col < 64 && (used >> col) & 1ull) ++col;
    if (col >= 64) return -1;
    colour[e] = col;
    n_colours = std::max(n_colours, col + 1);
  }
  return n_colours;
}

// ---- tile-configuration cache: fe_ks_tune's choice per (degree, n_q,
// precision, columns, complex, device), reused by contexts of the same shape
// whose configuration was not set explicitly.
namespace {
struct TuneKey {
  int p, nq, prec, cplx, sm_major, sm_minor, sms;
  int64_t ncols;
  bool operator<(const TuneKey& o) const {
    return std::tie(p, nq, prec, cplx, sm_major, sm_minor, sms, ncols) <
           std::tie(o.p, o.nq, o.prec, o.cplx, o.sm_major, o.sm_minor, o.sms, o.ncols);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune_cache;

TuneKey tune_key(const Ctx& c, int prec, int64_t ncols) {
  TuneKey k{c.p, c.nq, prec, c.cplx, 0, 0, 0, ncols};
  cudaDeviceGetAttribute(&k.sm_major, cudaDevAttrComputeCapabilityMajor, c.device);
  cudaDeviceGetAttribute(&k.sm_minor, cudaDevAttrComputeCapabilityMinor, c.device);
  cudaDeviceGetAttribute(&k.sms, cudaDevAttrMultiProcessorCount, c.device);
  return k;
}
}  // namespace

int* config_slot(Ctx& c, int prec) {
  return prec == FE_KS_F64    ? &c.cfg64
         : prec == FE_KS_F32  ? &c.cfg32
         : prec == FE_KS_F64E ? &c.cfgE
         : prec == FE_KS_BF16 ? &c.cfg_tc[0]
         : prec == FE_KS_F16  ? &c.cfg_tc[1]
                              : nullptr;
}

// tile configurations of a precision: 10 for the CUDA-core kernels; the BF16 and
// FP16 cell kernels have four (1 = warp-level MMA; 0, 2, 3 = tcgen05 with its two
// pipelines staggered by a point of the tile) where the tcgen05 kernel serves the
// context (real, n_q = n_p), else one
static int n_configs(const Ctx& c, int prec) {
  if (prec == FE_KS_F64 || prec == FE_KS_F32 || prec == FE_KS_F64E) return kLocalConfigs;
  if (prec == FE_KS_BF16 || prec == FE_KS_F16) return (!c.cplx && c.nq == c.np && c.tc5_cst) ? 4 : 1;
  return 1;
}

void tune_cache_store(const Ctx& c, int prec, int64_t ncols, int cfg) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[tune_key(c, prec, ncols)] = cfg;
}

// the cached configuration for this shape, unless the context's was set explicitly
void tune_cache_apply(Ctx& c, int prec, int64_t ncols) {
  int* slot = config_slot(c, prec);
  if (!slot || c.cfg_explicit[prec]) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune_cache.find(tune_key(c, prec, ncols));
  if (it != g_tune_cache.end()) *slot = it->second;
}

static fe_ks_status check_geometry_args(const fe_ks_problem* prob) {
  if (!prob) return fail(FE_KS_ERR_ARG, "problem is NULL");
  if (prob->degree < 1 || prob->degree > 8)
    return fail(FE_KS_ERR_UNSUPPORTED, "degree must be in 1..8");
  if (prob->n_q != prob->degree + 1 && prob->n_q != prob->degree + 3)
    return fail(FE_KS_ERR_UNSUPPORTED, "n_q must be n_p or n_p + 2 (degree + 1 or degree + 3)");
  if (prob->n_cells <= 0 || prob->n_cells > (int64_t)INT32_MAX)
    return fail(FE_KS_ERR_ARG, "n_cells out of range");
  if (!prob->cell_vertices) return fail(FE_KS_ERR_ARG, "cell_vertices is NULL");
  return FE_KS_OK;
}

}  // namespace feks

using namespace feks;

extern "C" {

const char* fe_ks_last_error(void) { return g_last_error.c_str(); }

fe_ks_status fe_ks_quadrature_points(const fe_ks_problem* prob, double* xq_out) {
  g_last_error.clear();
  fe_ks_status st = check_geometry_args(prob);
  if (st != FE_KS_OK) return st;
  if (!xq_out) return fail(FE_KS_ERR_ARG, "xq_out is NULL");
  const int nq = prob->n_q, nq3 = nq * nq * nq;
  double xg[kMaxN], wg[kMaxN];
  gauss_legendre(nq, xg, wg);
  parallel_for(prob->n_cells, [&](int64_t b, int64_t e) {
    for (int64_t c = b; c < e; ++c) {
      const double* V = prob->cell_vertices + 24 * c;
      for (int q = 0; q < nq3; ++q) {
        const double xi[3] = {xg[q % nq], xg[(q / nq) % nq], xg[q / (nq * nq)]};
        double x[3], J[3][3];
        trilinear(V, xi, x, J);
        for (int d = 0; d < 3; ++d) xq_out[(c * nq3 + q) * 3 + d] = x[d];
      }
    }
  });
  return FE_KS_OK;
}

fe_ks_status fe_ks_setup(const fe_ks_problem* prob, int terms_mask, int64_t n_v_max, void* cuda_stream,
                         fe_ks_ctx** out) {
  g_last_error.clear();
  if (!out) return fail(FE_KS_ERR_ARG, "out is NULL");
  *out = nullptr;
  fe_ks_status st = check_geometry_args(prob);
  if (st != FE_KS_OK) return st;
  if (!prob->cell_dofs) return fail(FE_KS_ERR_ARG, "cell_dofs is NULL");
  if (n_v_max < 1) return fail(FE_KS_ERR_ARG, "n_v_max must be >= 1");
  if (prob->n_dofs < 1 || prob->n_dofs > (int64_t)INT32_MAX) return fail(FE_KS_ERR_ARG, "n_dofs out of range");
  if ((terms_mask & FE_KS_TERM_L) && !prob->v_loc_q) return fail(FE_KS_ERR_ARG, "v_loc_q is NULL");
  if (terms_mask & ~FE_KS_TERM_ALL) return fail(FE_KS_ERR_ARG, "unknown bits in terms_mask");
  const bool want_nl = (terms_mask & FE_KS_TERM_NL) && prob->n_atoms > 0;
  if (want_nl) {
    if (prob->n_proj < 1 || prob->n_proj > 16) return fail(FE_KS_ERR_UNSUPPORTED, "n_proj must be in 1..16");
    if (!prob->atom_cell_ptr || !prob->atom_cells || !prob->image_shift || !prob->chi_q || !prob->h_coef)
      return fail(FE_KS_ERR_ARG, "nonlocal arrays are NULL");
  }
  if (prob->n_atoms < 0) return fail(FE_KS_ERR_ARG, "n_atoms < 0");

  auto* h = new fe_ks_ctx();
  Ctx* c = &h->c;
  c->p = prob->degree;
  c->np = prob->degree + 1;
  c->nq = prob->n_q;
  c->np3 = c->np * c->np * c->np;
  c->nq3 = c->nq * c->nq * c->nq;
  c->E = prob->n_cells;
  c->m = prob->n_dofs;
  c->n_v_max = n_v_max;
  c->terms = terms_mask;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&c->device);
  const double* kp = prob->kpt;
  c->cplx = (prob->force_complex != 0) || kp[0] != 0.0 || kp[1] != 0.0 || kp[2] != 0.0;
  c->gga = (terms_mask & FE_KS_TERM_G) && prob->v_gga_q != nullptr;
  c->ncoef = c->cplx ? kCoefCplx : kCoefReal;
  const int np = c->np, nq = c->nq, np3 = c->np3, nq3 = c->nq3;
  const int64_t E = c->E, m = c->m;

  // ---- mesh checks: DoF range and uniqueness inside a cell
  {
    std::string err;
    for (int64_t e = 0; e < E && err.empty(); ++e) {
      const int* d = prob->cell_dofs + e * np3;
      std::vector<int> s(d, d + np3);
      for (int i = 0; i < np3; ++i)
        if (s[i] < 0 || s[i] >= m) err = "cell_dofs entry out of range in cell " + std::to_string(e);
      std::sort(s.begin(), s.end());
      if (err.empty() && std::adjacent_find(s.begin(), s.end()) != s.end())
        err = "cell " + std::to_string(e) + " references a DoF twice (need >= 2 cells per periodic direction)";
    }
    if (!err.empty()) {
      delete h;
      return fail(FE_KS_ERR_MESH, err);
    }
  }

  // ---- 1D tables
  double xg[kMaxN], wg[kMaxN], xl[kMaxN], wl[kMaxN];
  gauss_legendre(nq, xg, wg);
  gauss_lobatto(np, xl, wl);
  build_eo_tables<double>(c->p, nq, &c->f64.tab);
  build_eo_tables<float>(c->p, nq, &c->f32.tab);
  build_eo_tables<ff2>(c->p, nq, &c->emu.tab);

  // ---- per-point coefficients (eq. reformcellmat with det J w_Q and J^-1 folded in)
  const int ncoef = c->ncoef;
  std::vector<double> coef((size_t)E * ncoef * nq3, 0.0);
  const double k2h = 0.5 * (kp[0] * kp[0] + kp[1] * kp[1] + kp[2] * kp[2]);
  std::atomic<int64_t> bad_det(-1);
  parallel_for(E, [&](int64_t b, int64_t e_end) {
    for (int64_t e = b; e < e_end; ++e) {
      const double* V = prob->cell_vertices + 24 * e;
      double* cf = coef.data() + (size_t)e * ncoef * nq3;
      for (int q = 0; q < nq3; ++q) {
        const int qx = q % nq, qy = (q / nq) % nq, qz = q / (nq * nq);
        const double xi[3] = {xg[qx], xg[qy], xg[qz]};
        double x[3], J[3][3], Ji[3][3];
        trilinear(V, xi, x, J);
        const double det = inverse3(J, Ji);
        if (!(det > 0.0)) {
          bad_det.store(e);
          continue;
        }
        const double wd = det * wg[qx] * wg[qy] * wg[qz];
        if (terms_mask & FE_KS_TERM_T) {
          double K[3][3];
          for (int s = 0; s < 3; ++s)
            for (int d = 0; d < 3; ++d) K[s][d] = Ji[s][0] * Ji[d][0] + Ji[s][1] * Ji[d][1] + Ji[s][2] * Ji[d][2];
          cf[0 * nq3 + q] = 0.5 * K[0][0] * wd;
          cf[1 * nq3 + q] = 0.5 * K[0][1] * wd;
          cf[2 * nq3 + q] = 0.5 * K[0][2] * wd;
          cf[3 * nq3 + q] = 0.5 * K[1][1] * wd;
          cf[4 * nq3 + q] = 0.5 * K[1][2] * wd;
          cf[5 * nq3 + q] = 0.5 * K[2][2] * wd;
        }
        if (terms_mask & FE_KS_TERM_L) cf[6 * nq3 + q] = (prob->v_loc_q[e * nq3 + q] + k2h) * wd;
        if (c->gga) {
          const double* g = prob->v_gga_q + (e * nq3 + q) * 3;
          for (int s = 0; s < 3; ++s) cf[(7 + s) * nq3 + q] = (Ji[s][0] * g[0] + Ji[s][1] * g[1] + Ji[s][2] * g[2]) * wd;
        }
        if (c->cplx && (terms_mask & FE_KS_TERM_K)) {
          for (int s = 0; s < 3; ++s)
            cf[(10 + s) * nq3 + q] = (Ji[s][0] * kp[0] + Ji[s][1] * kp[1] + Ji[s][2] * kp[2]) * wd;
        }
      }
    }
  });
  if (bad_det.load() >= 0) {
    delete h;
    return fail(FE_KS_ERR_MESH, "det J <= 0 at a quadrature point of cell " + std::to_string(bad_det.load()));
  }

  // ---- GLL-lumped mass D (Algorithm 4's diagonal approximation of M)
  std::vector<double> D(m, 0.0);
  {
    std::vector<double> detn((size_t)E * np3);
    parallel_for(E, [&](int64_t b, int64_t e_end) {
      for (int64_t e = b; e < e_end; ++e) {
        const double* V = prob->cell_vertices + 24 * e;
        for (int n = 0; n < np3; ++n) {
          const int i = n % np, j = (n / np) % np, k = n / (np * np);
          const double xi[3] = {xl[i], xl[j], xl[k]};
          double x[3], J[3][3], Ji[3][3];
          trilinear(V, xi, x, J);
          detn[e * np3 + n] = inverse3(J, Ji) * wl[i] * wl[j] * wl[k];
        }
      }
    });
    for (int64_t e = 0; e < E; ++e)
      for (int n = 0; n < np3; ++n) D[prob->cell_dofs[e * np3 + n]] += detn[e * np3 + n];
    for (int64_t i = 0; i < m; ++i)
      if (!(D[i] > 0.0)) {
        delete h;
        return fail(FE_KS_ERR_MESH, "DoF " + std::to_string(i) + " belongs to no cell (lumped mass <= 0)");
      }
  }

  // ---- greedy colouring: cells of one colour share no DoF (race-free scatter-add)
  std::vector<int> colour(E, -1);
  const int n_colours = feks::greedy_colouring(E, np3, m, prob->cell_dofs, colour.data());
  if (n_colours < 0) {
    delete h;
    return fail(FE_KS_ERR_UNSUPPORTED, "mesh needs more than 64 colours");
  }
  std::vector<int> colour_cells;
  c->colour_ptr.assign(n_colours + 1, 0);
  for (int col = 0; col < n_colours; ++col) {
    for (int64_t e = 0; e < E; ++e)
      if (colour[e] == col) colour_cells.push_back((int)e);
    c->colour_ptr[col + 1] = (int)colour_cells.size();
  }

  // ---- nonlocal projector matrices F^(a,e)[b][node] (eq. Vnonloc), cell -> pair CSR
  std::vector<double> F;
  std::vector<int> pair_atom, pair_cell, cell_pair_ptr, cell_pairs, atom_pair_ptr;
  if (want_nl) {
    c->n_atoms = prob->n_atoms;
    c->n_proj = prob->n_proj;
    const int nproj = prob->n_proj;
    const int64_t npairs = prob->atom_cell_ptr[prob->n_atoms];
    c->n_pairs = npairs;
    atom_pair_ptr.assign(prob->atom_cell_ptr, prob->atom_cell_ptr + prob->n_atoms + 1);
    for (int a = 0; a < prob->n_atoms; ++a) {
      if (atom_pair_ptr[a + 1] < atom_pair_ptr[a]) {
        delete h;
        return fail(FE_KS_ERR_ARG, "atom_cell_ptr is not monotone");
      }
      for (int t = atom_pair_ptr[a]; t < atom_pair_ptr[a + 1]; ++t) {
        if (prob->atom_cells[t] < 0 || prob->atom_cells[t] >= E) {
          delete h;
          return fail(FE_KS_ERR_MESH, "atom_cells entry out of range");
        }
        pair_atom.push_back(a);
        pair_cell.push_back(prob->atom_cells[t]);
      }
    }
    const int cw = c->cplx ? 2 : 1;
    F.assign((size_t)npairs * nproj * np3 * cw, 0.0);
    // N^1D[q][i] at the Gauss points
    double N[kMaxN][kMaxN], val[kMaxN], der[kMaxN];
    for (int q = 0; q < nq; ++q) {
      lagrange_eval(np, xl, xg[q], val, der);
      for (int i = 0; i < np; ++i) N[q][i] = val[i];
    }
    parallel_for(npairs, [&](int64_t b, int64_t e_end) {
      std::vector<std::complex<double>> g(nq3), t1((size_t)np * nq * nq), t2((size_t)np * np * nq);
      for (int64_t pr = b; pr < e_end; ++pr) {
        const int e = pair_cell[pr];
        const double* V = prob->cell_vertices + 24 * (int64_t)e;
        const double* Lr = prob->image_shift + 3 * pr;
        for (int bb = 0; bb < nproj; ++bb) {
          for (int q = 0; q < nq3; ++q) {
            const int qx = q % nq, qy = (q / nq) % nq, qz = q / (nq * nq);
            const double xi[3] = {xg[qx], xg[qy], xg[qz]};
            double x[3], J[3][3], Ji[3][3];
            trilinear(V, xi, x, J);
            const double wd = inverse3(J, Ji) * wg[qx] * wg[qy] * wg[qz];
            const double chi = prob->chi_q[((size_t)pr * nq3 + q) * nproj + bb];
            const double ph = -(kp[0] * (x[0] - Lr[0]) + kp[1] * (x[1] - Lr[1]) + kp[2] * (x[2] - Lr[2]));
            g[q] = std::complex<double>(std::cos(ph), std::sin(ph)) * (wd * chi);
          }
          // contract qx -> i, qy -> j, qz -> k with N^1D (sum factorisation of N^T)
          for (int qz = 0; qz < nq; ++qz)
            for (int qy = 0; qy < nq; ++qy)
              for (int i = 0; i < np; ++i) {
                std::complex<double> s = 0.0;
                for (int qx = 0; qx < nq; ++qx) s += N[qx][i] * g[qx + nq * (qy + nq * qz)];
                t1[i + np * (qy + nq * qz)] = s;
              }
          for (int qz = 0; qz < nq; ++qz)
            for (int j = 0; j < np; ++j)
              for (int i = 0; i < np; ++i) {
                std::complex<double> s = 0.0;
                for (int qy = 0; qy < nq; ++qy) s += N[qy][j] * t1[i + np * (qy + nq * qz)];
                t2[i + np * (j + np * qz)] = s;
              }
          for (int k = 0; k < np; ++k)
            for (int j = 0; j < np; ++j)
              for (int i = 0; i < np; ++i) {
                std::complex<double> s = 0.0;
                for (int qz = 0; qz < nq; ++qz) s += N[qz][k] * t2[i + np * (j + np * qz)];
                const size_t o = ((size_t)pr * nproj + bb) * np3 + i + np * (j + np * k);
                if (cw == 2) {
                  F[2 * o] = s.real();
                  F[2 * o + 1] = s.imag();
                } else {
                  F[o] = s.real();
                }
              }
        }
      }
    });
    cell_pair_ptr.assign(E + 1, 0);
    for (int64_t pr = 0; pr < npairs; ++pr) cell_pair_ptr[pair_cell[pr] + 1]++;
    for (int64_t e = 0; e < E; ++e) cell_pair_ptr[e + 1] += cell_pair_ptr[e];
    cell_pairs.assign(npairs, 0);
    std::vector<int> fp(cell_pair_ptr.begin(), cell_pair_ptr.end() - 1);
    for (int64_t pr = 0; pr < npairs; ++pr) cell_pairs[fp[pair_cell[pr]]++] = (int)pr;
  }

  // ---- upload
  auto chk = [&](fe_ks_status s) { return s == FE_KS_OK; };
  std::vector<float> tmp32;
  auto to32 = [&](const std::vector<double>& v) {
    tmp32.resize(v.size());
    for (size_t i = 0; i < v.size(); ++i) tmp32[i] = (float)v[i];
    return tmp32.data();
  };
  std::vector<double> ds(m);
  for (int64_t i = 0; i < m; ++i) ds[i] = 1.0 / std::sqrt(D[i]);
  std::vector<ff2> tmpff;
  auto toff = [&](const std::vector<double>& v) {
    tmpff.resize(v.size());
    for (size_t i = 0; i < v.size(); ++i) tmpff[i] = ff_from_double_host(v[i]);
    return tmpff.data();
  };
  bool ok = chk(upload(c, &c->cell_dofs, prob->cell_dofs, (size_t)E * np3)) &&
            chk(upload(c, &c->colour_cells, colour_cells.data(), colour_cells.size())) &&
            chk(upload(c, &c->f64.coef, coef.data(), coef.size())) &&
            chk(upload(c, &c->f32.coef, to32(coef), coef.size())) &&
            chk(upload(c, &c->f64.dscale, ds.data(), ds.size())) &&
            chk(upload(c, &c->f32.dscale, to32(ds), ds.size())) &&
            chk(upload(c, reinterpret_cast<ff2**>(&c->emu.coef), toff(coef), coef.size())) &&
            chk(upload(c, reinterpret_cast<ff2**>(&c->emu.dscale), toff(ds), ds.size()));
  if (ok) {
    std::vector<uint32_t> frag(kTcFragWords), frag16(kTcFragWords), fraglo(kTcFragWords);
    build_tc_frags(c->p, frag.data(), 0);
    build_tc_frags(c->p, frag16.data(), 1);
    build_tc_frags(c->p, fraglo.data(), 2);
    ok = chk(upload(c, &c->tc_frag, frag.data(), frag.size())) &&
         chk(upload(c, &c->tc_frag16, frag16.data(), frag16.size())) &&
         chk(upload(c, &c->tc_frag_lo, fraglo.data(), fraglo.size()));
    const int zero = 0;
    ok = ok && chk(upload(c, &c->dev_status, &zero, 1));
    if (ok && !c->cplx && c->nq == c->np) {   // the tcgen05 cell kernel's operator block
      std::vector<uint4> cst;
      build_tc5_const(c->p, false, cst);
      ok = chk(upload(c, &c->tc5_cst, cst.data(), cst.size()));
      build_tc5_const(c->p, true, cst);
      ok = ok && chk(upload(c, &c->tc5_cst16, cst.data(), cst.size()));
    }
  }
  if (ok && want_nl) {
    std::vector<double> hh(prob->h_coef, prob->h_coef + (size_t)prob->n_atoms * prob->n_proj);
    const size_t qn = (size_t)prob->n_atoms * prob->n_proj * n_v_max * (c->cplx ? 2 : 1);
    const size_t pn = (size_t)c->n_pairs * prob->n_proj * n_v_max * (c->cplx ? 2 : 1);
    ok = chk(upload(c, &c->f64.F, F.data(), F.size())) && chk(upload(c, &c->f32.F, to32(F), F.size())) &&
         chk(upload(c, reinterpret_cast<ff2**>(&c->emu.F), toff(F), F.size())) &&
         chk(upload(c, &c->h64, hh.data(), hh.size())) && chk(upload(c, &c->h32, to32(hh), hh.size())) &&
         chk(upload(c, &c->pair_atom, pair_atom.data(), pair_atom.size())) &&
         chk(upload(c, &c->pair_cell, pair_cell.data(), pair_cell.size())) &&
         chk(upload(c, &c->atom_pair_ptr, atom_pair_ptr.data(), atom_pair_ptr.size())) &&
         chk(upload(c, &c->cell_pair_ptr, cell_pair_ptr.data(), cell_pair_ptr.size())) &&
         chk(upload(c, &c->cell_pairs, cell_pairs.data(), cell_pairs.size())) &&
         chk(upload<double>(c, &c->f64.Q, nullptr, qn)) && chk(upload<float>(c, &c->f32.Q, nullptr, qn)) &&
         chk(upload<double>(c, &c->f64.part, nullptr, pn)) && chk(upload<float>(c, &c->f32.part, nullptr, pn));
    if (ok) {
      std::vector<uint2> fpack;
      build_tc_fpack(c->np, c->cplx != 0, prob->n_proj, c->n_pairs, F.data(), 0, fpack);
      ok = chk(upload(c, &c->tc_fpack, fpack.data(), fpack.size()));
      if (ok) {
        build_tc_fpack(c->np, c->cplx != 0, prob->n_proj, c->n_pairs, F.data(), 1, fpack);
        ok = chk(upload(c, &c->tc_fpack16, fpack.data(), fpack.size()));
      }
      if (ok) {
        build_tc_fpack(c->np, c->cplx != 0, prob->n_proj, c->n_pairs, F.data(), 2, fpack);
        ok = chk(upload(c, &c->tc_fpack_lo, fpack.data(), fpack.size()));
      }
    }
  }
  if (!ok) {
    std::string msg = g_last_error;
    for (void* p : c->allocations) cudaFree(p);
    delete h;
    return fail(msg.find("cudaMalloc") != std::string::npos ? FE_KS_ERR_OOM : FE_KS_ERR_CUDA, msg);
  }
  *out = h;
  return FE_KS_OK;
}

void fe_ks_destroy(fe_ks_ctx* ctx) {
  if (!ctx) return;
  Ctx& hc = ctx->c;
  if (hc.hs_in) {
    cudaStreamSynchronize(hc.hs_in);
    cudaStreamSynchronize(hc.hs_out);
    for (int b = 0; b < 2; ++b) {
      cudaEventDestroy(hc.h_in[b]);
      cudaEventDestroy(hc.h_done[b]);
      cudaEventDestroy(hc.h_out[b]);
    }
    cudaStreamDestroy(hc.hs_in);
    cudaStreamDestroy(hc.hs_out);
  }
  for (void* p : ctx->c.allocations) cudaFree(p);
  for (cudaEvent_t e : ctx->c.ev_pool) cudaEventDestroy(e);
  for (auto& r : ctx->c.ev_rec)
    for (cudaEvent_t e : r) cudaEventDestroy(e);
  delete ctx;
}

fe_ks_status fe_ks_set_profiling(fe_ks_ctx* ctx, int on) {
  if (!ctx) return fail(FE_KS_ERR_ARG, "ctx is NULL");
  ctx->c.profiling = on != 0;
  return FE_KS_OK;
}

fe_ks_status fe_ks_read_profile(fe_ks_ctx* ctx, double ms[3], int64_t launches[3]) {
  if (!ctx || !ms || !launches) return fail(FE_KS_ERR_ARG, "NULL argument");
  Ctx& c = ctx->c;
  for (int i = 0; i < 3; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  for (size_t r = 0; r < c.ev_rec.size(); ++r) {
    auto& ev = c.ev_rec[r];
    if (cudaEventSynchronize(ev[3]) != cudaSuccess) return fail(FE_KS_ERR_CUDA, "event synchronize failed");
    for (int i = 0; i < 3; ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
      ms[i] += t;
      launches[i] += c.ev_launches[r][i];
    }
    for (cudaEvent_t e : ev) c.ev_pool.push_back(e);
  }
  c.ev_rec.clear();
  c.ev_launches.clear();
  return FE_KS_OK;
}

fe_ks_status fe_ks_set_stream(fe_ks_ctx* ctx, void* cuda_stream) {
  if (!ctx) return fail(FE_KS_ERR_ARG, "ctx is NULL");
  ctx->c.stream = static_cast<cudaStream_t>(cuda_stream);
  return FE_KS_OK;
}

const double* fe_ks_dinv_sqrt(const fe_ks_ctx* ctx) { return ctx ? ctx->c.f64.dscale : nullptr; }

fe_ks_status fe_ks_info(const fe_ks_ctx* ctx, int64_t* n_dofs, int64_t* n_cells, int32_t* degree,
                        int32_t* is_complex, int32_t* n_colours, int64_t* n_pairs) {
  if (!ctx) return fail(FE_KS_ERR_ARG, "ctx is NULL");
  const Ctx& c = ctx->c;
  if (n_dofs) *n_dofs = c.m;
  if (n_cells) *n_cells = c.E;
  if (degree) *degree = c.p;
  if (is_complex) *is_complex = c.cplx;
  if (n_colours) *n_colours = (int32_t)c.colour_ptr.size() - 1;
  if (n_pairs) *n_pairs = c.n_pairs;
  return FE_KS_OK;
}

}  // extern "C"

namespace feks {

template <typename T>
fe_ks_status apply_core(Ctx& c, const T* X, T* Y, int64_t ncols, bool scaled, T alpha, bool zero_fill, int tc) {
  NvtxRange range(tc == 3   ? "fe_ks_apply bf16x2"
                  : tc == 2 ? "fe_ks_apply f16"
                  : tc == 1 ? "fe_ks_apply bf16"
                  : sizeof(T) == 8 ? "fe_ks_apply f64"
                                   : "fe_ks_apply f32");
  OpData<T>& od = *reinterpret_cast<OpData<T>*>(sizeof(T) == 8 ? (void*)&c.f64 : (void*)&c.f32);
  const T* hcoef = reinterpret_cast<const T*>(sizeof(T) == 8 ? (const void*)c.h64 : (const void*)c.h32);
  cudaStream_t s = c.stream;
  const size_t bytes = (size_t)c.m * ncols * sizeof(T);
  std::array<cudaEvent_t, 4> ev{};
  std::array<int, 3> nlaunch{zero_fill ? 1 : 0, 0, 0};
  auto mark = [&](int i) {
    if (!c.profiling) return;
    if (c.ev_pool.empty()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      c.ev_pool.push_back(e);
    }
    ev[i] = c.ev_pool.back();
    c.ev_pool.pop_back();
    cudaEventRecord(ev[i], s);
  };
  mark(0);
  if (zero_fill && cudaMemsetAsync(Y, 0, bytes, s) != cudaSuccess)
    return fail(FE_KS_ERR_CUDA, "cudaMemsetAsync failed");
  mark(1);
  if (tc && c.nq != c.np)
    return fail(FE_KS_ERR_UNSUPPORTED, "the tensor-core precisions need n_q = n_p (square 1D operators)");
  const bool nl = (c.terms & FE_KS_TERM_NL) && c.n_pairs > 0;
  if (nl) {
    ProjParams<T> pp{};
    pp.X = X;
    pp.ld = ncols;
    pp.ncols = (int)ncols;
    pp.cell_dofs = c.cell_dofs;
    pp.atom_pair_ptr = c.atom_pair_ptr;
    pp.pair_cell = c.pair_cell;
    pp.F = od.F;
    pp.h = hcoef;
    pp.dscale = scaled ? od.dscale : nullptr;
    pp.Q = od.Q;
    pp.n_proj = c.n_proj;
    pp.np3 = c.np3;
    pp.part = od.part;
    pp.n_pairs = c.n_pairs;
    cudaError_t err = launch_proj_pairs<T>(c, pp, c.n_atoms, s);
    if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("projection kernel: ") + cudaGetErrorString(err));
    nlaunch[1] = 1;
  }
  mark(2);
  LocalParams<T> lp{};
  lp.X = X;
  lp.Y = Y;
  lp.ld = ncols;
  lp.ncols = (int)ncols;
  lp.cell_dofs = c.cell_dofs;
  lp.coef = od.coef;
  lp.ncoef = c.ncoef;
  lp.gga = c.gga;
  lp.dscale = scaled ? od.dscale : nullptr;
  lp.cell_pair_ptr = nl ? c.cell_pair_ptr : nullptr;
  lp.cell_pairs = c.cell_pairs;
  lp.pair_atom = c.pair_atom;
  lp.F = od.F;
  lp.Q = od.Q;
  lp.n_proj = c.n_proj;
  lp.alpha = alpha;
  lp.tab = od.tab;
  for (size_t col = 0; col + 1 < c.colour_ptr.size(); ++col) {
    lp.cells = c.colour_cells + c.colour_ptr[col];
    lp.n_cells = c.colour_ptr[col + 1] - c.colour_ptr[col];
    cudaError_t err;
    if constexpr (std::is_same<T, float>::value)
      err = !tc ? launch_local<T, T>(c, lp, s)   // tc: n_q = n_p, checked above
            : use_tc5(c, tc) ? launch_tc5(c, lp, s, tc == 2, tc5_stagger(c.cfg_tc[tc - 1]))
                             : launch_tc(c, lp, s, tc);
    else
      err = launch_local<T, T>(c, lp, s);
    if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("local kernel: ") + cudaGetErrorString(err));
    if (lp.n_cells > 0) nlaunch[2]++;
  }
  mark(3);
  if (c.profiling) {
    c.ev_rec.push_back(ev);
    c.ev_launches.push_back(nlaunch);
  }
  return FE_KS_OK;
}

template fe_ks_status apply_core<double>(Ctx&, const double*, double*, int64_t, bool, double, bool, int);
template fe_ks_status apply_core<float>(Ctx&, const float*, float*, int64_t, bool, float, bool, int);

// FP64-accurate application computed in pairs of floats: FP64 projections,
// pair-of-floats cell kernel with FP64 gather / scatter (alpha is applied in
// the pair arithmetic).
fe_ks_status apply_core_emu(Ctx& c, const double* X, double* Y, int64_t ncols, bool scaled, double alpha,
                            bool zero_fill) {
  NvtxRange range("fe_ks_apply f64e");
  cudaStream_t s = c.stream;
  const size_t bytes = (size_t)c.m * ncols * sizeof(double);
  std::array<cudaEvent_t, 4> ev{};
  std::array<int, 3> nlaunch{zero_fill ? 1 : 0, 0, 0};
  auto mark = [&](int i) {
    if (!c.profiling) return;
    if (c.ev_pool.empty()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      c.ev_pool.push_back(e);
    }
    ev[i] = c.ev_pool.back();
    c.ev_pool.pop_back();
    cudaEventRecord(ev[i], s);
  };
  mark(0);
  if (zero_fill && cudaMemsetAsync(Y, 0, bytes, s) != cudaSuccess) return fail(FE_KS_ERR_CUDA, "cudaMemsetAsync failed");
  mark(1);
  const bool nl = (c.terms & FE_KS_TERM_NL) && c.n_pairs > 0;
  if (nl) {
    ProjParams<double> pp{};
    pp.X = X;
    pp.ld = ncols;
    pp.ncols = (int)ncols;
    pp.cell_dofs = c.cell_dofs;
    pp.atom_pair_ptr = c.atom_pair_ptr;
    pp.pair_cell = c.pair_cell;
    pp.F = c.f64.F;
    pp.h = c.h64;
    pp.dscale = scaled ? c.f64.dscale : nullptr;
    pp.Q = c.f64.Q;
    pp.n_proj = c.n_proj;
    pp.np3 = c.np3;
    pp.part = c.f64.part;
    pp.n_pairs = c.n_pairs;
    cudaError_t err = launch_proj_pairs_emu(c, pp, static_cast<const ff2*>(c.emu.F), c.n_atoms, s);
    if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("projection kernel: ") + cudaGetErrorString(err));
    nlaunch[1] = 1;
  }
  mark(2);
  LocalParams<ff2, double> lp{};
  lp.X = X;
  lp.Y = Y;
  lp.ld = ncols;
  lp.ncols = (int)ncols;
  lp.cell_dofs = c.cell_dofs;
  lp.coef = static_cast<const ff2*>(c.emu.coef);
  lp.ncoef = c.ncoef;
  lp.gga = c.gga;
  lp.dscale = scaled ? static_cast<const ff2*>(c.emu.dscale) : nullptr;
  lp.cell_pair_ptr = nl ? c.cell_pair_ptr : nullptr;
  lp.cell_pairs = c.cell_pairs;
  lp.pair_atom = c.pair_atom;
  lp.F = static_cast<const ff2*>(c.emu.F);
  lp.Q = c.f64.Q;
  lp.n_proj = c.n_proj;
  lp.alpha = ff_from_double_host(alpha);
  lp.tab = c.emu.tab;
  for (size_t col = 0; col + 1 < c.colour_ptr.size(); ++col) {
    lp.cells = c.colour_cells + c.colour_ptr[col];
    lp.n_cells = c.colour_ptr[col + 1] - c.colour_ptr[col];
    cudaError_t err = launch_local<ff2, double>(c, lp, s);
    if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("local kernel: ") + cudaGetErrorString(err));
    if (lp.n_cells > 0) nlaunch[2]++;
  }
  mark(3);
  if (c.profiling) {
    c.ev_rec.push_back(ev);
    c.ev_launches.push_back(nlaunch);
  }
  return FE_KS_OK;
}

template <typename T>
static fe_ks_status apply_impl(fe_ks_ctx* ctx, const void* Xv, void* Yv, int64_t n_v, bool scaled, int tc = 0) {
  using TS = typename std::conditional<std::is_same<T, ff2>::value, double, T>::type;
  g_last_error.clear();
  if (!ctx) return fail(FE_KS_ERR_ARG, "ctx is NULL");
  Ctx& c = ctx->c;
  if (!Xv || !Yv) return fail(FE_KS_ERR_ARG, "X or Y is NULL");
  if (n_v < 1 || n_v > c.n_v_max) return fail(FE_KS_ERR_ARG, "n_v must be in 1..n_v_max");
  if (((uintptr_t)Xv % sizeof(TS)) || ((uintptr_t)Yv % sizeof(TS)))
    return fail(FE_KS_ERR_ARG, "X and Y must be aligned to the scalar size");
  const int64_t ncols = n_v * (c.cplx ? 2 : 1);
  const size_t bytes = (size_t)c.m * ncols * sizeof(TS);
  const char* xb = static_cast<const char*>(Xv);
  const char* yb = static_cast<const char*>(Yv);
  if (xb < yb + bytes && yb < xb + bytes) return fail(FE_KS_ERR_ARG, "X and Y overlap");
  tune_cache_apply(c, std::is_same<T, ff2>::value ? FE_KS_F64E : (sizeof(T) == 8 ? FE_KS_F64 : FE_KS_F32), ncols);
  if constexpr (std::is_same<T, ff2>::value)
    return apply_core_emu(c, static_cast<const double*>(Xv), static_cast<double*>(Yv), ncols, scaled, 1.0, true);
  else
    return apply_core<T>(c, static_cast<const T*>(Xv), static_cast<T*>(Yv), ncols, scaled, T(1), true, tc);
}

}  // namespace feks

extern "C" {

fe_ks_status fe_ks_apply(fe_ks_ctx* ctx, const void* X, void* Y, int64_t n_v, int precision) {
  if (precision == FE_KS_F64) return apply_impl<double>(ctx, X, Y, n_v, false);
  if (precision == FE_KS_F64E) return apply_impl<ff2>(ctx, X, Y, n_v, false);
  if (precision == FE_KS_F32) return apply_impl<float>(ctx, X, Y, n_v, false);
  if (precision == FE_KS_BF16) return apply_impl<float>(ctx, X, Y, n_v, false, 1);
  if (precision == FE_KS_F16) return apply_impl<float>(ctx, X, Y, n_v, false, 2);
  if (precision == FE_KS_BF16X2) return apply_impl<float>(ctx, X, Y, n_v, false, 3);
  return fail(FE_KS_ERR_UNSUPPORTED, "unknown precision");
}

fe_ks_status fe_ks_set_config(fe_ks_ctx* ctx, int precision, int config) {
  if (!ctx) return fail(FE_KS_ERR_ARG, "ctx is NULL");
  int* slot = config_slot(ctx->c, precision);
  if (!slot) return fail(FE_KS_ERR_UNSUPPORTED, "precision without tile configurations");
  if (config < 0 || config >= n_configs(ctx->c, precision)) return fail(FE_KS_ERR_ARG, "config out of range");
  *slot = config;
  ctx->c.cfg_explicit[precision] = true;
  return FE_KS_OK;
}

fe_ks_status fe_ks_get_config(const fe_ks_ctx* ctx, int precision, int* config) {
  if (!ctx || !config) return fail(FE_KS_ERR_ARG, "NULL argument");
  const int* slot = config_slot(const_cast<Ctx&>(ctx->c), precision);
  if (!slot) return fail(FE_KS_ERR_UNSUPPORTED, "precision without tile configurations");
  *config = *slot;
  return FE_KS_OK;
}

fe_ks_status fe_ks_colour_cells(int64_t n_cells, int32_t np3, int64_t n_dofs, const int32_t* cell_dofs,
                                int32_t* colour, int32_t* n_colours) {
  set_error("");
  if (!cell_dofs || !colour || !n_colours) return fail(FE_KS_ERR_ARG, "NULL argument");
  if (n_cells < 1 || n_cells > (int64_t)INT32_MAX || np3 < 1 || n_dofs < 1 || n_dofs > (int64_t)INT32_MAX)
    return fail(FE_KS_ERR_ARG, "sizes out of range");
  for (int64_t i = 0; i < n_cells * np3; ++i)
    if (cell_dofs[i] < 0 || cell_dofs[i] >= n_dofs) return fail(FE_KS_ERR_MESH, "cell_dofs entry out of range");
  const int nc = greedy_colouring(n_cells, np3, n_dofs, cell_dofs, colour);
  if (nc < 0) return fail(FE_KS_ERR_UNSUPPORTED, "mesh needs more than 64 colours");
  *n_colours = nc;
  return FE_KS_OK;
}

fe_ks_status fe_ks_tune(fe_ks_ctx* ctx, const void* X, void* Y, int64_t n_v, int precision, int reps,
                        double* ms_per_config, int* best) {
  g_last_error.clear();
  if (!ctx || !X || !Y) return fail(FE_KS_ERR_ARG, "NULL argument");
  if (precision != FE_KS_F64 && precision != FE_KS_F32 && precision != FE_KS_F64E && precision != FE_KS_BF16 &&
      precision != FE_KS_F16 && precision != FE_KS_BF16X2)
    return fail(FE_KS_ERR_UNSUPPORTED, "unknown precision");
  if (reps < 1) reps = 1;
  Ctx& c = ctx->c;
  int single = 0;   // the split-precision kernel has one configuration
  int* slot = config_slot(c, precision);
  int& cfg = slot ? *slot : single;
  const bool tcp = precision == FE_KS_BF16 || precision == FE_KS_F16 || precision == FE_KS_BF16X2;
  const int n_conf = n_configs(c, precision);
  const int keep = cfg;
  bool* expl = slot ? &c.cfg_explicit[precision] : nullptr;
  const bool keep_expl = expl ? *expl : false;
  if (expl) *expl = true;   // the loop below sets the configuration itself
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best_ms = 1e300;
  int best_cfg = keep;
  for (int k = 0; k < kLocalConfigs; ++k) {
    if (k >= n_conf) {
      if (ms_per_config) ms_per_config[k] = -1.0;
      continue;
    }
    cfg = k;
    double ms = -1.0;
    fe_ks_status st = fe_ks_apply(ctx, X, Y, n_v, precision);   // warm-up, and rejects configs that cannot launch
    if (st == FE_KS_OK) {
      cudaEventRecord(e0, c.stream);
      for (int r = 0; r < reps && st == FE_KS_OK; ++r) st = fe_ks_apply(ctx, X, Y, n_v, precision);
      cudaEventRecord(e1, c.stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = FE_KS_ERR_CUDA;
      float t = 0.f;
      if (st == FE_KS_OK && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms = t / reps;
    } else {
      cudaGetLastError();   // clear a rejected launch configuration
      g_last_error.clear();
    }
    if (ms_per_config) ms_per_config[k] = ms;
    if (ms > 0 && ms < best_ms) {
      best_ms = ms;
      best_cfg = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (expl) *expl = keep_expl;
  cfg = best_cfg;
  if (best) *best = best_cfg;
  if (best_ms == 1e300) return fail(FE_KS_ERR_CUDA, "no tile configuration could be launched");
  if (!tcp) {
    c.cfg_explicit[precision] = true;
    tune_cache_store(c, precision, n_v * (c.cplx ? 2 : 1), best_cfg);
  }
  return FE_KS_OK;
}

fe_ks_status fe_ks_device_status(fe_ks_ctx* ctx, int* status) {
  g_last_error.clear();
  if (!ctx || !status) return fail(FE_KS_ERR_ARG, "NULL argument");
  Ctx& c = ctx->c;
  int v = 0;
  if (cudaStreamSynchronize(c.stream) != cudaSuccess ||
      cudaMemcpy(&v, c.dev_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(c.dev_status, 0, sizeof(int)) != cudaSuccess)
    return fail(FE_KS_ERR_CUDA, "reading the device status failed");
  *status = v;
  return FE_KS_OK;
}

fe_ks_status fe_ks_inject_fault(fe_ks_ctx* ctx, int kind) {
  g_last_error.clear();
  if (!ctx) return fail(FE_KS_ERR_ARG, "ctx is NULL");
  if (kind != 0 && kind != 1) return fail(FE_KS_ERR_ARG, "kind must be 0 (off) or 1");
  ctx->c.inject_fault = kind;
  return FE_KS_OK;
}

fe_ks_status fe_ks_apply_scaled(fe_ks_ctx* ctx, const void* X, void* Y, int64_t n_v, int precision) {
  if (precision == FE_KS_F64) return apply_impl<double>(ctx, X, Y, n_v, true);
  if (precision == FE_KS_F64E) return apply_impl<ff2>(ctx, X, Y, n_v, true);
  if (precision == FE_KS_F32) return apply_impl<float>(ctx, X, Y, n_v, true);
  if (precision == FE_KS_BF16) return apply_impl<float>(ctx, X, Y, n_v, true, 1);
  if (precision == FE_KS_F16) return apply_impl<float>(ctx, X, Y, n_v, true, 2);
  if (precision == FE_KS_BF16X2) return apply_impl<float>(ctx, X, Y, n_v, true, 3);
  return fail(FE_KS_ERR_UNSUPPORTED, "unknown precision");
}

// ---- host buffers: copy in, apply, copy out, pipelined across calls ----
// Storage bytes of one [m][n_v] block in the given precision (0: unknown precision).
static size_t host_block_bytes(const Ctx& c, int64_t n_v, int precision) {
  const size_t esz = (precision == FE_KS_F64 || precision == FE_KS_F64E) ? 8
                     : (precision == FE_KS_F32 || precision == FE_KS_BF16 || precision == FE_KS_F16 ||
                        precision == FE_KS_BF16X2)
                         ? 4
                                                                                                       : 0;
  return ((size_t)c.m * n_v * (c.cplx ? 2 : 1) * esz + 255) & ~(size_t)255;
}

fe_ks_status fe_ks_apply_host_workspace(const fe_ks_ctx* ctx, int64_t n_v, int precision, size_t* bytes) {
  if (!ctx || !bytes) return fail(FE_KS_ERR_ARG, "NULL argument");
  const size_t blk = host_block_bytes(ctx->c, n_v, precision);
  if (!blk) return fail(FE_KS_ERR_UNSUPPORTED, "unknown precision");
  *bytes = 4 * blk;   // two slots of (X, Y)
  return FE_KS_OK;
}

fe_ks_status fe_ks_apply_host(fe_ks_ctx* ctx, const void* X_host, void* Y_host, int64_t n_v, int precision,
                              void* work, size_t work_bytes) {
  set_error("");
  if (!ctx || !X_host || !Y_host || !work) return fail(FE_KS_ERR_ARG, "NULL argument");
  Ctx& c = ctx->c;
  if (n_v < 1 || n_v > c.n_v_max) return fail(FE_KS_ERR_ARG, "n_v must be in 1..n_v_max");
  const size_t blk = host_block_bytes(c, n_v, precision);
  if (!blk) return fail(FE_KS_ERR_UNSUPPORTED, "unknown precision");
  if (work_bytes < 4 * blk) return fail(FE_KS_ERR_ARG, "workspace smaller than fe_ks_apply_host_workspace");
  if ((uintptr_t)work % 256) return fail(FE_KS_ERR_ARG, "workspace must be 256-byte aligned");
  if (!c.hs_in) {   // first call: the context's copy streams and slot events
    if (cudaStreamCreateWithFlags(&c.hs_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c.hs_out, cudaStreamNonBlocking) != cudaSuccess)
      return fail(FE_KS_ERR_CUDA, "copy stream creation failed");
    for (int b = 0; b < 2; ++b)
      if (cudaEventCreateWithFlags(&c.h_in[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&c.h_done[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&c.h_out[b], cudaEventDisableTiming) != cudaSuccess)
        return fail(FE_KS_ERR_CUDA, "event creation failed");
    for (int b = 0; b < 2; ++b) {   // every slot starts free
      cudaEventRecord(c.h_done[b], c.hs_in);
      cudaEventRecord(c.h_out[b], c.hs_out);
    }
  }
  const int b = c.h_slot;
  char* base = static_cast<char*>(work) + (size_t)b * 2 * blk;
  void* Xd = base;
  void* Yd = base + blk;
  const size_t bytes = (size_t)c.m * n_v * (c.cplx ? 2 : 1) *
                       ((precision == FE_KS_F64 || precision == FE_KS_F64E) ? 8 : 4);
  // copy in once the slot's previous application has read its X
  cudaStreamWaitEvent(c.hs_in, c.h_done[b], 0);
  if (cudaMemcpyAsync(Xd, X_host, bytes, cudaMemcpyHostToDevice, c.hs_in) != cudaSuccess)
    return fail(FE_KS_ERR_CUDA, "host-to-device copy failed");
  cudaEventRecord(c.h_in[b], c.hs_in);
  // apply once X is in and the slot's previous Y has been copied out
  cudaStreamWaitEvent(c.stream, c.h_in[b], 0);
  cudaStreamWaitEvent(c.stream, c.h_out[b], 0);
  fe_ks_status st = fe_ks_apply(ctx, Xd, Yd, n_v, precision);
  if (st != FE_KS_OK) return st;
  cudaEventRecord(c.h_done[b], c.stream);
  // copy out after the application
  cudaStreamWaitEvent(c.hs_out, c.h_done[b], 0);
  if (cudaMemcpyAsync(Y_host, Yd, bytes, cudaMemcpyDeviceToHost, c.hs_out) != cudaSuccess)
    return fail(FE_KS_ERR_CUDA, "device-to-host copy failed");
  cudaEventRecord(c.h_out[b], c.hs_out);
  c.h_slot = 1 - b;
  return FE_KS_OK;
}

fe_ks_status fe_ks_host_wait(fe_ks_ctx* ctx) {
  if (!ctx) return fail(FE_KS_ERR_ARG, "ctx is NULL");
  Ctx& c = ctx->c;
  if (!c.hs_in) return FE_KS_OK;
  if (cudaStreamSynchronize(c.hs_in) != cudaSuccess || cudaStreamSynchronize(c.stream) != cudaSuccess ||
      cudaStreamSynchronize(c.hs_out) != cudaSuccess)
    return fail(FE_KS_ERR_CUDA, std::string("host pipeline: ") + cudaGetErrorString(cudaGetLastError()));
  return FE_KS_OK;
}

}  // extern "C"
