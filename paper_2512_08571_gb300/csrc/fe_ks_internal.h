// Internal declarations shared by the translation units of libfe_ks.so.
// Paper: Panigrahi & Motamarri, matrix-free FE Kohn-Sham operator (Sec. 3-4).
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fe_ks.h"
#include "fe_ks_ff.cuh"

namespace feks {

constexpr int kMaxN = 11;      // n_p <= 9, n_q <= 11 (n_q = n_p + 2 at p = 8)
constexpr int kMaxH = kMaxN / 2;

// Even-odd split of a centro-(anti)symmetric 1D matrix M (NO x NI) with
// M[NO-1-o][NI-1-i] = S * M[o][i]  (S = +1 for N^1D, -1 for D~^1D; Sec. 5.4,
// "even-odd decomposition").  For o < NO/2, i < NI/2:
//   E[o][i] = (M[o][i] + M[o][NI-1-i]) / 2,  E[o][NI/2] = M[o][NI/2] (NI odd)
//   O[o][i] = (M[o][i] - M[o][NI-1-i]) / 2
// and the middle row (NO odd) MID[i] = M[NO/2][i].
template <typename T>
struct EOMat {
  T E[kMaxH][kMaxH + 1];
  T O[kMaxH][kMaxH];
  T MID[kMaxH + 1];
};

// The four 1D operators of Algorithm 2: N^1D, (N^1D)^T, D~^1D, (D~^1D)^T.
template <typename T>
struct EOTables {
  EOMat<T> N, Nt, D, Dt;
};

// Coefficient slots per quadrature point (Sec. 3.1, eq. reformcellmat, with
// det J w_Q and J^{-1} folded in):
//   0..5  G_sd = 1/2 (J^-1 J^-T)_sd det J w      (00 01 02 11 12 22)
//   6     V^L  = (V_loc + |k|^2/2) det J w
//   7..9  V^G_s = (J^-1 V^G)_s det J w
//   10..12 V^K_s = (J^-1 k)_s det J w           (complex operators only)
constexpr int kCoefReal = 10;
constexpr int kCoefCplx = 13;

template <typename T>
struct OpData {
  T* coef = nullptr;       // [E][ncoef][n_q^3]
  T* F = nullptr;          // [n_pairs][n_proj][n_p^3] (complex: x2 interleaved)
  T* dscale = nullptr;     // [m] D^{-1/2}
  T* Q = nullptr;          // workspace [n_atoms][n_proj][ncols_max]
  T* part = nullptr;       // projection partials [n_pairs][n_proj][ncols_max]
  EOTables<T> tab;
};

// Kernel parameters of the fused local kernel (one colour of cells).  T is
// the arithmetic type, TS the storage type of X, Y and the projections Q
// (they differ only for the pair-of-floats FP64 variant).
template <typename T, typename TS = T>
struct LocalParams {
  const TS* X;
  TS* Y;
  int64_t ld;              // row pitch of X and Y in scalars (= ncols)
  int ncols;               // real columns (complex: 2 n_v)
  const int* cell_dofs;    // [E][n_p^3]
  const int* cells;        // cells of this colour
  int n_cells;
  const T* coef;
  int ncoef;
  int gga;                 // V^G coefficients present
  const T* dscale;         // D^{-1/2} or nullptr
  // nonlocal expansion fused into the scatter (Algorithm 1, F Delta T3)
  const int* cell_pair_ptr;  // [E+1] or nullptr
  const int* cell_pairs;
  const int* pair_atom;
  const T* F;
  const TS* Q;             // [n_atoms][n_proj][ld], already scaled by Delta
  int n_proj;
  T alpha;                 // Y += alpha * (H X) (1 for a plain application)
  EOTables<T> tab;
};

// Projection kernel parameters: Q[a][b][col] = h[a][b] sum conj(F) X.
template <typename T>
struct ProjParams {
  const T* X;
  int64_t ld;
  int ncols;
  const int* cell_dofs;
  const int* atom_pair_ptr;  // [n_atoms+1]
  const int* pair_cell;
  const T* F;
  const T* h;              // [n_atoms][n_proj]
  const T* dscale;
  T* Q;
  int n_proj;
  int np3;
  T* part = nullptr;       // pair partials [n_pairs][n_proj][ld] (pair form)
  int64_t n_pairs = 0;
};

struct Ctx {
  int p = 0, nq = 0, np = 0, np3 = 0, nq3 = 0;
  int cplx = 0, terms = 0, gga = 0, ncoef = 0;
  int cfg64 = 0, cfg32 = 0, cfgE = 0;   // tile configuration of the fused kernel per precision
  int rr_gram_tc = 1;                   // Rayleigh-Ritz Gram products on the tensor cores (pairs plan)
  int cfg_tc[2] = {0, 0};               // BF16, FP16 cell kernel: 1 = warp-level MMA; 0, 2, 3 = tcgen05 (where
                                        // supported) with its two pipelines staggered by a point of the tile
  bool cfg_explicit[6] = {};            // set by fe_ks_set_config / fe_ks_tune, per precision
  int64_t E = 0, m = 0, n_v_max = 0;
  int n_atoms = 0, n_proj = 0;
  int64_t n_pairs = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  // device tables
  int* cell_dofs = nullptr;
  int* colour_cells = nullptr;
  std::vector<int> colour_ptr;
  int* pair_atom = nullptr;
  int* pair_cell = nullptr;
  int* atom_pair_ptr = nullptr;
  int* cell_pair_ptr = nullptr;
  int* cell_pairs = nullptr;
  double* h64 = nullptr;
  float* h32 = nullptr;
  OpData<double> f64;
  OpData<float> f32;
  // pair-of-floats copies of the coefficients, projector matrices, D^{-1/2}
  // and 1D tables for the FP64-accurate FP32-pipe variant
  struct {
    void* coef = nullptr;
    void* F = nullptr;
    void* dscale = nullptr;
    EOTables<ff2> tab;
  } emu;
  // B fragments of the BF16 tensor-core cell kernel: [4 ops][2 tiles][32 lanes][2]
  uint32_t* tc_frag = nullptr;     // BF16
  uint32_t* tc_frag16 = nullptr;   // FP16
  uint2* tc_fpack = nullptr;       // F as expansion B fragments, BF16 (when the nonlocal term is present)
  uint2* tc_fpack16 = nullptr;     // the same in FP16
  uint32_t* tc_frag_lo = nullptr;  // BF16 remainders of the 1D operators (split precision FE_KS_BF16X2)
  uint2* tc_fpack_lo = nullptr;    // BF16 remainders of F (split precision)
  uint4* tc5_cst = nullptr;        // tcgen05 cell kernel: plane and z-sweep operators, BF16 (real, n_q = n_p)
  uint4* tc5_cst16 = nullptr;      // the same in FP16
  int* dev_status = nullptr;       // device word: 1 after a bounded wait in a cell kernel expired
  int inject_fault = 0;            // host-side fault injection into the tcgen05 cell kernel (tests)
  std::vector<void*> allocations;
  // host-buffer pipeline (fe_ks_apply_host): copy-in and copy-out streams and,
  // per workspace slot, events for "X copied in", "applied", "Y copied out"
  cudaStream_t hs_in = nullptr, hs_out = nullptr;
  cudaEvent_t h_in[2] = {}, h_done[2] = {}, h_out[2] = {};
  int h_slot = 0;
  // profiling: events recorded per application (start, after fill, after projection, after local)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::array<cudaEvent_t, 4>> ev_rec;
  std::vector<std::array<int, 3>> ev_launches;
};

// NVTX range for the duration of a scope (host side; visible in timeline tools)
struct NvtxRange {
  explicit NvtxRange(const char* name);
  ~NvtxRange();
};

// error reporting (thread-local message)
void set_error(const std::string& msg);
fe_ks_status fail(fe_ks_status code, const std::string& msg);

// greedy cell colouring (fe_ks_api.cu); returns the colour count or -1 (> 64)
int greedy_colouring(int64_t E, int np3, int64_t m, const int* cell_dofs, int* colour);

// host 1D tables (fe_ks_tables.cpp)
void gauss_legendre(int n, double* x, double* w);
void gauss_lobatto(int n, double* x, double* w);
void lagrange_eval(int n, const double* nodes, double x, double* val, double* der);
template <typename T>
void build_eo_tables(int p, int nq, EOTables<T>* out);
template <>
void build_eo_tables<ff2>(int p, int nq, EOTables<ff2>* out);
// B-operand fragments of the tensor-core cell kernel for degree p (n_q = p + 1):
// out[((op * 2 + tile) * 32 + lane) * 2 + reg], op 0 = N (nodes -> Gauss
// points), 1 = D (Gauss-point derivative of the nodal basis), 2 = N^T, 3 = D^T.
constexpr int kTcFragWords = 4 * 2 * 32 * 2;
// kind: 0 = BF16, 1 = FP16, 2 = the BF16 remainder x - bf16(x) (low part of the split)
void build_tc_frags(int p, uint32_t* out, int kind);
uint16_t bf16_bits(double x);   // nearest BF16 (ties to even), as its bit pattern
uint16_t bf16_lo_bits(double x);   // nearest BF16 of x - bf16(x)
uint16_t f16_bits(double x);    // nearest FP16 (ties to even), as its bit pattern
// The projector matrices F [pair][n_proj][n^3] (complex: x2 interleaved) as BF16
// B fragments of the tensor-core kernel's expansion MMAs:
// out[pair][row tile][half][8-column tile][K step][lane] (uint2 per lane).
void build_tc_fpack(int n, bool cplx, int n_proj, int64_t n_pairs, const double* F, int kind, std::vector<uint2>& out);

// Y (+)= alpha H X or alpha Hs X on the context's stream; zero_fill clears Y first.
// tc: FP32 storage with the tensor-core cell kernel (T = float only): 0 = off,
// 1 = BF16, 2 = FP16, 3 = BF16 hi + lo split (FE_KS_BF16X2).
template <typename T>
fe_ks_status apply_core(Ctx& c, const T* X, T* Y, int64_t ncols, bool scaled, T alpha, bool zero_fill,
                        int tc = 0);
fe_ks_status apply_core_emu(Ctx& c, const double* X, double* Y, int64_t ncols, bool scaled, double alpha,
                            bool zero_fill);

constexpr int kLocalConfigs = 10;

// Row chunk of the split Gram products: partials [chunk][n1][n2] of 8192 rows each,
// summed in chunk order by launch_gram_reduce (compensated; upper = mirror the
// upper triangle of a symmetric product).
constexpr int kGramChunkRows = 8192;
cudaError_t launch_gram_reduce(const double* part, double* C, int nchunks, int n1, int n2, int upper, cudaStream_t s);

// kernel launchers (fe_ks_local_pN.cu)
template <typename T, typename TS>
cudaError_t launch_local(const Ctx& c, const LocalParams<T, TS>& prm, cudaStream_t s);
template <typename T>
cudaError_t launch_proj(const Ctx& c, const ProjParams<T>& prm, int n_atoms, cudaStream_t s);
cudaError_t launch_proj_emu(const Ctx& c, const ProjParams<double>& prm, const ff2* F, int n_atoms, cudaStream_t s);
// pair form of the projection (needs prm.part and prm.n_pairs)
template <typename T>
cudaError_t launch_proj_pairs(const Ctx& c, const ProjParams<T>& prm, int n_atoms, cudaStream_t s);
cudaError_t launch_proj_pairs_emu(const Ctx& c, const ProjParams<double>& prm, const ff2* F, int n_atoms,
                                  cudaStream_t s);
// BF16 tensor-core cell kernel (fe_ks_tc.cu) for one colour of cells
cudaError_t launch_tc(const Ctx& c, const LocalParams<float>& lp, cudaStream_t s, int tc);
size_t tc_smem_bytes(int n, bool cplx);
// tcgen05 cell kernel (fe_ks_tc5.cu): real operators, n_q = n_p; f16 selects FP16 operands
cudaError_t launch_tc5(const Ctx& c, const LocalParams<float>& lp, cudaStream_t s, bool f16, int stagger);
void build_tc5_const(int p, bool f16, std::vector<uint4>& out);
// stagger point of the tcgen05 kernel's two pipelines for a 16-bit tile configuration (0, 2, 3)
inline int tc5_stagger(int cfg) { return cfg == 2 ? 0 : cfg == 3 ? 2 : 1; }
// true when the tcgen05 kernel serves this context and precision (tc: 1 = BF16, 2 = FP16)
inline bool use_tc5(const Ctx& c, int tc) {
  return (tc == 1 || tc == 2) && c.cfg_tc[tc - 1] != 1 && !c.cplx && c.nq == c.np && c.tc5_cst && c.tc5_cst16;
}

}  // namespace feks

// The opaque handle of the C interface.
struct fe_ks_ctx {
  feks::Ctx c;
};
