// Batched application of many independent operators in one persistent launch.
//
// Y_s = H_s X_s for systems s of uneven size, degree, vector count and
// precision (FP64 / FP32).  The host builds one work queue, phase-major:
//   phase 0        : zero-fill slices of every Y_s and the per-pair projection
//                    partials F^(a,e)^H X^(e) (eq. AXmatrixfreenonloc, first factor),
//   phase 1        : per-atom sums of the partials in pair order, scaled by Delta
//                    (systems with projectors only),
//   phase o + c    : the cells of colour c of every system (o = 2 with
//                    projectors, 1 without; Algorithm 2 on a tile of cells x
//                    columns, expansion and scatter-add fused).
// Persistent CTAs claim items in queue order with one atomic counter.  An
// item of phase k of system s first waits until every item of phase k - 1 of
// the same system has finished (per-(system, phase) completion counters with
// release/acquire ordering).  An item only ever waits on items earlier in the
// queue, which were claimed by running CTAs, so the queue drains without any
// co-residency assumption.  Every wait is bounded: on expiry the CTA sets the
// error flag and leaves; the host reports FE_KS_ERR_TIMEOUT.
//
// Tunables (fe_ks_batch_tune): columns per tile (the per-precision tile
// configuration of the fused kernel), cells per work item, and the number of
// items a CTA claims per atomic fetch.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "fe_ks_local.cuh"

namespace feks {

constexpr int kMaxSys = 16;
constexpr int kMaxPhase = 66;
constexpr int kBatchNT = 384;
enum : int { kItemZero = 0, kItemPair = 1, kItemLocal = 2, kItemSum = 3 };

struct BatchSys {
  int prec;        // FE_KS_F64 or FE_KS_F32
  int p;           // degree
  int cfg;         // tile configuration (0 or 1)
  int ncols;
  int64_t m;
  const void* X;
  void* Y;
  const int* cell_dofs;
  const int* colour_cells;
  const void* coef;
  int ncoef;
  int gga;
  const int* cell_pair_ptr;   // nullptr without projectors
  const int* cell_pairs;
  const int* pair_atom;
  const void* F;
  void* Q;
  const void* h;
  const int* atom_pair_ptr;
  const int* pair_cell;
  void* part;      // projection partials [pair][n_proj][ncols]
  int n_proj;
  int np3;
};

struct BatchParams {
  BatchSys sys[kMaxSys];
  EOTables<double> t64[9];
  EOTables<float> t32[9];
  const int4* items;
  int n_items;
  int* queue;
  int* done;         // [kMaxSys][kMaxPhase]
  const int* need;   // [kMaxSys][kMaxPhase]
  int* err;
  long long wait_cycles;
  int depth;
};

// Operand view of one system for the cell routine (field names of LocalParams).
template <typename T>
struct SysArgs {
  const T* X;
  T* Y;
  int64_t ld;
  int ncols;
  const int* cell_dofs;
  const T* coef;
  int ncoef;
  int gga;
  const T* dscale;
  const int* cell_pair_ptr;
  const int* cell_pairs;
  const int* pair_atom;
  const T* F;
  const T* Q;
  int n_proj;
  T alpha;
};

template <typename T>
__device__ __forceinline__ SysArgs<T> sys_args(const BatchSys& s) {
  SysArgs<T> a;
  a.X = static_cast<const T*>(s.X);
  a.Y = static_cast<T*>(s.Y);
  a.ld = s.ncols;
  a.ncols = s.ncols;
  a.cell_dofs = s.cell_dofs;
  a.coef = static_cast<const T*>(s.coef);
  a.ncoef = s.ncoef;
  a.gga = s.gga;
  a.dscale = nullptr;
  a.cell_pair_ptr = s.cell_pair_ptr;
  a.cell_pairs = s.cell_pairs;
  a.pair_atom = s.pair_atom;
  a.F = static_cast<const T*>(s.F);
  a.Q = static_cast<const T*>(s.Q);
  a.n_proj = s.n_proj;
  a.alpha = T(1);
  return a;
}

template <typename T>
__device__ void zero_item(const BatchSys& s, int row0, int rows) {
  T* Y = static_cast<T*>(s.Y) + (int64_t)row0 * s.ncols;
  const int64_t n = (int64_t)rows * s.ncols;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) Y[i] = T(0);
}

// Columns per projection item: the smallest of 32, 64, 128 that covers the
// columns (each divides the block size).
__host__ __device__ inline int batch_proj_cw(int ncols) { return ncols <= 32 ? 32 : ncols <= 64 ? 64 : 128; }

// Shared memory of a projection item: the pair's F block, the cell's DoF list
// and the slice reduction buffer.
template <typename T>
__host__ __device__ inline size_t batch_proj_bytes(int n_proj, int np3, int cw) {
  const size_t head = ((size_t)n_proj * np3 * sizeof(T) + (size_t)np3 * sizeof(int) + 15) & ~(size_t)15;
  return head + (size_t)(kBatchNT / cw) * n_proj * cw * sizeof(T);
}

// part[pr][b][col] = sum_node F[pr][b][node] x(d(node), col) for columns
// [col0, col0 + cw): one column per thread, kBatchNT / cw row slices reduced
// in shared memory in slice order.
template <typename T>
__device__ void pair_item(const BatchSys& s, int pr, int col0, int cw, unsigned char* smem) {
  const int np3 = s.np3, n_proj = s.n_proj;
  T* Fs = reinterpret_cast<T*>(smem);
  int* ds = reinterpret_cast<int*>(smem + (size_t)n_proj * np3 * sizeof(T));
  T* red = reinterpret_cast<T*>(smem + (((size_t)n_proj * np3 * sizeof(T) + (size_t)np3 * sizeof(int) + 15) & ~(size_t)15));
  const int rs = kBatchNT / cw;
  const int lc = threadIdx.x % cw, sl = threadIdx.x / cw;
  const int col = col0 + lc;
  const bool act = col < s.ncols;
  const T* X = static_cast<const T*>(s.X);
  const T* Fp = static_cast<const T*>(s.F) + (int64_t)pr * n_proj * np3;
  for (int i = threadIdx.x; i < n_proj * np3; i += kBatchNT) Fs[i] = Fp[i];
  const int cell = s.pair_cell[pr];
  for (int i = threadIdx.x; i < np3; i += kBatchNT) ds[i] = s.cell_dofs[(int64_t)cell * np3 + i];
  __syncthreads();
  T acc[16];
#pragma unroll
  for (int b = 0; b < 16; ++b) acc[b] = T(0);
  constexpr int RU = 4;
  for (int n0 = sl; n0 < np3; n0 += RU * rs) {
    T xs[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int node = n0 + u * rs;
      xs[u] = (node < np3 && act) ? X[(int64_t)ds[node] * s.ncols + col] : T(0);
    }
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int node = n0 + u * rs;
      if (node >= np3) break;
#pragma unroll
      for (int b = 0; b < 16; ++b)
        if (b < n_proj) acc[b] = fma(Fs[b * np3 + node], xs[u], acc[b]);
    }
  }
#pragma unroll
  for (int b = 0; b < 16; ++b)
    if (b < n_proj) red[((size_t)sl * n_proj + b) * cw + lc] = acc[b];
  __syncthreads();
  T* part = static_cast<T*>(s.part);
  for (int idx = threadIdx.x; idx < n_proj * cw; idx += kBatchNT) {
    const int b = idx / cw, c = idx % cw;
    T v = red[(size_t)b * cw + c];
    for (int k = 1; k < rs; ++k) v += red[((size_t)k * n_proj + b) * cw + c];
    if (col0 + c < s.ncols) part[((int64_t)pr * n_proj + b) * s.ncols + col0 + c] = v;
  }
}

// Q[a][b][col] = h[a][b] * sum over the pairs of atom a, in pair order, of part[pr][b][col]
template <typename T>
__device__ void sum_item(const BatchSys& s, int a, int col0, int cw) {
  const T* part = static_cast<const T*>(s.part);
  const T* h = static_cast<const T*>(s.h);
  T* Q = static_cast<T*>(s.Q);
  for (int idx = threadIdx.x; idx < s.n_proj * cw; idx += kBatchNT) {
    const int b = idx / cw, col = col0 + idx % cw;
    if (col >= s.ncols) continue;
    T v = T(0);
    for (int pr = s.atom_pair_ptr[a]; pr < s.atom_pair_ptr[a + 1]; ++pr)
      v += part[((int64_t)pr * s.n_proj + b) * s.ncols + col];
    Q[((int64_t)a * s.n_proj + b) * s.ncols + col] = v * h[a * s.n_proj + b];
  }
}

template <typename T, int P, int CFG>
__device__ __forceinline__ void local_cells(const BatchParams& bp, const BatchSys& s, const EOTables<T>& tb, int c0,
                                            int nc, int col0, unsigned char* smem) {
  constexpr int NQ = P + 1;
  const SysArgs<T> a = sys_args<T>(s);
  for (int k = 0; k < nc; ++k)
    cell_tile<T, P + 1, NQ, cfg_vt<NQ>(CFG), false, kBatchNT>(a, tb, s.colour_cells[c0 + k], col0, smem);
}

template <typename T>
__device__ __forceinline__ void local_item(const BatchParams& bp, const BatchSys& s, const EOTables<T>* tabs, int c0,
                                           int nc, int col0, unsigned char* smem) {
#define FEKS_LOCAL_CASE(P)                                                       \
  case P:                                                                        \
    if (s.cfg == 1)                                                              \
      local_cells<T, P, 1>(bp, s, tabs[P], c0, nc, col0, smem);                  \
    else                                                                         \
      local_cells<T, P, 0>(bp, s, tabs[P], c0, nc, col0, smem);                  \
    break;
  switch (s.p) {
    FEKS_LOCAL_CASE(4)
    FEKS_LOCAL_CASE(5)
    FEKS_LOCAL_CASE(6)
    FEKS_LOCAL_CASE(7)
    FEKS_LOCAL_CASE(8)
    default: break;
  }
#undef FEKS_LOCAL_CASE
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int MINB>
__global__ void __launch_bounds__(kBatchNT, MINB) fe_batched_kernel(const __grid_constant__ BatchParams bp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_base, s_stop;
  for (;;) {
    if (threadIdx.x == 0) {
      s_base = atomicAdd(bp.queue, bp.depth);
      s_stop = 0;
    }
    __syncthreads();
    const int base = s_base;
    if (base >= bp.n_items) break;
    for (int it = base; it < base + bp.depth && it < bp.n_items; ++it) {
      const int4 w = bp.items[it];
      const int sidx = w.x & 0xff, kind = (w.x >> 8) & 0xff, phase = w.x >> 16;
      const BatchSys& s = bp.sys[sidx];
      if (phase > 0 && threadIdx.x == 0) {
        const int* ctr = bp.done + sidx * kMaxPhase + phase - 1;
        const int need = bp.need[sidx * kMaxPhase + phase - 1];
        const long long t0 = clock64();
        while (ld_acquire(ctr) < need) {
          if (ld_acquire(bp.err) != 0 || clock64() - t0 > bp.wait_cycles) {
            atomicExch(bp.err, 1);
            s_stop = 1;
            break;
          }
          __nanosleep(256);
        }
        __threadfence();
      }
      __syncthreads();
      if (s_stop) return;   // bounded wait expired (or another CTA gave up): leave, the host reports it
      if (kind == kItemZero) {
        if (s.prec == FE_KS_F64)
          zero_item<double>(s, w.y, w.w);
        else
          zero_item<float>(s, w.y, w.w);
      } else if (kind == kItemPair) {
        if (s.prec == FE_KS_F64)
          pair_item<double>(s, w.y, w.z, w.w, smem);
        else
          pair_item<float>(s, w.y, w.z, w.w, smem);
      } else if (kind == kItemSum) {
        if (s.prec == FE_KS_F64)
          sum_item<double>(s, w.y, w.z, w.w);
        else
          sum_item<float>(s, w.y, w.z, w.w);
      } else {
        if (s.prec == FE_KS_F64)
          local_item<double>(bp, s, bp.t64, w.y, w.w, w.z, smem);
        else
          local_item<float>(bp, s, bp.t32, w.y, w.w, w.z, smem);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bp.done + sidx * kMaxPhase + phase, 1);
      }
    }
  }
}

// Shared memory of one system's cell tile (host side of CellShape).
template <typename T, int P>
static size_t cell_bytes_p(int cfg) {
  constexpr int NQ = P + 1;
  return cfg == 1 ? CellShape<T, P + 1, NQ, cfg_vt<NQ>(1), false>::bytes
                  : CellShape<T, P + 1, NQ, cfg_vt<NQ>(0), false>::bytes;
}
template <typename T>
static size_t cell_bytes(int p, int cfg) {
  switch (p) {
    case 4: return cell_bytes_p<T, 4>(cfg);
    case 5: return cell_bytes_p<T, 5>(cfg);
    case 6: return cell_bytes_p<T, 6>(cfg);
    case 7: return cell_bytes_p<T, 7>(cfg);
    case 8: return cell_bytes_p<T, 8>(cfg);
    default: return 0;
  }
}
static int vt_of(int p, int cfg) { return (p + 1 >= 7) ? (cfg ? 8 : 4) : (cfg ? 16 : 8); }

}  // namespace feks

using namespace feks;

struct fe_ks_batch {
  std::vector<fe_ks_ctx*> ctxs;
  std::vector<int64_t> n_v;
  std::vector<int> prec;
  std::vector<int> cfg;
  int cells_per_item = 1;
  int depth = 1;
  int blocks_per_sm = 1;     // 1: registers for every variant; 2: two CTAs per SM, some spills
  double wait_seconds = 2.0;
  int inject_missing = 0;
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  // device buffers (allocated at create / rebuild)
  int4* d_items = nullptr;
  int n_items = 0;
  int* d_need = nullptr;
  int* d_state = nullptr;   // [queue][err][done: kMaxSys*kMaxPhase]
  BatchParams host{};
  size_t smem = 0;
  int grid = 0;
  std::vector<size_t> item_capacity;
};

static fe_ks_status batch_build(fe_ks_batch* b) {
  std::vector<int4> items;
  std::vector<int> need(kMaxSys * kMaxPhase, 0);
  const int ns = (int)b->ctxs.size();
  int max_ph = 0;
  for (int s = 0; s < ns; ++s) max_ph = std::max<int>(max_ph, (int)b->ctxs[s]->c.colour_ptr.size() - 1 + 2);
  if (max_ph >= kMaxPhase) return fail(FE_KS_ERR_UNSUPPORTED, "too many colours for the batched launch");
  std::vector<std::vector<int4>> per_phase(max_ph + 1);
  size_t smem = 0;
  for (int s = 0; s < ns; ++s) {
    const Ctx& c = b->ctxs[s]->c;
    const int ncols = (int)b->n_v[s];
    const int vt = vt_of(c.p, b->cfg[s]);
    const size_t cb = b->prec[s] == FE_KS_F64 ? cell_bytes<double>(c.p, b->cfg[s]) : cell_bytes<float>(c.p, b->cfg[s]);
    if (cb == 0 || cb > 227 * 1024) return fail(FE_KS_ERR_UNSUPPORTED, "tile configuration does not fit");
    smem = std::max(smem, cb);
    // phase 0: zero-fill slices and projections
    const int rows = std::max(1, 65536 / ncols);
    for (int64_t r = 0; r < c.m; r += rows) {
      per_phase[0].push_back(make_int4(s | (kItemZero << 8), (int)r, 0, (int)std::min<int64_t>(rows, c.m - r)));
      need[s * kMaxPhase + 0]++;
    }
    const bool nl = (c.terms & FE_KS_TERM_NL) && c.n_pairs > 0;
    if (nl) {
      const int cw = batch_proj_cw(ncols);
      smem = std::max(smem, b->prec[s] == FE_KS_F64 ? batch_proj_bytes<double>(c.n_proj, c.np3, cw)
                                                    : batch_proj_bytes<float>(c.n_proj, c.np3, cw));
      for (int64_t pr = 0; pr < c.n_pairs; ++pr)
        for (int col = 0; col < ncols; col += cw) {
          per_phase[0].push_back(make_int4(s | (kItemPair << 8), (int)pr, col, cw));
          need[s * kMaxPhase + 0]++;
        }
      for (int a = 0; a < c.n_atoms; ++a)
        for (int col = 0; col < ncols; col += cw) {
          per_phase[1].push_back(make_int4(s | (kItemSum << 8) | (1 << 16), a, col, cw));
          need[s * kMaxPhase + 1]++;
        }
    }
    const int ph0 = nl ? 2 : 1;   // no empty phase: a colour waits on the phase just before it
    for (int col = 0; col + 1 < (int)c.colour_ptr.size(); ++col) {
      const int ph = col + ph0;
      for (int c0 = c.colour_ptr[col]; c0 < c.colour_ptr[col + 1]; c0 += b->cells_per_item) {
        const int nc = std::min(b->cells_per_item, c.colour_ptr[col + 1] - c0);
        for (int t = 0; t < ncols; t += vt) {
          per_phase[ph].push_back(make_int4(s | (kItemLocal << 8) | (ph << 16), c0, t, nc));
          need[s * kMaxPhase + ph]++;
        }
      }
    }
  }
  for (auto& v : per_phase) items.insert(items.end(), v.begin(), v.end());
  if (b->inject_missing) need[0]++;   // host-side fault injection: one item that is never published
  // (re)allocate device queue
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  if (cudaMalloc(&b->d_items, items.size() * sizeof(int4)) != cudaSuccess) return fail(FE_KS_ERR_OOM, "batch queue");
  cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_need, need.data(), need.size() * sizeof(int), cudaMemcpyHostToDevice);
  b->n_items = (int)items.size();
  b->smem = smem;
  if (cudaFuncSetAttribute(fe_batched_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(fe_batched_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return fail(FE_KS_ERR_CUDA, "batched kernel shared memory");
  int per_sm = 0;
  if (b->blocks_per_sm == 2)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fe_batched_kernel<2>, kBatchNT, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fe_batched_kernel<1>, kBatchNT, smem);
  b->grid = std::max(1, per_sm) * b->sms;
  // kernel parameters
  BatchParams& P = b->host;
  P = BatchParams{};
  for (int s = 0; s < ns; ++s) {
    const Ctx& c = b->ctxs[s]->c;
    BatchSys& d = P.sys[s];
    const bool f64 = b->prec[s] == FE_KS_F64;
    d.prec = b->prec[s];
    d.p = c.p;
    d.cfg = b->cfg[s];
    d.ncols = (int)b->n_v[s];
    d.m = c.m;
    d.cell_dofs = c.cell_dofs;
    d.colour_cells = c.colour_cells;
    d.coef = f64 ? (const void*)c.f64.coef : (const void*)c.f32.coef;
    d.ncoef = c.ncoef;
    d.gga = c.gga;
    const bool nl = (c.terms & FE_KS_TERM_NL) && c.n_pairs > 0;
    d.cell_pair_ptr = nl ? c.cell_pair_ptr : nullptr;
    d.cell_pairs = c.cell_pairs;
    d.pair_atom = c.pair_atom;
    d.F = f64 ? (const void*)c.f64.F : (const void*)c.f32.F;
    d.Q = f64 ? (void*)c.f64.Q : (void*)c.f32.Q;
    d.h = f64 ? (const void*)c.h64 : (const void*)c.h32;
    d.atom_pair_ptr = c.atom_pair_ptr;
    d.pair_cell = c.pair_cell;
    d.part = f64 ? (void*)c.f64.part : (void*)c.f32.part;
    d.n_proj = c.n_proj;
    d.np3 = c.np3;
    build_eo_tables<double>(c.p, c.nq, &P.t64[c.p]);
    build_eo_tables<float>(c.p, c.nq, &P.t32[c.p]);
  }
  P.items = b->d_items;
  P.n_items = b->n_items;
  P.queue = b->d_state;
  P.err = b->d_state + 1;
  P.done = b->d_state + 2;
  P.need = b->d_need;
  P.depth = b->depth;
  int khz = 0;
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, b->device);
  P.wait_cycles = (long long)(b->wait_seconds * (khz > 0 ? khz : 2000000) * 1e3);
  return FE_KS_OK;
}

extern "C" {

fe_ks_status fe_ks_batch_create(fe_ks_ctx* const* ctxs, int n_sys, const int64_t* n_v, const int* precision,
                                fe_ks_batch** out) {
  set_error("");
  if (!ctxs || !n_v || !precision || !out) return fail(FE_KS_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (n_sys < 1 || n_sys > kMaxSys) return fail(FE_KS_ERR_ARG, "n_sys must be in 1..16");
  for (int s = 0; s < n_sys; ++s) {
    if (!ctxs[s]) return fail(FE_KS_ERR_ARG, "NULL context");
    const Ctx& c = ctxs[s]->c;
    if (c.cplx) return fail(FE_KS_ERR_UNSUPPORTED, "the batched launch supports real operators");
    if (c.p < 4 || c.p > 8) return fail(FE_KS_ERR_UNSUPPORTED, "the batched launch supports degrees 4..8");
    if (c.nq != c.np) return fail(FE_KS_ERR_UNSUPPORTED, "the batched launch supports n_q = n_p");
    if (n_v[s] < 1 || n_v[s] > c.n_v_max) return fail(FE_KS_ERR_ARG, "n_v out of range");
    if (precision[s] != FE_KS_F64 && precision[s] != FE_KS_F32) return fail(FE_KS_ERR_ARG, "unknown precision");
    if (c.colour_ptr.size() - 1 > (size_t)kMaxPhase - 1) return fail(FE_KS_ERR_UNSUPPORTED, "too many colours");
    if (c.n_proj > 16) return fail(FE_KS_ERR_UNSUPPORTED, "n_proj > 16");
  }
  auto* b = new fe_ks_batch();
  b->ctxs.assign(ctxs, ctxs + n_sys);
  b->n_v.assign(n_v, n_v + n_sys);
  b->prec.assign(precision, precision + n_sys);
  b->cfg.assign(n_sys, 0);
  b->stream = ctxs[0]->c.stream;
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  if (cudaMalloc(&b->d_need, sizeof(int) * kMaxSys * kMaxPhase) != cudaSuccess ||
      cudaMalloc(&b->d_state, sizeof(int) * (2 + kMaxSys * kMaxPhase)) != cudaSuccess) {
    if (b->d_need) cudaFree(b->d_need);
    delete b;
    return fail(FE_KS_ERR_OOM, "batch state");
  }
  fe_ks_status st = batch_build(b);
  if (st != FE_KS_OK) {
    std::string msg = fe_ks_last_error();
    cudaFree(b->d_need);
    cudaFree(b->d_state);
    if (b->d_items) cudaFree(b->d_items);
    delete b;
    return fail(st, msg);
  }
  *out = b;
  return FE_KS_OK;
}

fe_ks_status fe_ks_batch_configure(fe_ks_batch* b, const int* tile_config, int cells_per_item, int depth,
                                   int blocks_per_sm, double wait_seconds, int inject_missing_item) {
  if (!b) return fail(FE_KS_ERR_ARG, "batch is NULL");
  if (blocks_per_sm != 1 && blocks_per_sm != 2) return fail(FE_KS_ERR_ARG, "blocks_per_sm must be 1 or 2");
  b->blocks_per_sm = blocks_per_sm;
  if (cells_per_item < 1 || cells_per_item > 64 || depth < 1 || depth > 16 || !(wait_seconds > 0))
    return fail(FE_KS_ERR_ARG, "cells_per_item in 1..64, depth in 1..16, wait_seconds > 0");
  if (tile_config)
    for (size_t s = 0; s < b->ctxs.size(); ++s) {
      if (tile_config[s] < 0 || tile_config[s] > 1) return fail(FE_KS_ERR_ARG, "tile_config must be 0 or 1");
      b->cfg[s] = tile_config[s];
    }
  b->cells_per_item = cells_per_item;
  b->depth = depth;
  b->wait_seconds = wait_seconds;
  b->inject_missing = inject_missing_item != 0;
  return batch_build(b);
}

fe_ks_status fe_ks_batch_apply(fe_ks_batch* b, const void* const* X, void* const* Y, void* cuda_stream) {
  if (!b || !X || !Y) return fail(FE_KS_ERR_ARG, "NULL argument");
  cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : b->stream;
  BatchParams P = b->host;
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    if (!X[i] || !Y[i]) return fail(FE_KS_ERR_ARG, "NULL X or Y");
    P.sys[i].X = X[i];
    P.sys[i].Y = Y[i];
  }
  if (cudaMemsetAsync(b->d_state, 0, sizeof(int) * (2 + kMaxSys * kMaxPhase), s) != cudaSuccess)
    return fail(FE_KS_ERR_CUDA, "reset of the batch counters failed");
  if (b->blocks_per_sm == 2)
    fe_batched_kernel<2><<<b->grid, kBatchNT, b->smem, s>>>(P);
  else
    fe_batched_kernel<1><<<b->grid, kBatchNT, b->smem, s>>>(P);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("batched kernel: ") + cudaGetErrorString(err));
  return FE_KS_OK;
}

fe_ks_status fe_ks_batch_status(fe_ks_batch* b) {
  if (!b) return fail(FE_KS_ERR_ARG, "batch is NULL");
  int err = 0;
  if (cudaMemcpy(&err, b->d_state + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(FE_KS_ERR_CUDA, "reading the batch status failed");
  if (err) return fail(FE_KS_ERR_TIMEOUT, "a batched work item waited longer than the configured limit");
  return FE_KS_OK;
}

fe_ks_status fe_ks_batch_info(const fe_ks_batch* b, int* n_items, int* grid, size_t* smem_bytes) {
  if (!b) return fail(FE_KS_ERR_ARG, "batch is NULL");
  if (n_items) *n_items = b->n_items;
  if (grid) *grid = b->grid;
  if (smem_bytes) *smem_bytes = b->smem;
  return FE_KS_OK;
}

void fe_ks_batch_destroy(fe_ks_batch* b) {
  if (!b) return;
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_need) cudaFree(b->d_need);
  if (b->d_state) cudaFree(b->d_state);
  delete b;
}

}  // extern "C"
