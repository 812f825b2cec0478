// Device side of the batched persistent launch: work-item routines and the
// persistent kernel, templated on the block size NT.  Included by one
// translation unit per block size (fe_ks_batched_k.cu) and, for the shared
// structures and the host-side size helpers, by fe_ks_batched.cu.
#pragma once
#include "fe_ks_local.cuh"

namespace feks {

constexpr int kMaxSys = 16;
constexpr int kMaxPhase = 66;
// Block sizes the persistent kernel is compiled for (one translation unit
// each); fe_ks_batch_configure picks one.  384 is the default; 256 serves the
// FP64 half of a split batch (fe_ks_batch_set_split).
constexpr int kBatchThreads[4] = {384, 512, 672, 256};
// Precision classes of a kernel object: every routine, or the FP64 / FP32 ones
// only (a split batch runs one persistent launch per class, concurrently).
enum : int { kClassAll = 0, kClassF64 = 1, kClassF32 = 2 };
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
// columns and divides the block size nt (672 = 21 x 32 takes 32).
__host__ __device__ inline int batch_proj_cw(int ncols, int nt) {
  const int cw = ncols <= 32 ? 32 : ncols <= 64 ? 64 : 128;
  return nt % cw == 0 ? cw : 32;
}

// Shared memory of a projection item: the pair's F block, the cell's DoF list
// and the slice reduction buffer.
template <typename T>
__host__ __device__ inline size_t batch_proj_bytes(int n_proj, int np3, int cw, int nt) {
  const size_t head = ((size_t)n_proj * np3 * sizeof(T) + (size_t)np3 * sizeof(int) + 15) & ~(size_t)15;
  return head + (size_t)(nt / cw) * n_proj * cw * sizeof(T);
}

// part[pr][b][col] = sum_node F[pr][b][node] x(d(node), col) for columns
// [col0, col0 + cw): one column per thread, NT / cw row slices reduced
// in shared memory in slice order.
template <typename T, int NT>
__device__ void pair_item(const BatchSys& s, int pr, int col0, int cw, unsigned char* smem) {
  const int np3 = s.np3, n_proj = s.n_proj;
  T* Fs = reinterpret_cast<T*>(smem);
  int* ds = reinterpret_cast<int*>(smem + (size_t)n_proj * np3 * sizeof(T));
  T* red = reinterpret_cast<T*>(smem + (((size_t)n_proj * np3 * sizeof(T) + (size_t)np3 * sizeof(int) + 15) & ~(size_t)15));
  const int rs = NT / cw;
  const int lc = threadIdx.x % cw, sl = threadIdx.x / cw;   // sl < rs: cw divides NT (batch_proj_cw)
  const int col = col0 + lc;
  const bool act = col < s.ncols;
  const T* X = static_cast<const T*>(s.X);
  const T* Fp = static_cast<const T*>(s.F) + (int64_t)pr * n_proj * np3;
  for (int i = threadIdx.x; i < n_proj * np3; i += NT) Fs[i] = Fp[i];
  const int cell = s.pair_cell[pr];
  for (int i = threadIdx.x; i < np3; i += NT) ds[i] = s.cell_dofs[(int64_t)cell * np3 + i];
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
  for (int idx = threadIdx.x; idx < n_proj * cw; idx += NT) {
    const int b = idx / cw, c = idx % cw;
    T v = red[(size_t)b * cw + c];
    for (int k = 1; k < rs; ++k) v += red[((size_t)k * n_proj + b) * cw + c];
    if (col0 + c < s.ncols) part[((int64_t)pr * n_proj + b) * s.ncols + col0 + c] = v;
  }
}

// Q[a][b][col] = h[a][b] * sum over the pairs of atom a, in pair order, of part[pr][b][col]
template <typename T, int NT>
__device__ void sum_item(const BatchSys& s, int a, int col0, int cw) {
  const T* part = static_cast<const T*>(s.part);
  const T* h = static_cast<const T*>(s.h);
  T* Q = static_cast<T*>(s.Q);
  for (int idx = threadIdx.x; idx < s.n_proj * cw; idx += NT) {
    const int b = idx / cw, col = col0 + idx % cw;
    if (col >= s.ncols) continue;
    T v = T(0);
    for (int pr = s.atom_pair_ptr[a]; pr < s.atom_pair_ptr[a + 1]; ++pr)
      v += part[((int64_t)pr * s.n_proj + b) * s.ncols + col];
    Q[((int64_t)a * s.n_proj + b) * s.ncols + col] = v * h[a * s.n_proj + b];
  }
}

template <typename T, int P, int CFG, int NT>
__device__ __forceinline__ void local_cells(const BatchSys& s, const EOTables<T>& tb, int c0, int nc, int col0,
                                            unsigned char* smem) {
  constexpr int NQ = P + 1;
  const SysArgs<T> a = sys_args<T>(s);
  for (int k = 0; k < nc; ++k)
    cell_tile<T, P + 1, NQ, cfg_vt<NQ>(CFG), false, NT>(a, tb, s.colour_cells[c0 + k], col0, smem);
}

template <typename T, int NT>
__device__ __forceinline__ void local_item(const BatchSys& s, const EOTables<T>* tabs, int c0, int nc, int col0,
                                           unsigned char* smem) {
#define FEKS_LOCAL_CASE(P)                                                  \
  case P:                                                                   \
    if (s.cfg == 1)                                                         \
      local_cells<T, P, 1, NT>(s, tabs[P], c0, nc, col0, smem);             \
    else                                                                    \
      local_cells<T, P, 0, NT>(s, tabs[P], c0, nc, col0, smem);             \
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

template <int NT, int MINB, int CLS = kClassAll>
__global__ void __launch_bounds__(NT, MINB) fe_batched_kernel(const __grid_constant__ BatchParams bp) {
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
      // a class object only holds its own routines (the host queues only its systems' items)
      if (s.prec == FE_KS_F64) {
        if constexpr (CLS != kClassF32) {
          if (kind == kItemZero)
            zero_item<double>(s, w.y, w.w);
          else if (kind == kItemPair)
            pair_item<double, NT>(s, w.y, w.z, w.w, smem);
          else if (kind == kItemSum)
            sum_item<double, NT>(s, w.y, w.z, w.w);
          else
            local_item<double, NT>(s, bp.t64, w.y, w.w, w.z, smem);
        }
      } else {
        if constexpr (CLS != kClassF64) {
          if (kind == kItemZero)
            zero_item<float>(s, w.y, w.w);
          else if (kind == kItemPair)
            pair_item<float, NT>(s, w.y, w.z, w.w, smem);
          else if (kind == kItemSum)
            sum_item<float, NT>(s, w.y, w.z, w.w);
          else
            local_item<float, NT>(s, bp.t32, w.y, w.w, w.z, smem);
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bp.done + sidx * kMaxPhase + phase, 1);
      }
    }
  }
}

// Per-block-size entry points, defined in fe_ks_batched_k.cu (one object per
// block size): shared-memory opt-in and occupancy, and the launch.
template <int NT>
cudaError_t batched_prepare(size_t smem, int blocks_per_sm, int* per_sm);
template <int NT>
cudaError_t batched_launch(const BatchParams& P, int grid, size_t smem, int blocks_per_sm, cudaStream_t s);
// one-class objects (one CTA per SM budget, so that the other class's object can share the SM)
template <int NT>
cudaError_t batched_prepare_class(int cls, size_t smem, int* per_sm);
template <int NT>
cudaError_t batched_launch_class(int cls, const BatchParams& P, int grid, size_t smem, cudaStream_t s);

}  // namespace feks
