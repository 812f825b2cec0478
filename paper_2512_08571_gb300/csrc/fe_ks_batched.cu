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
// Tunables (fe_ks_batch_configure): per system the column tile of the cell
// routine (narrow or wide), cells per work item, the number of items a CTA
// claims per atomic fetch, the block size (384, 512 or 672 threads, one
// kernel object each) and the resident CTAs per SM.  The device code is in
// fe_ks_batched.cuh.
//
// Split mode (fe_ks_batch_set_split): the FP64 systems' items and the FP32
// systems' items go to two queues, each drained by a persistent kernel object
// that holds only that precision's routines (its own register budget), and
// the two launches run concurrently (stream fork / join with events, so the
// pair still captures as one graph).  FP64 items keep the SM's FP64 pipe busy
// and FP32 items its FP32 pipe, so CTAs of the two objects sharing an SM
// overlap.  Items still wait only on earlier items of their own system, which
// sit in the same queue.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "fe_ks_batched.cuh"

namespace feks {

// Shared memory of one system's cell item (host side of CellShape).
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

static cudaError_t prepare_nt(int nt, size_t smem, int blocks_per_sm, int* per_sm) {
  switch (nt) {
    case 384: return batched_prepare<384>(smem, blocks_per_sm, per_sm);
    case 512: return batched_prepare<512>(smem, blocks_per_sm, per_sm);
    case 672: return batched_prepare<672>(smem, blocks_per_sm, per_sm);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t launch_nt(int nt, const BatchParams& P, int grid, size_t smem, int blocks_per_sm,
                             cudaStream_t s) {
  switch (nt) {
    case 384: return batched_launch<384>(P, grid, smem, blocks_per_sm, s);
    case 512: return batched_launch<512>(P, grid, smem, blocks_per_sm, s);
    case 672: return batched_launch<672>(P, grid, smem, blocks_per_sm, s);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t prepare_class_nt(int nt, int cls, size_t smem, int* per_sm) {
  switch (nt) {
    case 256: return batched_prepare_class<256>(cls, smem, per_sm);
    case 384: return batched_prepare_class<384>(cls, smem, per_sm);
    case 512: return batched_prepare_class<512>(cls, smem, per_sm);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t launch_class_nt(int nt, int cls, const BatchParams& P, int grid, size_t smem, cudaStream_t s) {
  switch (nt) {
    case 256: return batched_launch_class<256>(cls, P, grid, smem, s);
    case 384: return batched_launch_class<384>(cls, P, grid, smem, s);
    case 512: return batched_launch_class<512>(cls, P, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

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
  int nt = kBatchThreads[0]; // threads per CTA (one of kBatchThreads)
  double wait_seconds = 2.0;
  int inject_missing = 0;
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  // device buffers (allocated at create / rebuild)
  int4* d_items = nullptr;
  int n_items = 0;
  int* d_need = nullptr;
  int* d_state = nullptr;   // [queue][queue of the FP32 class][err][done: kMaxSys*kMaxPhase]
  BatchParams host{};
  size_t smem = 0;
  int grid = 0;
  std::vector<size_t> item_capacity;
  // split mode: block sizes of the FP64 and FP32 objects (0 = off), their queues and grids
  int split_nt[2] = {0, 0};
  int4* d_items_cls[2] = {nullptr, nullptr};
  int n_items_cls[2] = {0, 0};
  size_t smem_cls[2] = {0, 0};
  int grid_cls[2] = {0, 0};
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // direct systems (fe_ks_batch_set_direct): applied by their own tuned cell kernels, each
  // on a side stream of its own, concurrently with the persistent launch of the others
  std::vector<int> direct;
  std::vector<int> forced;   // systems the persistent routines do not cover: always direct
  std::vector<cudaStream_t> dstream;
  std::vector<cudaEvent_t> djoin;
  cudaEvent_t dfork = nullptr;
};

static constexpr int kStateWords = 3 + kMaxSys * kMaxPhase;

static bool batch_split(const fe_ks_batch* b) { return b->split_nt[0] > 0 && b->split_nt[1] > 0; }

static fe_ks_status batch_build(fe_ks_batch* b) {
  std::vector<int4> items;
  std::vector<int> need(kMaxSys * kMaxPhase, 0);
  const int ns = (int)b->ctxs.size();
  const bool split = batch_split(b);
  int max_ph = 0;
  for (int s = 0; s < ns; ++s)
    if (b->direct.empty() || !b->direct[s])
      max_ph = std::max<int>(max_ph, (int)b->ctxs[s]->c.colour_ptr.size() - 1 + 2);
  if (max_ph >= kMaxPhase) return fail(FE_KS_ERR_UNSUPPORTED, "too many colours for the batched launch");
  std::vector<std::vector<int4>> per_phase(max_ph + 1);
  std::vector<std::vector<int4>> per_phase_cls[2] = {std::vector<std::vector<int4>>(max_ph + 1),
                                                     std::vector<std::vector<int4>>(max_ph + 1)};
  size_t smem = 0;
  size_t smem_cls[2] = {0, 0};
  for (int s = 0; s < ns; ++s) {
    if (!b->direct.empty() && b->direct[s]) continue;   // applied by its own kernels, not from the queue
    const Ctx& c = b->ctxs[s]->c;
    const int ncols = (int)b->n_v[s];
    const int vt = vt_of(c.p, b->cfg[s]);
    const int cls = b->prec[s] == FE_KS_F64 ? 0 : 1;
    const int nt = split ? b->split_nt[cls] : b->nt;
    std::vector<std::vector<int4>>& pp = split ? per_phase_cls[cls] : per_phase;
    size_t& sm = split ? smem_cls[cls] : smem;
    const size_t cb = b->prec[s] == FE_KS_F64 ? cell_bytes<double>(c.p, b->cfg[s]) : cell_bytes<float>(c.p, b->cfg[s]);
    if (cb == 0 || cb > 227 * 1024) return fail(FE_KS_ERR_UNSUPPORTED, "tile configuration does not fit");
    sm = std::max(sm, cb);
    // phase 0: zero-fill slices and projections
    const int rows = std::max(1, 65536 / ncols);
    for (int64_t r = 0; r < c.m; r += rows) {
      pp[0].push_back(make_int4(s | (kItemZero << 8), (int)r, 0, (int)std::min<int64_t>(rows, c.m - r)));
      need[s * kMaxPhase + 0]++;
    }
    const bool nl = (c.terms & FE_KS_TERM_NL) && c.n_pairs > 0;
    if (nl) {
      const int cw = batch_proj_cw(ncols, nt);
      sm = std::max(sm, b->prec[s] == FE_KS_F64 ? batch_proj_bytes<double>(c.n_proj, c.np3, cw, nt)
                                                : batch_proj_bytes<float>(c.n_proj, c.np3, cw, nt));
      for (int64_t pr = 0; pr < c.n_pairs; ++pr)
        for (int col = 0; col < ncols; col += cw) {
          pp[0].push_back(make_int4(s | (kItemPair << 8), (int)pr, col, cw));
          need[s * kMaxPhase + 0]++;
        }
      for (int a = 0; a < c.n_atoms; ++a)
        for (int col = 0; col < ncols; col += cw) {
          pp[1].push_back(make_int4(s | (kItemSum << 8) | (1 << 16), a, col, cw));
          need[s * kMaxPhase + 1]++;
        }
    }
    const int ph0 = nl ? 2 : 1;   // no empty phase: a colour waits on the phase just before it
    for (int col = 0; col + 1 < (int)c.colour_ptr.size(); ++col) {
      const int ph = col + ph0;
      for (int c0 = c.colour_ptr[col]; c0 < c.colour_ptr[col + 1]; c0 += b->cells_per_item) {
        const int nc = std::min(b->cells_per_item, c.colour_ptr[col + 1] - c0);
        for (int t = 0; t < ncols; t += vt) {
          pp[ph].push_back(make_int4(s | (kItemLocal << 8) | (ph << 16), c0, t, nc));
          need[s * kMaxPhase + ph]++;
        }
      }
    }
  }
  if (b->inject_missing) need[0]++;   // host-side fault injection: one item that is never published
  cudaMemcpy(b->d_need, need.data(), need.size() * sizeof(int), cudaMemcpyHostToDevice);
  auto upload_items = [&](const std::vector<int4>& v, int4** dst) -> bool {
    if (*dst) cudaFree(*dst);
    *dst = nullptr;
    if (v.empty()) return true;
    if (cudaMalloc(dst, v.size() * sizeof(int4)) != cudaSuccess) return false;
    return cudaMemcpy(*dst, v.data(), v.size() * sizeof(int4), cudaMemcpyHostToDevice) == cudaSuccess;
  };
  if (split) {
    for (int k = 0; k < 2; ++k) {
      std::vector<int4> v;
      for (auto& ph : per_phase_cls[k]) v.insert(v.end(), ph.begin(), ph.end());
      if (!upload_items(v, &b->d_items_cls[k])) return fail(FE_KS_ERR_OOM, "batch queue");
      b->n_items_cls[k] = (int)v.size();
      b->smem_cls[k] = std::max<size_t>(smem_cls[k], 16);
      b->grid_cls[k] = 0;
      if (v.empty()) continue;
      int per_sm = 0;
      if (prepare_class_nt(b->split_nt[k], k == 0 ? kClassF64 : kClassF32, b->smem_cls[k], &per_sm) != cudaSuccess) {
        cudaGetLastError();
        return fail(FE_KS_ERR_CUDA, "batched class kernel shared memory / occupancy");
      }
      b->grid_cls[k] = std::max(1, per_sm) * b->sms;
    }
    b->n_items = b->n_items_cls[0] + b->n_items_cls[1];
    b->smem = std::max(b->smem_cls[0], b->smem_cls[1]);
    b->grid = b->grid_cls[0] + b->grid_cls[1];
  } else {
    for (auto& v : per_phase) items.insert(items.end(), v.begin(), v.end());
    if (!upload_items(items, &b->d_items)) return fail(FE_KS_ERR_OOM, "batch queue");
    b->n_items = (int)items.size();
    b->smem = std::max<size_t>(smem, 16);
    int per_sm = 0;
    if (prepare_nt(b->nt, b->smem, b->blocks_per_sm, &per_sm) != cudaSuccess) {
      cudaGetLastError();
      return fail(FE_KS_ERR_CUDA, "batched kernel shared memory / occupancy");
    }
    b->grid = std::max(1, per_sm) * b->sms;
  }
  // kernel parameters
  BatchParams& P = b->host;
  P = BatchParams{};
  for (int s = 0; s < ns; ++s) {
    if (!b->direct.empty() && b->direct[s]) continue;
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
  P.err = b->d_state + 2;
  P.done = b->d_state + 3;
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
  std::vector<int> forced(n_sys, 0);
  for (int s = 0; s < n_sys; ++s) {
    if (!ctxs[s]) return fail(FE_KS_ERR_ARG, "NULL context");
    const Ctx& c = ctxs[s]->c;
    if (n_v[s] < 1 || n_v[s] > c.n_v_max) return fail(FE_KS_ERR_ARG, "n_v out of range");
    const int pr = precision[s];
    if (pr != FE_KS_F64 && pr != FE_KS_F32 && pr != FE_KS_F64E && pr != FE_KS_BF16 && pr != FE_KS_F16 &&
        pr != FE_KS_BF16X2)
      return fail(FE_KS_ERR_ARG, "unknown precision");
    if ((pr == FE_KS_BF16 || pr == FE_KS_F16 || pr == FE_KS_BF16X2) && c.nq != c.np)
      return fail(FE_KS_ERR_UNSUPPORTED, "the tensor-core precisions need n_q = n_p");
    // the persistent routines cover real FP64 / FP32 systems of degree 4..8 with n_q = n_p;
    // every other system is applied by its own kernels on a side stream
    forced[s] = c.cplx || c.p < 4 || c.p > 8 || c.nq != c.np || (pr != FE_KS_F64 && pr != FE_KS_F32) ||
                c.colour_ptr.size() - 1 > (size_t)kMaxPhase - 3 || c.n_proj > 16;
  }
  auto* b = new fe_ks_batch();
  b->ctxs.assign(ctxs, ctxs + n_sys);
  b->n_v.assign(n_v, n_v + n_sys);
  b->prec.assign(precision, precision + n_sys);
  b->cfg.assign(n_sys, 0);
  b->forced = forced;
  b->direct = forced;
  b->stream = ctxs[0]->c.stream;
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  if (cudaMalloc(&b->d_need, sizeof(int) * kMaxSys * kMaxPhase) != cudaSuccess ||
      cudaMalloc(&b->d_state, sizeof(int) * kStateWords) != cudaSuccess) {
    if (b->d_need) cudaFree(b->d_need);
    delete b;
    return fail(FE_KS_ERR_OOM, "batch state");
  }
  if (std::count(forced.begin(), forced.end(), 1) > 0) {
    fe_ks_status st = fe_ks_batch_set_direct(b, nullptr);   // creates the side streams; keeps the forced flags
    if (st != FE_KS_OK) {
      std::string msg = fe_ks_last_error();
      fe_ks_batch_destroy(b);
      return fail(st, msg);
    }
    *out = b;
    return FE_KS_OK;
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
                                   int blocks_per_sm, double wait_seconds, int inject_missing_item,
                                   int threads_per_block) {
  if (!b) return fail(FE_KS_ERR_ARG, "batch is NULL");
  if (blocks_per_sm != 1 && blocks_per_sm != 2) return fail(FE_KS_ERR_ARG, "blocks_per_sm must be 1 or 2");
  if (threads_per_block != 0 && threads_per_block != kBatchThreads[0] && threads_per_block != kBatchThreads[1] &&
      threads_per_block != kBatchThreads[2])
    return fail(FE_KS_ERR_ARG, "threads_per_block must be 0 (default), 384, 512 or 672");
  if (cells_per_item < 1 || cells_per_item > 64 || depth < 1 || depth > 16 || !(wait_seconds > 0))
    return fail(FE_KS_ERR_ARG, "cells_per_item in 1..64, depth in 1..16, wait_seconds > 0");
  if (tile_config)
    for (size_t s = 0; s < b->ctxs.size(); ++s) {
      if (tile_config[s] < 0 || tile_config[s] > 1) return fail(FE_KS_ERR_ARG, "tile_config must be 0 or 1");
    }
  if (tile_config)
    for (size_t s = 0; s < b->ctxs.size(); ++s) b->cfg[s] = tile_config[s];
  b->blocks_per_sm = blocks_per_sm;
  if (threads_per_block) b->nt = threads_per_block;
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
  // direct systems first: fork one side stream per system from the caller's stream
  bool any_direct = false;
  for (size_t i = 0; i < b->direct.size(); ++i) any_direct = any_direct || b->direct[i];
  if (any_direct) {
    if (cudaEventRecord(b->dfork, s) != cudaSuccess) return fail(FE_KS_ERR_CUDA, "batch fork event");
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
      if (!b->direct[i]) continue;
      Ctx& c = b->ctxs[i]->c;
      if (cudaStreamWaitEvent(b->dstream[i], b->dfork, 0) != cudaSuccess) return fail(FE_KS_ERR_CUDA, "batch fork");
      const cudaStream_t keep = c.stream;
      c.stream = b->dstream[i];   // the context's own kernels, launched on the system's side stream
      const int64_t ncols = b->n_v[i] * (c.cplx ? 2 : 1);
      const int pr = b->prec[i];
      const fe_ks_status st =
          pr == FE_KS_F64    ? apply_core<double>(c, static_cast<const double*>(X[i]), static_cast<double*>(Y[i]), ncols,
                                                  false, 1.0, true)
          : pr == FE_KS_F64E ? apply_core_emu(c, static_cast<const double*>(X[i]), static_cast<double*>(Y[i]), ncols,
                                              false, 1.0, true)
                             : apply_core<float>(c, static_cast<const float*>(X[i]), static_cast<float*>(Y[i]), ncols,
                                                 false, 1.f, true,
                                                 pr == FE_KS_BF16 ? 1 : pr == FE_KS_F16 ? 2 : pr == FE_KS_BF16X2 ? 3 : 0);
      c.stream = keep;
      if (st != FE_KS_OK) return st;
      if (cudaEventRecord(b->djoin[i], b->dstream[i]) != cudaSuccess) return fail(FE_KS_ERR_CUDA, "batch join event");
    }
  }
  auto join_direct = [&]() -> fe_ks_status {
    for (size_t i = 0; i < b->direct.size(); ++i)
      if (b->direct[i] && cudaStreamWaitEvent(s, b->djoin[i], 0) != cudaSuccess)
        return fail(FE_KS_ERR_CUDA, "batch join");
    return FE_KS_OK;
  };
  if (b->n_items == 0) return join_direct();
  if (cudaMemsetAsync(b->d_state, 0, sizeof(int) * kStateWords, s) != cudaSuccess)
    return fail(FE_KS_ERR_CUDA, "reset of the batch counters failed");
  if (!batch_split(b)) {
    cudaError_t err = launch_nt(b->nt, P, b->grid, b->smem, b->blocks_per_sm, s);
    if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("batched kernel: ") + cudaGetErrorString(err));
    return join_direct();
  }
  // split: FP64 object on the caller's stream, FP32 object on the side stream, joined back
  cudaError_t err = cudaEventRecord(b->ev_fork, s);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(b->side, b->ev_fork, 0);
  for (int k = 0; k < 2 && err == cudaSuccess; ++k) {
    if (b->n_items_cls[k] == 0) continue;
    BatchParams Pk = P;
    Pk.items = b->d_items_cls[k];
    Pk.n_items = b->n_items_cls[k];
    Pk.queue = b->d_state + k;
    err = launch_class_nt(b->split_nt[k], k == 0 ? kClassF64 : kClassF32, Pk, b->grid_cls[k], b->smem_cls[k],
                          k == 0 ? s : b->side);
  }
  if (err == cudaSuccess) err = cudaEventRecord(b->ev_join, b->side);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(s, b->ev_join, 0);
  if (err != cudaSuccess) return fail(FE_KS_ERR_CUDA, std::string("batched class kernels: ") + cudaGetErrorString(err));
  return join_direct();
}

fe_ks_status fe_ks_batch_status(fe_ks_batch* b) {
  if (!b) return fail(FE_KS_ERR_ARG, "batch is NULL");
  int err = 0;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&err, b->d_state + 2, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(FE_KS_ERR_CUDA, "reading the batch status failed");
  if (err && b->n_items > 0) return fail(FE_KS_ERR_TIMEOUT, "a batched work item waited longer than the configured limit");
  return FE_KS_OK;
}

fe_ks_status fe_ks_batch_info(const fe_ks_batch* b, int* n_items, int* grid, size_t* smem_bytes) {
  if (!b) return fail(FE_KS_ERR_ARG, "batch is NULL");
  if (n_items) *n_items = b->n_items;
  if (grid) *grid = b->grid;
  if (smem_bytes) *smem_bytes = b->smem;
  return FE_KS_OK;
}

fe_ks_status fe_ks_batch_set_split(fe_ks_batch* b, int threads_f64, int threads_f32) {
  if (!b) return fail(FE_KS_ERR_ARG, "batch is NULL");
  auto ok = [](int t) { return t == 0 || t == 256 || t == 384 || t == 512; };
  if (!ok(threads_f64) || !ok(threads_f32) || ((threads_f64 == 0) != (threads_f32 == 0)))
    return fail(FE_KS_ERR_ARG, "threads must both be 0 (off) or both in {256, 384, 512}");
  if (threads_f64 && !b->side) {
    if (cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess)
      return fail(FE_KS_ERR_CUDA, "creating the split launch's stream and events failed");
  }
  b->split_nt[0] = threads_f64;
  b->split_nt[1] = threads_f32;
  return batch_build(b);
}

fe_ks_status fe_ks_batch_set_direct(fe_ks_batch* b, const int* direct) {
  if (!b) return fail(FE_KS_ERR_ARG, "batch is NULL");
  const size_t ns = b->ctxs.size();
  bool want = false;
  for (size_t i = 0; i < ns; ++i) want = want || (direct && direct[i]) || b->forced[i];
  if (want && b->dstream.empty()) {
    b->dstream.assign(ns, nullptr);
    b->djoin.assign(ns, nullptr);
    bool ok = cudaEventCreateWithFlags(&b->dfork, cudaEventDisableTiming) == cudaSuccess;
    for (size_t i = 0; i < ns && ok; ++i)
      ok = cudaStreamCreateWithFlags(&b->dstream[i], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&b->djoin[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return fail(FE_KS_ERR_CUDA, "creating the direct systems' streams and events failed");
  }
  b->direct.assign(ns, 0);
  for (size_t i = 0; i < ns; ++i) b->direct[i] = (direct && direct[i] != 0) || b->forced[i];
  return batch_build(b);
}

void fe_ks_batch_destroy(fe_ks_batch* b) {
  if (!b) return;
  for (size_t i = 0; i < b->dstream.size(); ++i) {
    if (b->dstream[i]) cudaStreamDestroy(b->dstream[i]);
    if (b->djoin[i]) cudaEventDestroy(b->djoin[i]);
  }
  if (b->dfork) cudaEventDestroy(b->dfork);
  for (int k = 0; k < 2; ++k)
    if (b->d_items_cls[k]) cudaFree(b->d_items_cls[k]);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_need) cudaFree(b->d_need);
  if (b->d_state) cudaFree(b->d_state);
  delete b;
}

}  // extern "C"
