/*
 * fe_ks.h -- C interface of the GB300 matrix-free finite-element Kohn-Sham
 * operator Y = H X (Panigrahi & Motamarri, "Matrix-free algorithms for fast
 * ab initio calculations on distributed CPU architectures using
 * finite-element discretization").
 *
 * H = H_loc + H_nloc is the FE-discretised Kohn-Sham Hamiltonian of a periodic
 * cell (Sec. 2.2, eq. FEeigen):
 *   H_loc = T + L + G - iK                                   (eq. Hloc)
 *     T_IJ = 1/2 int grad N_I . grad N_J
 *     L_IJ = int V^L N_I N_J,   V^L = V_loc + |k|^2/2         (eq. Vloc)
 *     G_IJ = int V^G . (grad N_I N_J + N_I grad N_J)
 *     K_IJ = int k . (N_I grad N_J)
 *   H_nloc,IJ = sum_a sum_b F^a_{b,I} h^a_b conj(F^a_{b,J})  (eq. Vnonloc)
 *     F^a_{b,I} = int sum_r exp(-ik.(x - L_r)) chi^a_b(x - R_a - L_r) N_I(x) dx
 * N_I are degree-p Lagrange functions on Gauss-Lobatto-Legendre nodes; the
 * integrals use the tensor Gauss rule with n_q points per direction
 * (eq. cellIntegrals).  The action is evaluated matrix-free: cell gather
 * Q C P X, sum-factorised contractions with N^1D and the collocation
 * derivative D~^1D, quadrature-point coefficients, transposed contractions and
 * scatter-add (eq. HX, eq. ggaReal / eq. ggaCmplx, Algorithms 1 and 2).
 *
 * Conventions (all entry points):
 *  - Multivectors are row-major [m][n_v] with the vector index fastest.
 *    Complex operators (k != 0) use interleaved complex numbers (re, im),
 *    i.e. [m][n_v] complex = [m][2 n_v] reals.  Pointers must be 16-byte
 *    aligned device pointers unless stated otherwise.
 *  - Calls are asynchronous on the context's CUDA stream.  Argument errors are
 *    reported synchronously; errors of kernels already in flight surface at
 *    the caller's next synchronisation, as for any CUDA launch.
 *  - No call after fe_ks_setup allocates device memory except where stated.
 *  - On error the call returns a negative fe_ks_status and fe_ks_last_error()
 *    returns a message (thread-local).  No C++ exception crosses the ABI.
 */
#ifndef FE_KS_H
#define FE_KS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fe_ks_ctx fe_ks_ctx;   /* opaque; owns the device copies of all tables */

typedef enum {
  FE_KS_OK = 0,
  FE_KS_ERR_ARG = -1,          /* invalid argument (null pointer, bad size, misalignment)   */
  FE_KS_ERR_MESH = -2,         /* invalid mesh: DoF index out of range, det J <= 0         */
  FE_KS_ERR_CUDA = -3,         /* a CUDA runtime call failed                                */
  FE_KS_ERR_OOM = -4,          /* device allocation failed during setup                     */
  FE_KS_ERR_TIMEOUT = -5,      /* a device-side bounded wait gave up (batched persistent)   */
  FE_KS_ERR_UNSUPPORTED = -6   /* valid request the library does not implement              */
} fe_ks_status;

/* Arithmetic of one application. */
typedef enum {
  FE_KS_F64 = 0,               /* FP64 storage and FP64 arithmetic (DFMA)                  */
  FE_KS_F32 = 1,               /* FP32 storage and FP32 arithmetic (FFMA)                  */
  FE_KS_F64E = 2,              /* FP64 storage, FP64-accurate result; the cell kernel and the
                                  projections work in pairs of floats (hi + lo, ~48 bits) on
                                  the FP32 pipe (apply / apply_scaled / tune / residual only) */
  FE_KS_BF16 = 3,              /* FP32 storage; the cell kernel's 1D contractions (N, D and
                                  their transposes) run on the tensor cores with BF16
                                  operands and FP32 accumulation, the quadrature-point terms,
                                  projections and scatter in FP32, the nonlocal expansion
                                  as BF16 MMAs (apply / apply_scaled / tune / filter) */
  FE_KS_F16 = 4,               /* as FE_KS_BF16 with FP16 operands (8x the precision): each
                                  column of a gathered cell tile is scaled by a power of two
                                  so that its largest entry is below 1/16, and unscaled at
                                  the scatter */
  FE_KS_BF16X2 = 5             /* as FE_KS_BF16 with split products: every 16-bit operand
                                  (the gathered and intermediate cell data, the 1D matrices,
                                  the projector blocks and projections of the expansion) is
                                  held as hi = bf16(x) plus lo = bf16(x - hi), about 16
                                  significant bits, and every product is hi*hi + hi*lo +
                                  lo*hi on the tensor cores with FP32 accumulation (the
                                  lo*lo term is dropped); error about 2^-16 per stage,
                                  i.e. near FP32 (apply / apply_scaled / tune / filter) */
} fe_ks_precision;

/* Terms of H that an application includes (terms_mask of fe_ks_setup). */
enum {
  FE_KS_TERM_T = 1,            /* kinetic 1/2 grad.grad                                     */
  FE_KS_TERM_L = 2,            /* local potential V_loc + |k|^2/2                          */
  FE_KS_TERM_G = 4,            /* GGA gradient term (needs v_gga_q)                        */
  FE_KS_TERM_K = 8,            /* Bloch -iK term (k != 0)                                   */
  FE_KS_TERM_NL = 16,          /* separable nonlocal pseudopotential                       */
  FE_KS_TERM_ALL = 31
};

/*
 * Problem description.  All pointers are HOST pointers, read during
 * fe_ks_setup only; the caller keeps ownership.
 *
 *  n_cells, n_dofs : E hexahedral cells, m global DoFs (after periodic
 *                    identification; the constraint map C is folded into
 *                    cell_dofs, Sec. 3.1 eq. HX).
 *  degree          : FE degree p, n_p = p + 1 GLL nodes per direction (2..8).
 *  n_q             : Gauss points per direction: n_q = n_p (square 1D
 *                    operators) or n_q = n_p + 2 (the paper's default for
 *                    accurate V_loc and V^G integrals, Sec. 6).  The tensor-core
 *                    precisions (FE_KS_BF16, FE_KS_F16) and the batched launch
 *                    need n_q = n_p and return FE_KS_ERR_UNSUPPORTED otherwise.
 *  cell_vertices   : [E][8][3] physical vertex coordinates; vertex slot
 *                    a + 2b + 4c sits at reference corner (2a-1, 2b-1, 2c-1);
 *                    the cell map is trilinear; coordinates are unwrapped per
 *                    cell (periodic images are not folded back).
 *  cell_dofs       : [E][n_p^3] global DoF of local node i + n_p (j + n_p k).
 *  v_loc_q         : [E][n_q^3] V_loc at the quadrature points returned by
 *                    fe_ks_quadrature_points, WITHOUT |k|^2/2 (setup adds it).
 *  v_gga_q         : [E][n_q^3][3] physical V^G at the quadrature points, or NULL.
 *  kpt             : Bloch vector k (bohr^-1).  Nonzero k makes the operator
 *                    complex; force_complex = 1 makes it complex at k = 0 too.
 *  n_atoms, n_proj : atoms carrying separable projectors, projectors per atom.
 *  atom_cell_ptr   : [n_atoms + 1] CSR offsets into atom_cells / image_shift.
 *  atom_cells      : [nnz] cells meeting the support of atom a (E(a) of Sec. 3);
 *                    a cell may appear twice with different lattice images.
 *  image_shift     : [nnz][3] lattice vector L_r of the atom image for that entry.
 *  chi_q           : [nnz][n_q^3][n_proj] projector values chi_b(x_Q - R_a - L_r)
 *                    at that cell's quadrature points (real).
 *  h_coef          : [n_atoms][n_proj] diagonal coefficients Delta^a (Ha).
 */
typedef struct {
  int64_t n_cells;
  int64_t n_dofs;
  int32_t degree;
  int32_t n_q;
  const double* cell_vertices;
  const int32_t* cell_dofs;
  const double* v_loc_q;
  const double* v_gga_q;
  double kpt[3];
  int32_t force_complex;
  int32_t n_atoms;
  int32_t n_proj;
  const int32_t* atom_cell_ptr;
  const int32_t* atom_cells;
  const double* image_shift;
  const double* chi_q;
  const double* h_coef;
} fe_ks_problem;

/*
 * Physical coordinates of all quadrature points, so the caller can evaluate
 * its fields there (Sec. 3.1, eq. cellIntegrals: tensor Gauss points mapped by
 * the trilinear cell map).  xq_out is a HOST buffer [E][n_q^3][3], point index
 * qx + n_q (qy + n_q qz).  Only n_cells, degree, n_q and cell_vertices are read.
 */
fe_ks_status fe_ks_quadrature_points(const fe_ks_problem* prob, double* xq_out);

/*
 * Build a context: 1D tables (Gauss / GLL by Newton iteration), per-point
 * coefficients (Sec. 3.1 eq. reformcellmat with the Jacobian scaling folded
 * in), cell-level projector matrices F^(a,e) (eq. Vnonloc), a conflict-free
 * colouring of the cells for the scatter-add, the GLL-lumped mass D, and all
 * device workspace for n_v_max vectors.  terms_mask selects the terms of H.
 * cuda_stream (cudaStream_t, may be NULL = legacy default stream) orders all
 * later calls.  Returns FE_KS_ERR_MESH for out-of-range DoFs or det J <= 0.
 */
fe_ks_status fe_ks_setup(const fe_ks_problem* prob, int terms_mask, int64_t n_v_max,
                         void* cuda_stream, fe_ks_ctx** out);

/*
 * Y = H X for n_v vectors (eq. HX).  X, Y: device [m][n_v] (complex:
 * interleaved) in the precision's storage type (double or float).  Y is
 * overwritten.  X and Y must not overlap.  1 <= n_v <= n_v_max.
 */
fe_ks_status fe_ks_apply(fe_ks_ctx* ctx, const void* X, void* Y, int64_t n_v, int precision);

/*
 * Y = Hs X with Hs = D^{-1/2} H D^{-1/2}, D the GLL-lumped mass (the diagonal
 * approximation of M used by Algorithm 4).  Same layout rules as fe_ks_apply.
 */
fe_ks_status fe_ks_apply_scaled(fe_ks_ctx* ctx, const void* X, void* Y, int64_t n_v,
                                int precision);

/*
 * Y = H X (eq. HX) with X and Y in HOST memory ([m][n_v] row-major, the precision's
 * storage type; pinned memory lets the copies run asynchronously).  The call
 * enqueues, and returns without waiting: copy X in on the context's copy-in
 * stream, fe_ks_apply on the context's stream, copy Y out on its copy-out
 * stream.  Consecutive calls alternate between two slots of the device
 * workspace, so call k's copies overlap the application of call k +- 1.
 * work: device memory of fe_ks_apply_host_workspace bytes (two slots of X and
 * Y), 256-byte aligned, owned by the caller and reused across calls.
 * The caller keeps X_host unchanged and leaves Y_host unread until
 * fe_ks_host_wait returns; that call blocks until every result enqueued so
 * far is in host memory.  The first call creates the two copy streams.
 * Errors as fe_ks_apply; FE_KS_ERR_ARG for a short or misaligned workspace.
 */
fe_ks_status fe_ks_apply_host_workspace(const fe_ks_ctx* ctx, int64_t n_v, int precision, size_t* bytes);
fe_ks_status fe_ks_apply_host(fe_ks_ctx* ctx, const void* X_host, void* Y_host, int64_t n_v, int precision,
                              void* work, size_t work_bytes);
fe_ks_status fe_ks_host_wait(fe_ks_ctx* ctx);

/*
 * Residual-based Chebyshev filter (R-ChFSI, Algorithm 4) of degree `degree`
 * on the standard form Hs = D^{-1/2} H D^{-1/2}: D is the GLL-lumped mass
 * (Algorithm 4's diagonal approximation of M), so in scaled variables M and
 * D become the identity.  The result is p(Hs) X for the degree-`degree`
 * Chebyshev polynomial that damps [lam_T, lam_max] (mapped onto [-1, 1]
 * around c = (lam_max + lam_T)/2 with half-width e = (lam_max - lam_T)/2)
 * and is 1 at lam_min.  It is evaluated in residual form: the three-term
 * Chebyshev recurrence is run on the part R = p_k(Hs) X - X p_k(Lam), which
 * is driven by the residual Y = Hs X - X Lam of the current Ritz pairs,
 * while the diagonal part p_k(Lam) follows the scalar recurrence on the
 * host; the output is R + X p(Lam).  The residual Y and the final combination are
 * FP64-accurate: residual_precision selects native FP64 (FE_KS_F64) or the
 * pair-of-floats kernel (FE_KS_F64E) for the residual's application.  The
 * degree - 1 applications inside the recurrence run in `precision`
 * (FE_KS_F64, FE_KS_F64E or FE_KS_F32), which is where the paper's R-ChFSI
 * tolerates inexact products.
 *  X     : device FP64 [m][n_v] (complex: interleaved), overwritten by the
 *          filtered block.
 *  ritz  : device FP64 [n_v] current Ritz values Lam (real).
 *  bounds: lam_min < lam_T < lam_max (spectrum lower bound, upper end of the
 *          wanted part, spectrum upper bound).
 *  work  : device workspace of at least fe_ks_cheb_filter_workspace bytes,
 *          256-byte aligned; owned by the caller, not retained.
 * Stream-ordered, allocates nothing, so it can be captured in a CUDA graph.
 */
fe_ks_status fe_ks_cheb_filter_workspace(const fe_ks_ctx* ctx, int64_t n_v, int precision, size_t* bytes);
fe_ks_status fe_ks_cheb_filter(fe_ks_ctx* ctx, double* X, const double* ritz, int64_t n_v, int degree,
                               double lam_min, double lam_T, double lam_max, int precision,
                               int residual_precision, void* work, size_t work_bytes);

/*
 * The same filter for the generalised problem H X = M X Lam with the
 * consistent mass M (eq. FEeigen; Algorithm 4 as printed: the residual
 * H X - M X Lam uses M, the recurrence applies H D^{-1} with D the GLL-lumped
 * mass, and the result is D^{-1} R_Y + X Lam_Y).  `mass` is a context of the
 * same mesh whose application is M: set up with V_loc = 1 - |k|^2/2 at every
 * quadrature point, no GGA field, no atoms, terms = FE_KS_TERM_L (then
 * (V_loc + |k|^2/2) det J w = det J w and the L term is exactly M).  X holds
 * the generalised eigenvector block (not the D^{1/2}-scaled one).  Internally
 * the recurrence runs on D^{-1/2} H D^{-1/2} in the variables D^{-1/2} R,
 * which is the printed recurrence exactly; the residual's applications of H
 * and M take `residual_precision`.  Same workspace, precisions, stream order
 * and errors as fe_ks_cheb_filter; FE_KS_ERR_ARG if `mass` does not match the
 * operator (DoF count, real/complex, device, n_v_max).
 */
fe_ks_status fe_ks_cheb_filter_ghep(fe_ks_ctx* ctx, fe_ks_ctx* mass, double* X, const double* ritz, int64_t n_v,
                                    int degree, double lam_min, double lam_T, double lam_max, int precision,
                                    int residual_precision, void* work, size_t work_bytes);

/*
 * Tile configuration of the fused cell kernel.  FE_KS_BF16 and FE_KS_F16 (real
 * operators, n_q = n_p): 0, 2, 3 = the 5th-generation tensor-core kernel
 * (tcgen05: the x-y plane products and the z sweeps of Algorithm 2 as four MMA
 * chains per cell and 4-vector tile, two pipelines per CTA, accumulators in
 * tensor memory), its second pipeline starting each work unit after the first
 * one's first plane product (0, the default), at once (2) or after its first
 * quadrature-point step (3); 1 = the warp-level MMA kernel (one sweep per
 * direction).  Complex operators and FE_KS_BF16X2 have the warp-level kernel
 * only.  FE_KS_F64, FE_KS_F32,
 * FE_KS_F64E:
 *   0..2  one CTA per (cell, column tile), 3 tile widths;
 *   3..4  one CTA per cell walking all column tiles, the next tile's rows of X
 *         staged by cp.async, reduction-based scatter;
 *   5..6  as 3..4 with 2 or 4 adjacent columns per thread;
 *   7..9  "lean" one-CTA-per-cell walks: a single staging buffer refilled
 *         with the next tile's rows as soon as the first sweep has read it,
 *         coefficients read through the L1 instead of staged, so two (7, 8)
 *         or three (9) CTAs share an SM (8 columns with 2 or 4 per thread;
 *         4 columns with 2 per thread).
 * 0 is the default; there are FE_KS_N_CONFIGS choices.
 *
 * fe_ks_tune times every configuration with fe_ks_apply on the caller's X and
 * Y (reps timed calls each, after one untimed call). It keeps the fastest for
 * this context and precision, and reports the milliseconds per call (-1 for
 * a configuration that cannot launch, e.g. shared memory too large) and the
 * choice. Y is overwritten. The choice also goes into an in-process cache
 * keyed by (degree, n_q, precision, columns, complex, device compute
 * capability and SM count). Other contexts of the same shape whose
 * configuration was not set explicitly use it at their next application.
 *
 * fe_ks_set_config sets the configuration directly (and explicitly);
 * fe_ks_get_config reads the current one.
 */
#define FE_KS_N_CONFIGS 10
fe_ks_status fe_ks_tune(fe_ks_ctx* ctx, const void* X, void* Y, int64_t n_v, int precision, int reps,
                        double* ms_per_config, int* best);
fe_ks_status fe_ks_set_config(fe_ks_ctx* ctx, int precision, int config);
fe_ks_status fe_ks_get_config(const fe_ks_ctx* ctx, int precision, int* config);

/*
 * Device status of the context's cell kernels: synchronises the context's
 * stream, returns in *status 1 if a bounded device-side wait of the tcgen05
 * cell kernel expired since the last call (its results are then not valid),
 * else 0, and clears the word.
 */
fe_ks_status fe_ks_device_status(fe_ks_ctx* ctx, int* status);

/*
 * Host-side fault injection for tests of the failure path (no GPU fault):
 * kind = 1 makes every later launch of the tcgen05 cell kernel on ctx skip the
 * issue and the commit of each pipeline's first plane product, with a short
 * wait limit; the pipelines' bounded waits then expire, the CTAs stop, free
 * their tensor memory and set the device status word (fe_ks_device_status
 * reports 1), and the application's Y is not valid.  kind = 0 turns it off;
 * the context stays usable.  FE_KS_ERR_ARG for another kind.
 */
fe_ks_status fe_ks_inject_fault(fe_ks_ctx* ctx, int kind);

/*
 * Cell-matrix (CM) baseline: the method the paper's matrix-free algorithms
 * are measured against (Sec. 3, eq. HX with precomputed H^(e)).  Real
 * operators only.
 *
 * fe_ks_cm_create builds, for every cell of ctx, the dense local cell matrix
 * H_loc^(e) (n_p^3 x n_p^3, row-major) of the terms ctx was set up with,
 * except the nonlocal one.  It runs ctx's own FP64 matrix-free cell kernel
 * on identity blocks over a disjoint per-cell numbering, so the two methods
 * agree up to rounding.  The matrices are stored in `precision` (FE_KS_F64:
 * E n_p^6 8 bytes, 59 GB at 24^3 cells p = 8; FE_KS_F32: half; FE_KS_BF16:
 * a quarter, rounded to nearest even).  Gather and product buffers for
 * n_v_max vectors are allocated at create.
 *
 * fe_ks_cm_apply computes Y = H X on ctx's stream: per colour, gather the
 * cells' rows of X, one batched library GEMM H_loc^(e) X^(e) over the
 * colour's cells, and a colour-exclusive scatter-add that also adds the
 * nonlocal expansion F Delta P (P from ctx's projection kernel).  X and Y are
 * device [m][n_v]: FP64 for FE_KS_F64, FP32 otherwise.  FE_KS_BF16 rounds the
 * gathered X to BF16 and runs the GEMM on the tensor cores (BF16 x BF16,
 * FP32 accumulation and result); the projection and expansion stay FP32.
 * The call allocates nothing.
 *
 * fe_ks_cm_info reports the setup time (ms) and the bytes held.
 *
 * Errors: FE_KS_ERR_UNSUPPORTED (complex operator, precision), FE_KS_ERR_OOM,
 * FE_KS_ERR_ARG, FE_KS_ERR_CUDA.  ctx must outlive the object.
 */
typedef struct fe_ks_cm fe_ks_cm;
fe_ks_status fe_ks_cm_create(fe_ks_ctx* ctx, int precision, int64_t n_v_max, fe_ks_cm** out);
fe_ks_status fe_ks_cm_apply(fe_ks_cm* cm, const void* X, void* Y, int64_t n_v);
fe_ks_status fe_ks_cm_info(const fe_ks_cm* cm, double* setup_ms, size_t* bytes);
void fe_ks_cm_destroy(fe_ks_cm* cm);

/*
 * Host-only: the greedy cell colouring the scatter-add relies on, i.e. the
 * assembly Q^T of Algorithm 1 done one colour at a time.
 *
 * Cells are taken in index order; each gets the smallest colour (0..63) not
 * used by a cell that shares one of its DoFs, so the cells of one colour
 * touch disjoint rows of Y and one launch per colour needs no atomics and is
 * deterministic.
 *
 * cell_dofs is [n_cells][np3] (host, caller-owned). colour receives [n_cells]
 * (host, caller-owned) and n_colours the colour count.
 *
 * Errors: FE_KS_ERR_MESH for an entry outside [0, n_dofs);
 * FE_KS_ERR_UNSUPPORTED when more than 64 colours would be needed;
 * FE_KS_ERR_ARG for NULL pointers or sizes out of range. Needs no GPU.
 */
fe_ks_status fe_ks_colour_cells(int64_t n_cells, int32_t np3, int64_t n_dofs, const int32_t* cell_dofs,
                                int32_t* colour, int32_t* n_colours);

/*
 * Batched application: Y_s = H_s X_s for up to 16 independent systems of
 * uneven size, degree, vector count and precision in ONE call.  Real FP64 /
 * FP32 systems of degree 4..8 with n_q = n_p go to ONE persistent kernel
 * launch: the work queue is phase-major -- zero-fill of every Y_s and the
 * per-atom projections first, then the cells of colour 0, 1, ... of every
 * system -- and a work item of system s waits (bounded) for the completion of
 * s's previous phase only, so systems overlap freely.  Every other system
 * (complex operators, n_q = n_p + 2, degrees 1..3, FE_KS_F64E / FE_KS_BF16 /
 * FE_KS_F16 / FE_KS_BF16X2) is a direct system (fe_ks_batch_set_direct below):
 * applied by its own kernels on a side stream, concurrently.
 *
 * fe_ks_batch_create builds the queue for the given contexts (owned by the
 * caller, must outlive the batch), vector counts and precisions; it allocates
 * the queue and counters (the only allocation), and the side streams when a
 * system is direct.  X[s] and Y[s] of a complex system hold interleaved
 * (re, im) columns, as for fe_ks_apply.
 * fe_ks_batch_configure sets the tunables -- tile configuration per system
 * (0/1: columns per tile), cells per work item, items claimed per fetch, resident CTAs per SM (1, or
 * 2 with a tighter register budget; 672-thread blocks run one per SM),
 * threads per block (384, 512 or 672; 0 keeps the current, initially 384) --
 * plus the bounded-wait limit in seconds, and inject_missing_item = 1 makes
 * the host count one phase-0 item that is never published (fault injection:
 * the launch then ends with FE_KS_ERR_TIMEOUT reported by fe_ks_batch_status).
 * fe_ks_batch_apply launches on cuda_stream (NULL: the first context's
 * stream) with X[s], Y[s] device arrays laid out as for fe_ks_apply; it is a
 * counter reset plus one kernel, so it can be captured into a CUDA graph.
 * fe_ks_batch_status synchronises with the device and reports a wait that
 * expired.
 */
typedef struct fe_ks_batch fe_ks_batch;
fe_ks_status fe_ks_batch_create(fe_ks_ctx* const* ctxs, int n_sys, const int64_t* n_v, const int* precision,
                                fe_ks_batch** out);
fe_ks_status fe_ks_batch_configure(fe_ks_batch* b, const int* tile_config, int cells_per_item, int depth,
                                   int blocks_per_sm, double wait_seconds, int inject_missing_item,
                                   int threads_per_block);
fe_ks_status fe_ks_batch_apply(fe_ks_batch* b, const void* const* X, void* const* Y, void* cuda_stream);
fe_ks_status fe_ks_batch_status(fe_ks_batch* b);
/*
 * Split mode of the batched launch: threads_f64 = threads_f32 = 0 turns it
 * off (the default); otherwise both are block sizes in {256, 384, 512}.  The
 * FP64 systems' items and the FP32 systems' items then go to two queues, each
 * drained by a persistent kernel object that holds only that precision's
 * routines (so each has the register budget of its own routines, capped at
 * half the register file), and fe_ks_batch_apply launches the two objects
 * concurrently: the FP64 one on cuda_stream, the FP32 one on a side stream
 * forked from and joined back into cuda_stream with events (still one graph
 * when captured).  An FP64 CTA and an FP32 CTA can then share an SM, one
 * loading its FP64 pipe and the other its FP32 pipe.  Dependencies are per
 * system as before; a system's items all sit in its class's queue.  The
 * first call creates the side stream and two events.  Rebuilds the queues
 * (as fe_ks_batch_configure does); the other tunables are kept.
 */
fe_ks_status fe_ks_batch_set_split(fe_ks_batch* b, int threads_f64, int threads_f32);
/*
 * Direct systems: direct[s] != 0 (host array of n_sys flags; NULL clears all)
 * takes system s out of the persistent queue.  fe_ks_batch_apply then applies
 * it with its own context's kernels (projection and one tuned cell-kernel
 * launch per colour, as fe_ks_apply does, in the context's current tile
 * configuration), each direct system on a side stream of its own forked from
 * cuda_stream with an event and joined back into it; the persistent launch of
 * the remaining systems (if any) runs on cuda_stream concurrently.  The whole
 * call still captures as one CUDA graph.  For a batch whose work is dominated
 * by a few large systems, whose own tuned launches beat any routine inside a
 * shared persistent kernel, while the small ones still gain from the queue.
 * During fe_ks_batch_apply a direct system's context has its stream switched to
 * the side stream and restored before the call returns.  The first call with
 * flags creates the streams and events.  Rebuilds the queue.
 */
fe_ks_status fe_ks_batch_set_direct(fe_ks_batch* b, const int* direct);
fe_ks_status fe_ks_batch_info(const fe_ks_batch* b, int* n_items, int* grid, size_t* smem_bytes);
void fe_ks_batch_destroy(fe_ks_batch* b);

/* Length-m device copy of D^{-1/2} in FP64 (owned by the context). */
const double* fe_ks_dinv_sqrt(const fe_ks_ctx* ctx);

/* Problem sizes as seen by the context. */
fe_ks_status fe_ks_info(const fe_ks_ctx* ctx, int64_t* n_dofs, int64_t* n_cells, int32_t* degree,
                        int32_t* is_complex, int32_t* n_colours, int64_t* n_pairs);

/*
 * Per-phase timing of later applications (CUDA events on the context's
 * stream, recorded around the zero-fill, the projection kernel and the fused
 * local kernels).  fe_ks_set_profiling(ctx, 1) starts recording (events are
 * created lazily, no device memory is allocated), 0 stops.
 * fe_ks_read_profile synchronises the recorded events and returns, for
 * phases 0 = zero-fill, 1 = nonlocal projection, 2 = fused local kernel, the
 * total milliseconds ms[3] and the number of kernel launches launches[3] since
 * the last read, then clears them.
 */
fe_ks_status fe_ks_set_profiling(fe_ks_ctx* ctx, int on);
fe_ks_status fe_ks_read_profile(fe_ks_ctx* ctx, double ms[3], int64_t launches[3]);

/*
 * Diagnostic: FP64 (precision = FE_KS_F64) or FP32 FMA throughput of the
 * current device in TFLOP/s (2 flops per FMA), from a bounded register-only
 * FMA loop on 4 CTAs per SM; precision = FE_KS_BF16 measures the warp-level
 * tensor-core rate (mma.sync m16n8k16, BF16 operands, FP32 accumulation)
 * that the tensor-core cell kernel uses.  Allocates and frees a small device buffer.
 */
fe_ks_status fe_ks_measure_fma_peak(int precision, double* tflops);

/*
 * Allocation-free nonlocal term (no counterpart in the paper; an interface
 * for callers that cannot call cudaMalloc).
 *
 * Who needs it: callers whose device memory is owned by another allocator
 * (a framework's memory pool that must account for every byte), or code that
 * runs where a cudaMalloc would implicitly synchronise the device or exceed a
 * fixed memory budget.  They pass every input and output; this call allocates
 * nothing (no cudaMalloc / cudaFree, no allocating library routine) and keeps
 * its only scratch -- the per-atom projections diag(h_a) F_a^H X -- in a
 * file-scope device array of 4 MiB (524288 doubles) that every GPU which
 * loads the library holds until the process exits.
 *
 *   Y += sum_a F_a diag(h_a) F_a^H X          (FP64; eq. Vnonloc)
 *
 *  X, Y          : device FP64 [n_dofs][n_v] (complex: interleaved, is_complex = 1);
 *                  Y is accumulated into (zero it first for the bare term).
 *  cell_dofs     : device [E][(degree+1)^3] global DoF of each cell node.
 *  atom_pair_ptr : device [n_atoms + 1] CSR offsets of each atom's (cell, image) entries.
 *  pair_cell     : device [n_pairs] cell of each entry; pair_atom: device [n_pairs] its atom,
 *                  which must agree with the CSR ranges (pair_atom[j] = a for
 *                  atom_pair_ptr[a] <= j < atom_pair_ptr[a + 1]); the projection reads the
 *                  ranges and the expansion reads pair_atom, and the call does not check
 *                  that they agree.
 *  F             : device [n_pairs][n_proj][(degree+1)^3] projector matrices
 *                  F^(a,e) (complex: interleaved re, im per entry).
 *  h_coef        : device [n_atoms][n_proj] coefficients Delta^a.
 * Limit: n_atoms * n_proj * n_v * (1 + is_complex) <= 524288, else
 * FE_KS_ERR_ARG with a message naming the limit.  The first call on a device
 * looks up the scratch address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share
 * the one scratch array, which keeps the last call's contents (every entry a
 * call reads is written by that call first): calls that overlap on the GPU
 * (different streams, or other devices' threads using the same device) race.
 * Pairs of different cells share DoFs, so the expansion adds into Y with FP64
 * atomics in no fixed order: results can differ from run to run in rounding
 * only (every other apply path of the library is bitwise deterministic).
 * A device index of 64 or more returns FE_KS_ERR_UNSUPPORTED.
 */
fe_ks_status fe_ks_nonlocal_apply_static(const double* X, double* Y, int64_t n_v, int32_t is_complex,
                                         int32_t degree, int64_t n_dofs, const int32_t* cell_dofs,
                                         int32_t n_atoms, int32_t n_proj, const int32_t* atom_pair_ptr,
                                         const int32_t* pair_cell, const int32_t* pair_atom, int64_t n_pairs,
                                         const double* F, const double* h_coef, void* cuda_stream);

/*
 * Column-major FP64 GEMM C = alpha op(A) op(B) + beta C through cuBLAS, for
 * the Rayleigh-Ritz step of Algorithm 3 (Gram matrices and the rotation of
 * the filtered block).  emulated = 1 asks cuBLAS for its FP64 emulation on
 * integer tensor cores (fixed-point slices); FE_KS_ERR_UNSUPPORTED if
 * unavailable.  trans_* = 1 transposes.  The first call on a device creates
 * a cuBLAS handle (which allocates); stream-ordered on cuda_stream.
 */
fe_ks_status fe_ks_gemm_f64(int trans_a, int trans_b, int64_t m, int64_t n, int64_t k, double alpha,
                            const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                            int64_t ldc, int emulated, void* cuda_stream);

/*
 * FP64-accurate dense products for the Rayleigh-Ritz step, computed in pairs
 * of floats on the FP32 pipe (compensated dot products: exact FMA products,
 * error-free sums), FP64 in and out:
 *   fe_ks_gram_ff  : C[n1][n2] = Y^T Z for row-major Y [m][n1], Z [m][n2];
 *                    the m dimension is split in chunks of 8192 rows whose
 *                    partial sums are added in a fixed order (deterministic);
 *                    work: device buffer of fe_ks_gram_ff_workspace bytes.
 *   fe_ks_gram_ff_sym: the same for n1 = n2 = n when Y^T Z is known to be
 *                    symmetric: only the 64 x 64 tiles on or above the
 *                    diagonal are computed and the result is mirrored
 *                    (exactly symmetric; same workspace).
 *   fe_ks_rotate_ff: X[m][k] = Y[m][n] E[n][k], all row-major.
 * Real operators only; stream-ordered on cuda_stream; no allocation.
 */
fe_ks_status fe_ks_gram_ff_workspace(int64_t m, int n1, int n2, size_t* bytes);
fe_ks_status fe_ks_gram_ff(const double* Y, const double* Z, double* C, int64_t m, int n1, int n2, void* work,
                           size_t work_bytes, void* cuda_stream);
fe_ks_status fe_ks_gram_ff_sym(const double* Y, const double* Z, double* C, int64_t m, int n, void* work,
                               size_t work_bytes, void* cuda_stream);
fe_ks_status fe_ks_rotate_ff(const double* Y, const double* E, double* X, int64_t m, int n, int k,
                             void* cuda_stream);

/*
 * Rayleigh-Ritz step of Algorithm 3 on span(X), the FP64-accurate projection
 * the R-ChFSI outer loop performs after each filter (Sec. 5.5: the filter may
 * run in low precision, this step may not).  Standard form (mass == NULL):
 * Op = Hs = D^{-1/2} H D^{-1/2} and metric I.  Generalised form (eq. FEeigen):
 * Op = H and metric M, `mass` being a context whose application is M (see
 * fe_ks_cheb_filter_ghep).  It solves (X^T Op X) E = (X^T M X) E Lam, with
 * E^T (X^T M X) E = I, and overwrites X by X E and ritz by Lam (ascending):
 *   S = X^T M X; S' = d S d with d = diag(S)^{-1/2}; S' = L L^T (Cholesky);
 *   A = X^T Op X; L^{-1} (d A d) L^{-T} = W Lam W^T; E = d L^{-T} W.
 * The tall products (X^T M X, X^T Op X, X E) and the applications take
 * `precision`: FE_KS_F64E = the library's pair-of-floats Gram and rotation
 * kernels and pair-of-floats applications (FP64-accurate on the FP32 pipe);
 * FE_KS_F64 = native FP64 applications and cuBLAS FP64 GEMMs (the plain
 * FP64 comparator).  The n_v x n_v Cholesky, scaling and triangular solves
 * are the library's kernels; the n_v x n_v symmetric eigensolve is
 * cuSOLVER's syevd.  If a pivot of S' falls below 1e-10 (X nearly
 * rank-deficient) the step first orthonormalises X in the metric by shifted
 * CholeskyQR3 (three Cholesky-QR passes, the first with a shift) and projects
 * onto the orthonormal block; *path (may be NULL) returns 0 for the Cholesky
 * path and 1 for that fallback.
 *  X      : device FP64 [m][n_v] row-major, in/out (real operators only).
 *  ritz   : device FP64 [n_v], out.
 *  work   : device, >= fe_ks_rayleigh_ritz_workspace bytes, 256-byte aligned,
 *           caller-owned, must not overlap X.
 * The call synchronises the context's stream twice (it reads the Cholesky
 * status and the eigensolver status).  The first call on a device (also
 * through the workspace query) creates a cuSOLVER handle, which allocates.
 * Errors: FE_KS_ERR_UNSUPPORTED for complex operators; FE_KS_ERR_ARG for an X
 * that even the shifted Cholesky QR cannot orthonormalise, bad sizes, a short
 * workspace or overlap; FE_KS_ERR_CUDA.
 */
fe_ks_status fe_ks_rayleigh_ritz_workspace(const fe_ks_ctx* ctx, int64_t n_v, int precision, size_t* bytes);
fe_ks_status fe_ks_rayleigh_ritz(fe_ks_ctx* ctx, fe_ks_ctx* mass, double* X, double* ritz, int64_t n_v, int precision,
                                 void* work, size_t work_bytes, int* path);

/*
 * Upper bound of the spectrum of Hs = D^{-1/2} H D^{-1/2} for the filter's
 * lam_max (Algorithm 4 takes the bounds as inputs; the paper gives no method):
 * `steps` steps of the symmetric Lanczos recurrence from the start vector v0,
 *   v_1 = v0/|v0|;  w = Hs v_j - alpha_j v_j - beta_{j-1} v_{j-1},
 *   alpha_j = v_j^H Hs v_j,  beta_j = |w|,  v_{j+1} = w / beta_j,
 * then lam_max = theta_max(T_k) + |beta_k| with T_k the k x k tridiagonal
 * matrix of the coefficients (the standard safe bound).  The recurrence runs
 * on the device (applications in `precision`, FE_KS_F64 or FE_KS_F64E;
 * fixed-order reductions, so the result is deterministic); the host then
 * reads the 2k coefficients (one stream synchronisation) and finds
 * theta_max by Sturm-sequence bisection.  A beta that vanishes exactly
 * stops the recurrence there (k < steps, reported in *steps_done).
 *  v0     : device FP64 [m] (complex operators: [m] interleaved complex).
 *  lam_max: host, out.  alpha, beta: host [steps] or NULL, out (the first k used).
 *  work   : device, >= fe_ks_lanczos_bound_workspace bytes (three vectors and
 *           the reduction scratch), 256-byte aligned, caller-owned.
 */
fe_ks_status fe_ks_lanczos_bound_workspace(const fe_ks_ctx* ctx, int steps, size_t* bytes);
fe_ks_status fe_ks_lanczos_bound(fe_ks_ctx* ctx, const double* v0, int steps, int precision, void* work,
                                 size_t work_bytes, double* lam_max, double* alpha, double* beta, int* steps_done);

/*
 * FP64-accurate symmetric Gram product C = Y^T Z (n x n, known symmetric, e.g.
 * Y^T M Y or Y^T H Y of Rayleigh-Ritz) on the 5th-generation tensor cores:
 * every FP64 value is cut, relative to its column's largest exponent over a
 * chunk of 32 rows, into eight exact 7-bit slices held as BF16; the slice
 * products run as tcgen05 BF16 MMAs with FP32 accumulation in six groups by
 * slice order, so that every group that matters stays an exact integer; each
 * chunk is scaled and accumulated in pairs of floats; chunk groups of 8192
 * rows are added in a fixed order (compensated).  Error a few units of 2^-52
 * of sum_r |Y_ri Z_rj|, deterministic, C
 * exactly symmetric.  Y, Z: device FP64 [m][n] row-major.  work: device,
 * >= fe_ks_gram_tc_workspace bytes, 256-byte aligned.  The kernel flags a
 * chunk whose scale 2^(E_i + E_j) (E the exponents of the two columns) falls
 * outside the FP32 range (columns of magnitude far from 1: below about 2^-60
 * or above 2^60 together); fe_ks_gram_tc_status (which synchronises) returns
 * bit 0 = a bounded wait expired, bit 1 = such a chunk; in either case C is
 * not valid and fe_ks_gram_ff_sym is the fallback.  Stream-ordered, no
 * allocation.
 */
fe_ks_status fe_ks_gram_tc_workspace(int64_t m, int n, size_t* bytes);
fe_ks_status fe_ks_gram_tc_sym(const double* Y, const double* Z, double* C, int64_t m, int n, void* work,
                               size_t work_bytes, void* cuda_stream);
fe_ks_status fe_ks_gram_tc_status(const void* work, int* status);

/*
 * FP64-accurate rotation X = Y E (Y [m][n], E [n][k], X [m][k], all row-major
 * device FP64) on the tensor cores by the same exact slices: each row of Y and
 * each column of E is cut relative to its own largest exponent over a chunk of
 * 32 of the n contraction indices.  X must not overlap Y or E.  flags: device
 * int[2], set to (a bounded wait expired, a chunk scale left the FP32 range);
 * if either is set after the stream reaches the call, X is not valid.
 * Stream-ordered, no allocation.
 */
fe_ks_status fe_ks_rotate_tc(const double* Y, const double* E, double* X, int64_t m, int n, int k, int* flags,
                             void* cuda_stream);

/*
 * Which kernel the pair-of-floats Rayleigh-Ritz step (precision FE_KS_F64E of
 * fe_ks_rayleigh_ritz) uses for its two Gram products: 1 (default) the
 * tensor-core one above (falling back to the pair-of-floats kernel for a call
 * whose status is not 0), 0 the pair-of-floats one.
 */
fe_ks_status fe_ks_set_rr_gram(fe_ks_ctx* ctx, int tensor_cores);

/* Change the stream used by later calls. */
fe_ks_status fe_ks_set_stream(fe_ks_ctx* ctx, void* cuda_stream);

/* Message of the last failed call on this thread ("" if none). */
const char* fe_ks_last_error(void);

/* Free the context and all device memory it owns (NULL is ignored). */
void fe_ks_destroy(fe_ks_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FE_KS_H */
