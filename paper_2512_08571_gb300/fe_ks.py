"""ctypes binding of libfe_ks.so (argument marshalling only).

Every function mirrors an entry point of ``include/fe_ks.h`` under the same
name; all work happens in the library's CUDA kernels.  There is no fallback:
if the shared library is missing or fails to load, importing the binding
raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfe_ks.so")

FE_KS_OK = 0
STATUS_NAMES = {0: "FE_KS_OK", -1: "FE_KS_ERR_ARG", -2: "FE_KS_ERR_MESH", -3: "FE_KS_ERR_CUDA",
                -4: "FE_KS_ERR_OOM", -5: "FE_KS_ERR_TIMEOUT", -6: "FE_KS_ERR_UNSUPPORTED"}
FE_KS_F64, FE_KS_F32, FE_KS_F64E, FE_KS_BF16, FE_KS_F16, FE_KS_BF16X2 = 0, 1, 2, 3, 4, 5
TERM_T, TERM_L, TERM_G, TERM_K, TERM_NL, TERM_ALL = 1, 2, 4, 8, 16, 31




class FeKsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class fe_ks_problem(ctypes.Structure):
    _fields_ = [
        ("n_cells", ctypes.c_int64), ("n_dofs", ctypes.c_int64),
        ("degree", ctypes.c_int32), ("n_q", ctypes.c_int32),
        ("cell_vertices", ctypes.c_void_p), ("cell_dofs", ctypes.c_void_p),
        ("v_loc_q", ctypes.c_void_p), ("v_gga_q", ctypes.c_void_p),
        ("kpt", ctypes.c_double * 3), ("force_complex", ctypes.c_int32),
        ("n_atoms", ctypes.c_int32), ("n_proj", ctypes.c_int32),
        ("atom_cell_ptr", ctypes.c_void_p), ("atom_cells", ctypes.c_void_p),
        ("image_shift", ctypes.c_void_p), ("chi_q", ctypes.c_void_p), ("h_coef", ctypes.c_void_p),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfe_ks.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.fe_ks_quadrature_points.argtypes = [P(fe_ks_problem), vp]
    lib.fe_ks_setup.argtypes = [P(fe_ks_problem), ctypes.c_int, i64, vp, P(vp)]
    lib.fe_ks_apply.argtypes = [vp, vp, vp, i64, ctypes.c_int]
    lib.fe_ks_apply_scaled.argtypes = [vp, vp, vp, i64, ctypes.c_int]
    lib.fe_ks_apply_host_workspace.argtypes = [vp, i64, ctypes.c_int, P(ctypes.c_size_t)]
    lib.fe_ks_apply_host.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp, ctypes.c_size_t]
    lib.fe_ks_host_wait.argtypes = [vp]
    lib.fe_ks_dinv_sqrt.argtypes = [vp]
    lib.fe_ks_dinv_sqrt.restype = vp
    lib.fe_ks_info.argtypes = [vp, P(i64), P(i64), P(i32), P(i32), P(i32), P(i64)]
    lib.fe_ks_set_stream.argtypes = [vp, vp]
    lib.fe_ks_last_error.restype = ctypes.c_char_p
    lib.fe_ks_set_profiling.argtypes = [vp, ctypes.c_int]
    lib.fe_ks_read_profile.argtypes = [vp, P(ctypes.c_double), P(i64)]
    lib.fe_ks_measure_fma_peak.argtypes = [ctypes.c_int, P(ctypes.c_double)]
    lib.fe_ks_cheb_filter_workspace.argtypes = [vp, i64, ctypes.c_int, P(ctypes.c_size_t)]
    lib.fe_ks_cheb_filter.argtypes = [vp, vp, vp, i64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t]
    lib.fe_ks_cheb_filter_ghep.argtypes = [vp, vp, vp, vp, i64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t]
    lib.fe_ks_nonlocal_apply_static.argtypes = [vp, vp, i64, i32, i32, i64, vp, i32, i32, vp, vp, vp, i64,
                                                vp, vp, vp]
    lib.fe_ks_tune.argtypes = [vp, vp, vp, i64, ctypes.c_int, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_int)]
    lib.fe_ks_set_config.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.fe_ks_get_config.argtypes = [vp, ctypes.c_int, P(ctypes.c_int)]
    lib.fe_ks_device_status.argtypes = [vp, P(ctypes.c_int)]
    lib.fe_ks_inject_fault.argtypes = [vp, ctypes.c_int]
    lib.fe_ks_cm_create.argtypes = [vp, ctypes.c_int, i64, P(vp)]
    lib.fe_ks_cm_apply.argtypes = [vp, vp, vp, i64]
    lib.fe_ks_cm_info.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_size_t)]
    lib.fe_ks_cm_destroy.argtypes = [vp]
    lib.fe_ks_cm_destroy.restype = None
    lib.fe_ks_colour_cells.argtypes = [i64, i32, i64, vp, vp, P(i32)]
    lib.fe_ks_batch_create.argtypes = [P(vp), ctypes.c_int, P(i64), P(ctypes.c_int), P(vp)]
    lib.fe_ks_batch_configure.argtypes = [vp, P(ctypes.c_int), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_int, ctypes.c_int]
    lib.fe_ks_batch_apply.argtypes = [vp, P(vp), P(vp), vp]
    lib.fe_ks_batch_status.argtypes = [vp]
    lib.fe_ks_batch_set_split.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.fe_ks_batch_set_direct.argtypes = [vp, P(ctypes.c_int)]
    lib.fe_ks_batch_info.argtypes = [vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_size_t)]
    lib.fe_ks_batch_destroy.argtypes = [vp]
    lib.fe_ks_batch_destroy.restype = None
    lib.fe_ks_gemm_f64.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, i64, ctypes.c_double, vp, i64, vp, i64,
                                   ctypes.c_double, vp, i64, ctypes.c_int, vp]
    lib.fe_ks_gram_ff_workspace.argtypes = [i64, ctypes.c_int, ctypes.c_int, P(ctypes.c_size_t)]
    lib.fe_ks_gram_ff.argtypes = [vp, vp, vp, i64, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t, vp]
    lib.fe_ks_gram_ff_sym.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp, ctypes.c_size_t, vp]
    lib.fe_ks_rotate_ff.argtypes = [vp, vp, vp, i64, ctypes.c_int, ctypes.c_int, vp]
    lib.fe_ks_rayleigh_ritz_workspace.argtypes = [vp, i64, ctypes.c_int, P(ctypes.c_size_t)]
    lib.fe_ks_rayleigh_ritz.argtypes = [vp, vp, vp, vp, i64, ctypes.c_int, vp, ctypes.c_size_t, P(ctypes.c_int)]
    lib.fe_ks_lanczos_bound_workspace.argtypes = [vp, ctypes.c_int, P(ctypes.c_size_t)]
    lib.fe_ks_lanczos_bound.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t,
                                        P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                                        P(ctypes.c_int)]
    lib.fe_ks_gram_tc_workspace.argtypes = [i64, ctypes.c_int, P(ctypes.c_size_t)]
    lib.fe_ks_gram_tc_sym.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp, ctypes.c_size_t, vp]
    lib.fe_ks_gram_tc_status.argtypes = [vp, P(ctypes.c_int)]
    lib.fe_ks_set_rr_gram.argtypes = [vp, ctypes.c_int]
    lib.fe_ks_rotate_tc.argtypes = [vp, vp, vp, i64, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.fe_ks_destroy.argtypes = [vp]
    lib.fe_ks_destroy.restype = None
    for name in ("fe_ks_quadrature_points", "fe_ks_setup", "fe_ks_apply", "fe_ks_apply_scaled",
                 "fe_ks_apply_host_workspace", "fe_ks_apply_host", "fe_ks_host_wait",
                 "fe_ks_info", "fe_ks_set_stream", "fe_ks_set_profiling", "fe_ks_read_profile",
                 "fe_ks_measure_fma_peak", "fe_ks_cheb_filter_workspace", "fe_ks_cheb_filter",
                 "fe_ks_nonlocal_apply_static", "fe_ks_tune", "fe_ks_set_config", "fe_ks_batch_create",
                 "fe_ks_batch_configure", "fe_ks_batch_apply", "fe_ks_batch_status", "fe_ks_batch_info",
                 "fe_ks_gemm_f64", "fe_ks_gram_ff_workspace", "fe_ks_gram_ff", "fe_ks_rotate_ff",
                 "fe_ks_gram_ff_sym", "fe_ks_rayleigh_ritz_workspace", "fe_ks_rayleigh_ritz",
                 "fe_ks_lanczos_bound_workspace", "fe_ks_lanczos_bound", "fe_ks_batch_set_split",
                 "fe_ks_gram_tc_workspace", "fe_ks_gram_tc_sym", "fe_ks_gram_tc_status", "fe_ks_set_rr_gram",
                 "fe_ks_rotate_tc"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


_lib = _load()


def lib():
    return _lib


def _check(status):
    if status != FE_KS_OK:
        raise FeKsError(status, _lib.fe_ks_last_error().decode())


def _ptr(a):
    """Data pointer of a C-contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous (row-major [m][n_v])")
        return a.ctypes.data
    if hasattr(a, "is_contiguous") and not a.is_contiguous():
        raise ValueError("tensor must be contiguous (row-major [m][n_v])")
    return a.data_ptr()


def fe_ks_quadrature_points(prob):
    xq = np.empty((prob.n_cells, prob.n_q ** 3, 3), dtype=np.float64)
    _check(_lib.fe_ks_quadrature_points(ctypes.byref(prob), xq.ctypes.data))
    return xq


def fe_ks_setup(prob, terms_mask=TERM_ALL, n_v_max=1, stream=None):
    ctx = ctypes.c_void_p()
    _check(_lib.fe_ks_setup(ctypes.byref(prob), terms_mask, n_v_max, stream, ctypes.byref(ctx)))
    return ctx


def fe_ks_apply(ctx, X, Y, n_v, precision):
    _check(_lib.fe_ks_apply(ctx, _ptr(X), _ptr(Y), n_v, precision))


def fe_ks_apply_scaled(ctx, X, Y, n_v, precision):
    _check(_lib.fe_ks_apply_scaled(ctx, _ptr(X), _ptr(Y), n_v, precision))


def fe_ks_apply_host_workspace(ctx, n_v, precision):
    out = ctypes.c_size_t()
    _check(_lib.fe_ks_apply_host_workspace(ctx, n_v, precision, ctypes.byref(out)))
    return out.value


def fe_ks_apply_host(ctx, X_host, Y_host, n_v, precision, work, work_bytes):
    """Enqueue Y_host = H X_host (host arrays / CPU tensors); results are final after fe_ks_host_wait."""
    _check(_lib.fe_ks_apply_host(ctx, _ptr(X_host), _ptr(Y_host), n_v, precision, _ptr(work), work_bytes))


def fe_ks_host_wait(ctx):
    _check(_lib.fe_ks_host_wait(ctx))


def fe_ks_cheb_filter_workspace(ctx, n_v, precision):
    out = ctypes.c_size_t()
    _check(_lib.fe_ks_cheb_filter_workspace(ctx, n_v, precision, ctypes.byref(out)))
    return out.value


def fe_ks_cheb_filter(ctx, X, ritz, n_v, degree, lam_min, lam_T, lam_max, precision, work, work_bytes,
                      residual_precision=FE_KS_F64):
    _check(_lib.fe_ks_cheb_filter(ctx, _ptr(X), _ptr(ritz), n_v, degree, lam_min, lam_T, lam_max, precision,
                                  residual_precision, _ptr(work), work_bytes))


def fe_ks_cheb_filter_ghep(ctx, mass, X, ritz, n_v, degree, lam_min, lam_T, lam_max, precision, work, work_bytes,
                           residual_precision=FE_KS_F64):
    _check(_lib.fe_ks_cheb_filter_ghep(ctx, mass, _ptr(X), _ptr(ritz), n_v, degree, lam_min, lam_T, lam_max,
                                       precision, residual_precision, _ptr(work), work_bytes))


def fe_ks_nonlocal_apply_static(X, Y, n_v, is_complex, degree, n_dofs, cell_dofs, n_atoms, n_proj,
                                atom_pair_ptr, pair_cell, pair_atom, n_pairs, F, h_coef, stream=None):
    _check(_lib.fe_ks_nonlocal_apply_static(_ptr(X), _ptr(Y), n_v, int(is_complex), degree, n_dofs,
                                            _ptr(cell_dofs), n_atoms, n_proj, _ptr(atom_pair_ptr),
                                            _ptr(pair_cell), _ptr(pair_atom), n_pairs, _ptr(F), _ptr(h_coef),
                                            stream))


N_CONFIGS = 10


def fe_ks_tune(ctx, X, Y, n_v, precision, reps=3):
    """Time every tile configuration on (X, Y); keep the fastest. Returns (best, [ms per config])."""
    ms = (ctypes.c_double * N_CONFIGS)()
    best = ctypes.c_int()
    _check(_lib.fe_ks_tune(ctx, _ptr(X), _ptr(Y), n_v, precision, reps, ms, ctypes.byref(best)))
    return best.value, list(ms)


def fe_ks_set_config(ctx, precision, config):
    _check(_lib.fe_ks_set_config(ctx, precision, config))


def fe_ks_get_config(ctx, precision):
    out = ctypes.c_int()
    _check(_lib.fe_ks_get_config(ctx, precision, ctypes.byref(out)))
    return out.value


def fe_ks_device_status(ctx):
    """1 if a bounded device-side wait of the tcgen05 cell kernel expired since the last call (synchronises)."""
    out = ctypes.c_int()
    _check(_lib.fe_ks_device_status(ctx, ctypes.byref(out)))
    return out.value


def fe_ks_inject_fault(ctx, kind):
    """Host-side fault injection into the tcgen05 cell kernel (1 = on, 0 = off); tests only."""
    _check(_lib.fe_ks_inject_fault(ctx, kind))


def fe_ks_cm_create(ctx, precision, n_v_max):
    out = ctypes.c_void_p()
    _check(_lib.fe_ks_cm_create(ctx, precision, n_v_max, ctypes.byref(out)))
    return out


def fe_ks_cm_apply(cm, X, Y, n_v):
    _check(_lib.fe_ks_cm_apply(cm, _ptr(X), _ptr(Y), n_v))


def fe_ks_cm_info(cm):
    ms, nb = ctypes.c_double(), ctypes.c_size_t()
    _check(_lib.fe_ks_cm_info(cm, ctypes.byref(ms), ctypes.byref(nb)))
    return dict(setup_ms=ms.value, bytes=nb.value)


def fe_ks_cm_destroy(cm):
    _lib.fe_ks_cm_destroy(cm)


def fe_ks_colour_cells(cell_dofs, n_dofs):
    """Host colouring of the cells ([n_cells][np3] int32 numpy array): (colour per cell, count)."""
    import numpy as np
    cd = np.ascontiguousarray(cell_dofs, dtype=np.int32)
    colour = np.empty(cd.shape[0], dtype=np.int32)
    n = ctypes.c_int32()
    _check(_lib.fe_ks_colour_cells(cd.shape[0], cd.shape[1], n_dofs, cd.ctypes.data, colour.ctypes.data,
                                   ctypes.byref(n)))
    return colour, n.value


def fe_ks_batch_create(ctxs, n_v, precision):
    n = len(ctxs)
    arr = (ctypes.c_void_p * n)(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    nv = (ctypes.c_int64 * n)(*n_v)
    pr = (ctypes.c_int * n)(*precision)
    out = ctypes.c_void_p()
    _check(_lib.fe_ks_batch_create(arr, n, nv, pr, ctypes.byref(out)))
    return out


def fe_ks_batch_configure(batch, tile_config=None, cells_per_item=1, depth=1, wait_seconds=2.0,
                          inject_missing_item=False, blocks_per_sm=1, threads=0):
    tc = None if tile_config is None else (ctypes.c_int * len(tile_config))(*tile_config)
    _check(_lib.fe_ks_batch_configure(batch, tc, cells_per_item, depth, blocks_per_sm, wait_seconds,
                                      int(inject_missing_item), threads))


def fe_ks_batch_apply(batch, Xs, Ys, stream=None):
    n = len(Xs)
    xa = (ctypes.c_void_p * n)(*[_ptr(x) for x in Xs])
    ya = (ctypes.c_void_p * n)(*[_ptr(y) for y in Ys])
    _check(_lib.fe_ks_batch_apply(batch, xa, ya, stream))


def fe_ks_batch_set_split(batch, threads_f64, threads_f32):
    _check(_lib.fe_ks_batch_set_split(batch, threads_f64, threads_f32))


def fe_ks_batch_set_direct(batch, direct=None):
    """Systems flagged in `direct` run their own tuned kernels on side streams (None: none)."""
    arr = None if direct is None else (ctypes.c_int * len(direct))(*[int(bool(d)) for d in direct])
    _check(_lib.fe_ks_batch_set_direct(batch, arr))


def fe_ks_batch_status(batch):
    _check(_lib.fe_ks_batch_status(batch))


def fe_ks_batch_info(batch):
    n, g, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
    _check(_lib.fe_ks_batch_info(batch, ctypes.byref(n), ctypes.byref(g), ctypes.byref(s)))
    return dict(n_items=n.value, grid=g.value, smem_bytes=s.value)


def fe_ks_batch_destroy(batch):
    _lib.fe_ks_batch_destroy(batch)


def fe_ks_gemm_f64(trans_a, trans_b, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, emulated=False, stream=None):
    _check(_lib.fe_ks_gemm_f64(int(trans_a), int(trans_b), m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb, beta,
                               _ptr(C), ldc, int(emulated), stream))


def row_gram(Y, Z, emulated=False, stream=None):
    """Y^T Z for row-major real FP64 Y [m][n1], Z [m][n2] (contiguous device tensors) -> [n1][n2]."""
    import torch
    m, n1 = Y.shape
    n2 = Z.shape[1]
    C = torch.empty((n2, n1), dtype=torch.float64, device=Y.device)     # column-major (n1 x n2)
    # column-major views: Yc (n1 x m, ld n1), Zc (n2 x m, ld n2); C = Yc Zc^T
    fe_ks_gemm_f64(0, 1, n1, n2, m, 1.0, Y, n1, Z, n2, 0.0, C, n1, emulated, stream)
    return C.T


def row_rotate(Y, E, emulated=False, stream=None):
    """Y E for row-major real FP64 Y [m][n], E [n][k] (contiguous device tensors) -> [m][k] row-major."""
    import torch
    m, n = Y.shape
    k = E.shape[1]
    Ec = E.contiguous()
    X = torch.empty((m, k), dtype=torch.float64, device=Y.device)
    # row-major X = Y E  <=>  column-major Xc (k x m) = Ec (k x n) Yc (n x m)
    fe_ks_gemm_f64(0, 0, k, m, n, 1.0, Ec, k, Y, n, 0.0, X, k, emulated, stream)
    return X


def fe_ks_gram_ff(Y, Z, stream=None, work=None, symmetric=False):
    """Y^T Z (row-major FP64 device tensors [m][n1], [m][n2]) in pairs of floats -> [n1][n2].
    symmetric=True: the product is known to be symmetric (n1 = n2); half the tiles are computed."""
    import torch
    m, n1 = Y.shape
    n2 = Z.shape[1]
    nb = ctypes.c_size_t()
    _check(_lib.fe_ks_gram_ff_workspace(m, n1, n2, ctypes.byref(nb)))
    if work is None or work.numel() < nb.value:
        work = torch.empty(nb.value, dtype=torch.uint8, device=Y.device)
    C = torch.empty((n1, n2), dtype=torch.float64, device=Y.device)
    if symmetric:
        _check(_lib.fe_ks_gram_ff_sym(_ptr(Y), _ptr(Z), _ptr(C), m, n1, _ptr(work), nb.value, stream))
    else:
        _check(_lib.fe_ks_gram_ff(_ptr(Y), _ptr(Z), _ptr(C), m, n1, n2, _ptr(work), nb.value, stream))
    return C



def fe_ks_gram_tc_sym(Y, Z, stream=None, work=None):
    """Y^T Z for row-major FP64 device tensors [m][n] whose product is symmetric, on the
    tensor cores (exact 8-bit slices).  Returns (C [n][n], status: 0 = valid)."""
    import torch
    m, n = Y.shape
    nb = ctypes.c_size_t()
    _check(_lib.fe_ks_gram_tc_workspace(m, n, ctypes.byref(nb)))
    if work is None or work.numel() < nb.value + 256:
        work = torch.empty(nb.value + 256, dtype=torch.uint8, device=Y.device)
    off = (-work.data_ptr()) % 256
    view = work[off:off + nb.value]
    C = torch.empty((n, n), dtype=torch.float64, device=Y.device)
    _check(_lib.fe_ks_gram_tc_sym(_ptr(Y), _ptr(Z), _ptr(C), m, n, _ptr(view), nb.value, stream))
    st = ctypes.c_int()
    _check(_lib.fe_ks_gram_tc_status(_ptr(view), ctypes.byref(st)))
    return C, st.value


def fe_ks_rotate_tc(Y, E, stream=None):
    """Y E (row-major FP64 device tensors [m][n], [n][k]) on the tensor cores -> ([m][k], flags)."""
    import torch
    m, n = Y.shape
    k = E.shape[1]
    X = torch.empty((m, k), dtype=torch.float64, device=Y.device)
    flags = torch.zeros(2, dtype=torch.int32, device=Y.device)
    _check(_lib.fe_ks_rotate_tc(_ptr(Y), _ptr(E.contiguous()), _ptr(X), m, n, k, _ptr(flags), stream))
    return X, flags.cpu().tolist()


def fe_ks_set_rr_gram(ctx, tensor_cores):
    _check(_lib.fe_ks_set_rr_gram(ctx, int(bool(tensor_cores))))


def fe_ks_rotate_ff(Y, E, stream=None):
    """Y E (row-major FP64 device tensors [m][n], [n][k]) in pairs of floats -> [m][k]."""
    import torch
    m, n = Y.shape
    k = E.shape[1]
    X = torch.empty((m, k), dtype=torch.float64, device=Y.device)
    _check(_lib.fe_ks_rotate_ff(_ptr(Y), _ptr(E.contiguous()), _ptr(X), m, n, k, stream))
    return X


def fe_ks_rayleigh_ritz_workspace(ctx, n_v, precision):
    out = ctypes.c_size_t()
    _check(_lib.fe_ks_rayleigh_ritz_workspace(ctx, n_v, precision, ctypes.byref(out)))
    return out.value


def fe_ks_rayleigh_ritz(ctx, X, ritz, n_v, precision, work, work_bytes, mass=None):
    """Rayleigh-Ritz on span(X) in place (X <- X E, ritz <- Lam); returns the path taken
    (0 Cholesky, 1 shifted Cholesky QR)."""
    path = ctypes.c_int()
    _check(_lib.fe_ks_rayleigh_ritz(ctx, mass, _ptr(X), _ptr(ritz), n_v, precision, _ptr(work), work_bytes,
                                    ctypes.byref(path)))
    return path.value


def fe_ks_lanczos_bound_workspace(ctx, steps):
    out = ctypes.c_size_t()
    _check(_lib.fe_ks_lanczos_bound_workspace(ctx, steps, ctypes.byref(out)))
    return out.value


def fe_ks_lanczos_bound(ctx, v0, steps, precision, work, work_bytes):
    """Lanczos upper bound of Hs from the device vector v0: (lam_max, alphas, betas)."""
    lm = ctypes.c_double()
    a = (ctypes.c_double * steps)()
    b = (ctypes.c_double * steps)()
    k = ctypes.c_int()
    _check(_lib.fe_ks_lanczos_bound(ctx, _ptr(v0), steps, precision, _ptr(work), work_bytes, ctypes.byref(lm),
                                    a, b, ctypes.byref(k)))
    return lm.value, list(a)[:k.value], list(b)[:k.value]


def fe_ks_dinv_sqrt(ctx):
    return _lib.fe_ks_dinv_sqrt(ctx)


def fe_ks_info(ctx):
    m, E, npairs = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    p, cplx, ncol = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.fe_ks_info(ctx, ctypes.byref(m), ctypes.byref(E), ctypes.byref(p), ctypes.byref(cplx),
                           ctypes.byref(ncol), ctypes.byref(npairs)))
    return dict(n_dofs=m.value, n_cells=E.value, degree=p.value, complex=bool(cplx.value),
                n_colours=ncol.value, n_pairs=npairs.value)


def fe_ks_set_profiling(ctx, on):
    _check(_lib.fe_ks_set_profiling(ctx, int(bool(on))))


def fe_ks_read_profile(ctx):
    """{phase: (ms, launches)} for phases 'fill', 'proj', 'local' since the last read."""
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_int64 * 3)()
    _check(_lib.fe_ks_read_profile(ctx, ms, n))
    return {k: (ms[i], n[i]) for i, k in enumerate(("fill", "proj", "local"))}


def fe_ks_measure_fma_peak(precision):
    out = ctypes.c_double()
    _check(_lib.fe_ks_measure_fma_peak(precision, ctypes.byref(out)))
    return out.value


def fe_ks_set_stream(ctx, stream):
    _check(_lib.fe_ks_set_stream(ctx, stream))


def fe_ks_last_error():
    return _lib.fe_ks_last_error().decode()


def fe_ks_destroy(ctx):
    _lib.fe_ks_destroy(ctx)
