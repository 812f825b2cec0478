"""Full-size parity on sampled rows: the workloads at their benchmark sizes
(C2: 12^3 cells p=6 N_v=64; C3: 16^3 p=7 complex N_v=128; C4: 24^3 p=8 N_v=256;
AE: 24^3 p=8 complex without projectors, N_v=64; C4 with n_q = n_p + 2),
every precision including the 16-bit tensor-core ones,
applied on the GPU in the benchmark's launch configuration, compared with the
oracle's row-restricted evaluation: all nodes of one cell (interior, face, edge
and corner DoFs) plus interior nodes of six random cells.  Tolerances as in
test_parity_apply (per column over the sampled rows).  Also at full size: the
cell-matrix baseline at C4, the six C5 systems in one batched launch, and one
R-ChFSI filter pass at C4 (FP32 and pairs-of-floats recurrences against the
FP64 one, a property that holds at any size)."""
import dataclasses

import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from synth.host_problem import HostProblem
from oracle.operator import Problem
from synth import CONFIGS
from gpu_util import RowCache, needed_rows, fill_device, parity_err, torch_dtype

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {fk.FE_KS_F64: 1e-12, fk.FE_KS_F32: 1e-5, fk.FE_KS_F64E: 1e-12,
       fk.FE_KS_BF16: 2.0 ** -5, fk.FE_KS_F16: 2.0 ** -8,
       fk.FE_KS_BF16X2: 2.0 ** -13}   # 8 u of the 16-bit types (test_parity_bf16)


def _rows(P, wl, seed):
    rng = np.random.default_rng(seed)
    e0 = int(rng.integers(P.E))
    npn = wl.p + 1
    rows = [P.dofs[e0]] + [P.dofs[e][[npn * npn + npn + 1]] for e in rng.integers(0, P.E, 6)]
    return np.unique(np.concatenate(rows))


def _workload(key):
    if key == "C4q":
        return dataclasses.replace(CONFIGS["C4"], nq=CONFIGS["C4"].p + 3, name="C4q")
    return CONFIGS[key]


@pytest.mark.parametrize("key", ["C2", "C3", "C4", "AE", "C4q"])
def test_full_size_sampled_rows(key):
    wl = _workload(key)
    hp = HostProblem(wl)
    P = Problem(wl)
    rows = _rows(P, wl, 7 + len(key))
    need = needed_rows(P, rows)
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, torch.cuda.current_stream().cuda_stream)
    try:
        precisions = [fk.FE_KS_F64, fk.FE_KS_F32, fk.FE_KS_F64E]
        if wl.nq == wl.p + 1:      # the tensor-core kernel needs square 1D operators
            precisions += [fk.FE_KS_BF16, fk.FE_KS_F16, fk.FE_KS_BF16X2]
        for precision in precisions:
            dt = torch_dtype(precision, hp.complex)
            X = torch.empty((hp.m, wl.n_v), dtype=dt, device="cuda")
            npdt = {torch.float64: np.float64, torch.float32: np.float32,
                    torch.complex128: np.complex128, torch.complex64: np.complex64}[dt]
            fill_device(wl, wl.n_v, X, npdt)
            Y = torch.full_like(X, float("nan"))
            fk.fe_ks_apply(ctx, X, Y, wl.n_v, precision)
            torch.cuda.synchronize()
            Yg = Y[torch.from_numpy(rows).cuda()].cpu().numpy()
            del X, Y
            torch.cuda.empty_cache()
            Xl = RowCache(wl, need, round_to=npdt)
            Yref = P.apply_rows(Xl, rows)
            err = parity_err(Yg, Yref)
            assert err <= TOL[precision], (key, precision, err)
    finally:
        fk.fe_ks_destroy(ctx)


def test_cell_matrix_full_size_sampled_rows():
    """The cell-matrix baseline at C4 (58.8 GB of FP64 cell matrices), as the bench runs it."""
    wl = CONFIGS["C4"]
    hp = HostProblem(wl)
    P = Problem(wl)
    rows = _rows(P, wl, 41)
    need = needed_rows(P, rows)
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, torch.cuda.current_stream().cuda_stream)
    refs = {}   # one oracle evaluation per input rounding (FP32 and BF16 both read FP32 X)
    try:
        for precision, tol in ((fk.FE_KS_F64, 1e-12), (fk.FE_KS_F32, 1e-5), (fk.FE_KS_BF16, 2.0 ** -5)):
            dt = torch.float64 if precision == fk.FE_KS_F64 else torch.float32
            npdt = np.float64 if precision == fk.FE_KS_F64 else np.float32
            X = torch.empty((hp.m, wl.n_v), dtype=dt, device="cuda")
            fill_device(wl, wl.n_v, X, npdt)
            Y = torch.full_like(X, float("nan"))
            cm = fk.fe_ks_cm_create(ctx, precision, wl.n_v)
            try:
                fk.fe_ks_cm_apply(cm, X, Y, wl.n_v)
                torch.cuda.synchronize()
            finally:
                fk.fe_ks_cm_destroy(cm)
            Yg = Y[torch.from_numpy(rows).cuda()].cpu().numpy()
            del X, Y
            torch.cuda.empty_cache()
            if npdt not in refs:
                refs[npdt] = P.apply_rows(RowCache(wl, need, round_to=npdt), rows)
            err = parity_err(Yg, refs[npdt])
            assert err <= tol, (precision, err)
    finally:
        fk.fe_ks_destroy(ctx)


@pytest.mark.parametrize("threads,occ", [(384, 1), (512, 2)])
def test_batched_c5_full_size_sampled_rows(threads, occ):
    """The six C5 systems (6^3..20^3 cells, p = 4..8, N_v = 16..512, FP64 / FP32) in one
    persistent launch with the settings the bench's tuner picks (wide tiles, 2 cells per item,
    2 items per fetch), each system's sampled rows against the oracle."""
    from synth import batched_systems
    stream = torch.cuda.current_stream().cuda_stream
    wls = batched_systems()
    prec = [fk.FE_KS_F64 if wl.precision == "f64" else fk.FE_KS_F32 for wl in wls]
    hps = [HostProblem(wl) for wl in wls]
    ctxs = [fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, stream) for hp, wl in zip(hps, wls)]
    try:
        Xs, Ys = [], []
        for wl, pr in zip(wls, prec):
            dt = torch.float64 if pr == fk.FE_KS_F64 else torch.float32
            X = torch.empty((wl.n_dofs, wl.n_v), dtype=dt, device="cuda")
            fill_device(wl, wl.n_v, X, np.float64 if pr == fk.FE_KS_F64 else np.float32)
            Xs.append(X)
            Ys.append(torch.full_like(X, float("nan")))
        b = fk.fe_ks_batch_create(ctxs, [wl.n_v for wl in wls], prec)
        try:
            fk.fe_ks_batch_configure(b, [1] * len(wls), 2, 2, 2.0, False, blocks_per_sm=occ, threads=threads)
            fk.fe_ks_batch_apply(b, Xs, Ys, stream)
            fk.fe_ks_batch_status(b)
        finally:
            fk.fe_ks_batch_destroy(b)
        for s, (wl, pr, Y) in enumerate(zip(wls, prec, Ys)):
            P = Problem(wl)
            npdt = np.float64 if pr == fk.FE_KS_F64 else np.float32
            rows = _rows(P, wl, 50 + s)
            Yg = Y[torch.from_numpy(rows).cuda()].cpu().numpy()
            Yref = P.apply_rows(RowCache(wl, needed_rows(P, rows), round_to=npdt), rows)
            err = parity_err(Yg, Yref)
            assert err <= (1e-12 if pr == fk.FE_KS_F64 else 1e-5), (s, err)
    finally:
        for c in ctxs:
            fk.fe_ks_destroy(c)


def test_filter_pass_full_size():
    """One degree-20 R-ChFSI filter pass at C4 (the bench's pass): the FP32 recurrence stays
    within 2e-4 and the pairs-of-floats recurrence within 1e-12 of the FP64 one, per column
    and element-wise (the bounds of the small-size comparison with the oracle's Algorithm 4)."""
    from paper_2512_08571_gb300.chfsi import RChFSI
    wl = CONFIGS["C4"]
    hp = HostProblem(wl)
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, torch.cuda.current_stream().cuda_stream)
    try:
        X0 = torch.empty((hp.m, wl.n_v), dtype=torch.float64, device="cuda")
        fill_device(wl, wl.n_v, X0, np.float64)
        ref = RChFSI(ctx, hp.m, wl.n_v, False, degree=20, precision=fk.FE_KS_F64, exact=fk.FE_KS_F64)
        lmax = ref.lanczos_upper_bound()
        lam, X = ref.rayleigh_ritz(X0)
        del X0
        X64 = X.clone()
        ref.filter(X64, lam)
        del ref
        torch.cuda.empty_cache()
        for prec, exact, tol in ((fk.FE_KS_F32, fk.FE_KS_F64E, 2e-4), (fk.FE_KS_F64E, fk.FE_KS_F64E, 1e-12)):
            sol = RChFSI(ctx, hp.m, wl.n_v, False, degree=20, precision=prec, exact=exact, gemm_pairs=True)
            sol.lmax = lmax
            Xp = X.clone()
            sol.filter(Xp, lam)
            torch.cuda.synchronize()
            d = Xp - X64
            err = max(float(torch.max(torch.linalg.vector_norm(d, dim=0) / torch.linalg.vector_norm(X64, dim=0))),
                      float(torch.max(d.abs().amax(0) / X64.abs().amax(0))))
            del d
            assert err < tol, (prec, err)
            del sol, Xp
            torch.cuda.empty_cache()
    finally:
        fk.fe_ks_destroy(ctx)
