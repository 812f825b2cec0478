"""GPU parity of the cell-matrix baseline (fe_ks_cm_*) against the FP64 oracle.

The cell-matrix method (Sec. 3) applies the same operator as the matrix-free
kernels, one dense H_loc^(e) per cell plus the separable nonlocal term, so it
takes the same tolerances as fe_ks_apply: 1e-12 per column in FP64, 1e-5 in
FP32 on the FP32-rounded input.
"""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from synth.host_problem import HostProblem
from oracle.operator import Problem
from synth import CONFIGS, trial_vectors
from gpu_util import gpu_apply, parity_err, round_input

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# BF16 (tensor-core GEMM on BF16-rounded H^(e) and X^(e), FP32 accumulation): 8 units of
# BF16 rounding, as for the matrix-free tensor-core path
TOL = {fk.FE_KS_F64: 1e-12, fk.FE_KS_F32: 1e-5, fk.FE_KS_BF16: 8 * 2.0 ** -8}

SMALL = {
    "C1": CONFIGS["C1"],
    "C2s": CONFIGS["C2"].scaled(n=6, n_v=7),            # GGA, jittered mesh, ragged columns
    "C4s": CONFIGS["C4"].scaled(n=4, n_v=5, n_atoms=6),  # GGA + nonlocal projectors
    "C4v": CONFIGS["C4"].scaled(n=4, n_v=16, n_atoms=6),
}


@pytest.fixture(scope="module")
def cases():
    return {k: (wl, HostProblem(wl), Problem(wl), trial_vectors(wl)) for k, wl in SMALL.items()}


def cm_apply(hp, X, precision, terms=fk.TERM_ALL, n_v_max=None):
    n_v = X.shape[1]
    ctx = fk.fe_ks_setup(hp.struct, terms, n_v if n_v_max is None else n_v_max,
                         torch.cuda.current_stream().cuda_stream)
    try:
        cm = fk.fe_ks_cm_create(ctx, precision, n_v if n_v_max is None else n_v_max)
        try:
            dt = torch.float64 if precision == fk.FE_KS_F64 else torch.float32
            Xd = torch.from_numpy(np.ascontiguousarray(X)).to("cuda").to(dt)
            Yd = torch.full_like(Xd, float("nan"))
            fk.fe_ks_cm_apply(cm, Xd, Yd, n_v)
            torch.cuda.synchronize()
            info = fk.fe_ks_cm_info(cm)
            return Yd.cpu().numpy(), info["setup_ms"], info["bytes"]
        finally:
            fk.fe_ks_cm_destroy(cm)
    finally:
        fk.fe_ks_destroy(ctx)


@pytest.mark.parametrize("precision", [fk.FE_KS_F64, fk.FE_KS_F32, fk.FE_KS_BF16])
@pytest.mark.parametrize("key", list(SMALL))
def test_cell_matrix_matches_oracle(cases, key, precision):
    wl, hp, P, X = cases[key]
    Xin = round_input(X, precision)
    Y, ms, nbytes = cm_apply(hp, Xin, precision)
    err = parity_err(Y, P.apply(Xin))
    assert err <= TOL[precision], err
    esz = {fk.FE_KS_F64: 8, fk.FE_KS_F32: 4, fk.FE_KS_BF16: 2}[precision]
    assert nbytes >= wl.n_cells * (wl.p + 1) ** 6 * esz   # every cell matrix is held
    assert ms > 0.0


@pytest.mark.parametrize("key", ["C2s", "C4s"])
def test_cell_matrix_equals_matrix_free(cases, key):
    """Same operator, two algorithms: FP64 results agree to rounding."""
    wl, hp, P, X = cases[key]
    Ycm, _, _ = cm_apply(hp, X, fk.FE_KS_F64)
    Ymf = gpu_apply(hp, X, fk.FE_KS_F64)
    assert parity_err(Ycm, Ymf) <= 1e-13


def test_cell_matrix_terms_and_fewer_columns(cases):
    """Kinetic-only operator and n_v below the buffers' n_v_max."""
    wl, hp, P, X = cases["C4s"]
    Xs = X[:, :3]
    zero = lambda x: np.zeros(np.asarray(x).shape[:-1])
    P_T = Problem(wl, vloc=zero, vgga=None, with_atoms=False)
    Y, _, _ = cm_apply(hp, Xs, fk.FE_KS_F64, terms=fk.TERM_T, n_v_max=X.shape[1])
    assert parity_err(Y, P_T.apply(Xs)) <= 1e-12


def test_cell_matrix_rejects_bad_arguments(cases):
    wl, hp, P, X = cases["C1"]
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, 4, torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(fk.FeKsError):
            fk.fe_ks_cm_create(ctx, fk.FE_KS_F16, 4)
        with pytest.raises(fk.FeKsError):
            fk.fe_ks_cm_create(ctx, fk.FE_KS_F64, 5)   # above the context's n_v_max
        cm = fk.fe_ks_cm_create(ctx, fk.FE_KS_F64, 2)
        try:
            Xd = torch.zeros(wl.n_dofs, 4, dtype=torch.float64, device="cuda")
            with pytest.raises(fk.FeKsError):
                fk.fe_ks_cm_apply(cm, Xd, Xd.clone(), 3)   # above the baseline's n_v_max
        finally:
            fk.fe_ks_cm_destroy(cm)
    finally:
        fk.fe_ks_destroy(ctx)


def test_cell_matrix_rejects_complex():
    wl = CONFIGS["C3"].scaled(n=2, n_v=2, n_atoms=2)
    hp = HostProblem(wl)
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, 2, torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(fk.FeKsError):
            fk.fe_ks_cm_create(ctx, fk.FE_KS_F64, 2)
    finally:
        fk.fe_ks_destroy(ctx)
