"""GPU parity at n_q = n_p + 2, the paper's default quadrature (Sec. 6): the 1D
interpolation N is n_q x n_p (not square) and the gradient D~ is n_q x n_q.

Same tolerances as at n_q = n_p: 1e-12 per column in FP64 and in pairs of
floats, 1e-5 in FP32 on the FP32-rounded input.  The tensor-core precisions
and the batched launch refuse n_q != n_p.
"""
import dataclasses

import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from synth.host_problem import HostProblem
from oracle.operator import Problem
from synth import CONFIGS, trial_vectors
from gpu_util import gpu_apply, parity_err, round_input

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {fk.FE_KS_F64: 1e-12, fk.FE_KS_F32: 1e-5, fk.FE_KS_F64E: 1e-12}
PREC = [fk.FE_KS_F64, fk.FE_KS_F32, fk.FE_KS_F64E]


def _nq2(wl, **kw):
    w = wl.scaled(**kw)
    return dataclasses.replace(w, nq=w.p + 3, name=w.name + "-q2")


SMALL = {
    "C1q": _nq2(CONFIGS["C1"], n=3, n_v=5),                 # p = 4, n_q = 7
    "C2q": _nq2(CONFIGS["C2"], n=4, n_v=7),                 # p = 6, n_q = 9, jitter, GGA, atoms
    "C3q": _nq2(CONFIGS["C3"], n=3, n_v=3, n_atoms=4),      # p = 7, n_q = 10, complex
    "C4q": _nq2(CONFIGS["C4"], n=3, n_v=8, n_atoms=6),      # p = 8, n_q = 11, aligned columns
}


@pytest.fixture(scope="module")
def cases():
    return {k: (wl, HostProblem(wl), Problem(wl), trial_vectors(wl)) for k, wl in SMALL.items()}


@pytest.mark.parametrize("precision", PREC)
@pytest.mark.parametrize("key", list(SMALL))
def test_apply_nq_np2_matches_oracle(cases, key, precision):
    wl, hp, P, X = cases[key]
    Xin = round_input(X, precision)
    err = parity_err(gpu_apply(hp, Xin, precision), P.apply(Xin))
    assert err <= TOL[precision], err


@pytest.mark.parametrize("key", ["C2q", "C4q"])
def test_every_fitting_tile_configuration(cases, key):
    """Configurations whose tiles fit in shared memory at n_q = n_p + 2 agree; the others
    are reported as not runnable by the tuner (time -1) instead of launching."""
    wl, hp, P, X = cases[key]
    n_v = X.shape[1]
    for precision in PREC:
        Xin = round_input(X, precision)
        Yref = P.apply(Xin)
        ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, n_v, torch.cuda.current_stream().cuda_stream)
        try:
            dt = torch.float64 if precision != fk.FE_KS_F32 else torch.float32
            Xd = torch.from_numpy(np.ascontiguousarray(Xin)).to("cuda").to(dt)
            Yd = torch.empty_like(Xd)
            best, ms = fk.fe_ks_tune(ctx, Xd, Yd, n_v, precision, reps=1)
            runnable = [c for c, t in enumerate(ms) if t > 0]
            assert 0 in runnable and best in runnable
            for cfg in runnable:
                fk.fe_ks_set_config(ctx, precision, cfg)
                Yd.fill_(float("nan"))
                fk.fe_ks_apply(ctx, Xd, Yd, n_v, precision)
                torch.cuda.synchronize()
                err = parity_err(Yd.cpu().numpy(), Yref)
                assert err <= TOL[precision], (precision, cfg, err)
        finally:
            fk.fe_ks_destroy(ctx)


def test_scaled_apply_nq_np2(cases):
    """H~ = D^{-1/2} H D^{-1/2}: D is the GLL-lumped mass, independent of n_q."""
    wl, hp, P, X = cases["C2q"]
    d = 1.0 / np.sqrt(P.lumped_mass())
    Y = gpu_apply(hp, X, fk.FE_KS_F64, scaled=True)
    Yref = d[:, None] * P.apply(d[:, None] * X)
    assert parity_err(Y, Yref) <= 1e-12


def test_tensor_core_precisions_refuse_nq_np2(cases):
    wl, hp, P, X = cases["C4q"]
    for precision in (fk.FE_KS_BF16, fk.FE_KS_F16, fk.FE_KS_BF16X2):
        with pytest.raises(fk.FeKsError, match="UNSUPPORTED"):
            gpu_apply(hp, X.astype(np.float32), precision)


def test_cell_matrix_nq_np2(cases):
    """The cell-matrix baseline built from the n_q = n_p + 2 operator."""
    wl, hp, P, X = cases["C4q"]
    n_v = X.shape[1]
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, n_v, torch.cuda.current_stream().cuda_stream)
    try:
        cm = fk.fe_ks_cm_create(ctx, fk.FE_KS_F64, n_v)
        try:
            Xd = torch.from_numpy(X).to("cuda")
            Yd = torch.empty_like(Xd)
            fk.fe_ks_cm_apply(cm, Xd, Yd, n_v)
            torch.cuda.synchronize()
            assert parity_err(Yd.cpu().numpy(), P.apply(X)) <= 1e-12
        finally:
            fk.fe_ks_cm_destroy(cm)
    finally:
        fk.fe_ks_destroy(ctx)
