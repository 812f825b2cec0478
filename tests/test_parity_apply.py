"""GPU parity of fe_ks_apply against the FP64 oracle (eq. HX, Algorithms 1-2).

Tolerances: relative error per column (max over columns of
||Y_v - Y_v^ref|| / ||Y_v^ref||) <= 1e-12 for FP64 and for the FP64-accurate
pair-of-floats variant (FE_KS_F64E), <= 1e-5 for FP32; the FP32 case feeds the
oracle the FP32-rounded input, so only the arithmetic differs.
"""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from synth.host_problem import HostProblem
from oracle.operator import Problem
from synth import CONFIGS, Workload, trial_vectors
from gpu_util import gpu_apply, parity_err, round_input

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {fk.FE_KS_F64: 1e-12, fk.FE_KS_F32: 1e-5, fk.FE_KS_F64E: 1e-12}
PREC = [fk.FE_KS_F64, fk.FE_KS_F32, fk.FE_KS_F64E]

# parity-sized versions of the four operator workloads (several tiles, ragged column tails)
SMALL = {
    "C1": CONFIGS["C1"],
    "C2s": CONFIGS["C2"].scaled(n=6, n_v=7),
    "C3s": CONFIGS["C3"].scaled(n=4, n_v=3, n_atoms=4),
    "C4s": CONFIGS["C4"].scaled(n=4, n_v=5, n_atoms=6),
    # column counts whose rows are 16-byte aligned (vectorised staging path)
    "C4v": CONFIGS["C4"].scaled(n=4, n_v=16, n_atoms=6),
    "C3v": CONFIGS["C3"].scaled(n=4, n_v=4, n_atoms=4),
}


@pytest.fixture(scope="module")
def cases():
    out = {}
    for key, wl in SMALL.items():
        out[key] = (wl, HostProblem(wl), Problem(wl), trial_vectors(wl))
    return out


@pytest.mark.parametrize("precision", PREC)
@pytest.mark.parametrize("key", list(SMALL))
def test_apply_matches_oracle(cases, key, precision):
    wl, hp, P, X = cases[key]
    Xin = round_input(X, precision)
    Y = gpu_apply(hp, Xin, precision)
    Yref = P.apply(Xin)
    err = parity_err(Y, Yref)
    assert err <= TOL[precision], err


@pytest.mark.parametrize("config", range(fk.N_CONFIGS))
@pytest.mark.parametrize("key", ["C2s", "C3s", "C4s", "C4v", "C3v"])
def test_every_tile_configuration(cases, key, config):
    """Every tile configuration the tuner may pick gives the same answer."""
    wl, hp, P, X = cases[key]
    for precision in PREC:
        Xin = round_input(X, precision)
        try:
            Y = gpu_apply(hp, Xin, precision, config=config)
        except fk.FeKsError as exc:          # configuration too large for this degree/precision
            assert "configuration" in str(exc) or "invalid" in str(exc), exc
            continue
        err = parity_err(Y, P.apply(Xin))
        assert err <= TOL[precision], (config, precision, err)


@pytest.mark.parametrize("precision", PREC)
def test_apply_scaled_matches_oracle(cases, precision):
    wl, hp, P, X = cases["C2s"]
    Xin = round_input(X, precision)
    s = 1.0 / np.sqrt(P.lumped_mass())
    Y = gpu_apply(hp, Xin, precision, scaled=True)
    Yref = s[:, None] * P.apply(s[:, None] * Xin)
    err = parity_err(Y, Yref)
    assert err <= TOL[precision], err


@pytest.mark.parametrize("p", range(1, 9))
def test_every_degree_kinetic_and_local(p):
    wl = Workload(f"deg{p}", L=4.0 + p, n=2 if p > 2 else 3, p=p, nq=p + 1, n_v=3, jitter=0.08, seed=900 + p)
    hp = HostProblem(wl)
    P = Problem(wl)
    X = trial_vectors(wl)
    Y = gpu_apply(hp, X, fk.FE_KS_F64)
    err = parity_err(Y, P.apply(X))
    assert err <= 1e-12, err


def test_term_subsets(cases):
    wl, hp, P, X = cases["C2s"]
    zero = lambda x: np.zeros(np.asarray(x).shape[:-1])
    P_T = Problem(wl, vloc=zero, vgga=None, with_atoms=False)
    Y = gpu_apply(hp, X, fk.FE_KS_F64, terms=fk.TERM_T)
    assert parity_err(Y, P_T.apply(X)) <= 1e-12
    P_TL = Problem(wl, vgga=None, with_atoms=False)
    Y = gpu_apply(hp, X, fk.FE_KS_F64, terms=fk.TERM_T | fk.TERM_L)
    assert parity_err(Y, P_TL.apply(X)) <= 1e-12
    P_loc = Problem(wl, with_atoms=False)
    Y = gpu_apply(hp, X, fk.FE_KS_F64, terms=fk.TERM_ALL & ~fk.TERM_NL)
    assert parity_err(Y, P_loc.apply(X)) <= 1e-12


def test_single_vector_and_bitwise_determinism(cases):
    wl, hp, P, X = cases["C3s"]
    Ys = gpu_apply(hp, X[:, :1], fk.FE_KS_F64, repeat=2)
    assert np.array_equal(Ys[0], Ys[1])
    assert parity_err(Ys[0], P.apply(X[:, :1])) <= 1e-12


def test_zero_input_gives_zero(cases):
    wl, hp, P, X = cases["C4s"]
    Y = gpu_apply(hp, np.zeros_like(X), fk.FE_KS_F64)
    assert np.all(Y == 0.0)


def test_invalid_calls_are_rejected(cases):
    wl, hp, P, X = cases["C1"]
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, 4, torch.cuda.current_stream().cuda_stream)
    try:
        Xd = torch.zeros((hp.m, 8), dtype=torch.float64, device="cuda")
        Yd = torch.zeros_like(Xd)
        with pytest.raises(fk.FeKsError, match="n_v"):
            fk.fe_ks_apply(ctx, Xd, Yd, 8, fk.FE_KS_F64)       # above n_v_max
        with pytest.raises(fk.FeKsError, match="overlap"):
            fk.fe_ks_apply(ctx, Xd, Xd, 4, fk.FE_KS_F64)
        with pytest.raises(fk.FeKsError, match="precision"):
            fk.fe_ks_apply(ctx, Xd, Yd, 4, 7)
    finally:
        fk.fe_ks_destroy(ctx)


@pytest.mark.parametrize("precision", PREC)
@pytest.mark.parametrize("key", ["C2s", "C3s", "C4s"])
def test_nonlocal_term_isolated(cases, key, precision):
    """Y(all terms) - Y(local terms) against the oracle's nonlocal term: the term is
    1e-5..1e-4 of |H X| for random blocks, so it is checked on its own.  The
    difference carries the storage rounding of the full result, u |H X| / |NL|
    relative to the term (<= 1e-16 x 1e5 for FP64, 6e-8 x 1e5 for FP32)."""
    wl, hp, P, X = cases[key]
    Xin = round_input(X, precision)
    Y_all = gpu_apply(hp, Xin, precision)
    Y_loc = gpu_apply(hp, Xin, precision, terms=fk.TERM_ALL & ~fk.TERM_NL)
    ref = P.apply(Xin) - Problem(wl, with_atoms=False).apply(Xin)
    tol = {fk.FE_KS_F64: 1e-9, fk.FE_KS_F64E: 1e-9, fk.FE_KS_F32: 1e-2}[precision]
    assert parity_err(Y_all - Y_loc, ref) <= tol
