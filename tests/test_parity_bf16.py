"""GPU parity of the tensor-core cell kernel (FE_KS_BF16) against the FP64 oracle.

FE_KS_BF16 keeps X and Y in FP32 and runs the 1D contractions of Algorithm 2
as BF16 x BF16 products with FP32 accumulation.  Tolerance derivation: a BF16
rounding has relative error <= u = 2^-8 (8 significant bits).  A value reaches
the output through at most six roundings of data (the gathered X, the x and
y sweeps, the quadrature-point values, the transposed z and y sweeps) and the
rounded entries of three 1D matrices; for the trial blocks used here (uniform
random columns, dominated by the kinetic term) the result does not cancel
against its intermediates, so the first-order bound is (6 + 3) u = 0.035 per
element and a column norm is no worse.  The tests hold the per-column
relative error (max over columns) to 8 u = 2^-5 = 0.03125, which the measured
errors clear by a wide margin; the input the oracle sees is the FP32-rounded
one, so only the arithmetic differs.
"""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from paper_2512_08571_gb300.problem import HostProblem
from oracle.operator import Problem
from synth import CONFIGS, Workload, trial_vectors
from gpu_util import gpu_apply, rel_err_cols, round_input

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8
TOL = 8 * U_BF16
BF = fk.FE_KS_BF16

SMALL = {
    "C1": CONFIGS["C1"],
    "C2s": CONFIGS["C2"].scaled(n=6, n_v=7),
    "C3s": CONFIGS["C3"].scaled(n=4, n_v=3, n_atoms=4),
    "C4s": CONFIGS["C4"].scaled(n=4, n_v=5, n_atoms=6),
    "C4v": CONFIGS["C4"].scaled(n=4, n_v=16, n_atoms=6),
    "C3v": CONFIGS["C3"].scaled(n=4, n_v=12, n_atoms=4),
    # more column tiles than one CTA takes, ragged last tile
    "C4w": CONFIGS["C4"].scaled(n=3, n_v=37, n_atoms=3),
}


@pytest.fixture(scope="module")
def cases():
    return {k: (wl, HostProblem(wl), Problem(wl), trial_vectors(wl)) for k, wl in SMALL.items()}


@pytest.mark.parametrize("key", list(SMALL))
def test_bf16_matches_oracle(cases, key):
    wl, hp, P, X = cases[key]
    Xin = round_input(X, BF)
    Y = gpu_apply(hp, Xin, BF)
    err = rel_err_cols(Y, P.apply(Xin))
    print(f"{key}: BF16 tensor-core rel err {err:.3e} (tolerance {TOL:.3e})")
    assert err <= TOL, err


def test_bf16_scaled_matches_oracle(cases):
    wl, hp, P, X = cases["C2s"]
    Xin = round_input(X, BF)
    s = 1.0 / np.sqrt(P.lumped_mass())
    Y = gpu_apply(hp, Xin, BF, scaled=True)
    err = rel_err_cols(Y, s[:, None] * P.apply(s[:, None] * Xin))
    assert err <= TOL, err


@pytest.mark.parametrize("p", range(1, 9))
def test_bf16_every_degree(p):
    wl = Workload(f"deg{p}", L=4.0 + p, n=2 if p > 2 else 3, p=p, nq=p + 1, n_v=11, jitter=0.08, gga=True,
                  seed=900 + p)
    hp = HostProblem(wl)
    P = Problem(wl)
    X = round_input(trial_vectors(wl), BF)
    err = rel_err_cols(gpu_apply(hp, X, BF), P.apply(X))
    assert err <= TOL, (p, err)


def test_bf16_term_subsets(cases):
    wl, hp, P, X = cases["C2s"]
    X = round_input(X, BF)
    zero = lambda x: np.zeros(np.asarray(x).shape[:-1])
    P_T = Problem(wl, vloc=zero, vgga=None, with_atoms=False)
    assert rel_err_cols(gpu_apply(hp, X, BF, terms=fk.TERM_T), P_T.apply(X)) <= TOL
    P_loc = Problem(wl, with_atoms=False)
    assert rel_err_cols(gpu_apply(hp, X, BF, terms=fk.TERM_ALL & ~fk.TERM_NL), P_loc.apply(X)) <= TOL


def test_bf16_deterministic_and_zero(cases):
    wl, hp, P, X = cases["C4v"]
    X = round_input(X, BF)
    Ys = gpu_apply(hp, X, BF, repeat=2)
    assert np.array_equal(Ys[0], Ys[1])
    assert np.all(gpu_apply(hp, np.zeros_like(X), BF) == 0.0)


def test_bf16_close_to_fp32_kernel(cases):
    """The tensor-core result sits within the BF16 bound of the FP32 CUDA-core kernel's."""
    wl, hp, P, X = cases["C3v"]
    X = round_input(X, BF)
    Yb = gpu_apply(hp, X, BF)
    Yf = gpu_apply(hp, X, fk.FE_KS_F32)
    assert rel_err_cols(Yb, Yf) <= TOL
    assert rel_err_cols(Yb, Yf) > 1e-6   # really a different (lower-precision) arithmetic


@pytest.mark.parametrize("key", ["C2s", "C3s", "C4s"])
def test_bf16_nonlocal_term_isolated(cases, key):
    """The nonlocal term alone: for random trial blocks it is 1e-5..1e-4 of |H X|,
    below the BF16 tolerance of the whole result, so it is checked on its own as
    Y(all terms) - Y(local terms).  Both runs use the same kernel on the same
    input, so the local parts agree to FP32 rounding of the accumulators
    (u_32 |H X| / |NL| <= 6e-8 x 1e5 = 6e-3 relative to the term), and the
    nonlocal part carries the BF16 rounding of F and Q (2 u)."""
    wl, hp, P, X = cases[key]
    X = round_input(X, BF)
    Y_all = gpu_apply(hp, X, BF)
    Y_loc = gpu_apply(hp, X, BF, terms=fk.TERM_ALL & ~fk.TERM_NL)
    ref = P.apply(X) - Problem(wl, with_atoms=False).apply(X)
    err = rel_err_cols(Y_all - Y_loc, ref)
    print(f"{key}: BF16 nonlocal term rel err {err:.3e}")
    assert err <= TOL, err
