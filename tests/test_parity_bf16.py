"""GPU parity of the tensor-core cell kernel (FE_KS_BF16, FE_KS_F16) against the
FP64 oracle.

Both keep X and Y in FP32 and run the 1D contractions of Algorithm 2 as 16-bit
products with FP32 accumulation (FP16 with a power-of-two scale per cell tile).
Tolerance derivation: a rounding to the 16-bit type has relative error <= u
(2^-8 for BF16's 8 significant bits, 2^-11 for FP16's 11).  A value reaches
the output through at most six roundings of data (the gathered X, the x and
y sweeps, the quadrature-point values, the transposed z and y sweeps) and the
rounded entries of three 1D matrices; for the trial blocks used here (uniform
random columns, dominated by the kinetic term) the result does not cancel
against its intermediates, so the first-order bound is (6 + 3) u = 0.035 per
element and a column norm is no worse.  The tests hold the per-column
relative error (max over columns) to 8 u = 2^-5 = 0.03125, which the measured
errors clear by a wide margin; the input the oracle sees is the FP32-rounded
one, so only the arithmetic differs.  The same bound with u = 2^-11 holds
for FP16.  The split precision FE_KS_BF16X2 holds every 16-bit operand as
hi + lo (hi = bf16(x), lo = bf16(x - hi)): the pair carries x to a relative
error of 2^-16, and the dropped lo * lo term of each product is below 2^-16 of
it, so the same count of roundings with u = 2^-16 gives 8 u = 2^-13.
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

U = {fk.FE_KS_BF16: 2.0 ** -8, fk.FE_KS_F16: 2.0 ** -11, fk.FE_KS_BF16X2: 2.0 ** -16}
TOL16 = {prec: 8 * u for prec, u in U.items()}
TOL = TOL16[fk.FE_KS_BF16]
BF = fk.FE_KS_BF16
TC = [fk.FE_KS_BF16, fk.FE_KS_F16, fk.FE_KS_BF16X2]
NAME = {fk.FE_KS_BF16: "BF16", fk.FE_KS_F16: "FP16", fk.FE_KS_BF16X2: "BF16x2"}

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


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("key", list(SMALL))
def test_bf16_matches_oracle(cases, key, prec):
    wl, hp, P, X = cases[key]
    Xin = round_input(X, prec)
    Y = gpu_apply(hp, Xin, prec)
    err = parity_err(Y, P.apply(Xin))
    print(f"{key}: {NAME[prec]} tensor-core rel err {err:.3e} (tolerance {TOL16[prec]:.3e})")
    assert err <= TOL16[prec], err


@pytest.mark.parametrize("scale", [1e-7, 1e5])
def test_f16_tile_scaling_range(cases, scale):
    """FP16 has a narrow range: blocks scaled far below (1e-7: subnormal in FP16)
    and above (1e5: the intermediates would overflow 65504) keep the relative
    error of the unscaled block, because every cell tile is scaled by a power
    of two before the 16-bit rounding and unscaled after."""
    wl, hp, P, X = cases["C4v"]
    Xin = round_input(X * scale, fk.FE_KS_F16)
    Y = gpu_apply(hp, Xin, fk.FE_KS_F16)
    assert np.all(np.isfinite(Y))
    err = parity_err(Y, P.apply(Xin))
    assert err <= TOL16[fk.FE_KS_F16], (scale, err)


def test_bf16_scaled_matches_oracle(cases):
    wl, hp, P, X = cases["C2s"]
    Xin = round_input(X, BF)
    s = 1.0 / np.sqrt(P.lumped_mass())
    Y = gpu_apply(hp, Xin, BF, scaled=True)
    err = parity_err(Y, s[:, None] * P.apply(s[:, None] * Xin))
    assert err <= TOL, err


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("p", range(1, 9))
def test_bf16_every_degree(p, prec):
    wl = Workload(f"deg{p}", L=4.0 + p, n=2 if p > 2 else 3, p=p, nq=p + 1, n_v=11, jitter=0.08, gga=True,
                  seed=900 + p)
    hp = HostProblem(wl)
    P = Problem(wl)
    X = round_input(trial_vectors(wl), prec)
    err = parity_err(gpu_apply(hp, X, prec), P.apply(X))
    assert err <= TOL16[prec], (p, err)


def test_bf16_term_subsets(cases):
    wl, hp, P, X = cases["C2s"]
    X = round_input(X, BF)
    zero = lambda x: np.zeros(np.asarray(x).shape[:-1])
    P_T = Problem(wl, vloc=zero, vgga=None, with_atoms=False)
    assert parity_err(gpu_apply(hp, X, BF, terms=fk.TERM_T), P_T.apply(X)) <= TOL
    P_loc = Problem(wl, with_atoms=False)
    assert parity_err(gpu_apply(hp, X, BF, terms=fk.TERM_ALL & ~fk.TERM_NL), P_loc.apply(X)) <= TOL


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
    assert parity_err(Yb, Yf) <= TOL
    assert parity_err(Yb, Yf) > 1e-6   # really a different (lower-precision) arithmetic


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("key", ["C2s", "C3s", "C4s"])
def test_bf16_nonlocal_term_isolated(cases, key, prec):
    """The nonlocal term alone: for random trial blocks it is 1e-5..1e-4 of |H X|,
    below the BF16 tolerance of the whole result, so it is checked on its own as
    Y(all terms) - Y(local terms).  Both runs use the same kernel on the same
    input, so the local parts agree to FP32 rounding of the accumulators
    (u_32 |H X| / |NL| <= 6e-8 x 1e5 = 6e-3 relative to the term), and the
    nonlocal part carries the 16-bit rounding of F and Q (2 u)."""
    wl, hp, P, X = cases[key]
    X = round_input(X, prec)
    Y_all = gpu_apply(hp, X, prec)
    Y_loc = gpu_apply(hp, X, prec, terms=fk.TERM_ALL & ~fk.TERM_NL)
    ref = P.apply(X) - Problem(wl, with_atoms=False).apply(X)
    err = parity_err(Y_all - Y_loc, ref)
    print(f"{key}: {NAME[prec]} nonlocal term rel err {err:.3e}")
    # FP32 rounding of the accumulators relative to the term (6e-3, see above) bounds FP16 too
    assert err <= max(TOL16[prec], 1e-2), err


@pytest.mark.parametrize("prec", TC)
def test_columns_of_very_different_size(cases, prec):
    """Columns of one tile spanning 15 orders of magnitude (as converged and
    unconverged vectors do inside the eigensolver) keep each column's relative
    error: FP16 scales every column by its own power of two."""
    wl, hp, P, X = cases["C4v"]
    Xs = X * (10.0 ** -np.arange(X.shape[1]))[None, :]
    Xin = round_input(Xs, prec)
    Y = gpu_apply(hp, Xin, prec)
    err = parity_err(Y, P.apply(Xin))
    assert err <= TOL16[prec], err


def test_split_precision_is_near_fp32(cases):
    """BF16x2 really carries the extra digits: on every case its error is at least
    16 times smaller than single BF16's (the bound ratio is 2^8)."""
    for key in ("C2s", "C4v", "C3v"):
        wl, hp, P, X = cases[key]
        Xin = round_input(X, BF)
        ref = P.apply(Xin)
        e1 = parity_err(gpu_apply(hp, Xin, BF), ref)
        e2 = parity_err(gpu_apply(hp, Xin, fk.FE_KS_BF16X2), ref)
        assert e2 * 16 <= e1, (key, e1, e2)
