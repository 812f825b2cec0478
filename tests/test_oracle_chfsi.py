"""Pins of the oracle's R-ChFSI filter (Algorithm 4), Rayleigh-Ritz (Algorithm 3),
Lanczos bound, and the paper's FLOP model (eq. flopRealMF / eq. flopComplexMF)."""
import numpy as np
import pytest

from oracle import chfsi, flops
from oracle.operator import Problem
from synth import Workload, trial_vectors


def _sym(n, seed, complex_=False):
    rng = np.random.default_rng(seed)
    ev = np.sort(rng.uniform(-3.0, 20.0, n))
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if complex_ else 0))
    return (Q * ev) @ Q.conj().T, ev, Q


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("degree", [2, 5, 12])
def test_filter_equals_chebyshev_closed_form(degree, complex_):
    """Algorithm 4 (residual form) equals T_m((H-c)/e)/T_m((lmin-c)/e) X (numpy chebval)."""
    H, ev, Q = _sym(60, 1 + degree, complex_)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((60, 6)) + (1j * rng.standard_normal((60, 6)) if complex_ else 0)
    lam = np.sort(rng.uniform(-3.0, 2.0, 6))           # arbitrary "Ritz values": the identity is exact
    lmin, lT, lmax = -3.5, 2.0, 20.5
    got = chfsi.filter_rchfsi(lambda V: H @ V, X, lam, degree, lmin, lT, lmax)
    want = chfsi.filter_reference_polynomial(ev, Q, X, degree, lmin, lT, lmax)
    assert np.max(np.abs(got - want)) < 1e-10 * np.max(np.abs(want))


def test_lanczos_upper_bound():
    H, ev, _ = _sym(200, 9)
    ub = chfsi.lanczos_upper_bound(lambda V: H @ V, np.random.default_rng(0).standard_normal(200), 10)
    assert ub >= ev[-1] - 1e-12
    assert ub < ev[-1] + 0.5 * (ev[-1] - ev[0])


def test_rchfsi_converges_to_lowest_eigenvalues_of_fe_operator():
    wl = Workload("eig", L=9.0, n=3, p=3, nq=4, n_v=12, jitter=0.1, gga=True, n_atoms=2, seed=21)
    P = Problem(wl)
    H = P.assemble("H").toarray()
    D = P.lumped_mass()
    s = 1.0 / np.sqrt(D)
    Hs = s[:, None] * H * s[None, :]
    want = np.linalg.eigvalsh(Hs)[:8]
    X0 = trial_vectors(wl, n_v=12)
    lam, X, res = chfsi.rchfsi(lambda V: Hs @ V, X0, degree=12, n_iter=40, tol=1e-10)
    np.testing.assert_allclose(lam[:8], want, atol=1e-8)
    assert np.max(res[:8]) < 1e-7


@pytest.mark.parametrize("n_p,n_q", [(5, 5), (7, 7), (9, 9), (8, 10), (5, 7)])
def test_flop_model_stage_sum_equals_closed_form(n_p, n_q):
    """The per-stage counts printed before eq. flopRealMF / flopComplexMF sum to the printed totals."""
    args = (n_p, n_q, 7, 11, 13)
    assert sum(flops.mf_real_stages(*args).values()) == flops.mf_real_total(*args)
    assert sum(flops.mf_complex_stages(*args).values()) == flops.mf_complex_total(*args)


def test_flop_model_leading_order():
    """About 12 n_p^4 FLOP per vector per cell at leading order (Sec. 5.4), 2 n_p^6 for CM."""
    n = 200
    per = flops.mf_real_total(n, n, 1, 1, 0) / n ** 4
    assert 11.5 < per < 12.6
    assert flops.cm_real_total(n, 1, 1, 0) == 2 * n ** 6


# ---- generalised form (consistent mass M, D^{-1} in the recurrence)

@pytest.mark.parametrize("degree", [3, 9])
def test_ghep_filter_with_diagonal_mass_is_the_scaled_standard_filter(degree):
    """With M = D (diagonal), Algorithm 4 for the GHEP is the standard-form filter
    on Hs = D^{-1/2} H D^{-1/2} in the variables D^{1/2} X:
        D^{1/2} filter_ghep(H, D, D^{-1}; X) = filter_std(Hs; D^{1/2} X).
    A D^{-1} in the wrong place (residual, recurrence or final step) breaks it."""
    H, _, _ = _sym(50, 30 + degree)
    rng = np.random.default_rng(5)
    D = rng.uniform(0.5, 2.0, 50)
    X = rng.standard_normal((50, 5))
    lam = np.sort(rng.uniform(-3.0, 1.0, 5))
    lmin, lT, lmax = -3.5, 1.0, 45.0
    got = chfsi.filter_rchfsi_ghep(lambda V: H @ V, lambda V: D[:, None] * V, 1.0 / D, X, lam, degree, lmin, lT, lmax)
    s = 1.0 / np.sqrt(D)
    Hs = s[:, None] * H * s[None, :]
    want = chfsi.filter_rchfsi(lambda V: Hs @ V, np.sqrt(D)[:, None] * X, lam, degree, lmin, lT, lmax)
    assert np.max(np.abs(np.sqrt(D)[:, None] * got - want)) < 1e-10 * np.max(np.abs(want))


def test_ghep_filter_keeps_exact_eigenpairs():
    """Exact generalised eigenpairs make the residual H X - M X Lam vanish, so the
    filter returns each column scaled (by Lam_Y), whatever D is."""
    import scipy.linalg as sl
    rng = np.random.default_rng(7)
    H, _, _ = _sym(40, 11)
    B = rng.standard_normal((40, 40))
    M = B @ B.T / 40 + np.eye(40)
    ev, V = sl.eigh(H, M)
    X, lam = V[:, :4], ev[:4]
    D = np.diag(M).copy()
    out = chfsi.filter_rchfsi_ghep(lambda Z: H @ Z, lambda Z: M @ Z, 1.0 / D, X, lam, 8, ev[0] - 0.5, ev[6], ev[-1] * 1.01)
    for j in range(4):
        a = out[:, j] @ X[:, j] / (X[:, j] @ X[:, j])
        assert np.linalg.norm(out[:, j] - a * X[:, j]) < 1e-9 * np.linalg.norm(out[:, j])


def test_rchfsi_ghep_converges_to_generalised_eigenvalues_of_fe_operator():
    """The lowest eigenvalues of H u = eps M u (eq. FEeigen) with the consistent
    mass, against scipy's dense generalised eigensolver."""
    import scipy.linalg as sl
    wl = Workload("eigg", L=9.0, n=3, p=3, nq=4, n_v=12, jitter=0.1, gga=True, n_atoms=2, seed=22)
    P = Problem(wl)
    H = P.assemble("H").toarray()
    M = P.assemble("M").toarray()
    want = sl.eigh(0.5 * (H + H.T), 0.5 * (M + M.T), eigvals_only=True)[:8]
    X0 = trial_vectors(wl, n_v=12)
    lam, X, res = chfsi.rchfsi_ghep(lambda V: H @ V, lambda V: M @ V, 1.0 / P.lumped_mass(), X0, degree=12,
                                    n_iter=60, tol=1e-10)
    np.testing.assert_allclose(lam[:8], want, atol=1e-8)
    assert np.max(res[:8]) < 1e-7
