"""Rayleigh-Ritz (Algorithm 3) and the Lanczos bound behind the C interface, against the oracle.

* fe_ks_lanczos_bound: the k Lanczos coefficients and the bound
  theta_max(T_k) + |beta_k| equal the oracle's recurrence on the dense
  Hs = D^{-1/2} H D^{-1/2} from the same start vector.  Tolerance 1e-12 of
  max |alpha|: perturbing Hs entry-wise at the FP64 rounding level (1e-15 |Hs|)
  moves the ten coefficients of this workload by at most 2e-15 of max |alpha|.
* fe_ks_rayleigh_ritz (FP64 with library GEMMs, and pairs of floats with the
  library's own kernels): the Ritz values equal the oracle's (dense generalised
  eigensolve of the projected pencil) within 1e-12 of max |lam|; what is not
  unique (the eigenvector basis) is checked for validity: X^T X = I, X^T Hs X =
  diag(lam), and each returned vector of a simple Ritz value is parallel to the
  oracle's.  The same for the generalised pair (H, M) with a mass context.
* A block with two nearly parallel columns takes the shifted CholeskyQR3 path
  and still returns an orthonormal Ritz basis whose values match a Householder
  QR reference.
"""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from synth.host_problem import HostProblem, mass_problem
from oracle import chfsi as ochfsi
from oracle.operator import Problem
from synth import Workload, trial_vectors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WL = Workload("eig", L=6.0, n=2, p=8, nq=9, n_v=16, gga=True, n_atoms=2, seed=4321)


@pytest.fixture(scope="module")
def dense():
    P = Problem(WL)
    H = P.assemble("H").toarray()
    H = 0.5 * (H + H.T)
    M = P.assemble("M").toarray()
    M = 0.5 * (M + M.T)
    s = 1.0 / np.sqrt(P.lumped_mass())
    Hs = s[:, None] * H * s[None, :]
    return P, H, M, 0.5 * (Hs + Hs.T)


@pytest.fixture(scope="module")
def gpu():
    hp = HostProblem(WL)
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, WL.n_v, torch.cuda.current_stream().cuda_stream)
    yield hp, ctx
    fk.fe_ks_destroy(ctx)


def _work(nb):
    buf = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    off = (-buf.data_ptr()) % 256
    return buf, buf[off:off + nb]


@pytest.mark.parametrize("precision", [fk.FE_KS_F64, fk.FE_KS_F64E])
def test_lanczos_bound_matches_oracle(dense, gpu, precision):
    P, H, M, Hs = dense
    hp, ctx = gpu
    v0 = np.random.default_rng(11).standard_normal(hp.m)
    alphas, betas, bound = ochfsi.lanczos_coefficients(lambda V: Hs @ V, v0, 10)
    nb = fk.fe_ks_lanczos_bound_workspace(ctx, 10)
    _, work = _work(nb)
    lmax, a, b = fk.fe_ks_lanczos_bound(ctx, torch.from_numpy(v0).cuda(), 10, precision, work, nb)
    scale = np.max(np.abs(alphas))
    assert len(a) == 10
    assert np.max(np.abs(np.array(a) - alphas)) <= 1e-12 * scale
    assert np.max(np.abs(np.array(b) - betas)) <= 1e-12 * scale
    assert abs(lmax - bound) <= 1e-12 * scale
    assert lmax >= np.linalg.eigvalsh(Hs)[-1] - 1e-9      # it is an upper bound here


def _check_ritz(X, lam, lam_ref, X_ref, op, metric):
    scale = np.max(np.abs(lam_ref))
    assert np.max(np.abs(lam - lam_ref)) <= 1e-12 * scale, np.max(np.abs(lam - lam_ref))
    n = X.shape[1]
    G = X.T @ metric(X)
    assert np.max(np.abs(G - np.eye(n))) <= 1e-12
    A = X.T @ op(X)
    assert np.max(np.abs(A - np.diag(lam))) <= 1e-12 * scale
    gaps = np.abs(lam_ref[:, None] - lam_ref[None, :]) + np.eye(n) * 1e300
    for j in range(n):
        if gaps[j].min() > 1e-6 * scale:                 # simple Ritz value: the vector is unique up to sign
            c = abs(X[:, j] @ metric(X_ref[:, j:j + 1])[:, 0])
            assert c >= 1.0 - 1e-9, (j, c)


@pytest.mark.parametrize("precision", [fk.FE_KS_F64, fk.FE_KS_F64E])
def test_rayleigh_ritz_matches_oracle(dense, gpu, precision):
    P, H, M, Hs = dense
    hp, ctx = gpu
    Y = trial_vectors(WL)
    lam_ref, X_ref = ochfsi.rayleigh_ritz(lambda V: Hs @ V, Y)
    X_ref = X_ref / np.sqrt(np.sum(X_ref * X_ref, axis=0))[None, :]
    nb = fk.fe_ks_rayleigh_ritz_workspace(ctx, WL.n_v, precision)
    _, work = _work(nb)
    Xd = torch.from_numpy(Y.copy()).cuda()
    lam = torch.empty(WL.n_v, dtype=torch.float64, device="cuda")
    path = fk.fe_ks_rayleigh_ritz(ctx, Xd, lam, WL.n_v, precision, work, nb)
    torch.cuda.synchronize()
    assert path == 0
    _check_ritz(Xd.cpu().numpy(), lam.cpu().numpy(), lam_ref, X_ref, lambda V: Hs @ V, lambda V: V)


def test_rayleigh_ritz_generalised_matches_oracle(dense, gpu):
    P, H, M, Hs = dense
    hp, ctx = gpu
    hm = mass_problem(WL)
    mctx = fk.fe_ks_setup(hm.struct, fk.TERM_L, WL.n_v, torch.cuda.current_stream().cuda_stream)
    try:
        Y = trial_vectors(WL, seed_purpose=7)
        lam_ref, X_ref = ochfsi.rayleigh_ritz_ghep(lambda V: H @ V, lambda V: M @ V, Y)
        nb = fk.fe_ks_rayleigh_ritz_workspace(ctx, WL.n_v, fk.FE_KS_F64E)
        _, work = _work(nb)
        Xd = torch.from_numpy(Y.copy()).cuda()
        lam = torch.empty(WL.n_v, dtype=torch.float64, device="cuda")
        fk.fe_ks_rayleigh_ritz(ctx, Xd, lam, WL.n_v, fk.FE_KS_F64E, work, nb, mass=mctx)
        torch.cuda.synchronize()
        _check_ritz(Xd.cpu().numpy(), lam.cpu().numpy(), lam_ref, X_ref, lambda V: H @ V, lambda V: M @ V)
    finally:
        fk.fe_ks_destroy(mctx)


@pytest.mark.parametrize("precision", [fk.FE_KS_F64, fk.FE_KS_F64E])
def test_rayleigh_ritz_nearly_dependent_block_takes_cholesky_qr(dense, gpu, precision):
    P, H, M, Hs = dense
    hp, ctx = gpu
    rng = np.random.default_rng(5)
    Y = trial_vectors(WL)
    Y[:, 1] = Y[:, 0] + 1e-7 * rng.standard_normal(hp.m)     # pivot of the scaled Gram matrix ~1e-14
    Q, _ = np.linalg.qr(Y)                                     # Householder reference basis
    lam_ref = np.linalg.eigvalsh(Q.T @ Hs @ Q)
    nb = fk.fe_ks_rayleigh_ritz_workspace(ctx, WL.n_v, precision)
    _, work = _work(nb)
    Xd = torch.from_numpy(Y).cuda()
    lam = torch.empty(WL.n_v, dtype=torch.float64, device="cuda")
    path = fk.fe_ks_rayleigh_ritz(ctx, Xd, lam, WL.n_v, precision, work, nb)
    torch.cuda.synchronize()
    assert path == 1
    X, lam = Xd.cpu().numpy(), lam.cpu().numpy()
    scale = np.max(np.abs(lam_ref))
    # the near-dependent direction is known to ~1e-16 / 1e-7 relative, so the values to ~1e-9
    assert np.max(np.abs(lam - lam_ref)) <= 1e-7 * scale
    assert np.max(np.abs(X.T @ X - np.eye(WL.n_v))) <= 1e-12
    assert np.max(np.abs(X.T @ Hs @ X - np.diag(lam))) <= 1e-11 * scale


def test_rayleigh_ritz_arguments(gpu):
    hp, ctx = gpu
    nb = fk.fe_ks_rayleigh_ritz_workspace(ctx, WL.n_v, fk.FE_KS_F64E)
    _, work = _work(nb)
    X = torch.zeros((hp.m, WL.n_v), dtype=torch.float64, device="cuda")
    lam = torch.empty(WL.n_v, dtype=torch.float64, device="cuda")
    with pytest.raises(fk.FeKsError, match="workspace"):
        fk.fe_ks_rayleigh_ritz(ctx, X, lam, WL.n_v, fk.FE_KS_F64E, work, nb - 256)
    with pytest.raises(fk.FeKsError, match="precision"):
        fk.fe_ks_rayleigh_ritz(ctx, X, lam, WL.n_v, fk.FE_KS_F32, work, nb)
    with pytest.raises(fk.FeKsError, match="rank-deficient|Cholesky"):
        fk.fe_ks_rayleigh_ritz(ctx, X, lam, WL.n_v, fk.FE_KS_F64E, work, nb)   # X = 0


def test_rayleigh_ritz_refuses_complex():
    wl = Workload("eigc", L=6.0, n=2, p=4, nq=5, n_v=4, kfrac=(0.3, 0.0, 0.0), complex=True, seed=7)
    hp = HostProblem(wl)
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(fk.FeKsError, match="real operators"):
            fk.fe_ks_rayleigh_ritz_workspace(ctx, wl.n_v, fk.FE_KS_F64)
    finally:
        fk.fe_ks_destroy(ctx)
