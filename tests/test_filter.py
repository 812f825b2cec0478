"""GPU R-ChFSI filter (Algorithm 4) and eigensolver (Algorithm 3) against the oracle.

* One filter pass on the GPU (FP64 and FP32 recurrence) equals the oracle's
  Algorithm 4 on the same block with the same bounds (FP64 and pairs of
  floats: 1e-12 relative, per column and element-wise; FP32: the recurrence
  error stays relative to the residual part R).
* Converged eigenvalues of the all-FP64 and the mixed (FP32, BF16 or FP16
  recurrence) eigensolver match the dense eigenvalues of
  Hs = D^{-1/2} H D^{-1/2} from the oracle within 1e-8 Ha (the lowest
  N_v - 6 of N_v, the rest being the usual buffer of the subspace iteration).
"""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from synth.host_problem import HostProblem
from oracle import chfsi as ochfsi
from oracle.operator import Problem
from synth import Workload, trial_vectors
from gpu_util import parity_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WL = Workload("eig", L=6.0, n=2, p=8, nq=9, n_v=16, gga=True, n_atoms=2, seed=4321)


@pytest.fixture(scope="module")
def dense():
    P = Problem(WL)
    H = P.assemble("H").toarray()
    s = 1.0 / np.sqrt(P.lumped_mass())
    Hs = s[:, None] * H * s[None, :]
    Hs = 0.5 * (Hs + Hs.T)
    return P, Hs, np.linalg.eigvalsh(Hs)


@pytest.fixture(scope="module")
def gpu():
    hp = HostProblem(WL)
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, WL.n_v, torch.cuda.current_stream().cuda_stream)
    yield hp, ctx
    fk.fe_ks_destroy(ctx)


@pytest.mark.parametrize("precision,tol,resid", [(fk.FE_KS_F64, 1e-12, fk.FE_KS_F64),
                                                (fk.FE_KS_F64E, 1e-12, fk.FE_KS_F64E),
                                                (fk.FE_KS_F32, 2e-4, fk.FE_KS_F64),
                                                (fk.FE_KS_F32, 2e-4, fk.FE_KS_F64E)])
def test_one_filter_pass_matches_oracle(dense, gpu, precision, tol, resid):
    P, Hs, ev = dense
    hp, ctx = gpu
    X = np.linalg.qr(trial_vectors(WL))[0]
    lam = np.sort(np.random.default_rng(3).uniform(ev[0], ev[8], WL.n_v))
    lmin, lT, lmax = ev[0] - 0.1, ev[12], ev[-1] * 1.01
    want = ochfsi.filter_rchfsi(lambda V: Hs @ V, X, lam, 12, lmin, lT, lmax)
    Xd = torch.from_numpy(X).cuda()
    lamd = torch.from_numpy(lam).cuda()
    nb = fk.fe_ks_cheb_filter_workspace(ctx, WL.n_v, precision)
    work = torch.empty(nb, dtype=torch.uint8, device="cuda")
    fk.fe_ks_cheb_filter(ctx, Xd, lamd, WL.n_v, 12, lmin, lT, lmax, precision, work, nb, residual_precision=resid)
    torch.cuda.synchronize()
    got = Xd.cpu().numpy()
    err = parity_err(got, want)
    assert err < tol, err


@pytest.mark.parametrize("precision,exact,pairs", [(fk.FE_KS_F64, fk.FE_KS_F64, False),
                                                   (fk.FE_KS_F32, fk.FE_KS_F64, False),
                                                   (fk.FE_KS_F32, fk.FE_KS_F64E, True),
                                                   (fk.FE_KS_BF16, fk.FE_KS_F64E, True),
                                                   (fk.FE_KS_F16, fk.FE_KS_F64E, True),
                                                   (fk.FE_KS_BF16X2, fk.FE_KS_F64E, True)])
def test_eigensolver_converges_to_oracle_eigenvalues(dense, gpu, precision, exact, pairs):
    """Converged eigenvalues within 1e-8 Ha of the dense oracle for every recurrence
    arithmetic, the 16-bit tensor-core ones included: the residual the filter
    starts from and the Rayleigh-Ritz step stay FP64-accurate, so the
    recurrence's rounding only slows convergence, it does not bias the limit."""
    from paper_2512_08571_gb300.chfsi import RChFSI
    P, Hs, ev = dense
    hp, ctx = gpu
    n_conv = WL.n_v - 6
    solver = RChFSI(ctx, hp.m, WL.n_v, False, degree=20, precision=precision, exact=exact, gemm_pairs=pairs)
    lmax = solver.lanczos_upper_bound()
    assert lmax >= ev[-1] - 1e-9
    X0 = torch.from_numpy(trial_vectors(WL)).cuda()
    n_iter = 60 if precision in (fk.FE_KS_F64, fk.FE_KS_F32) else 100
    lam, X, res, its = solver.run(X0, n_iter=n_iter, tol=1e-9, n_check=n_conv)
    lam = lam.cpu().numpy()
    assert float(res[:n_conv].max()) < 1e-9, (its, res[:n_conv].max().item())
    np.testing.assert_allclose(lam[:n_conv], ev[:n_conv], atol=1e-8, rtol=0)


def test_filter_rejects_bad_bounds(gpu):
    hp, ctx = gpu
    X = torch.zeros((hp.m, WL.n_v), dtype=torch.float64, device="cuda")
    lam = torch.zeros(WL.n_v, dtype=torch.float64, device="cuda")
    nb = fk.fe_ks_cheb_filter_workspace(ctx, WL.n_v, fk.FE_KS_F64)
    work = torch.empty(nb, dtype=torch.uint8, device="cuda")
    with pytest.raises(fk.FeKsError, match="lam_min"):
        fk.fe_ks_cheb_filter(ctx, X, lam, WL.n_v, 5, 1.0, 0.5, 2.0, fk.FE_KS_F64, work, nb)
    with pytest.raises(fk.FeKsError, match="workspace"):
        fk.fe_ks_cheb_filter(ctx, X, lam, WL.n_v, 5, 0.0, 0.5, 2.0, fk.FE_KS_F64, work, nb - 8)


# ---- generalised problem H X = M X Lam with the consistent mass (eq. FEeigen)

@pytest.fixture(scope="module")
def dense_ghep():
    import scipy.linalg as sl
    P = Problem(WL)
    H = P.assemble("H").toarray()
    M = P.assemble("M").toarray()
    H, M = 0.5 * (H + H.T), 0.5 * (M + M.T)
    return P, H, M, 1.0 / P.lumped_mass(), sl.eigh(H, M, eigvals_only=True)


@pytest.fixture(scope="module")
def gpu_mass():
    from synth.host_problem import mass_problem
    hp = mass_problem(WL)
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_L, WL.n_v, torch.cuda.current_stream().cuda_stream)
    yield hp, ctx
    fk.fe_ks_destroy(ctx)


def test_mass_context_applies_the_consistent_mass(dense_ghep, gpu_mass):
    P, H, M, Dinv, ev = dense_ghep
    hp, mctx = gpu_mass
    X = trial_vectors(WL)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.empty_like(Xd)
    fk.fe_ks_apply(mctx, Xd, Yd, WL.n_v, fk.FE_KS_F64)
    want = M @ X
    err = parity_err(Yd.cpu().numpy(), want)
    assert err < 1e-12, err


@pytest.mark.parametrize("precision,tol,resid", [(fk.FE_KS_F64, 1e-12, fk.FE_KS_F64),
                                                (fk.FE_KS_F32, 2e-4, fk.FE_KS_F64E)])
def test_one_ghep_filter_pass_matches_oracle(dense_ghep, gpu, gpu_mass, precision, tol, resid):
    """fe_ks_cheb_filter_ghep against the oracle's Algorithm 4 for the generalised problem."""
    P, H, M, Dinv, ev = dense_ghep
    hp, ctx = gpu
    _, mctx = gpu_mass
    X = np.linalg.qr(trial_vectors(WL))[0]
    lam = np.sort(np.random.default_rng(4).uniform(ev[0], ev[8], WL.n_v))
    s = np.sqrt(Dinv)
    lmax = np.linalg.eigvalsh(s[:, None] * H * s[None, :])[-1] * 1.01
    lmin, lT = ev[0] - 0.1, ev[12]
    want = ochfsi.filter_rchfsi_ghep(lambda V: H @ V, lambda V: M @ V, Dinv, X, lam, 12, lmin, lT, lmax)
    Xd = torch.from_numpy(X).cuda()
    lamd = torch.from_numpy(lam).cuda()
    nb = fk.fe_ks_cheb_filter_workspace(ctx, WL.n_v, precision)
    work = torch.empty(nb, dtype=torch.uint8, device="cuda")
    fk.fe_ks_cheb_filter_ghep(ctx, mctx, Xd, lamd, WL.n_v, 12, lmin, lT, lmax, precision, work, nb,
                              residual_precision=resid)
    torch.cuda.synchronize()
    got = Xd.cpu().numpy()
    err = parity_err(got, want)
    assert err < tol, err


@pytest.mark.parametrize("precision,exact,pairs", [(fk.FE_KS_F64, fk.FE_KS_F64, False),
                                                   (fk.FE_KS_F32, fk.FE_KS_F64E, True),
                                                   (fk.FE_KS_BF16, fk.FE_KS_F64E, True)])
def test_ghep_eigensolver_converges_to_generalised_eigenvalues(dense_ghep, gpu, gpu_mass, precision, exact, pairs):
    """Algorithm 3 with the consistent mass: converged eigenvalues within 1e-8 Ha of
    scipy's dense generalised eigensolver on the oracle's assembled H and M."""
    from paper_2512_08571_gb300.chfsi import RChFSI
    P, H, M, Dinv, ev = dense_ghep
    hp, ctx = gpu
    _, mctx = gpu_mass
    n_conv = WL.n_v - 6
    solver = RChFSI(ctx, hp.m, WL.n_v, False, degree=20, precision=precision, exact=exact, gemm_pairs=pairs,
                    mass_ctx=mctx)
    X0 = torch.from_numpy(trial_vectors(WL)).cuda()
    lam, X, res, its = solver.run(X0, n_iter=100, tol=1e-9, n_check=n_conv)
    lam = lam.cpu().numpy()
    assert float(res[:n_conv].max()) < 1e-9, (its, res[:n_conv].max().item())
    np.testing.assert_allclose(lam[:n_conv], ev[:n_conv], atol=1e-8, rtol=0)
