"""GPU parity of the 5th-generation tensor-core cell kernel (tcgen05; tile
configuration 0 of FE_KS_BF16 and FE_KS_F16 for real operators with n_q = n_p)
against the FP64 oracle, beside the warp-level MMA kernel (configuration 1).

The tcgen05 kernel runs Algorithm 2 as four products per cell and 8-vector
tile: the x-y plane operators N(x)N, D(x)N, N(x)D on the in-plane nodes, the z
sweep, the quadrature-point step in FP32, the transposed z sweep and the
transposed plane product.  A value reaches the output through four roundings
of data (the gathered X, the plane products, the quadrature-point values, the
transposed z sweep) and the rounded entries of two operator matrices (a plane
entry N[a'][a] N[b'][b] is rounded once), fewer than the warp-level kernel's
six and three, so the tolerance derived for that kernel, 8 u per column and
per element (u = 2^-8 BF16, 2^-11 FP16), covers it.
"""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from synth.host_problem import HostProblem
from oracle.operator import Problem
from synth import CONFIGS, Workload, trial_vectors
from gpu_util import gpu_apply, parity_err, round_input, torch_dtype

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = {fk.FE_KS_BF16: 2.0 ** -8, fk.FE_KS_F16: 2.0 ** -11}
TOL = {prec: 8 * u for prec, u in U.items()}
PRECS = [fk.FE_KS_BF16, fk.FE_KS_F16]

SMALL = {
    "C1": CONFIGS["C1"],
    "C2s": CONFIGS["C2"].scaled(n=6, n_v=7),
    "C4s": CONFIGS["C4"].scaled(n=4, n_v=5, n_atoms=6),
    "C4v": CONFIGS["C4"].scaled(n=4, n_v=16, n_atoms=6),
    # many column tiles split over work units, ragged last tile
    "C4w": CONFIGS["C4"].scaled(n=3, n_v=37, n_atoms=3),
}


@pytest.fixture(scope="module")
def cases():
    return {k: (wl, HostProblem(wl), Problem(wl), trial_vectors(wl)) for k, wl in SMALL.items()}


def apply_status(hp, X, prec, config, scaled=False, terms=fk.TERM_ALL):
    """Apply with a given configuration; also return the device status word."""
    n_v = X.shape[1]
    ctx = fk.fe_ks_setup(hp.struct, terms, n_v, torch.cuda.current_stream().cuda_stream)
    try:
        fk.fe_ks_set_config(ctx, prec, config)
        Xd = torch.from_numpy(np.ascontiguousarray(X)).to("cuda").to(torch_dtype(prec, hp.complex))
        Yd = torch.full_like(Xd, float("nan"))
        (fk.fe_ks_apply_scaled if scaled else fk.fe_ks_apply)(ctx, Xd, Yd, n_v, prec)
        status = fk.fe_ks_device_status(ctx)
        return Yd.cpu().numpy(), status
    finally:
        fk.fe_ks_destroy(ctx)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("config", [0, 1, 2, 3])
@pytest.mark.parametrize("key", list(SMALL))
def test_both_kernels_match_oracle(cases, key, config, prec):
    """Configurations 0, 2, 3: the tcgen05 kernel with its pipelines staggered after the
    first plane product, not at all, after the first quadrature-point step; 1: the
    warp-level one."""
    wl, hp, P, X = cases[key]
    Xin = round_input(X, prec)
    Y, status = apply_status(hp, Xin, prec, config)
    assert status == 0
    err = parity_err(Y, P.apply(Xin))
    print(f"{key}: config {config} prec {prec} err {err:.3e}")
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
def test_tcgen05_every_degree(p, prec):
    """n = 2..9 points per direction: one, two or six GEMM2 row tiles, one or two
    GEMM1 tiles, K and N paddings of every kind; all terms with atoms."""
    wl = Workload(f"tc5deg{p}", L=4.0 + p, n=2 if p > 2 else 3, p=p, nq=p + 1, n_v=11, jitter=0.08, gga=True,
                  n_atoms=3, seed=300 + p)
    hp, P = HostProblem(wl), Problem(wl)
    Xin = round_input(trial_vectors(wl), prec)
    Y, status = apply_status(hp, Xin, prec, 0)
    assert status == 0
    err = parity_err(Y, P.apply(Xin))
    assert err <= TOL[prec], (p, err)


@pytest.mark.parametrize("prec", PRECS)
def test_tcgen05_scaled_matches_oracle(cases, prec):
    wl, hp, P, X = cases["C4v"]
    Xin = round_input(X, prec)
    Y, status = apply_status(hp, Xin, prec, 0, scaled=True)
    assert status == 0
    s = 1.0 / np.sqrt(P.lumped_mass())
    err = parity_err(Y, s[:, None] * P.apply(s[:, None] * Xin))
    assert err <= TOL[prec], err


def test_tcgen05_term_subsets(cases):
    """Kinetic term alone (the G slots of the quadrature-point step), all local
    terms (V^L and the V^G rows and columns), and the nonlocal term as the
    difference of the two (the FP32 expansion F Delta P on the accumulators)."""
    wl, hp, P, X = cases["C4s"]
    prec = fk.FE_KS_BF16
    Xin = round_input(X, prec)
    zero = lambda x: np.zeros(np.asarray(x).shape[:-1])
    P_T = Problem(wl, vloc=zero, vgga=None, with_atoms=False)
    P_loc = Problem(wl, with_atoms=False)
    Y_T, st1 = apply_status(hp, Xin, prec, 0, terms=fk.TERM_T)
    Y_loc, st2 = apply_status(hp, Xin, prec, 0, terms=fk.TERM_ALL & ~fk.TERM_NL)
    Y_all, st3 = apply_status(hp, Xin, prec, 0)
    assert st1 == st2 == st3 == 0
    assert parity_err(Y_T, P_T.apply(Xin)) <= TOL[prec]
    assert parity_err(Y_loc, P_loc.apply(Xin)) <= TOL[prec]
    ref_nl = P.apply(Xin) - P_loc.apply(Xin)
    # the local parts of the two runs agree to FP32 rounding of the accumulators;
    # the expansion itself is FP32 here (F and Delta-scaled projections unrounded)
    assert parity_err(Y_all - Y_loc, ref_nl) <= 1e-2


def test_tcgen05_bitwise_deterministic(cases):
    wl, hp, P, X = cases["C4w"]
    Xin = round_input(X, fk.FE_KS_BF16)
    Ys = gpu_apply(hp, Xin, fk.FE_KS_BF16, repeat=2, config=0)
    assert np.array_equal(Ys[0], Ys[1])


@pytest.mark.parametrize("scale", [1e-7, 1e5])
def test_tcgen05_f16_column_scaling_range(cases, scale):
    wl, hp, P, X = cases["C4v"]
    Xin = round_input(X * scale, fk.FE_KS_F16)
    Y, status = apply_status(hp, Xin, fk.FE_KS_F16, 0)
    assert status == 0 and np.all(np.isfinite(Y))
    assert parity_err(Y, P.apply(Xin)) <= TOL[fk.FE_KS_F16]


def test_configuration_interface(cases):
    """Real n_q = n_p contexts: four BF16/FP16 configurations, tcgen05 the default,
    the tuner times both; complex contexts have the warp-level kernel only."""
    wl, hp, P, X = cases["C4s"]
    n_v = X.shape[1]
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, n_v, torch.cuda.current_stream().cuda_stream)
    try:
        assert fk.fe_ks_get_config(ctx, fk.FE_KS_BF16) == 0
        assert fk.fe_ks_get_config(ctx, fk.FE_KS_F16) == 0
        with pytest.raises(fk.FeKsError):
            fk.fe_ks_set_config(ctx, fk.FE_KS_BF16, 4)
        Xd = torch.from_numpy(round_input(X, fk.FE_KS_BF16)).to("cuda").float()
        Yd = torch.empty_like(Xd)
        best, ms = fk.fe_ks_tune(ctx, Xd, Yd, n_v, fk.FE_KS_BF16, reps=1)
        assert best in (0, 1, 2, 3) and all(m > 0 for m in ms[:4]) and all(m == -1.0 for m in ms[4:])
        assert fk.fe_ks_get_config(ctx, fk.FE_KS_BF16) == best
    finally:
        fk.fe_ks_destroy(ctx)
    wlc = CONFIGS["C3"].scaled(n=3, n_v=2, n_atoms=2)
    hpc = HostProblem(wlc)
    ctx = fk.fe_ks_setup(hpc.struct, fk.TERM_ALL, 2, torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(fk.FeKsError):
            fk.fe_ks_set_config(ctx, fk.FE_KS_BF16, 1)
        assert fk.fe_ks_device_status(ctx) == 0
    finally:
        fk.fe_ks_destroy(ctx)


def test_expired_wait_reports_status_and_context_recovers(cases):
    """Failure path without a GPU fault: with the host-side injection each pipeline's first
    plane product is never issued or committed, so its bounded waits (short limit) run
    out; the kernel stops cleanly, fe_ks_device_status reports it, and the next
    application on the same context is correct."""
    wl, hp, P, X = cases["C4v"]
    prec = fk.FE_KS_BF16
    Xin = round_input(X, prec)
    n_v = X.shape[1]
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, n_v, torch.cuda.current_stream().cuda_stream)
    try:
        Xd = torch.from_numpy(np.ascontiguousarray(Xin)).to("cuda").float()
        Yd = torch.empty_like(Xd)
        fk.fe_ks_inject_fault(ctx, 1)
        fk.fe_ks_apply(ctx, Xd, Yd, n_v, prec)
        assert fk.fe_ks_device_status(ctx) == 1
        fk.fe_ks_inject_fault(ctx, 0)
        Yd.fill_(float("nan"))
        fk.fe_ks_apply(ctx, Xd, Yd, n_v, prec)
        assert fk.fe_ks_device_status(ctx) == 0
        assert parity_err(Yd.cpu().numpy(), P.apply(Xin)) <= TOL[prec]
        with pytest.raises(fk.FeKsError, match="ERR_ARG"):
            fk.fe_ks_inject_fault(ctx, 2)
    finally:
        fk.fe_ks_destroy(ctx)
