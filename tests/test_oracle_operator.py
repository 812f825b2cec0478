"""Pins of the oracle's operator (Sec. 2.2 eq. Hloc, eq. Vloc, eq. Vnonloc; Sec. 3.1 eq. HX).

Each test checks the oracle against something other than itself: exact
polynomial integrals (sympy), closed forms (plane-wave eigenvalues
|G+k|^2/2, volume, projector moments by 1D radial quadrature), invariants
(null space, Hermiticity, H(-k) = conj H(k), constant shift, translation).
"""
import math

import numpy as np
import pytest

from oracle.operator import Problem
from synth import CONFIGS, Workload, trial_vectors, projector_values, PROJ_RC, PROJ_SIGMA


def _zero(x):
    return np.zeros(np.asarray(x).shape[:-1])


def _single_cell(A, b, p, kpt=(0, 0, 0), vloc=_zero, vgga=None, nq=None):
    """One affine cell x = A xi + b with its own (non-periodic) DoFs."""
    verts = np.zeros((1, 8, 3))
    for v in range(8):
        xi = np.array([2 * (v & 1) - 1, 2 * ((v >> 1) & 1) - 1, 2 * ((v >> 2) & 1) - 1], float)
        verts[0, v] = A @ xi + b
    wl = Workload("cell", L=100.0, n=1, p=p, nq=p + 1 if nq is None else nq, n_v=1)
    dofs = np.arange((p + 1) ** 3)[None, :]
    return Problem(wl, verts=verts, dofs=dofs, vloc=vloc, vgga=vgga, kpt=kpt)


def test_polynomial_exactness_affine_cell():
    """u^T M v, u^T T v, u^T L v, u^T G v, u^T K v equal exact integrals (sympy)."""
    sp = pytest.importorskip("sympy")
    rng = np.random.default_rng(7)
    p = 3
    A = np.array([[1.3, 0.2, -0.1], [0.1, 0.9, 0.3], [-0.2, 0.15, 1.1]])
    b = np.array([0.5, -0.25, 1.0])
    X1, X2, X3 = sp.symbols("x1 x2 x3")
    xs = (X1, X2, X3)

    def rand_poly(deg):
        expr = 0
        for i in range(deg + 1):
            for j in range(deg + 1 - i):
                for k in range(deg + 1 - i - j):
                    expr += sp.Rational(int(rng.integers(-9, 10)), 7) * X1 ** i * X2 ** j * X3 ** k
        return expr

    u, v = rand_poly(p), rand_poly(p)
    vl_c = [sp.Rational(3, 2), sp.Rational(-1, 3), sp.Rational(2, 5), sp.Rational(1, 4)]
    VL = vl_c[0] + vl_c[1] * X1 + vl_c[2] * X2 + vl_c[3] * X3
    VG = [sp.Rational(1, 3) + sp.Rational(1, 5) * X2, sp.Rational(-2, 7) + sp.Rational(1, 3) * X3,
          sp.Rational(1, 2) - sp.Rational(1, 4) * X1]
    kv = [sp.Rational(3, 10), sp.Rational(-1, 5), sp.Rational(7, 10)]

    # exact integrals over the parallelepiped via xi-substitution
    E1, E2, E3 = sp.symbols("e1 e2 e3")
    Ar = [[sp.nsimplify(A[i, j]) for j in range(3)] for i in range(3)]
    br = [sp.nsimplify(b[i]) for i in range(3)]
    sub = {xs[i]: sum(Ar[i][j] * (E1, E2, E3)[j] for j in range(3)) + br[i] for i in range(3)}
    detA = sp.Matrix(Ar).det()

    def integ(f):
        g = sp.expand(f.subs(sub, simultaneous=True))
        return float(abs(detA) * sp.integrate(g, (E1, -1, 1), (E2, -1, 1), (E3, -1, 1)))

    grad = lambda f: [sp.diff(f, x) for x in xs]
    gu, gv = grad(u), grad(v)
    exact = {
        "M": integ(u * v),
        "T": integ(sp.Rational(1, 2) * sum(gu[i] * gv[i] for i in range(3))),
        "L": integ(VL * u * v),
        "G": integ(sum(VG[i] * (gu[i] * v + u * gv[i]) for i in range(3))),
        "K": integ(u * sum(kv[i] * gv[i] for i in range(3))),
    }
    fu = sp.lambdify(xs, u, "numpy")
    fv = sp.lambdify(xs, v, "numpy")
    vlf = lambda x: (float(vl_c[0]) + float(vl_c[1]) * x[..., 0] + float(vl_c[2]) * x[..., 1]
                     + float(vl_c[3]) * x[..., 2])
    vgf = lambda x: np.stack([1 / 3 + 0.2 * x[..., 1], -2 / 7 + x[..., 2] / 3, 0.5 - 0.25 * x[..., 0]], -1)
    kvec = np.array([float(k) for k in kv])
    P = _single_cell(A, b, p, kpt=kvec, vloc=vlf, vgga=vgf)
    xn = P.node_coords()[0]
    uu = fu(xn[:, 0], xn[:, 1], xn[:, 2]) * np.ones(len(xn))
    vv = fv(xn[:, 0], xn[:, 1], xn[:, 2]) * np.ones(len(xn))
    got = {
        "M": uu @ P.mass_matrix(0) @ vv,
        "T": np.real(uu @ P.cell_matrix(0, terms=("T",)) @ vv),
        "L": np.real(uu @ P.cell_matrix(0, terms=("L",)) @ vv) - 0.5 * kvec @ kvec * exact["M"],
        "G": np.real(uu @ P.cell_matrix(0, terms=("G",)) @ vv),
        "K": -np.imag(uu @ P.cell_matrix(0, terms=("K",)) @ vv),   # H_K = -i K
    }
    for key in exact:
        assert abs(got[key] - exact[key]) <= 1e-11 * max(1.0, abs(exact[key])), (key, got[key], exact[key])
    # the K orientation: u^T K v != v^T K u for these fields
    assert abs(exact["K"] - integ(v * sum(kv[i] * gu[i] for i in range(3)))) > 1e-3


def test_quadrature_order_n_p_plus_2():
    """n_q = n_p + 2 (the paper's default quadrature, Sec. 6) integrates u V v exactly for
    a quartic V_loc (total degree 3 + 3 + 4 = 10 <= 2 n_q - 1 = 11 at p = 3), while the
    n_q = n_p rule (exact to degree 7) does not.  Pins that the oracle's quadrature order
    follows n_q and not the degree."""
    sp = pytest.importorskip("sympy")
    rng = np.random.default_rng(11)
    p = 3
    A = np.array([[1.1, 0.1, 0.0], [-0.2, 0.8, 0.25], [0.05, -0.1, 1.2]])
    b = np.array([0.3, -0.6, 0.2])
    X1, X2, X3 = sp.symbols("x1 x2 x3")
    xs = (X1, X2, X3)

    def rand_poly(deg):
        expr = 0
        for i in range(deg + 1):
            for j in range(deg + 1 - i):
                for k in range(deg + 1 - i - j):
                    expr += sp.Rational(int(rng.integers(-9, 10)), 5) * X1 ** i * X2 ** j * X3 ** k
        return expr

    u, v = rand_poly(p), rand_poly(p)
    VL = 1 + X1 ** 2 * X2 ** 2 - sp.Rational(1, 2) * X3 ** 4 + X1 * X2 * X3
    E1, E2, E3 = sp.symbols("e1 e2 e3")
    Ar = [[sp.nsimplify(A[i, j]) for j in range(3)] for i in range(3)]
    br = [sp.nsimplify(b[i]) for i in range(3)]
    sub = {xs[i]: sum(Ar[i][j] * (E1, E2, E3)[j] for j in range(3)) + br[i] for i in range(3)}
    detA = sp.Matrix(Ar).det()

    def integ(f):
        g = sp.expand(f.subs(sub, simultaneous=True))
        return float(abs(detA) * sp.integrate(g, (E1, -1, 1), (E2, -1, 1), (E3, -1, 1)))

    gu, gv = [sp.diff(u, x) for x in xs], [sp.diff(v, x) for x in xs]
    exact_L = integ(VL * u * v)
    exact_T = integ(sp.Rational(1, 2) * sum(gu[i] * gv[i] for i in range(3)))
    fu, fv, fvl = (sp.lambdify(xs, f, "numpy") for f in (u, v, VL))
    vlf = lambda x: fvl(x[..., 0], x[..., 1], x[..., 2]) * np.ones(x.shape[:-1])
    got = {}
    for nq in (p + 1, p + 3):
        P = _single_cell(A, b, p, vloc=vlf, nq=nq)
        xn = P.node_coords()[0]
        uu = fu(xn[:, 0], xn[:, 1], xn[:, 2]) * np.ones(len(xn))
        vv = fv(xn[:, 0], xn[:, 1], xn[:, 2]) * np.ones(len(xn))
        got[nq] = (np.real(uu @ P.cell_matrix(0, terms=("L",)) @ vv),
                   np.real(uu @ P.cell_matrix(0, terms=("T",)) @ vv))
    assert abs(got[p + 3][0] - exact_L) <= 1e-11 * abs(exact_L)
    assert abs(got[p + 3][1] - exact_T) <= 1e-11 * abs(exact_T)
    assert abs(got[p + 1][1] - exact_T) <= 1e-11 * abs(exact_T)       # T: degree 4 per direction
    assert abs(got[p + 1][0] - exact_L) > 1e-6 * abs(exact_L)          # the low rule misses the quartic


def _periodic(n=3, p=4, L=10.0, jitter=0.0, kfrac=(0, 0, 0), gga=False, n_atoms=0, seed=11, nqx=0):
    return Workload("t", L=L, n=n, p=p, nq=p + 1 + nqx, n_v=4, jitter=jitter, kfrac=kfrac,
                    gga=gga, n_atoms=n_atoms, complex=any(kfrac), seed=seed)


# The identities below hold for any Gauss rule with n_q >= n_p: they are checked for the
# square rule and for n_q = n_p + 2.
@pytest.mark.parametrize("nqx", [0, 2])
def test_volume_and_null_space_jittered(nqx):
    wl = _periodic(n=3, p=3, jitter=0.1, gga=True, nqx=nqx)
    P = Problem(wl, vloc=_zero, vgga=lambda x: np.broadcast_to(np.array([0.3, -0.7, 0.2]), x.shape))
    one = np.ones((P.m, 1))
    Y = np.zeros((P.m, 1))
    M1 = np.zeros((P.m, 1))
    for e in range(P.E):
        d = P.dofs[e]
        Y[d] += np.real(P.cell_matrix(e, terms=("T", "G"))) @ one[d]
        M1[d] += P.mass_matrix(e) @ one[d]
    assert np.max(np.abs(Y)) < 1e-12            # T 1 = 0 and, for constant V^G, G 1 = 0
    assert abs(M1.sum() - wl.L ** 3) < 1e-9 * wl.L ** 3       # 1^T M 1 = volume
    assert abs(P.lumped_mass().sum() - wl.L ** 3) < 1e-9 * wl.L ** 3


@pytest.mark.parametrize("p,jitter", [(1, 0.0), (2, 0.0), (3, 0.1), (4, 0.12), (5, 0.1)])
def test_lumped_mass_is_the_row_sum_of_the_consistent_mass(p, jitter):
    """D_I (GLL weights times det J at the node) equals sum_J M_IJ = int N_I dV wherever the
    GLL rule integrates N_I det J exactly: N_I has degree p per variable, det J of a trilinear
    cell degree <= 2 (0 when the cell is affine), and the (p + 1)-point GLL rule is exact to
    degree 2 p - 1, so affine cells for every p and jittered cells for p >= 3.  Unlike the
    volume check, this holds node by node, so a misplaced weight or det J evaluated at the
    wrong node (an axis swap keeps the sum) fails it."""
    wl = _periodic(n=3, p=p, jitter=jitter)
    P = Problem(wl, vloc=_zero, vgga=None)
    one = np.ones(P.m)
    M1 = np.zeros(P.m)
    for e in range(P.E):
        d = P.dofs[e]
        M1[d] += P.mass_matrix(e) @ one[d]
    D = P.lumped_mass()
    assert np.max(np.abs(D - M1)) <= 1e-13 * np.max(M1)


@pytest.mark.parametrize("nqx", [0, 2])
def test_k_shift_null_space(nqx):
    """V = V^G = 0, no atoms: H(k) 1 = |k|^2/2 M 1."""
    wl = _periodic(n=2, p=3, jitter=0.1, kfrac=(0.25, 0.1, -0.3), nqx=nqx)
    P = Problem(wl, vloc=_zero, vgga=None)
    one = np.ones((P.m, 1))
    Y = P.apply(one)
    M1 = np.zeros((P.m, 1))
    for e in range(P.E):
        M1[P.dofs[e]] += P.mass_matrix(e) @ one[P.dofs[e]]
    k2 = P.kpt @ P.kpt
    np.testing.assert_allclose(Y, 0.5 * k2 * M1, atol=1e-12)


@pytest.mark.parametrize("jitter", [0.0, 0.1])
def test_plane_wave_rayleigh_quotients(jitter):
    """Rayleigh quotients of interpolated plane waves exp(iG.x) approach |G+k|^2/2.

    With the opposite sign of the K term they would approach |G-k|^2/2 instead.
    """
    kfrac = (0.3, 0.0, 0.0)
    errs = []
    for n in (2, 4):
        wl = _periodic(n=n, p=3, jitter=jitter, kfrac=kfrac)
        P = Problem(wl, vloc=_zero, vgga=None)
        xn = P.node_coords()
        X = np.zeros(P.m, dtype=complex)
        G = np.array([2 * math.pi / wl.L, 0.0, 0.0])
        for e in range(P.E):
            X[P.dofs[e]] = np.exp(1j * xn[e] @ G)
        HX = P.apply(X[:, None])[:, 0]
        MX = np.zeros(P.m, dtype=complex)
        for e in range(P.E):
            MX[P.dofs[e]] += P.mass_matrix(e) @ X[P.dofs[e]]
        rq = np.real(np.vdot(X, HX) / np.vdot(X, MX))
        want = 0.5 * np.sum((G + P.kpt) ** 2)
        wrong = 0.5 * np.sum((G - P.kpt) ** 2)
        errs.append(abs(rq - want))
        assert abs(rq - want) < 0.02 * abs(want - wrong)
    assert errs[1] < errs[0] / 8            # converges under refinement (O(h^2p) in theory)


def test_plane_wave_spectrum_k0():
    """Lowest generalized eigenvalues of (T, M) on a periodic box: 0 (x1), (2pi/L)^2/2 (x6), (x12)."""
    import scipy.linalg as sl
    wl = _periodic(n=3, p=4, L=10.0)
    P = Problem(wl, vloc=_zero, vgga=None)
    H = P.assemble("H").toarray()
    M = P.assemble("M").toarray()
    ev = sl.eigh(H, M, eigvals_only=True)[:20]
    g2 = 0.5 * (2 * math.pi / wl.L) ** 2
    np.testing.assert_allclose(ev[0], 0.0, atol=1e-10)
    np.testing.assert_allclose(ev[1:7], g2, rtol=3e-5)            # O(h^2p) discretisation error
    np.testing.assert_allclose(ev[7:19], 2 * g2, rtol=3e-4)
    assert np.ptp(ev[1:7]) < 1e-10 and np.ptp(ev[7:19]) < 1e-9   # exact cubic degeneracy
    assert ev[19] > 2.9 * g2            # next shell |G|^2 = 3 (2 pi / L)^2


@pytest.mark.parametrize("nqx", [0, 2])
def test_constant_shift_affine(nqx):
    wl = _periodic(n=2, p=3, nqx=nqx)
    c = -1.75
    P0 = Problem(wl, vloc=_zero, vgga=None)
    Pc = Problem(wl, vloc=lambda x: np.full(np.asarray(x).shape[:-1], c), vgga=None)
    X = trial_vectors(wl, n_v=3)
    MX = np.zeros_like(X)
    for e in range(P0.E):
        MX[P0.dofs[e]] += P0.mass_matrix(e) @ X[P0.dofs[e]]
    np.testing.assert_allclose(Pc.apply(X) - P0.apply(X), c * MX, atol=1e-12)


def _small_full(complex_=True, jitter=0.1, nqx=0):
    kf = (0.25, 0.1, 0.0) if complex_ else (0, 0, 0)
    return Workload("small", L=9.0, n=3, p=3, nq=4 + nqx, n_v=3, jitter=jitter, kfrac=kf, gga=True,
                    n_atoms=2, complex=complex_, seed=77)


@pytest.mark.parametrize("nqx", [0, 2])
def test_hermiticity_and_conjugate_k(nqx):
    wl = _small_full(True, nqx=nqx)
    P = Problem(wl)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((P.m, 2)) + 1j * rng.standard_normal((P.m, 2))
    Yv = rng.standard_normal((P.m, 2)) + 1j * rng.standard_normal((P.m, 2))
    HX, HY = P.apply(X), P.apply(Yv)
    lhs = X.conj().T @ HY
    rhs = HX.conj().T @ Yv
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(lhs))
    Pm = Problem(wl, kpt=-wl.kpt)
    # H(-k) = conj(H(k)) for real fields: H(-k) X = conj(H(k) conj(X))
    np.testing.assert_allclose(Pm.apply(X), np.conj(P.apply(np.conj(X))), atol=1e-11)


def test_translation_covariance():
    """Shifting V, V^G and atoms by one cell permutes Y (uniform grid, k = 0)."""
    wl = _small_full(False, jitter=0.0)
    P = Problem(wl)
    sh = np.array([wl.h, 0.0, 0.0])
    Ps = Problem(wl, vloc=lambda x: P.vloc(np.asarray(x) - sh),
                 vgga=lambda x: P.vgga(np.asarray(x) - sh), R=P.R + sh, h=P.h)
    M = wl.n * wl.p
    idx = np.arange(P.m)
    I, J, K = idx % M, (idx // M) % M, idx // (M * M)
    perm = ((I + wl.p) % M) + M * (J + M * K)        # node shifted by one cell in x
    X = trial_vectors(wl, n_v=2)
    Xs = np.empty_like(X)
    Xs[perm] = X
    Y = P.apply(X)
    Ys = Ps.apply(Xs)
    np.testing.assert_allclose(Ys[perm], Y, atol=1e-11)


def test_projector_moments_against_radial_integrals():
    """sum_I F_{s,I} = int chi_s and sum_e sum_i F_{px,i} x_i = int x chi_px (partition of unity)."""
    from scipy.integrate import quad
    wl = Workload("nl", L=10.0, n=8, p=6, nq=7, n_v=1, n_atoms=1, seed=5)
    R = np.array([[5.1, 4.9, 5.05]])
    P = Problem(wl, vloc=_zero, vgga=None, R=R, h=np.ones((1, 9)))
    g = lambda r: math.exp(-r * r / (2 * PROJ_SIGMA ** 2)) * (1 - (r / PROJ_RC) ** 2) ** 3
    c0 = 0.5 / math.sqrt(math.pi)
    c1 = math.sqrt(3 / (4 * math.pi))
    s_exact = c0 * quad(lambda r: 4 * math.pi * r * r * g(r), 0, PROJ_RC, epsabs=1e-14)[0]
    px_exact = c1 * quad(lambda r: 4 * math.pi / 3 * r ** 4 * g(r), 0, PROJ_RC, epsabs=1e-14)[0]
    xn = P.node_coords()
    _, cells, Fs = P.projector_blocks()[0]
    s_sum = sum(F[:, 0].sum() for F in Fs)
    px_sum = sum(F[:, 3] @ (xn[e][:, 0] - R[0, 0]) for e, F in zip(cells, Fs))
    z_sum = sum(F[:, 0] @ (xn[e][:, 0] - R[0, 0]) for e, F in zip(cells, Fs))
    assert abs(s_sum - s_exact) < 2e-5 * abs(s_exact)
    assert abs(px_sum - px_exact) < 2e-5 * abs(px_exact)
    assert abs(z_sum) < 1e-5 * abs(s_exact)          # odd moment of an s projector vanishes


def test_nonlocal_dense_vs_separable_and_psd():
    wl = _small_full(True)
    P = Problem(wl, vloc=_zero, vgga=None)
    P.h = np.abs(P.h)
    X = trial_vectors(wl, n_v=2)
    Ynl = P.apply(X, local=False)
    import scipy.sparse as sp
    Hn = (P.assemble("H") - sum(
        sp.csr_matrix((P.cell_matrix(e).ravel(), (np.repeat(P.dofs[e], P.dofs[e].size),
                       np.tile(P.dofs[e], P.dofs[e].size))), shape=(P.m, P.m))
        for e in range(P.E))).toarray()
    np.testing.assert_allclose(Hn @ X, Ynl, atol=1e-12)
    ev = np.linalg.eigvalsh(Hn)
    assert ev.min() > -1e-12 * ev.max()                   # PSD for h >= 0
    assert np.sum(ev > 1e-10 * ev.max()) <= 9 * P.R.shape[0]   # rank <= n_s


def test_sampled_rows_equal_full_apply():
    wl = _small_full(True)
    P = Problem(wl)
    X = trial_vectors(wl, n_v=2)
    rows = np.random.default_rng(1).choice(P.m, 17, replace=False)
    np.testing.assert_allclose(P.apply_rows(X, rows), P.apply(X)[rows], atol=1e-12)


def test_projector_bloch_phase_against_fourier_transform():
    """sum_J conj(F_{s,J}) u_J for u = exp(iG.x) equals exp(i q.R) chi_s^(q), q = k + G.

    chi_s^(q) = 4 pi c0 int r^2 g(r) sin(qr)/(qr) dr by 1D quadrature.  The
    opposite phase convention would give q = G - k instead.
    """
    from scipy.integrate import quad
    L = 10.0
    wl = Workload("nlk", L=L, n=8, p=6, nq=7, n_v=1, n_atoms=1, kfrac=(0.3, 0.1, 0.0),
                  complex=True, seed=5)
    R = np.array([[5.1, 4.9, 5.05]])
    P = Problem(wl, vloc=_zero, vgga=None, R=R, h=np.ones((1, 9)))
    G = np.array([2 * math.pi / L, 0.0, 0.0])
    xn = P.node_coords()
    _, cells, Fs = P.projector_blocks()[0]
    coef = sum(np.conj(F[:, 0]) @ np.exp(1j * xn[e] @ G) for e, F in zip(cells, Fs))
    g = lambda r: math.exp(-r * r / (2 * PROJ_SIGMA ** 2)) * (1 - (r / PROJ_RC) ** 2) ** 3
    c0 = 0.5 / math.sqrt(math.pi)

    def chihat(q):
        qn = np.linalg.norm(q)
        return 4 * math.pi * c0 * quad(lambda r: r * r * g(r) * math.sin(qn * r) / (qn * r),
                                       0, PROJ_RC, epsabs=1e-14)[0]
    q = P.kpt + G
    want = np.exp(1j * q @ R[0]) * chihat(q)
    qw = G - P.kpt
    wrong = np.exp(1j * qw @ R[0]) * chihat(qw)
    assert abs(coef - want) < 1e-5 * abs(want)
    assert abs(wrong - want) > 1e-2 * abs(want)
