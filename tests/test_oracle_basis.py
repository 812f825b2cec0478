"""Pins of the oracle's 1D tables (Sec. 2.2 eq. FEdiscr, Sec. 3.1 eq. cellIntegrals, Sec. 3.2 D = D~ N)."""
import numpy as np
import pytest

from oracle import basis


@pytest.mark.parametrize("n", range(1, 13))
def test_gauss_matches_library(n):
    x, w = basis.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xr, atol=2e-15)
    np.testing.assert_allclose(w, wr, atol=2e-15)


@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_exact_on_monomials(n):
    x, w = basis.gauss_legendre(n)
    for d in range(2 * n):
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(np.sum(w * x ** d) - exact) < 1e-14
    d = 2 * n  # first degree that is not integrated exactly
    exact = 2.0 / (d + 1)
    assert abs(np.sum(w * x ** d) - exact) > 1e-6


@pytest.mark.parametrize("npts", range(2, 11))
def test_gll_nodes_are_roots_and_exact(npts):
    x, w = basis.gauss_lobatto(npts)
    p = npts - 1
    assert x[0] == -1.0 and x[-1] == 1.0
    assert np.all(np.diff(x) > 0)
    np.testing.assert_allclose(x, -x[::-1], atol=1e-15)
    # interior nodes are the roots of P'_p, checked with numpy's Legendre class
    dP = np.polynomial.legendre.Legendre.basis(p).deriv()
    np.testing.assert_allclose(dP(x[1:-1]), 0.0, atol=1e-11)
    for d in range(2 * npts - 2):          # GLL exact to degree 2n-3
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(np.sum(w * x ** d) - exact) < 1e-14


@pytest.mark.parametrize("p,nq", [(1, 2), (4, 5), (6, 7), (7, 8), (8, 9), (8, 10), (4, 6)])
def test_lagrange_tables(p, nq):
    t = basis.tables(p, nq)
    xg, xq = t["xi_gll"], t["xi_q"]
    V, dV = basis.lagrange(xg, xg)
    np.testing.assert_allclose(V, np.eye(p + 1), atol=1e-14)        # L_i(x_j) = delta_ij
    np.testing.assert_allclose(t["N1D"].sum(axis=1), 1.0, atol=1e-14)   # partition of unity
    np.testing.assert_allclose(t["dN1D"].sum(axis=1), 0.0, atol=1e-12)
    # derivatives against numpy polynomial fits of each Lagrange basis function
    for i in range(p + 1):
        e = np.zeros(p + 1)
        e[i] = 1.0
        poly = np.polynomial.Polynomial.fit(xg, e, p, domain=[-1, 1], window=[-1, 1])
        np.testing.assert_allclose(t["N1D"][:, i], poly(xq), atol=1e-11)
        np.testing.assert_allclose(t["dN1D"][:, i], poly.deriv()(xq), atol=1e-9)
    # exact collocation factorisation D = D~ N when n_q >= n_p (Sec. 3.2)
    np.testing.assert_allclose(t["Dt1D"] @ t["N1D"], t["dN1D"], atol=1e-12)
    # centro-symmetry used by the even-odd decomposition
    np.testing.assert_allclose(t["N1D"], t["N1D"][::-1, ::-1], atol=1e-14)
    np.testing.assert_allclose(t["Dt1D"], -t["Dt1D"][::-1, ::-1], atol=1e-11)
