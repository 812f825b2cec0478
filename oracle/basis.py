"""1D tables of the FE discretisation: quadrature rules and Lagrange bases.

TEST INFRASTRUCTURE (oracle): see ``oracle/__init__.py``.

* Gauss-Legendre rule with n_q points on [-1, 1] (Sec. 3.1, eq. cellIntegrals).
* Gauss-Lobatto-Legendre (GLL) nodes: the FE nodal points of a degree-p
  spectral element (Sec. 2.2, eq. FEdiscr: "C^0 Lagrange interpolants
  constructed using GLL nodal points").
* Lagrange basis values and derivatives on an arbitrary node set, written as
  the textbook product formula (no barycentric tricks), so that
  N1D[q, i] = L_i(xi_q) (Sec. 3.2: the n_q x n_p matrix N^1D) and the
  collocation derivative Dt1D[q, r] = dL~_r/dxi (xi_q) on the Gauss points
  (Sec. 3.2, the factorisation D = D~ N).

Nodes are found with Newton's method on Legendre polynomials evaluated by the
three-term recurrence (textbook; checked in the tests against numpy's
``leggauss`` and against exactness on monomials).
"""
import numpy as np


def legendre(n, x):
    """Return (P_n(x), P_n'(x)) by the Bonnet recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    # derivative from P_n and P_{n-1}: (1-x^2) P_n' = n (P_{n-1} - x P_n)
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (p0 - x * p1) / (1.0 - x * x)
    # at x = +-1 the formula is 0/0; P_n'(+-1) = (+-1)^(n-1) n(n+1)/2
    end = np.abs(np.abs(x) - 1.0) < 1e-300
    if np.any(end):
        dp = np.where(end, np.sign(x) ** (n - 1) * n * (n + 1) / 2.0, dp)
    return p1, dp


def gauss_legendre(nq):
    """Gauss-Legendre points (ascending) and weights for an n_q-point rule."""
    i = np.arange(nq)
    x = -np.cos(np.pi * (i + 0.75) / (nq + 0.5))  # classical initial guess
    for _ in range(100):
        p, dp = legendre(nq, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    _, dp = legendre(nq, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return x, w


def gauss_lobatto(npts):
    """GLL nodes (ascending) and weights: -1, +1 and the roots of P'_{n-1}."""
    p = npts - 1
    if p < 1:
        raise ValueError("need at least 2 GLL points")
    i = np.arange(npts)
    x = -np.cos(np.pi * i / p)  # Chebyshev-Gauss-Lobatto initial guess
    inner = x[1:-1].copy()
    for _ in range(100):
        pp, dpp = legendre(p, inner)
        # second derivative from Legendre's equation:
        # (1-x^2) P'' - 2x P' + p(p+1) P = 0
        d2 = (2.0 * inner * dpp - p * (p + 1) * pp) / (1.0 - inner * inner)
        dx = dpp / d2
        inner = inner - dx
        if inner.size == 0 or np.max(np.abs(dx)) < 1e-16:
            break
    x = np.concatenate([[-1.0], inner, [1.0]])
    pp, _ = legendre(p, x)
    w = 2.0 / (p * (p + 1) * pp * pp)
    return x, w


def lagrange(nodes, x):
    """Values V[q, i] = L_i(x_q) and derivatives dV[q, i] = L_i'(x_q).

    L_i(x) = prod_{j != i} (x - x_j) / (x_i - x_j);
    L_i'(x) = sum_{k != i} 1/(x_i - x_k) prod_{j != i, k} (x - x_j)/(x_i - x_j).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    V = np.ones((x.size, n))
    dV = np.zeros((x.size, n))
    for i in range(n):
        for j in range(n):
            if j != i:
                V[:, i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
        for k in range(n):
            if k == i:
                continue
            term = np.full(x.size, 1.0 / (nodes[i] - nodes[k]))
            for j in range(n):
                if j != i and j != k:
                    term = term * (x - nodes[j]) / (nodes[i] - nodes[j])
            dV[:, i] += term
    return V, dV


def tables(p, nq):
    """The 1D tables of Sec. 3.2 for degree p (n_p = p+1 GLL nodes) and n_q Gauss points.

    Returns dict with
      xi_gll, w_gll : GLL nodes/weights (n_p)
      xi_q, w_q     : Gauss points/weights (n_q)
      N1D [n_q, n_p]: basis values at Gauss points
      dN1D[n_q, n_p]: basis derivatives at Gauss points
      Dt1D[n_q, n_q]: collocation derivative on the Gauss points
    """
    xg, wg = gauss_lobatto(p + 1)
    xq, wq = gauss_legendre(nq)
    N1D, dN1D = lagrange(xg, xq)
    _, Dt1D = lagrange(xq, xq)
    return dict(xi_gll=xg, w_gll=wg, xi_q=xq, w_q=wq, N1D=N1D, dN1D=dN1D, Dt1D=Dt1D)
