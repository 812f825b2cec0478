"""Residual-based Chebyshev filtered subspace iteration (R-ChFSI): standard form
and, at the end of this file, the generalised form with the consistent mass.

TEST INFRASTRUCTURE (oracle): see ``oracle/__init__.py``.

The eigenproblem is the standard Hermitian problem for
    Hs = D^{-1/2} H D^{-1/2},
D being the GLL-lumped mass matrix (the diagonal approximation of M that
Algorithm 4 works with).  In these scaled variables D and M both become the
identity.

What the filter computes (Algorithm 4).  Map the unwanted interval
[lT, lmax] onto [-1, 1] by t -> (t - c)/e with c = (lmax + lT)/2 and
e = (lmax - lT)/2.  The filter of degree m is p_m(Hs) X with
    p_k(t) = T_k((t - c)/e) / T_k((lmin - c)/e),
T_k the Chebyshev polynomials of the first kind: p_k damps the unwanted
interval and is 1 at lmin.  Normalised this way, the block X_k = p_k(Hs) X
obeys the three-term recurrence
    X_{k+1} = (2 s_{k+1} / e) (Hs - c) X_k - s_k s_{k+1} X_{k-1},
    s_1 = e / (lmin - c),  s_{k+1} = 1 / (2 / s_1 - s_k),
with X_0 = X and X_1 = (s_1 / e)(Hs - c) X.

The residual-based form splits X_k = R_k + X L_k, where L_k = p_k(Lam) is
diagonal in the current Ritz values Lam.  With the residual Y = Hs X - X Lam
one has (Hs - c) X L_k = Y L_k + X (Lam - c) L_k, so the two parts follow
separate recurrences:
    R_{k+1} = (2 s_{k+1} / e) [(Hs - c) R_k + Y L_k] - s_k s_{k+1} R_{k-1},
    L_{k+1} = (2 s_{k+1} / e) (Lam - c) L_k - s_k s_{k+1} L_{k-1},
from R_0 = 0, L_0 = I, R_1 = (s_1 / e) Y, L_1 = (s_1 / e)(Lam - c).  The
filtered block is R_m + X L_m.  The matrix products act only on R_k, which
shrinks as X converges; that is why the paper can take them in low precision.
(The paper calls the degree p; it is m here.)  Algorithm 3 is the outer loop:
filter, then Rayleigh-Ritz on the filtered block.

The spectral bounds are inputs in the paper.  Here lmax is the standard safe
Lanczos bound theta_max(T_k) + |beta_k| after k steps, lmin the smallest and
lT the largest current Ritz value.
"""
import numpy as np


def _chebyshev_scalars(degree, lmin, lT, lmax):
    """c, e and the normalisation ratios s_1 .. s_degree of the shifted, scaled
    Chebyshev recurrence (see the module docstring)."""
    e = (lmax - lT) / 2.0
    c = (lmax + lT) / 2.0
    s = [None, e / (lmin - c)]
    for _ in range(2, degree + 1):
        s.append(1.0 / (2.0 / s[1] - s[-1]))
    return c, e, s


def filter_rchfsi(apply_Hs, X, lam, degree, lmin, lT, lmax):
    """Algorithm 4 in standard form: R_m + X L_m for X_m = p_m(Hs) X.
    apply_Hs(V) -> Hs V; lam = current Ritz values [n_v]."""
    c, e, s = _chebyshev_scalars(degree, lmin, lT, lmax)
    Y = apply_Hs(X) - X * lam[None, :]                  # residual of the Ritz pairs
    R_prev, L_prev = np.zeros_like(Y), np.ones_like(lam)             # k = 0
    R_cur, L_cur = (s[1] / e) * Y, (s[1] / e) * (lam - c)            # k = 1
    for k in range(1, degree):
        a, b = 2.0 * s[k + 1] / e, s[k] * s[k + 1]
        R_next = a * (apply_Hs(R_cur) - c * R_cur + Y * L_cur[None, :]) - b * R_prev
        L_next = a * (lam - c) * L_cur - b * L_prev
        R_prev, R_cur = R_cur, R_next
        L_prev, L_cur = L_cur, L_next
    return R_cur + X * L_cur[None, :]


def filter_reference_polynomial(evals, evecs, X, degree, lmin, lT, lmax):
    """Closed form of the same filter: p(Hs) X with p(t) = T_m((t-c)/e) / T_m((lmin-c)/e).

    T_m is the Chebyshev polynomial of the first kind (numpy.polynomial).
    """
    from numpy.polynomial import chebyshev as C
    e = (lmax - lT) / 2.0
    c = (lmax + lT) / 2.0
    coef = np.zeros(degree + 1)
    coef[-1] = 1.0
    scale = C.chebval((lmin - c) / e, coef)
    pv = C.chebval((evals - c) / e, coef) / scale
    return evecs @ (pv[:, None] * (evecs.conj().T @ X))


def lanczos_upper_bound(apply_Hs, v0, steps=10):
    """Upper bound of the spectrum of Hs: theta_max(T_k) + |beta_k| after k Lanczos steps."""
    return lanczos_coefficients(apply_Hs, v0, steps)[2]


def lanczos_coefficients(apply_Hs, v0, steps=10):
    """k steps of the symmetric Lanczos recurrence from v0: (alphas, betas, bound) with the
    bound theta_max(T_k) + |beta_k| of lanczos_upper_bound."""
    v = v0 / np.linalg.norm(v0)
    v_prev = np.zeros_like(v)
    alphas, betas = [], []
    beta = 0.0
    for _ in range(steps):
        w = apply_Hs(v[:, None])[:, 0]
        alpha = np.real(np.vdot(v, w))
        w = w - alpha * v - beta * v_prev
        beta = np.linalg.norm(w)
        alphas.append(alpha)
        betas.append(beta)
        if beta == 0.0:
            break
        v_prev, v = v, w / beta
    T = np.diag(alphas) + np.diag(betas[:-1], 1) + np.diag(betas[:-1], -1)
    return np.array(alphas), np.array(betas), float(np.max(np.linalg.eigvalsh(T)) + abs(betas[-1]))


def rayleigh_ritz(apply_Hs, Y):
    """Algorithm 3's Rayleigh-Ritz step in standard form: (Y^H Hs Y) E = (Y^H Y) E Lam."""
    import scipy.linalg as sl
    S = Y.conj().T @ Y
    Hp = Y.conj().T @ apply_Hs(Y)
    Hp = 0.5 * (Hp + Hp.conj().T)
    S = 0.5 * (S + S.conj().T)
    lam, E = sl.eigh(Hp, S)
    return lam, Y @ E


def rchfsi(apply_Hs, X0, degree, n_iter, lanczos_steps=10, seed=0, tol=None):
    """Algorithm 3: repeat (filter, Rayleigh-Ritz).  Returns (Ritz values, vectors, residual norms)."""
    rng = np.random.default_rng(seed)
    lmax = lanczos_upper_bound(apply_Hs, rng.standard_normal(X0.shape[0]).astype(X0.dtype),
                               lanczos_steps)
    X, _ = np.linalg.qr(X0)
    lam, X = rayleigh_ritz(apply_Hs, X)
    res = None
    for _ in range(n_iter):
        Yf = filter_rchfsi(apply_Hs, X, lam, degree, lam[0], lam[-1], lmax)
        lam, X = rayleigh_ritz(apply_Hs, Yf)
        X = X / np.linalg.norm(X, axis=0)[None, :]
        R = apply_Hs(X) - X * lam[None, :]
        res = np.linalg.norm(R, axis=0)
        if tol is not None and np.max(res) < tol:
            break
    return lam, X, res


# ------------------------------------------------------------------------
# Generalised form: H X = M X Lam with the consistent mass M (eq. FEeigen),
# Algorithm 4 as printed: the residual uses M, the recurrence applies H D^{-1}
# (D the GLL-lumped approximation of M), and the result maps back with D^{-1}.

def filter_rchfsi_ghep(apply_H, apply_M, Dinv, X, lam, degree, lmin, lT, lmax):
    """Algorithm 4 for the GHEP.  apply_H / apply_M: V -> H V / M V; Dinv: the
    diagonal of D^{-1} [m]; lam = current Ritz values [n_v].

    The same two recurrences as the standard form, with the residual taken
    against the consistent mass, Y = H X - M X Lam, the product in the R
    recurrence being H D^{-1} R_k (R_k lives in the residual space, D^{-1} maps
    it back to the solution space), and the filtered block D^{-1} R_m + X L_m."""
    c, e, s = _chebyshev_scalars(degree, lmin, lT, lmax)
    Y = apply_H(X) - apply_M(X) * lam[None, :]
    R_prev, L_prev = np.zeros_like(Y), np.ones_like(lam)
    R_cur, L_cur = (s[1] / e) * Y, (s[1] / e) * (lam - c)
    for k in range(1, degree):
        a, b = 2.0 * s[k + 1] / e, s[k] * s[k + 1]
        R_next = a * (apply_H(Dinv[:, None] * R_cur) - c * R_cur + Y * L_cur[None, :]) - b * R_prev
        L_next = a * (lam - c) * L_cur - b * L_prev
        R_prev, R_cur = R_cur, R_next
        L_prev, L_cur = L_cur, L_next
    return Dinv[:, None] * R_cur + X * L_cur[None, :]


def rayleigh_ritz_ghep(apply_H, apply_M, Y):
    """Algorithm 3's Rayleigh-Ritz step: (Y^H H Y) E = (Y^H M Y) E Lam; X = Y E."""
    import scipy.linalg as sl
    S = Y.conj().T @ apply_M(Y)
    Hp = Y.conj().T @ apply_H(Y)
    Hp = 0.5 * (Hp + Hp.conj().T)
    S = 0.5 * (S + S.conj().T)
    lam, E = sl.eigh(Hp, S)
    return lam, Y @ E


def rchfsi_ghep(apply_H, apply_M, Dinv, X0, degree, n_iter, lanczos_steps=10, seed=0, tol=None):
    """Algorithm 3 for the GHEP.  The spectral upper bound is the Lanczos bound
    of D^{-1/2} H D^{-1/2} (the operator the recurrence effectively runs on).
    Returns (Ritz values, vectors, norms of H x - lam M x)."""
    rng = np.random.default_rng(seed)
    s = np.sqrt(Dinv)
    lmax = lanczos_upper_bound(lambda V: s[:, None] * apply_H(s[:, None] * V),
                               rng.standard_normal(X0.shape[0]).astype(X0.dtype), lanczos_steps)
    X, _ = np.linalg.qr(X0)
    lam, X = rayleigh_ritz_ghep(apply_H, apply_M, X)
    res = None
    for _ in range(n_iter):
        Yf = filter_rchfsi_ghep(apply_H, apply_M, Dinv, X, lam, degree, lam[0], lam[-1], lmax)
        lam, X = rayleigh_ritz_ghep(apply_H, apply_M, Yf)
        R = apply_H(X) - apply_M(X) * lam[None, :]
        res = np.linalg.norm(R, axis=0) / np.linalg.norm(X, axis=0)
        if tol is not None and np.max(res) < tol:
            break
    return lam, X, res
