"""Residual-based Chebyshev filtered subspace iteration (R-ChFSI): standard form
and, at the end of this file, the generalised form with the consistent mass.

TEST INFRASTRUCTURE (oracle): see ``oracle/__init__.py``.

The eigenproblem is the standard Hermitian problem for
    Hs = D^{-1/2} H D^{-1/2},
D being the GLL-lumped mass matrix (the diagonal approximation of M that
Algorithm 4 uses as D^{-1}).  In these scaled variables D -> I and M -> I, so
Algorithm 4 is used with both replaced by the identity:

  e = (lmax - lT)/2, c = (lmax + lT)/2, sigma = e / (lmin - c), sigma1 = sigma,
  gamma = 2 / sigma1
  Y  = Hs X - X Lam
  R_X = 0, R_Y = (sigma1/e) Y, Lam_X = I, Lam_Y = (sigma1/e)(Lam - c I)
  for k = 2..m:
      sigma2 = 1 / (gamma - sigma)
      R_X   <- (2 sigma2/e) [ (Hs - c I) R_Y + Y Lam_Y ] - sigma sigma2 R_X
      Lam_X <- (2 sigma2/e) Lam_Y (Lam - c I) - sigma sigma2 Lam_X
      swap(R_X, R_Y); swap(Lam_X, Lam_Y); sigma = sigma2
  X <- R_Y + X Lam_Y

(Algorithm 4; m is the filter degree, called p in the paper.)  The outer loop
is Algorithm 3: filter, then Rayleigh-Ritz on the filtered block.

The spectral bounds are inputs in the paper.  Here lmax is the standard safe
Lanczos bound theta_max(T_k) + |beta_k| after k steps, lmin the smallest and
lT the largest current Ritz value.
"""
import numpy as np


def filter_rchfsi(apply_Hs, X, lam, degree, lmin, lT, lmax):
    """Algorithm 4 in standard form.  apply_Hs(V) -> Hs V; lam = current Ritz values [n_v]."""
    e = (lmax - lT) / 2.0
    c = (lmax + lT) / 2.0
    sigma = e / (lmin - c)
    sigma1 = sigma
    gamma = 2.0 / sigma1
    Y = apply_Hs(X) - X * lam[None, :]
    RX = np.zeros_like(Y)
    RY = (sigma1 / e) * Y
    LX = np.ones_like(lam)
    LY = (sigma1 / e) * (lam - c)
    for _ in range(2, degree + 1):
        sigma2 = 1.0 / (gamma - sigma)
        RX = (2.0 * sigma2 / e) * (apply_Hs(RY) - c * RY + Y * LY[None, :]) - sigma * sigma2 * RX
        LX = (2.0 * sigma2 / e) * LY * (lam - c) - sigma * sigma2 * LX
        RX, RY = RY, RX
        LX, LY = LY, LX
        sigma = sigma2
    return RY + X * LY[None, :]


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
    return float(np.max(np.linalg.eigvalsh(T)) + abs(betas[-1]))


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
    diagonal of D^{-1} [m]; lam = current Ritz values [n_v]."""
    e = (lmax - lT) / 2.0
    c = (lmax + lT) / 2.0
    sigma = e / (lmin - c)
    sigma1 = sigma
    gamma = 2.0 / sigma1
    Y = apply_H(X) - apply_M(X) * lam[None, :]
    RX = np.zeros_like(Y)
    RY = (sigma1 / e) * Y
    LX = np.ones_like(lam)
    LY = (sigma1 / e) * (lam - c)
    for _ in range(2, degree + 1):
        sigma2 = 1.0 / (gamma - sigma)
        RX = (2.0 * sigma2 / e) * (apply_H(Dinv[:, None] * RY) - c * RY + Y * LY[None, :]) - sigma * sigma2 * RX
        LX = (2.0 * sigma2 / e) * LY * (lam - c) - sigma * sigma2 * LX
        RX, RY = RY, RX
        LX, LY = LY, LX
        sigma = sigma2
    return Dinv[:, None] * RY + X * LY[None, :]


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
