"""R-ChFSI eigensolver driver on the GPU (Algorithm 3 around Algorithm 4).

The caller's side of ``fe_ks_cheb_filter``: the outer subspace iteration of
Algorithm 3 in the standard form Hs = D^{-1/2} H D^{-1/2} (D the GLL-lumped
mass), or, given a context whose application is the consistent mass M, for
the generalised problem H X = M X Lam (``fe_ks_cheb_filter_ghep``; the
Rayleigh-Ritz step then solves (Y^H H Y) E = (Y^H M Y) E Lam).  Each
iteration filters the block with the library's residual-based Chebyshev
filter and then performs the FP64-accurate Rayleigh-Ritz step.  For real
operators every step is a library call: fe_ks_lanczos_bound (the upper bound
theta_max + |beta_k| after k Lanczos steps), fe_ks_cheb_filter and
fe_ks_rayleigh_ritz.  Complex operators keep the Rayleigh-Ritz step in
dense torch calls on the device (the library's Rayleigh-Ritz is real only).
The lower bound and the wanted-spectrum edge are the current Ritz values.
"""
import torch

from . import fe_ks as fk


class RChFSI:
    """precision: arithmetic of the filter's recurrence (FE_KS_F32, FE_KS_BF16, FE_KS_F64 or FE_KS_F64E);
    exact: the FP64-accurate path used for the filter's residual, Lanczos, Rayleigh-Ritz and
    residual norms (FE_KS_F64 native, or FE_KS_F64E pairs of floats);
    gemm_pairs: Rayleigh-Ritz Gram matrices and rotation in pairs of floats (FP64-accurate,
    FP32 pipe) instead of FP64 cuBLAS; gemm_emulated: cuBLAS's FP64 emulation;
    mass_ctx: a context whose application is M (``problem.mass_problem`` set up with
    FE_KS_TERM_L) to solve the generalised problem instead of the standard form."""

    def __init__(self, ctx, m, n_v, cplx, degree=20, precision=fk.FE_KS_F32, lanczos_steps=10,
                 exact=fk.FE_KS_F64, gemm_emulated=False, gemm_pairs=False, mass_ctx=None):
        self.ctx, self.m, self.n_v, self.cplx = ctx, m, n_v, cplx
        self.mass = mass_ctx
        self.degree, self.precision, self.lanczos_steps = degree, precision, lanczos_steps
        self.exact = exact
        self.gemm_emulated = gemm_emulated and not cplx
        self.gemm_pairs = gemm_pairs and not cplx
        self._gram_work = None
        self._lz = None
        self._rr = None
        self.rr_path = None
        self.dt = torch.complex128 if cplx else torch.float64
        self.dev = torch.device("cuda", torch.cuda.current_device())
        nb = fk.fe_ks_cheb_filter_workspace(ctx, n_v, precision)
        self.work = torch.empty(nb + 256, dtype=torch.uint8, device=self.dev)
        off = (-self.work.data_ptr()) % 256
        self.work_view = self.work[off:off + nb]
        self.work_bytes = nb
        self.tmp = torch.empty((m, n_v), dtype=self.dt, device=self.dev)
        self.lmax = None

    def apply_scaled(self, V, out=None):
        V = V.contiguous()
        out = torch.empty(V.shape, dtype=V.dtype, device=V.device) if out is None else out
        fk.fe_ks_apply_scaled(self.ctx, V, out, V.shape[1], self.exact)
        return out

    def apply_op(self, V, out=None):
        """The operator of the Rayleigh-Ritz step: Hs (standard form) or H (generalised)."""
        if self.mass is None:
            return self.apply_scaled(V, out)
        V = V.contiguous()
        out = torch.empty(V.shape, dtype=V.dtype, device=V.device) if out is None else out
        fk.fe_ks_apply(self.ctx, V, out, V.shape[1], self.exact)
        return out

    def apply_metric(self, V):
        """The metric of the Rayleigh-Ritz step: I (standard form) or M (generalised)."""
        if self.mass is None:
            return V
        V = V.contiguous()
        out = torch.empty(V.shape, dtype=V.dtype, device=V.device)
        fk.fe_ks_apply(self.mass, V, out, V.shape[1], self.exact)
        return out

    def _aligned(self, nbytes):
        buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.dev)
        off = (-buf.data_ptr()) % 256
        return buf, buf[off:off + nbytes]

    def lanczos_upper_bound(self, seed=0):
        """fe_ks_lanczos_bound from a seeded normal start vector."""
        g = torch.Generator(device=self.dev)
        g.manual_seed(seed)
        v = torch.randn((self.m, 1), generator=g, device=self.dev, dtype=torch.float64).to(self.dt).contiguous()
        if self._lz is None:
            nb = fk.fe_ks_lanczos_bound_workspace(self.ctx, self.lanczos_steps)
            self._lz = self._aligned(nb) + (nb,)
        _, view, nb = self._lz
        self.lmax, self.lanczos_alpha, self.lanczos_beta = fk.fe_ks_lanczos_bound(
            self.ctx, v, self.lanczos_steps, self.exact, view, nb)
        return self.lmax

    def lanczos_upper_bound_torch(self, seed=0):
        """The same bound with dense torch calls (kept for comparison)."""
        g = torch.Generator(device=self.dev)
        g.manual_seed(seed)
        v = torch.randn((self.m, 1), generator=g, device=self.dev, dtype=torch.float64).to(self.dt)
        v /= torch.linalg.vector_norm(v)
        v_prev = torch.zeros_like(v)
        w = torch.empty_like(v)
        alphas, betas, beta = [], [], 0.0
        for _ in range(self.lanczos_steps):
            self.apply_scaled(v, w)
            alpha = torch.real(torch.vdot(v[:, 0], w[:, 0])).item()
            w = w - alpha * v - beta * v_prev
            beta = torch.linalg.vector_norm(w).item()
            alphas.append(alpha)
            betas.append(beta)
            if beta == 0.0:
                break
            v_prev, v = v, w / beta
            w = torch.empty_like(v)
        k = len(alphas)
        T = torch.zeros((k, k), dtype=torch.float64)
        for i in range(k):
            T[i, i] = alphas[i]
            if i + 1 < k:
                T[i, i + 1] = T[i + 1, i] = betas[i]
        self.lmax = float(torch.linalg.eigvalsh(T).max().item() + abs(betas[-1]))
        return self.lmax

    def rayleigh_ritz(self, Y):
        """Rayleigh-Ritz on span(Y); returns (Lam, Y E) (real operators: fe_ks_rayleigh_ritz, in place)."""
        if self.cplx or self.gemm_emulated:
            return self.rayleigh_ritz_torch(Y)
        Y = Y.contiguous()
        prec = fk.FE_KS_F64E if self.gemm_pairs else fk.FE_KS_F64
        if self._rr is None or self._rr[0] != prec:
            nb = fk.fe_ks_rayleigh_ritz_workspace(self.ctx, self.n_v, prec)
            self._rr = (prec, nb) + self._aligned(nb)
        _, nb, _, view = self._rr
        lam = torch.empty(self.n_v, dtype=torch.float64, device=self.dev)
        self.rr_path = fk.fe_ks_rayleigh_ritz(self.ctx, Y, lam, self.n_v, prec, view, nb, mass=self.mass)
        return lam, Y

    def rayleigh_ritz_torch(self, Y):
        """Rayleigh-Ritz on span(Y): (Y^H Hs Y) E = (Y^H Y) E Lam, returns (Lam, Y E).

        Cholesky of the Gram matrix S = Y^H Y = L L^H reduces it to the standard
        problem L^-1 (Y^H Hs Y) L^-H W = W Lam with E = L^-H W (three FP64 GEMMs).
        A Householder QR is used instead when S is too ill-conditioned for Cholesky.
        """
        Y = Y.contiguous()
        S = self._gram(Y, self.apply_metric(Y), symmetric=True)
        S = 0.5 * (S + S.conj().T)
        L, info = torch.linalg.cholesky_ex(S)
        d = torch.real(torch.diagonal(L)) if int(info.item()) == 0 else None
        if d is None or float(d.min()) <= 1e-6 * float(d.max()):
            return self._rayleigh_ritz_qr(Y)
        HY = self.apply_op(Y, self.tmp)
        A = self._gram(Y, HY, symmetric=True)
        T1 = torch.linalg.solve_triangular(L, A, upper=False)
        B = torch.linalg.solve_triangular(L, T1.conj().T, upper=False).conj().T
        B = 0.5 * (B + B.conj().T)
        lam, W = torch.linalg.eigh(B)
        E = torch.linalg.solve_triangular(L.conj().T, W, upper=True)
        return lam.to(torch.float64).contiguous(), self._rotate(Y, E)

    def _gram(self, Y, Z, symmetric=False):
        """Y^H Z; symmetric=True when the product is known to be Hermitian (Y^H M Y, Y^H H Y):
        the pair-of-floats kernel then computes the tiles on and above the diagonal and
        mirrors them.  (cuBLAS's one-triangle FP64 form, syrkx, measured slower than its
        GEMM on this part, so the FP64 plan keeps the GEMM.)"""
        st = torch.cuda.current_stream().cuda_stream
        if self.gemm_pairs:
            return fk.fe_ks_gram_ff(Y, Z.contiguous(), stream=st, symmetric=symmetric)
        if self.gemm_emulated:
            return fk.row_gram(Y, Z, emulated=True, stream=st)
        return Y.conj().T @ Z

    def _rotate(self, Y, E):
        if self.gemm_pairs:
            return fk.fe_ks_rotate_ff(Y, E.contiguous(), stream=torch.cuda.current_stream().cuda_stream)
        if self.gemm_emulated:
            return fk.row_rotate(Y, E.contiguous(), emulated=True, stream=torch.cuda.current_stream().cuda_stream)
        return (Y @ E).contiguous()

    def _rayleigh_ritz_qr(self, Y):
        Q, _ = torch.linalg.qr(Y)
        Q = Q.contiguous()          # QR returns column-major factors; the C ABI is row-major
        HQ = self.apply_op(Q, self.tmp)
        A = Q.conj().T @ HQ
        A = 0.5 * (A + A.conj().T)
        if self.mass is not None:   # generalised: Cholesky of the (well-conditioned) Q^H M Q
            S = Q.conj().T @ self.apply_metric(Q)
            L = torch.linalg.cholesky(0.5 * (S + S.conj().T))
            B = torch.linalg.solve_triangular(L, torch.linalg.solve_triangular(L, A, upper=False).conj().T,
                                              upper=False).conj().T
            lam, W = torch.linalg.eigh(0.5 * (B + B.conj().T))
            W = torch.linalg.solve_triangular(L.conj().T, W, upper=True)
            return lam.to(torch.float64).contiguous(), (Q @ W).contiguous()
        lam, W = torch.linalg.eigh(A)
        return lam.to(torch.float64).contiguous(), (Q @ W).contiguous()

    def residual_norms(self, X, lam):
        """|Hs x - lam x| (standard form), |H x - lam M x| / |x| (generalised)."""
        if self.mass is None:
            R = self.apply_scaled(X, self.tmp) - X * lam[None, :].to(X.dtype)
            return torch.linalg.vector_norm(R, dim=0)
        R = self.apply_op(X, self.tmp) - self.apply_metric(X) * lam[None, :].to(X.dtype)
        return torch.linalg.vector_norm(R, dim=0) / torch.linalg.vector_norm(X, dim=0)

    def filter(self, X, lam):
        lmin, lT = float(lam[0].item()), float(lam[-1].item())
        if not lmin < lT < self.lmax:
            raise RuntimeError("spectral bounds out of order")
        if self.mass is None:
            fk.fe_ks_cheb_filter(self.ctx, X, lam, self.n_v, self.degree, lmin, lT, self.lmax, self.precision,
                                 self.work_view, self.work_bytes, residual_precision=self.exact)
        else:
            fk.fe_ks_cheb_filter_ghep(self.ctx, self.mass, X, lam, self.n_v, self.degree, lmin, lT, self.lmax,
                                      self.precision, self.work_view, self.work_bytes,
                                      residual_precision=self.exact)
        return X

    def run(self, X0, n_iter, tol=None, n_check=None):
        """Algorithm 3: Rayleigh-Ritz on X0, then (filter, Rayleigh-Ritz) n_iter times."""
        if self.lmax is None:
            self.lanczos_upper_bound()
        lam, X = self.rayleigh_ritz(X0)
        res = None
        n_check = self.n_v if n_check is None else n_check
        self.res_history = []   # largest residual norm of the checked pairs after each pass
        for it in range(n_iter):
            X = self.filter(X, lam)
            lam, X = self.rayleigh_ritz(X)
            if tol is not None:
                res = self.residual_norms(X, lam)
                self.res_history.append(float(res[:n_check].max()))
                if self.res_history[-1] < tol:
                    return lam, X, res, it + 1
        if res is None:
            res = self.residual_norms(X, lam)
        return lam, X, res, n_iter
