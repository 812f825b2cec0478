"""Plain FP64 assembly and action of the FE Kohn-Sham Hamiltonian.

TEST INFRASTRUCTURE (oracle): see ``oracle/__init__.py``.

This follows the paper's *definitions*, not its matrix-free algorithm:

* H_loc = T + L + G - iK with (Sec. 2.2, eq. Hloc / Sec. 3.1, eq. HlocIntegral)
    T_IJ = 1/2 int grad N_I . grad N_J
    L_IJ = int V^L N_I N_J,          V^L = V_loc + |k|^2 / 2   (eq. Vloc)
    G_IJ = int V^G . (grad N_I N_J + N_I grad N_J)
    K_IJ = int k . (N_I grad N_J)
  evaluated with the tensor Gauss rule of eq. cellIntegrals, using physical
  gradients grad N = J^{-T} grad_xi N of the trilinear cell map (J = dx/dxi),
  i.e. without the collocation factorisation D = D~ N of Sec. 3.2.
* H_nloc,IJ = sum_a sum_b F_{b,I} h_b conj(F_{b,J}) with
    F_{b,I} = int sum_r exp(-i k.(x - L_r)) chi_b(x - R_a - L_r) N_I(x) dx
  (eq. Vnonloc), summed over all 27 neighbouring lattice images.
* Y = H X = sum_e Q_e^T H^(e) Q_e X + F diag(h) F^H X (eq. HX), Q_e being the
  cell -> global DoF map after periodic identification.  Applying precomputed
  cell matrices cell by cell is the paper's cell-matrix (CM) baseline
  (Sec. 3.1; Sec. 5.4 "Cell-Matrix Action").
"""
import numpy as np

from . import basis
from synth import (make_mesh, vloc_fn, vgga_fn, atoms, projector_values,
                   lattice_images, PROJ_RC)


class Problem:
    """All inputs of one workload, as the oracle sees them (no GPU data)."""

    def __init__(self, wl, with_atoms=True, verts=None, dofs=None, vloc=None, vgga="wl",
                 R=None, h=None, kpt=None):
        self.wl = wl
        self.p, self.nq, self.np_ = wl.p, wl.nq, wl.p + 1
        if verts is None:
            self.verts, self.dofs, self.m = make_mesh(wl)
        else:
            self.verts, self.dofs = np.asarray(verts, float), np.asarray(dofs)
            self.m = int(self.dofs.max()) + 1
        self.E = self.verts.shape[0]
        self.kpt = wl.kpt if kpt is None else np.asarray(kpt, float)
        self.complex = bool(wl.complex) or bool(np.any(self.kpt != 0))
        self.vloc = vloc_fn(wl) if vloc is None else vloc
        self.vgga = vgga_fn(wl) if isinstance(vgga, str) else vgga
        if R is not None:
            self.R, self.h = np.asarray(R, float).reshape(-1, 3), np.asarray(h, float).reshape(-1, 9)
        elif with_atoms and wl.n_atoms > 0:
            self.R, self.h = atoms(wl)
        else:
            self.R, self.h = np.zeros((0, 3)), np.zeros((0, 9))
        self.t = basis.tables(self.p, self.nq)
        self._cell_cache = {}

    def node_coords(self):
        """Physical coordinates [E, n_p^3, 3] of every cell's nodes (unwrapped per cell)."""
        t, npn = self.t, self.np_
        li = np.arange(npn)
        kk, jj, ii = np.meshgrid(li, li, li, indexing="ij")
        xi = np.stack([t["xi_gll"][ii.ravel()], t["xi_gll"][jj.ravel()], t["xi_gll"][kk.ravel()]], axis=1)
        return np.stack([self.trilinear(e, xi)[0] for e in range(self.E)])

    # ----------------------------------------------------------- geometry
    def trilinear(self, e, xi):
        """x(xi) [Q,3] and J = dx/dxi [Q,3,3] of cell e at reference points xi [Q,3]."""
        X = self.verts[e]
        x = np.zeros((xi.shape[0], 3))
        J = np.zeros((xi.shape[0], 3, 3))
        for v in range(8):
            s = np.array([2 * (v & 1) - 1, 2 * ((v >> 1) & 1) - 1, 2 * ((v >> 2) & 1) - 1], float)
            f = (1.0 + s[None, :] * xi) / 2.0                  # [Q,3] factors
            phi = f[:, 0] * f[:, 1] * f[:, 2]
            dphi = np.stack([s[0] / 2 * f[:, 1] * f[:, 2],
                             s[1] / 2 * f[:, 0] * f[:, 2],
                             s[2] / 2 * f[:, 0] * f[:, 1]], axis=1)   # [Q,3] d/dxi_d
            x += phi[:, None] * X[v][None, :]
            J += X[v][None, :, None] * dphi[:, None, :]
        return x, J

    def cell(self, e, grads=True):
        """Quadrature data of cell e (cached): points, weights*detJ, N and physical grad N."""
        hit = self._cell_cache.get(e)
        if hit is not None and (not grads or "g" in hit):
            return hit
        t, nq, npn = self.t, self.nq, self.np_
        q = np.arange(nq)
        qz, qy, qx = np.meshgrid(q, q, q, indexing="ij")
        qx, qy, qz = qx.ravel(), qy.ravel(), qz.ravel()        # Q = qx + nq(qy + nq qz)
        xi = np.stack([t["xi_q"][qx], t["xi_q"][qy], t["xi_q"][qz]], axis=1)
        w = t["w_q"][qx] * t["w_q"][qy] * t["w_q"][qz]
        x, J = self.trilinear(e, xi)
        detJ = np.linalg.det(J)
        li = np.arange(npn)
        kk, jj, ii = np.meshgrid(li, li, li, indexing="ij")
        ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()        # I = i + np(j + np k)
        N, dN = t["N1D"], t["dN1D"]
        Bx, By, Bz = N[qx][:, ii], N[qy][:, jj], N[qz][:, kk]
        B = Bx * By * Bz                                       # [Q, I]
        out = dict(x=x, wdet=w * detJ, detJ=detJ, B=B)
        if grads:
            Jinv = np.linalg.inv(J)
            gref = np.stack([dN[qx][:, ii] * By * Bz,
                             Bx * dN[qy][:, jj] * Bz,
                             Bx * By * dN[qz][:, kk]], axis=0)     # [3, Q, I]  d/dxi_d
            # grad_x N = J^{-T} grad_xi N : component c = sum_d Jinv[d, c] d/dxi_d
            out["g"] = np.einsum("qdc,dqi->cqi", Jinv, gref)
        if len(self._cell_cache) < 512:
            self._cell_cache[e] = out
        return out

    # ------------------------------------------------------- cell matrices
    def cell_matrix(self, e, terms=("T", "L", "G", "K"), rows=None):
        """H^(e) = T + L + G - iK (eq. Hloccell), real when k = 0; optionally only rows `rows`."""
        c = self.cell(e)
        wd, B, g = c["wdet"], c["B"], c["g"]
        sel = slice(None) if rows is None else np.asarray(rows)
        k = self.kpt
        H = np.zeros((B[:, sel].shape[1], B.shape[1]))
        if "T" in terms:
            for d in range(3):
                H += 0.5 * g[d][:, sel].T @ (wd[:, None] * g[d])
        if "L" in terms:
            VL = self.vloc(c["x"]) + 0.5 * float(k @ k)
            H += B[:, sel].T @ ((wd * VL)[:, None] * B)
        if "G" in terms and self.vgga is not None:
            VG = self.vgga(c["x"])                              # [Q,3]
            gv = np.einsum("qc,cqi->qi", VG, g)                 # V^G . grad N_I at Q
            H += gv[:, sel].T @ (wd[:, None] * B)               # int (V^G.grad N_I) N_J
            H += B[:, sel].T @ (wd[:, None] * gv)               # int N_I (V^G.grad N_J)
        if self.complex:
            H = H.astype(np.complex128)
            if "K" in terms:
                kg = np.einsum("c,cqi->qi", k, g)               # k . grad N_J at Q
                H -= 1j * (B[:, sel].T @ (wd[:, None] * kg))    # int N_I (k . grad N_J)
        return H

    def mass_matrix(self, e):
        c = self.cell(e, grads=False)
        return c["B"].T @ (c["wdet"][:, None] * c["B"])

    # ------------------------------------------------------------ nonlocal
    def atom_cells(self, a):
        """Cells whose centroid is within rc + cell radius of some image of atom a."""
        cen = self.verts.mean(axis=1)
        rad = np.max(np.linalg.norm(self.verts - cen[:, None, :], axis=-1), axis=1)
        imgs = lattice_images(self.wl.L)
        d = np.linalg.norm(cen[:, None, :] - (self.R[a] + imgs)[None], axis=-1)
        return np.nonzero(np.min(d - rad[:, None], axis=1) < PROJ_RC)[0]

    def projector_matrix(self, a, e):
        """F^(a,e)[I, b] = int_e sum_r exp(-ik.(x-L_r)) chi_b(x - R_a - L_r) N_I dx."""
        c = self.cell(e, grads=False)
        x = c["x"]
        acc = np.zeros((x.shape[0], 9), dtype=np.complex128 if self.complex else np.float64)
        for Lr in lattice_images(self.wl.L):
            chi = projector_values(x - self.R[a] - Lr)
            if not np.any(chi):
                continue
            if self.complex:
                ph = np.exp(-1j * ((x - Lr) @ self.kpt))
                acc += ph[:, None] * chi
            else:
                acc += chi
        return c["B"].T @ (c["wdet"][:, None] * acc)            # [I, 9]

    def projector_block(self, a):
        """(a, cells, [F^(a,e) for e in cells]) for atom a (cached)."""
        if not hasattr(self, "_proj"):
            self._proj = {}
        if a not in self._proj:
            cells = self.atom_cells(a)
            self._proj[a] = (a, cells, [self.projector_matrix(a, e) for e in cells])
        return self._proj[a]

    def projector_blocks(self):
        """[(a, cells, [F^(a,e)])] for all atoms."""
        return [self.projector_block(a) for a in range(self.R.shape[0])]

    # -------------------------------------------------------------- action
    def apply(self, X, local=True, nonlocal_=True, cells=None):
        """Y = H X by the cell-matrix method (exact up to rounding)."""
        X = np.asarray(X)
        dt = np.complex128 if (self.complex or np.iscomplexobj(X)) else np.float64
        Y = np.zeros(X.shape, dtype=dt)
        if local:
            for e in (range(self.E) if cells is None else cells):
                d = self.dofs[e]
                Y[d] += self.cell_matrix(e) @ X[d]
        if nonlocal_ and self.R.shape[0] > 0:
            for a, cl, Fs in self.projector_blocks():
                P = sum(F.conj().T @ X[self.dofs[e]] for e, F in zip(cl, Fs))
                P = self.h[a][:, None] * P
                for e, F in zip(cl, Fs):
                    Y[self.dofs[e]] += F @ P
        return Y

    def apply_rows(self, X, rows):
        """Rows Y[rows, :] of Y = H X, computed only from the cells touching them.

        X may be any object with ``shape``, ``dtype`` and row indexing ``X[idx]``.
        """
        if not hasattr(X, "dtype"):
            X = np.asarray(X)
        rows = np.asarray(rows)
        dt = np.complex128 if (self.complex or np.issubdtype(X.dtype, np.complexfloating)) else np.float64
        out = np.zeros((rows.size, X.shape[1]), dtype=dt)
        pos = {int(r): i for i, r in enumerate(rows)}
        hit = np.isin(self.dofs, rows)
        for e in np.nonzero(hit.any(axis=1))[0]:
            loc = np.nonzero(hit[e])[0]
            contrib = self.cell_matrix(e, rows=loc) @ X[self.dofs[e]]
            for li, row in zip(loc, contrib):
                out[pos[int(self.dofs[e][li])]] += row
        if self.R.shape[0] > 0:
            hit_cells = np.nonzero(hit.any(axis=1))[0]
            for a in range(self.R.shape[0]):
                if not np.isin(self.atom_cells(a), hit_cells).any():
                    continue
                _, cl, Fs = self.projector_block(a)
                touch = [i for i, e in enumerate(cl) if hit[e].any()]
                P = sum(F.conj().T @ X[self.dofs[e]] for e, F in zip(cl, Fs))
                P = self.h[a][:, None] * P
                for i in touch:
                    e, F = cl[i], Fs[i]
                    loc = np.nonzero(hit[e])[0]
                    contrib = F[loc] @ P
                    for li, row in zip(loc, contrib):
                        out[pos[int(self.dofs[e][li])]] += row
        return out

    # ---------------------------------------------------- assembled matrices
    def assemble(self, what="H"):
        """Assembled sparse matrix (scipy CSR): 'H' (local + nonlocal) or 'M'."""
        import scipy.sparse as sp
        rows, cols, vals = [], [], []
        for e in range(self.E):
            d = self.dofs[e]
            A = self.cell_matrix(e) if what == "H" else self.mass_matrix(e)
            rows.append(np.repeat(d, d.size))
            cols.append(np.tile(d, d.size))
            vals.append(A.ravel())
        A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.m, self.m))
        if what == "H" and self.R.shape[0] > 0:
            for a, cl, Fs in self.projector_blocks():
                F = np.zeros((self.m, 9), dtype=np.complex128 if self.complex else np.float64)
                for e, Fe in zip(cl, Fs):
                    F[self.dofs[e]] += Fe
                nz = np.nonzero(np.any(F != 0, axis=1))[0]
                Fz = F[nz]
                blk = Fz @ (self.h[a][:, None] * Fz.conj().T)
                A = A + sp.csr_matrix((blk.ravel(), (np.repeat(nz, nz.size), np.tile(nz, nz.size))),
                                      shape=(self.m, self.m))
        return A.tocsr()

    def lumped_mass(self):
        """GLL-lumped mass D_I = sum_{e ni I} w^GLL_i w^GLL_j w^GLL_k det J(xi_I) (Algorithm 4's D)."""
        t, npn = self.t, self.np_
        li = np.arange(npn)
        kk, jj, ii = np.meshgrid(li, li, li, indexing="ij")
        ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
        xi = np.stack([t["xi_gll"][ii], t["xi_gll"][jj], t["xi_gll"][kk]], axis=1)
        w = t["w_gll"][ii] * t["w_gll"][jj] * t["w_gll"][kk]
        D = np.zeros(self.m)
        for e in range(self.E):
            _, J = self.trilinear(e, xi)
            np.add.at(D, self.dofs[e], w * np.linalg.det(J))
        return D
