"""Seeded synthetic workloads (periodic hexahedral meshes, fields, atoms, X).

The paper's material benchmarks (Al nanoparticles, BCC Mo, benzamide, BCC Li
with DFT-FE meshes and pseudopotentials) are not available; these inputs stand
in for them with the paper's shapes: FE degree 4..8, n_q = n_p Gauss points,
real and complex (Bloch) operators, GGA term and l <= 2 separable projectors.

Conventions shared with the C interface:
  * cell e = cx + n (cy + n cz) on an n x n x n periodic grid of side L;
  * cell vertex slot v = a + 2 b + 4 c for the reference corner
    (xi, eta, zeta) = (2a-1, 2b-1, 2c-1); coordinates are unwrapped per cell
    (a cell on the +x face has vertices beyond L, not wrapped to 0);
  * cell node (i, j, k), i fastest, local index i + n_p (j + n_p k);
  * global DoF of node (I, J, K) on the (n p)^3 periodic node lattice is
    I + M (J + M K) with M = n p (periodic identification, no phase).
"""
import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload", "CONFIGS", "batched_systems", "make_mesh", "vloc_fn", "vgga_fn",
    "atoms", "projector_values", "atom_cell_pairs", "trial_vectors", "N_PROJ",
    "PROJ_L", "PROJ_RC", "PROJ_SIGMA", "lattice_images", "trial_chunk", "TRIAL_CHUNK",
]

N_PROJ = 9                     # l = 0, 1, 2 -> 1 + 3 + 5 real projectors
PROJ_L = np.array([0, 1, 1, 1, 2, 2, 2, 2, 2])
PROJ_SIGMA = 0.8               # bohr, Gaussian radial width
PROJ_RC = 2.5                  # bohr, hard support radius


@dataclass
class Workload:
    name: str
    L: float                   # periodic cube side (bohr)
    n: int                     # cells per direction
    p: int                     # FE degree (n_p = p + 1)
    nq: int                    # Gauss points per direction
    n_v: int                   # vectors
    jitter: float = 0.0        # vertex jitter as a fraction of h
    kfrac: tuple = (0.0, 0.0, 0.0)   # k = kfrac * 2 pi / L
    gga: bool = False
    n_atoms: int = 0
    complex: bool = False
    seed: int = 0
    precision: str = "f64"

    @property
    def h(self):
        return self.L / self.n

    @property
    def n_p(self):
        return self.p + 1

    @property
    def n_cells(self):
        return self.n ** 3

    @property
    def n_dofs(self):
        return (self.n * self.p) ** 3

    @property
    def kpt(self):
        return np.array(self.kfrac, dtype=np.float64) * 2.0 * math.pi / self.L

    def scaled(self, n=None, n_v=None, n_atoms=None, name=None):
        """Same recipe on a smaller grid / vector count (parity-sized cases)."""
        import dataclasses
        n = self.n if n is None else n
        return dataclasses.replace(
            self, n=n, L=self.h * n,
            n_v=self.n_v if n_v is None else n_v,
            n_atoms=self.n_atoms if n_atoms is None else n_atoms,
            name=name or f"{self.name}-n{n}")


CONFIGS = {
    "C1": Workload("C1", L=10.0, n=4, p=4, nq=5, n_v=8, seed=1000),
    "C2": Workload("C2", L=20.0, n=12, p=6, nq=7, n_v=64, jitter=0.1, gga=True,
                   n_atoms=16, seed=2000),
    "C3": Workload("C3", L=24.0, n=16, p=7, nq=8, n_v=128, kfrac=(0.25, 0.1, 0.0),
                   gga=True, n_atoms=32, complex=True, seed=3000),
    "C4": Workload("C4", L=30.0, n=24, p=8, nq=9, n_v=256, gga=True, n_atoms=64,
                   seed=4000),
    # all-electron-like: a Bloch-periodic complex operator without pseudopotential
    # projectors, few vectors on a large mesh (the regime of the paper's benzamide
    # and BCC Li runs, FEOrder 8, N_v = 64)
    "AE": Workload("AE", L=30.0, n=24, p=8, nq=9, n_v=64, kfrac=(0.25, 0.25, 0.25), gga=True,
                   complex=True, seed=6000),
}


def batched_systems():
    """Six independent periodic systems of uneven size, degree and N_v."""
    grids = (6, 8, 10, 12, 16, 20)
    degs = (4, 5, 6, 6, 7, 8)
    nvs = (16, 32, 64, 128, 256, 512)
    nat = (4, 12, 20, 28, 38, 48)
    prec = ("f64", "f32", "f64", "f32", "f64", "f32")
    return [Workload(f"C5.{s}", L=1.5 * grids[s], n=grids[s], p=degs[s], nq=degs[s] + 1,
                     n_v=nvs[s], gga=True, n_atoms=nat[s], seed=5000 + 100 * s,
                     precision=prec[s])
            for s in range(6)]


def _rng(wl, purpose):
    return np.random.default_rng(wl.seed + purpose)


def make_mesh(wl):
    """Return (vertices [E,8,3] float64, cell_dofs [E, n_p^3] int32, n_dofs)."""
    n, p, h = wl.n, wl.p, wl.h
    rng = _rng(wl, 1)
    jit = rng.uniform(-wl.jitter * h, wl.jitter * h, size=(n, n, n, 3)) if wl.jitter > 0 \
        else np.zeros((n, n, n, 3))
    c = np.arange(n)
    cz, cy, cx = np.meshgrid(c, c, c, indexing="ij")
    cx, cy, cz = cx.ravel(), cy.ravel(), cz.ravel()       # e = cx + n(cy + n cz)
    verts = np.empty((n ** 3, 8, 3))
    for v in range(8):
        a, b, cc = v & 1, (v >> 1) & 1, (v >> 2) & 1
        gx, gy, gz = cx + a, cy + b, cz + cc
        base = np.stack([gx, gy, gz], axis=1) * h
        verts[:, v, :] = base + jit[gz % n, gy % n, gx % n]
    M = n * p
    npn = p + 1
    li = np.arange(npn)
    kk, jj, ii = np.meshgrid(li, li, li, indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()        # local i fastest
    I = (cx[:, None] * p + ii[None, :]) % M
    J = (cy[:, None] * p + jj[None, :]) % M
    K = (cz[:, None] * p + kk[None, :]) % M
    dofs = (I + M * (J + M * K)).astype(np.int32)
    return verts, dofs, M ** 3


def lattice_images(L):
    """The 27 lattice vectors L_r with components in {-L, 0, L}."""
    r = np.array([-1.0, 0.0, 1.0]) * L
    g = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    return g


def vloc_fn(wl):
    """V_loc(x): sum of 4 seeded negative Gaussians, periodised over 27 images.

    The 27-image sum of an isotropic Gaussian factorises into a product over
    the three axes of 3-image 1D sums, which is how it is evaluated.
    """
    rng = _rng(wl, 2)
    A = rng.uniform(1.0, 5.0, 4)
    s = rng.uniform(0.5, 1.5, 4)
    c = rng.uniform(0.0, wl.L, (4, 3))
    shifts = np.array([-1.0, 0.0, 1.0]) * wl.L

    def f(x):
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros(x.shape[:-1])
        for g in range(4):
            prod = np.ones(x.shape[:-1])
            for ax in range(3):
                d = x[..., ax] - c[g, ax]
                acc = np.zeros(x.shape[:-1])
                for sh in shifts:
                    acc += np.exp(-(d - sh) ** 2 / (2.0 * s[g] ** 2))
                prod *= acc
            out -= A[g] * prod
        return out
    return f


def vgga_fn(wl):
    """V^G(x): smooth periodic vector field sum_j a_j sin(2 pi n_j.x / L + phi_j)."""
    if not wl.gga:
        return None
    rng = _rng(wl, 3)
    a = rng.uniform(-0.5, 0.5, (3, 3))
    choices = np.array([[i & 1, (i >> 1) & 1, (i >> 2) & 1] for i in range(1, 8)], dtype=float)
    nj = choices[rng.integers(0, 7, 3)]
    phi = rng.uniform(0.0, 2 * math.pi, 3)

    def f(x):
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros(x.shape[:-1] + (3,))
        for j in range(3):
            arg = 2 * math.pi * (x @ nj[j]) / wl.L + phi[j]
            out += np.sin(arg)[..., None] * a[j]
        return out
    return f


def atoms(wl):
    """Atom positions [A,3] in the box and projector coefficients h [A, 9].

    One coefficient per (atom, l), uniform in [-2, 2] Ha, shared over m.
    """
    rng = _rng(wl, 4)
    R = rng.uniform(0.0, wl.L, (wl.n_atoms, 3))
    hl = rng.uniform(-2.0, 2.0, (wl.n_atoms, 3))
    h = hl[:, PROJ_L]
    return R, h


def projector_values(d):
    """chi_lm(d) for displacement d [...,3] from the atom: [..., 9].

    Radial part g(r) = exp(-r^2 / (2 sigma^2)) (1 - (r/rc)^2)^3 for r < rc, 0
    otherwise (smooth compact support, sigma = 0.8, rc = 2.5 bohr), times the
    real solid harmonics r^l Y_lm for l = 0, 1, 2 with orthonormal Y_lm.
    """
    d = np.asarray(d, dtype=np.float64)
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    r2 = x * x + y * y + z * z
    t = np.clip(1.0 - r2 / PROJ_RC ** 2, 0.0, None)
    g = np.exp(-r2 / (2.0 * PROJ_SIGMA ** 2)) * t ** 3
    c0 = 0.5 / math.sqrt(math.pi)
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    c2 = 0.5 * math.sqrt(15.0 / math.pi)
    c20 = 0.25 * math.sqrt(5.0 / math.pi)
    c22 = 0.25 * math.sqrt(15.0 / math.pi)
    S = np.stack([
        np.full_like(x, c0),
        c1 * y, c1 * z, c1 * x,
        c2 * x * y, c2 * y * z, c20 * (3 * z * z - r2), c2 * x * z, c22 * (x * x - y * y),
    ], axis=-1)
    return g[..., None] * S


def atom_cell_pairs(wl, verts, R):
    """(atom, cell, image) triples that may meet an atom's projector support.

    Returns (atom_cell_ptr [A+1] int32, atom_cells [nnz] int32,
    image_shift [nnz,3]) in CSR order by atom.  A triple is listed when the
    image R_a + L_r of the atom lies within rc + (cell radius) of the cell
    centroid; on small boxes one cell can meet two images of the same atom and
    is then listed once per image.  The choice is conservative: cells outside
    the support only add zeros.
    """
    cen = verts.mean(axis=1)
    rad = np.max(np.linalg.norm(verts - cen[:, None, :], axis=-1), axis=1)
    imgs = lattice_images(wl.L)
    ptr, cells, shifts = [0], [], []
    for a in range(R.shape[0]):
        d = cen[:, None, :] - (R[a][None, None, :] + imgs[None, :, :])
        dist = np.linalg.norm(d, axis=-1)                 # [E, 27]
        ce, im = np.nonzero(dist < PROJ_RC + rad[:, None])
        cells.extend(ce.tolist())
        shifts.extend(imgs[im].tolist())
        ptr.append(len(cells))
    return (np.array(ptr, dtype=np.int32), np.array(cells, dtype=np.int32),
            np.array(shifts, dtype=np.float64).reshape(-1, 3))


TRIAL_CHUNK = 1 << 16


def trial_vectors(wl, n_v=None, seed_purpose=5, rows=None, dtype=np.float64):
    """X [m, n_v], entries uniform in [-1, 1] (complex: re and im independent).

    Rows are drawn in fixed chunks of 65536 rows, chunk c from
    default_rng(seed + purpose + 7919 c), so any subset of rows (``rows``) or
    any chunk can be regenerated without drawing the whole matrix.
    """
    n_v = wl.n_v if n_v is None else n_v
    m = wl.n_dofs
    if rows is None:
        out = np.empty((m, n_v), dtype=np.complex128 if wl.complex else dtype)
        for c0 in range(0, m, TRIAL_CHUNK):
            out[c0:c0 + TRIAL_CHUNK] = trial_chunk(wl, n_v, c0 // TRIAL_CHUNK, seed_purpose)
        return out
    rows = np.asarray(rows)
    out = np.empty((rows.size, n_v), dtype=np.complex128 if wl.complex else np.float64)
    chunks = rows // TRIAL_CHUNK
    for c in np.unique(chunks):
        blk = trial_chunk(wl, n_v, int(c), seed_purpose)
        sel = chunks == c
        out[sel] = blk[rows[sel] - int(c) * TRIAL_CHUNK]
    return out


def trial_chunk(wl, n_v, c, seed_purpose=5):
    """Rows [c*65536, min(m, (c+1)*65536)) of the trial block X."""
    rng = np.random.default_rng(wl.seed + seed_purpose + 7919 * c)
    r = min(wl.n_dofs, (c + 1) * TRIAL_CHUNK) - c * TRIAL_CHUNK
    X = rng.uniform(-1.0, 1.0, (r, n_v))
    if wl.complex:
        X = X + 1j * rng.uniform(-1.0, 1.0, (r, n_v))
    return X
