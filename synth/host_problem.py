"""Assemble an ``fe_ks_problem`` from a seeded synthetic workload.

The caller's side of the interface, used by the tests, the benchmark and the
smoke run: mesh arrays from the generators of this folder, quadrature points
from the library (``fe_ks_quadrature_points``), the synthetic fields evaluated
there, and the atom/cell/image triples with projector values at the library's
quadrature points.  It holds none of the method's arithmetic.  It is not
imported by ``synth/__init__`` (the oracle imports that package and must not
load the GPU library).
"""
import numpy as np

from paper_2512_08571_gb300 import fe_ks as _fk
from .workloads import (make_mesh, vloc_fn, vgga_fn, atoms, projector_values, atom_cell_pairs, N_PROJ)


class HostProblem:
    """Owns the numpy arrays behind a ``fe_ks_problem`` struct."""

    def __init__(self, wl, with_atoms=True, vloc=None, vgga="wl", R=None, h=None, kpt=None):
        self.wl = wl
        self.verts, self.dofs, self.m = make_mesh(wl)
        self.verts = np.ascontiguousarray(self.verts, dtype=np.float64)
        self.dofs = np.ascontiguousarray(self.dofs, dtype=np.int32)
        self.kpt = np.asarray(wl.kpt if kpt is None else kpt, dtype=np.float64)
        s = _fk.fe_ks_problem()
        s.n_cells, s.n_dofs, s.degree, s.n_q = self.verts.shape[0], self.m, wl.p, wl.nq
        s.cell_vertices = self.verts.ctypes.data
        s.cell_dofs = self.dofs.ctypes.data
        xq = _fk.fe_ks_quadrature_points(s)
        self.xq = xq
        vl = vloc_fn(wl) if vloc is None else vloc
        self.v_loc_q = np.ascontiguousarray(vl(xq), dtype=np.float64)
        vg = vgga_fn(wl) if isinstance(vgga, str) else vgga
        self.v_gga_q = None if vg is None else np.ascontiguousarray(vg(xq), dtype=np.float64)
        s.v_loc_q = self.v_loc_q.ctypes.data
        s.v_gga_q = None if self.v_gga_q is None else self.v_gga_q.ctypes.data
        for d in range(3):
            s.kpt[d] = float(self.kpt[d])
        s.force_complex = int(bool(wl.complex))
        if R is None and with_atoms and wl.n_atoms > 0:
            R, h = atoms(wl)
        if R is not None and len(R) > 0:
            self.R = np.asarray(R, dtype=np.float64).reshape(-1, 3)
            self.h = np.ascontiguousarray(np.asarray(h, dtype=np.float64).reshape(-1, N_PROJ))
            ptr, cells, shifts = atom_cell_pairs(wl, self.verts, self.R)
            self.atom_cell_ptr = np.ascontiguousarray(ptr, dtype=np.int32)
            self.atom_cells = np.ascontiguousarray(cells, dtype=np.int32)
            self.image_shift = np.ascontiguousarray(shifts, dtype=np.float64)
            atom_of = np.repeat(np.arange(len(self.R)), np.diff(ptr))
            disp = xq[cells] - (self.R[atom_of] + shifts)[:, None, :]
            self.chi_q = np.ascontiguousarray(projector_values(disp), dtype=np.float64)
            s.n_atoms, s.n_proj = len(self.R), N_PROJ
            s.atom_cell_ptr = self.atom_cell_ptr.ctypes.data
            s.atom_cells = self.atom_cells.ctypes.data
            s.image_shift = self.image_shift.ctypes.data
            s.chi_q = self.chi_q.ctypes.data
            s.h_coef = self.h.ctypes.data
        else:
            self.R = np.zeros((0, 3))
            s.n_atoms, s.n_proj = 0, N_PROJ
        self.struct = s

    @property
    def complex(self):
        return bool(self.wl.complex) or bool(np.any(self.kpt != 0))


def mass_problem(wl):
    """The same mesh as ``HostProblem(wl)`` with V_loc = 1 - |k|^2/2, no GGA field and
    no atoms: set up with terms = FE_KS_TERM_L its application is the consistent
    mass matrix M (the L term's (V_loc + |k|^2/2) det J w becomes det J w)."""
    import numpy as _np
    k2 = 0.5 * float(_np.dot(_np.asarray(wl.kpt, dtype=float), _np.asarray(wl.kpt, dtype=float)))
    return HostProblem(wl, with_atoms=False, vloc=lambda xq: _np.full(xq.shape[:-1], 1.0 - k2), vgga=None)
