"""The C ABI loads, exports every entry point the header declares, and rejects
bad problems on the host before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from synth.host_problem import HostProblem
from oracle.operator import Problem
from synth import CONFIGS, Workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"\b(fe_ks_\w+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    lib = ctypes.CDLL(fk.LIB_PATH)
    names = _declared()
    assert "fe_ks_apply" in names and "fe_ks_setup" in names
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("nqx", [0, 2])
def test_quadrature_points_match_oracle_geometry(nqx):
    import dataclasses
    wl = CONFIGS["C2"].scaled(n=3)
    wl = dataclasses.replace(wl, nq=wl.p + 1 + nqx)
    hp = HostProblem(wl)
    P = Problem(wl)
    for e in (0, 7, 26):
        np.testing.assert_allclose(hp.xq[e], P.cell(e, grads=False)["x"], atol=1e-13)


def _struct(wl):
    return HostProblem(Workload(wl.name, L=wl.L, n=wl.n, p=wl.p, nq=wl.nq, n_v=1, seed=wl.seed))


def test_setup_rejects_bad_problems_on_host():
    hp = _struct(CONFIGS["C1"])
    s = hp.struct
    with pytest.raises(fk.FeKsError, match="UNSUPPORTED"):
        s.n_q = s.degree + 2      # only n_q = n_p and n_p + 2 are built
        fk.fe_ks_setup(s, fk.TERM_ALL, 1)
    s.n_q = s.degree + 1
    with pytest.raises(fk.FeKsError, match="ERR_ARG"):
        fk.fe_ks_setup(s, fk.TERM_ALL, 0)
    bad = hp.dofs.copy()
    bad[3, 5] = hp.m
    s.cell_dofs = bad.ctypes.data
    with pytest.raises(fk.FeKsError, match="MESH"):
        fk.fe_ks_setup(s, fk.TERM_ALL, 1)
    dup = hp.dofs.copy()
    dup[2, 1] = dup[2, 0]
    s.cell_dofs = dup.ctypes.data
    with pytest.raises(fk.FeKsError, match="twice"):
        fk.fe_ks_setup(s, fk.TERM_ALL, 1)
    s.cell_dofs = hp.dofs.ctypes.data
    with pytest.raises(fk.FeKsError, match="ERR_ARG"):
        fk.fe_ks_apply(None, None, None, 1, fk.FE_KS_F64)
