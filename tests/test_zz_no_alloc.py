"""fe_ks_nonlocal_apply_static: the allocation-free nonlocal entry point.

It exists for callers that cannot call cudaMalloc (device memory owned by
another allocator, or a code path where an allocation would synchronise the
device or break a memory budget): they pass every input and output, and the
call keeps its scratch in a static device array.  Its output must equal the
existing entry point's nonlocal term (fe_ks_apply with FE_KS_TERM_NL only)
and the oracle's nonlocal term F diag(h) F^H X, within the FP64 tolerance of
the other parity tests (per column and element-wise), on two calls in a row
with different inputs; and the second call must leave the device's free
memory unchanged.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from synth.host_problem import HostProblem
from oracle.operator import Problem
from synth import CONFIGS, trial_vectors
from gpu_util import gpu_apply, parity_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tables(P):
    """Per-(atom, cell) projector matrices F^(a,e) [n_proj][node] and CSR tables."""
    ptr, cells, atom, Fs = [0], [], [], []
    for a in range(P.R.shape[0]):
        _, cl, Fa = P.projector_block(a)
        for e, F in zip(cl, Fa):
            cells.append(e)
            atom.append(a)
            Fs.append(np.ascontiguousarray(F.T))
        ptr.append(len(cells))
    F = np.stack(Fs)
    if np.iscomplexobj(F):
        F = np.ascontiguousarray(F).view(np.float64)     # interleaved (re, im)
    return (np.array(ptr, np.int32), np.array(cells, np.int32), np.array(atom, np.int32),
            np.ascontiguousarray(F, dtype=np.float64))


@pytest.mark.parametrize("wl", [CONFIGS["C2"].scaled(n=6, n_v=7),
                                CONFIGS["C3"].scaled(n=4, n_v=3, n_atoms=4)], ids=["real", "complex"])
def test_static_scratch_matches_existing_entry_point(wl):
    hp = HostProblem(wl)
    P = Problem(wl)
    ptr, cells, atom, F = _tables(P)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_dofs, d_ptr, d_cells, d_atom, d_F = dev(hp.dofs), dev(ptr), dev(cells), dev(atom), dev(F)
    d_h = dev(P.h.astype(np.float64))
    cplx = hp.complex
    stream = torch.cuda.current_stream().cuda_stream
    free_after = []
    for seed in (5, 6):                       # two calls in a row, different inputs
        X = trial_vectors(wl, seed_purpose=seed)
        want = gpu_apply(hp, X, fk.FE_KS_F64, terms=fk.TERM_NL)
        oracle_nl = P.apply(X, local=False, nonlocal_=True)
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.zeros_like(Xd)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        fk.fe_ks_nonlocal_apply_static(Xd, Yd, wl.n_v, cplx, wl.p, hp.m, d_dofs, P.R.shape[0], 9, d_ptr,
                                       d_cells, d_atom, len(cells), d_F, d_h, stream)
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info()[0] - free_before)
        got = Yd.cpu().numpy()
        err = parity_err(got, want)
        assert err <= 1e-12, (seed, err)
        err_o = parity_err(got, oracle_nl)
        assert err_o <= 1e-12, (seed, err_o)
    # the first call may load the module's kernels; the second allocates nothing at all
    assert free_after[1] == 0, free_after


def test_static_scratch_rejects_oversize():
    wl = CONFIGS["C2"].scaled(n=6, n_v=7)
    hp = HostProblem(wl)
    X = torch.zeros((hp.m, 4000), dtype=torch.float64, device="cuda")
    Y = torch.zeros_like(X)
    one = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(fk.FeKsError, match="static scratch"):
        fk.fe_ks_nonlocal_apply_static(X, Y, 4000, 0, wl.p, hp.m, one, 16, 9, one, one, one, 1,
                                       X, X, None)
