"""Full-size parity on sampled rows: the workloads at their benchmark sizes
(C2: 12^3 cells p=6 N_v=64; C3: 16^3 p=7 complex N_v=128; C4: 24^3 p=8 N_v=256;
AE: 24^3 p=8 complex without projectors, N_v=64), every precision including
the 16-bit tensor-core ones,
applied on the GPU in the benchmark's launch configuration, compared with the
oracle's row-restricted evaluation: all nodes of one cell (interior, face, edge
and corner DoFs) plus interior nodes of six random cells.  Tolerances as in
test_parity_apply (per column over the sampled rows)."""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from paper_2512_08571_gb300.problem import HostProblem
from oracle.operator import Problem
from synth import CONFIGS
from gpu_util import RowCache, needed_rows, fill_device, rel_err_cols, torch_dtype

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {fk.FE_KS_F64: 1e-12, fk.FE_KS_F32: 1e-5, fk.FE_KS_F64E: 1e-12,
       fk.FE_KS_BF16: 2.0 ** -5, fk.FE_KS_F16: 2.0 ** -8}   # 8 u of the 16-bit types (test_parity_bf16)


def _rows(P, wl, seed):
    rng = np.random.default_rng(seed)
    e0 = int(rng.integers(P.E))
    npn = wl.p + 1
    rows = [P.dofs[e0]] + [P.dofs[e][[npn * npn + npn + 1]] for e in rng.integers(0, P.E, 6)]
    return np.unique(np.concatenate(rows))


@pytest.mark.parametrize("key", ["C2", "C3", "C4", "AE"])
def test_full_size_sampled_rows(key):
    wl = CONFIGS[key]
    hp = HostProblem(wl)
    P = Problem(wl)
    rows = _rows(P, wl, 7 + len(key))
    need = needed_rows(P, rows)
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, torch.cuda.current_stream().cuda_stream)
    try:
        for precision in (fk.FE_KS_F64, fk.FE_KS_F32, fk.FE_KS_F64E, fk.FE_KS_BF16, fk.FE_KS_F16):
            dt = torch_dtype(precision, hp.complex)
            X = torch.empty((hp.m, wl.n_v), dtype=dt, device="cuda")
            npdt = {torch.float64: np.float64, torch.float32: np.float32,
                    torch.complex128: np.complex128, torch.complex64: np.complex64}[dt]
            fill_device(wl, wl.n_v, X, npdt)
            Y = torch.full_like(X, float("nan"))
            fk.fe_ks_apply(ctx, X, Y, wl.n_v, precision)
            torch.cuda.synchronize()
            Yg = Y[torch.from_numpy(rows).cuda()].cpu().numpy()
            del X, Y
            torch.cuda.empty_cache()
            Xl = RowCache(wl, need, round_to=npdt)
            Yref = P.apply_rows(Xl, rows)
            err = rel_err_cols(Yg, Yref)
            assert err <= TOL[precision], (key, precision, err)
    finally:
        fk.fe_ks_destroy(ctx)
