"""Bad input values (fault injection on the host side): a NaN planted in one
entry of X reaches only the rows of Y whose cells touch that DoF, in that
column; every other entry equals the clean application bit for bit (the
columns are independent, the FP16 scale is per column), and the context
stays usable afterwards.
"""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from synth.host_problem import HostProblem
from synth import CONFIGS, trial_vectors
from gpu_util import round_input, torch_dtype

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [fk.FE_KS_F64, fk.FE_KS_F32, fk.FE_KS_BF16, fk.FE_KS_F16, fk.FE_KS_BF16X2])
def test_nan_in_x_stays_local(precision):
    wl = CONFIGS["C1"].scaled(n=3, n_v=3)
    hp = HostProblem(wl)
    X = round_input(trial_vectors(wl), precision)
    r0, col = 17, 1
    touched = np.unique(hp.dofs[np.any(hp.dofs == r0, axis=1)].ravel())
    dt = torch_dtype(precision, hp.complex)
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, torch.cuda.current_stream().cuda_stream)
    try:
        Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda().to(dt)
        clean = torch.empty_like(Xd)
        fk.fe_ks_apply(ctx, Xd, clean, wl.n_v, precision)
        Xbad = Xd.clone()
        Xbad[r0, col] = float("nan")
        Y = torch.empty_like(Xd)
        fk.fe_ks_apply(ctx, Xbad, Y, wl.n_v, precision)
        again = torch.empty_like(Xd)
        fk.fe_ks_apply(ctx, Xd, again, wl.n_v, precision)      # the context is still usable
        torch.cuda.synchronize()
        Y, clean, again = Y.cpu().numpy(), clean.cpu().numpy(), again.cpu().numpy()
    finally:
        fk.fe_ks_destroy(ctx)
    assert np.array_equal(again, clean)
    nan_rows = np.nonzero(np.isnan(Y[:, col]))[0]
    assert r0 in nan_rows and set(nan_rows.tolist()) <= set(touched.tolist())
    keep = np.ones(Y.shape, dtype=bool)
    keep[touched, col] = False
    assert np.array_equal(Y[keep], clean[keep])
