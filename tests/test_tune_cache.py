"""The tile-configuration cache: a context of the same shape picks up another
context's tuned configuration at its next application, unless its own was
set explicitly; the choice never changes the result beyond rounding."""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from synth.host_problem import HostProblem
from synth import CONFIGS, trial_vectors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_tuned_configuration_is_shared_by_same_shape_contexts():
    wl = CONFIGS["C4"].scaled(n=4, n_v=16, n_atoms=3)
    hp = HostProblem(wl)
    st = torch.cuda.current_stream().cuda_stream
    X = torch.from_numpy(trial_vectors(wl).astype(np.float32)).cuda()
    Y = torch.empty_like(X)
    a = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, st)
    b = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, st)
    c = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, st)
    try:
        fk.fe_ks_set_config(c, fk.FE_KS_F32, 2)                 # explicit: keeps its own
        best, ms = fk.fe_ks_tune(a, X, Y, wl.n_v, fk.FE_KS_F32, reps=1)
        assert fk.fe_ks_get_config(a, fk.FE_KS_F32) == best
        assert fk.fe_ks_get_config(b, fk.FE_KS_F32) == 0        # not applied yet
        fk.fe_ks_apply(b, X, Y, wl.n_v, fk.FE_KS_F32)
        assert fk.fe_ks_get_config(b, fk.FE_KS_F32) == best
        Yc = torch.empty_like(X)
        fk.fe_ks_apply(c, X, Yc, wl.n_v, fk.FE_KS_F32)
        assert fk.fe_ks_get_config(c, fk.FE_KS_F32) == 2
        torch.cuda.synchronize()
        d = (Y - Yc).norm(dim=0) / Yc.norm(dim=0)
        assert float(d.max()) < 1e-5
    finally:
        for ctx in (a, b, c):
            fk.fe_ks_destroy(ctx)
