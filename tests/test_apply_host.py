"""fe_ks_apply_host: Y = H X with host buffers, pipelined across calls.

Several calls with different inputs are in flight before one fe_ks_host_wait;
each result must equal, bit for bit, fe_ks_apply of the same input on device
buffers (same kernels, same colour order), and the oracle within the
fe_ks_apply tolerances.  Pinned and pageable host memory both work.
"""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from synth.host_problem import HostProblem
from oracle.operator import Problem
from synth import CONFIGS, trial_vectors
from gpu_util import gpu_apply, parity_err, round_input, torch_dtype

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {fk.FE_KS_F64: 1e-12, fk.FE_KS_F32: 1e-5}


@pytest.mark.parametrize("key,precision", [("C2s", fk.FE_KS_F64), ("C2s", fk.FE_KS_F32), ("C3s", fk.FE_KS_F64)])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_pipeline_matches_device_apply(key, precision, pinned):
    wl = {"C2s": CONFIGS["C2"].scaled(n=6, n_v=7),
          "C3s": CONFIGS["C3"].scaled(n=4, n_v=3, n_atoms=4)}[key]
    hp = HostProblem(wl)
    X0 = round_input(trial_vectors(wl), precision)
    inputs = [X0, 0.5 * X0 + 0.25, X0[::-1].copy()]            # three different blocks in flight
    inputs = [round_input(x, precision) for x in inputs]
    dt = torch_dtype(precision, hp.complex)
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, torch.cuda.current_stream().cuda_stream)
    try:
        wb = fk.fe_ks_apply_host_workspace(ctx, wl.n_v, precision)
        work = torch.empty(wb, dtype=torch.uint8, device="cuda")
        Xh = [torch.from_numpy(np.ascontiguousarray(x)).to(dt) for x in inputs]
        Yh = [torch.full_like(x, float("nan")) for x in Xh]
        if pinned:
            Xh = [x.pin_memory() for x in Xh]
            Yh = [y.pin_memory() for y in Yh]
        for x, y in zip(Xh, Yh):
            fk.fe_ks_apply_host(ctx, x, y, wl.n_v, precision, work, wb)
        fk.fe_ks_host_wait(ctx)
        with pytest.raises(fk.FeKsError, match="ERR_ARG"):
            fk.fe_ks_apply_host(ctx, Xh[0], Yh[0], wl.n_v, precision, work, wb - 256)
    finally:
        fk.fe_ks_destroy(ctx)
    P = Problem(wl)
    for x, y in zip(inputs, Yh):
        want = gpu_apply(hp, x, precision)
        got = y.numpy()
        assert np.array_equal(got, want)
        assert parity_err(got, P.apply(x)) <= TOL[precision]
