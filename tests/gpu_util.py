"""Helpers shared by the GPU parity tests (test-side glue, no method arithmetic)."""
import numpy as np

from paper_2512_08571_gb300 import fe_ks as fk
from synth.host_problem import HostProblem


def rel_err_cols(Y, Yref):
    """max over columns of ||Y_v - Yref_v||_2 / ||Yref_v||_2."""
    num = np.linalg.norm(Y - Yref, axis=0)
    den = np.linalg.norm(Yref, axis=0)
    return float(np.max(num / np.maximum(den, 1e-300)))


def max_abs_rel(Y, Yref):
    """Element-wise error: max over entries (i, v) of |Y_iv - Yref_iv| / max_i |Yref_iv|.

    A wrong value at a few DoFs (one face or corner node, one atom-cell pair)
    hides under the square root of a column norm but not here."""
    num = np.abs(Y - Yref)
    den = np.max(np.abs(Yref), axis=0)
    return float(np.max(num / np.maximum(den, 1e-300)[None, :]))


def parity_err(Y, Yref):
    """The larger of the per-column norm error and the element-wise error: a parity
    tolerance asserted on this value holds for both."""
    Y, Yref = np.asarray(Y), np.asarray(Yref)
    return max(rel_err_cols(Y, Yref), max_abs_rel(Y, Yref))


def torch_dtype(precision, cplx):
    import torch
    if precision in (fk.FE_KS_F64, fk.FE_KS_F64E):
        return torch.complex128 if cplx else torch.float64
    return torch.complex64 if cplx else torch.float32


def round_input(X, precision):
    """The input the GPU actually sees, promoted back to FP64 for the oracle."""
    if precision in (fk.FE_KS_F32, fk.FE_KS_BF16, fk.FE_KS_F16, fk.FE_KS_BF16X2):   # FP32 storage
        return X.astype(np.complex64 if np.iscomplexobj(X) else np.float32).astype(
            np.complex128 if np.iscomplexobj(X) else np.float64)
    return X


def gpu_apply(hp, X, precision, scaled=False, terms=fk.TERM_ALL, repeat=1, config=None):
    import torch
    n_v = X.shape[1]
    ctx = fk.fe_ks_setup(hp.struct, terms, n_v, torch.cuda.current_stream().cuda_stream)
    try:
        if config is not None:
            fk.fe_ks_set_config(ctx, precision, config)
        dt = torch_dtype(precision, hp.complex)
        Xd = torch.from_numpy(np.ascontiguousarray(X)).to("cuda").to(dt)
        outs = []
        for _ in range(repeat):
            Yd = torch.full_like(Xd, float("nan"))
            (fk.fe_ks_apply_scaled if scaled else fk.fe_ks_apply)(ctx, Xd, Yd, n_v, precision)
            torch.cuda.synchronize()
            outs.append(Yd.cpu().numpy())
        return outs if repeat > 1 else outs[0]
    finally:
        fk.fe_ks_destroy(ctx)


class RowCache:
    """Rows of the seeded trial block X, generated once for a known row set.

    Supports ``X[idx]`` for global row indices inside the set, so the oracle's
    sampled-row evaluation can run at full size without materialising X.
    """

    def __init__(self, wl, rows, n_v=None, round_to=None):
        from synth import trial_vectors
        self.rows = np.unique(np.asarray(rows))
        vals = trial_vectors(wl, n_v=n_v, rows=self.rows)
        if round_to is not None:
            vals = vals.astype(round_to).astype(vals.dtype)
        self.vals = vals
        self.dtype = vals.dtype
        self.shape = (wl.n_dofs, vals.shape[1])

    def __getitem__(self, idx):
        pos = np.searchsorted(self.rows, np.asarray(idx))
        return self.vals[pos]


def needed_rows(P, rows):
    """Global rows the oracle reads to evaluate Y[rows] (touched cells and atom supports)."""
    rows = np.asarray(rows)
    hit = np.isin(P.dofs, rows).any(axis=1)
    cells = set(np.nonzero(hit)[0].tolist())
    for a in range(P.R.shape[0]):
        ac = P.atom_cells(a)
        if np.any(hit[ac]):
            cells |= set(ac.tolist())
    return np.unique(P.dofs[sorted(cells)])


def fill_device(wl, n_v, X_dev, dtype_np):
    """Copy the seeded trial block into a device tensor chunk by chunk."""
    import torch
    from synth import trial_chunk, TRIAL_CHUNK
    for c in range((wl.n_dofs + TRIAL_CHUNK - 1) // TRIAL_CHUNK):
        blk = trial_chunk(wl, n_v, c)
        r0 = c * TRIAL_CHUNK
        X_dev[r0:r0 + blk.shape[0]].copy_(torch.from_numpy(blk.astype(dtype_np)))
