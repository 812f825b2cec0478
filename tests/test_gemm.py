"""Rayleigh-Ritz GEMMs through cuBLAS (native FP64 and its FP64 emulation)
against torch's FP64 matmul on the same device arrays."""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("emulated", [False, True])
def test_row_gram_and_rotate(emulated):
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    Y = torch.rand((20000, 48), generator=g, device="cuda", dtype=torch.float64) * 2 - 1
    Z = torch.rand((20000, 48), generator=g, device="cuda", dtype=torch.float64) * 2 - 1
    E = torch.rand((48, 40), generator=g, device="cuda", dtype=torch.float64) * 2 - 1
    try:
        C = fk.row_gram(Y, Z, emulated=emulated)
    except fk.FeKsError as exc:
        if emulated and "UNSUPPORTED" in str(exc):
            pytest.skip("cuBLAS FP64 emulation not available on this device")
        raise
    ref = Y.T @ Z
    scale = (Y.abs().T @ Z.abs()).max().item()
    assert (C - ref).abs().max().item() <= 1e-13 * scale
    X = fk.row_rotate(Y, E, emulated=emulated)
    refx = Y @ E
    assert (X - refx).abs().max().item() <= 1e-13 * (Y.abs() @ E.abs()).max().item()
