"""Rayleigh-Ritz GEMMs through cuBLAS (native FP64 and its FP64 emulation)
against torch's FP64 matmul on the same device arrays."""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _time(fn, reps=3):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


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


@pytest.mark.parametrize("m,n", [(20000, 48), (8192 * 3 + 77, 130)])
def test_symmetric_grams(m, n):
    """Y^T Y and Y^T (D Y) with D diagonal: the one-triangle pair-of-floats form equals the
    full product within the FP64-accurate bound and is exactly symmetric, and it equals the
    full pair-of-floats product bit for bit on and above the diagonal (130 = two 64-wide tiles
    and a ragged one)."""
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    Y = torch.rand((m, n), generator=g, device="cuda", dtype=torch.float64) * 2 - 1
    d = torch.rand((m, 1), generator=g, device="cuda", dtype=torch.float64) + 0.5
    # Sums of same-sign terms (the diagonal of Y^T Y) do not cancel, so the pair accumulator's
    # low word grows with the sum: its float roundings, renormalised every 4 terms, add about
    # sqrt(8192) x 2^-47 = 6.4e-13 of the sum over one 8192-row chunk; 1e-12 covers that.
    for Z in (Y, d * Y):            # Y^T Y and Y^T D Y: symmetric products
        ref = Y.T @ Z
        scale = (Y.abs().T @ Z.abs()).max().item()
        C = fk.fe_ks_gram_ff(Y, Z, symmetric=True)
        assert torch.equal(C, C.T)
        assert (C - ref).abs().max().item() <= 1e-12 * scale
        full = fk.fe_ks_gram_ff(Y, Z)
        sym = fk.fe_ks_gram_ff(Y, Z, symmetric=True)
        iu = torch.triu_indices(n, n, device="cuda")
        assert torch.equal(sym[iu[0], iu[1]], full[iu[0], iu[1]])
    with pytest.raises(fk.FeKsError, match="ERR_ARG"):
        fk._check(fk._lib.fe_ks_gram_ff_sym(None, None, None, m, n, None, 0, None))


def test_pair_of_floats_gram_and_rotation():
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    for m, n1, n2 in ((20000, 48, 48), (8192 * 3 + 77, 40, 70)):
        Y = torch.rand((m, n1), generator=g, device="cuda", dtype=torch.float64) * 2 - 1
        Z = torch.rand((m, n2), generator=g, device="cuda", dtype=torch.float64) * 2 - 1
        C = fk.fe_ks_gram_ff(Y, Z)
        ref = Y.T @ Z
        scale = (Y.abs().T @ Z.abs()).max().item()
        assert (C - ref).abs().max().item() <= 1e-13 * scale
        E = torch.rand((n1, n2), generator=g, device="cuda", dtype=torch.float64) * 2 - 1
        X = fk.fe_ks_rotate_ff(Y, E)
        refx = Y @ E
        assert (X - refx).abs().max().item() <= 1e-13 * (Y.abs() @ E.abs()).max().item()


def test_report_gram_speed():
    """Not a pass/fail check of speed: records native vs emulated FP64 Gram time."""
    Y = torch.rand((2_000_000, 256), device="cuda", dtype=torch.float64)
    nat = _time(lambda: fk.row_gram(Y, Y, emulated=False))
    try:
        emu = _time(lambda: fk.row_gram(Y, Y, emulated=True))
    except fk.FeKsError:
        emu = float("nan")
    pairs = _time(lambda: fk.fe_ks_gram_ff(Y, Y))
    E = torch.rand((256, 256), device="cuda", dtype=torch.float64)
    rot_nat = _time(lambda: Y @ E)
    rot_pairs = _time(lambda: fk.fe_ks_rotate_ff(Y, E))
    print(f"\nGram 2e6 x 256: native FP64 {nat:.1f} ms, emulated {emu:.1f} ms, pairs of floats {pairs:.1f} ms; "
          f"rotation: native {rot_nat:.1f} ms, pairs {rot_pairs:.1f} ms")
