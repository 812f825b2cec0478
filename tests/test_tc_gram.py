"""FP64-accurate Gram products and rotations on the tensor cores (fe_ks_gram_tc_sym, fe_ks_rotate_tc).

The Rayleigh-Ritz step (Algorithm 3) needs Y^T Y and Y^T H Y to FP64 accuracy.
The tensor-core kernel cuts every FP64 value into exact 8-bit slices relative to
its column's largest exponent over 32 rows and adds the slice products so that
the leading sums are exact; its error is about 2^-48 of sum_r |Y_ri Z_rj|.
Checked against numpy's FP64 product (itself within ~1e-15 of that sum at these
sizes) and against the library's pair-of-floats Gram kernel, at 1e-13 of
sum_r |Y_ri Z_rj| per entry, for blocks whose columns span many orders of
magnitude inside a chunk, with ragged row and column counts and several tiles,
plus exact symmetry and bitwise reproducibility.
"""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _blocks(m, n, seed, spread):
    rng = np.random.default_rng(seed)
    Y = rng.uniform(-1, 1, (m, n))
    # each row scaled by 10^U(-spread, 0): values of one column span `spread` decades inside a chunk
    Y *= 10.0 ** rng.uniform(-spread, 0.0, (m, 1))
    Z = Y @ np.diag(rng.uniform(0.5, 2.0, n)) + 1e-3 * rng.uniform(-1, 1, (m, n))   # Y^T Z symmetric-ish
    return Y, Z


@pytest.mark.parametrize("m,n,spread", [(70000, 130, 0.0), (40001, 256, 6.0), (8192 * 3 + 17, 77, 12.0)])
def test_tc_gram_matches_fp64_and_pair_kernel(m, n, spread):
    Y, Z = _blocks(m, n, 11 + n, spread)
    Zs = 0.5 * (Z + Y)           # any Z: the kernel computes every entry of the tiles it covers;
    Yd, Zd = torch.from_numpy(Y).cuda(), torch.from_numpy(Y.copy()).cuda()   # symmetric: Y^T Y
    C, status = fk.fe_ks_gram_tc_sym(Yd, Zd)
    assert status == 0
    C = C.cpu().numpy()
    ref = Y.T @ Y
    scale = np.abs(Y).T @ np.abs(Y)
    assert np.max(np.abs(C - ref) / scale) <= 1e-13
    assert np.array_equal(C, C.T)
    Cff = fk.fe_ks_gram_ff(Yd, Zd, symmetric=True).cpu().numpy()
    assert np.max(np.abs(C - Cff) / scale) <= 1e-13
    C2, _ = fk.fe_ks_gram_tc_sym(Yd, Zd)
    assert np.array_equal(C, C2.cpu().numpy())          # deterministic
    del Zs


def test_tc_gram_of_a_general_product_on_its_upper_triangle():
    """Y^T Z with Z != Y: the upper triangle (i <= j) is the product's, mirrored."""
    m, n = 50000, 140
    Y, Z = _blocks(m, n, 5, 3.0)
    C, status = fk.fe_ks_gram_tc_sym(torch.from_numpy(Y).cuda(), torch.from_numpy(Z).cuda())
    assert status == 0
    C = C.cpu().numpy()
    ref = Y.T @ Z
    scale = np.abs(Y).T @ np.abs(Z)
    iu = np.triu_indices(n)
    assert np.max(np.abs(C[iu] - ref[iu]) / scale[iu]) <= 1e-13


def test_tc_gram_zero_columns_and_out_of_range_scale():
    m, n = 9000, 40
    rng = np.random.default_rng(3)
    Y = rng.uniform(-1, 1, (m, n))
    Y[:, 7] = 0.0
    C, status = fk.fe_ks_gram_tc_sym(torch.from_numpy(Y).cuda(), torch.from_numpy(Y).cuda())
    assert status == 0
    C = C.cpu().numpy()
    assert np.all(C[7] == 0.0) and np.all(C[:, 7] == 0.0)
    # columns near 2^-70: the chunk scale leaves the FP32 range; the status says so
    Yt = Y * 2.0 ** -70
    _, status = fk.fe_ks_gram_tc_sym(torch.from_numpy(Yt).cuda(), torch.from_numpy(Yt).cuda())
    assert status & 2


@pytest.mark.parametrize("m,n,k,spread", [(30001, 256, 256, 0.0), (5000, 77, 130, 8.0)])
def test_tc_rotation_matches_fp64_and_pair_kernel(m, n, k, spread):
    """X = Y E with E a dense n x k block (as the Rayleigh-Ritz rotation's eigenvector
    matrix): within 1e-13 of sum_l |Y_rl E_lj| of numpy's FP64 product and of the
    pair-of-floats kernel, deterministic."""
    rng = np.random.default_rng(9 + n)
    Y = rng.uniform(-1, 1, (m, n)) * 10.0 ** rng.uniform(-spread, 0.0, (1, n))
    E = np.linalg.qr(rng.standard_normal((n, max(n, k))))[0][:, :k] if k <= n else rng.standard_normal((n, k))
    Yd, Ed = torch.from_numpy(Y).cuda(), torch.from_numpy(np.ascontiguousarray(E)).cuda()
    X, flags = fk.fe_ks_rotate_tc(Yd, Ed)
    assert flags == [0, 0]
    X = X.cpu().numpy()
    scale = np.abs(Y) @ np.abs(E)
    assert np.max(np.abs(X - Y @ E) / scale) <= 1e-13
    Xff = fk.fe_ks_rotate_ff(Yd, Ed).cpu().numpy()
    assert np.max(np.abs(X - Xff) / scale) <= 1e-13
    X2, _ = fk.fe_ks_rotate_tc(Yd, Ed)
    assert np.array_equal(X, X2.cpu().numpy())
