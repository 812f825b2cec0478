"""Host colouring behind the race-free scatter-add (assembly Q^T of Algorithm 1,
one launch per colour).  Needs no GPU: fe_ks_colour_cells is host code.

Checked on the periodic meshes of the workloads (several grid sizes and
degrees) against the definition: every cell has a colour, no two cells of a
colour share a DoF, and greedy index-order colouring of a periodic grid with
an even number of cells per direction needs exactly 2^3 = 8 colours (27 for
3 cells per direction, where every cell touches every other).
"""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from synth import Workload, make_mesh


@pytest.mark.parametrize("n,p", [(2, 1), (3, 2), (4, 4), (4, 8), (5, 3), (6, 2), (8, 1)])
def test_colouring_is_conflict_free(n, p):
    wl = Workload(f"col{n}{p}", L=2.0 * n, n=n, p=p, nq=p + 1, n_v=1, jitter=0.05, seed=77 + n)
    _, dofs, m = make_mesh(wl)
    colour, nc = fk.fe_ks_colour_cells(dofs, m)
    assert colour.shape == (n ** 3,)
    assert colour.min() == 0 and colour.max() == nc - 1 and nc <= 64
    for c in range(nc):
        cells = np.nonzero(colour == c)[0]
        d = dofs[cells].ravel()
        assert np.unique(d).size == d.size, f"colour {c} shares a DoF"
    if n % 2 == 0 and n >= 4:
        assert nc == 8
    if n == 3:
        assert nc == 27


def test_colouring_is_greedy_minimal_per_cell():
    """Each cell's colour is the smallest not used by an earlier neighbour."""
    wl = Workload("colg", L=10.0, n=5, p=2, nq=3, n_v=1, seed=5)
    _, dofs, m = make_mesh(wl)
    colour, _ = fk.fe_ks_colour_cells(dofs, m)
    sets = [set(r.tolist()) for r in dofs]
    for e in range(len(sets)):
        used = {int(colour[o]) for o in range(e) if sets[o] & sets[e]}
        assert colour[e] == min(set(range(65)) - used)


def test_colouring_rejects_bad_tables():
    dofs = np.array([[0, 1], [1, 2]], dtype=np.int32)
    with pytest.raises(fk.FeKsError):
        fk.fe_ks_colour_cells(dofs, 2)          # entry 2 out of range
    with pytest.raises(fk.FeKsError):
        fk.fe_ks_colour_cells(np.zeros((0, 8), dtype=np.int32), 4)
