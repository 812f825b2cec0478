"""Batched persistent launch (many uneven systems in one kernel) on the GPU.

Systems follow the C5 recipe (degrees 4..8, uneven grids and vector counts,
FP64 / FP32 alternating, GGA + projectors) on parity-sized grids.  Each
system's result must equal its own fe_ks_apply (and, for FP64, the oracle),
for every tunable setting, when captured in a CUDA graph and replayed, and
the bounded waits must turn a never-published work item into
FE_KS_ERR_TIMEOUT without losing the context.
"""
import numpy as np
import pytest

from paper_2512_08571_gb300 import fe_ks as fk
from synth.host_problem import HostProblem
from oracle.operator import Problem
from synth import Workload, trial_vectors
from gpu_util import parity_err, torch_dtype

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRIDS = (2, 3, 2, 3, 2, 2)
DEGS = (4, 5, 6, 6, 7, 8)
NVS = (3, 5, 8, 6, 4, 7)
PREC = (fk.FE_KS_F64, fk.FE_KS_F32, fk.FE_KS_F64, fk.FE_KS_F32, fk.FE_KS_F64, fk.FE_KS_F32)
TOL = {fk.FE_KS_F64: 1e-12, fk.FE_KS_F32: 1e-5}


def _systems():
    return [Workload(f"b{s}", L=3.0 * GRIDS[s], n=GRIDS[s], p=DEGS[s], nq=DEGS[s] + 1, n_v=NVS[s], gga=True,
                     n_atoms=1 + s % 3, jitter=0.05 * (s % 2), seed=7000 + 10 * s) for s in range(6)]


@pytest.fixture(scope="module")
def batch_setup():
    stream = torch.cuda.current_stream().cuda_stream
    wls = _systems()
    hps = [HostProblem(wl) for wl in wls]
    ctxs = [fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, stream) for hp, wl in zip(hps, wls)]
    Xs, Ys, refs = [], [], []
    for s, (wl, hp, ctx) in enumerate(zip(wls, hps, ctxs)):
        dt = torch_dtype(PREC[s], False)
        X = torch.from_numpy(trial_vectors(wl)).cuda().to(dt)
        Y = torch.empty_like(X)
        fk.fe_ks_apply(ctx, X, Y, wl.n_v, PREC[s])
        Xs.append(X)
        Ys.append(torch.empty_like(X))
        refs.append(Y.clone())
    torch.cuda.synchronize()
    b = fk.fe_ks_batch_create(ctxs, [wl.n_v for wl in wls], list(PREC))
    yield wls, hps, ctxs, Xs, Ys, refs, b
    fk.fe_ks_batch_destroy(b)
    for c in ctxs:
        fk.fe_ks_destroy(c)


def _check(Ys, refs):
    for s, (Y, R) in enumerate(zip(Ys, refs)):
        err = parity_err(Y.double().cpu().numpy(), R.double().cpu().numpy())
        assert err <= TOL[PREC[s]], (s, err)


@pytest.mark.parametrize("tile,cells,depth,occ", [(0, 1, 1, 1), (1, 1, 1, 2), (0, 3, 2, 2), (1, 2, 4, 1)])
def test_batched_equals_individual_applications(batch_setup, tile, cells, depth, occ):
    wls, hps, ctxs, Xs, Ys, refs, b = batch_setup
    fk.fe_ks_batch_configure(b, [tile] * 6, cells, depth, 2.0, False, blocks_per_sm=occ)
    for Y in Ys:
        Y.fill_(float("nan"))
    fk.fe_ks_batch_apply(b, Xs, Ys, torch.cuda.current_stream().cuda_stream)
    fk.fe_ks_batch_status(b)
    _check(Ys, refs)


@pytest.mark.parametrize("threads,occ", [(384, 1), (512, 1), (512, 2), (672, 1)])
@pytest.mark.parametrize("cells", [1, 2])
def test_batched_block_sizes(batch_setup, threads, occ, cells):
    """Every block size the kernel is built for (the projection items' column width must
    divide it: 672 = 21 x 32), mixed tile configurations, ragged column counts."""
    wls, hps, ctxs, Xs, Ys, refs, b = batch_setup
    tiles = [(s // 2) % 2 for s in range(6)]
    fk.fe_ks_batch_configure(b, tiles, cells, 2, 2.0, False, blocks_per_sm=occ, threads=threads)
    for Y in Ys:
        Y.fill_(float("nan"))
    fk.fe_ks_batch_apply(b, Xs, Ys, torch.cuda.current_stream().cuda_stream)
    fk.fe_ks_batch_status(b)
    _check(Ys, refs)
    fk.fe_ks_batch_configure(b, [0] * 6, 1, 1, 2.0, False, threads=384)


def test_aligned_rows_and_wide_projection_items():
    """Column counts that are multiples of 4 and above 32 (64-column projection items),
    every block size, against each system's own fe_ks_apply."""
    stream = torch.cuda.current_stream().cuda_stream
    spec = [(5, 2, 8, fk.FE_KS_F32), (8, 2, 48, fk.FE_KS_F32), (6, 2, 40, fk.FE_KS_F64)]
    wls = [Workload(f"a{s}", L=6.0, n=n, p=p, nq=p + 1, n_v=nv, gga=True, n_atoms=2, seed=7500 + s)
           for s, (p, n, nv, _) in enumerate(spec)]
    hps = [HostProblem(wl) for wl in wls]   # owns the arrays behind each problem struct
    ctxs = [fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, stream) for hp, wl in zip(hps, wls)]
    try:
        Xs, Ys, refs = [], [], []
        for wl, ctx, (_, _, _, pr) in zip(wls, ctxs, spec):
            X = torch.from_numpy(trial_vectors(wl)).cuda().to(torch_dtype(pr, False))
            R = torch.empty_like(X)
            fk.fe_ks_apply(ctx, X, R, wl.n_v, pr)
            Xs.append(X)
            Ys.append(torch.full_like(X, float("nan")))
            refs.append(R)
        b = fk.fe_ks_batch_create(ctxs, [wl.n_v for wl in wls], [sp[3] for sp in spec])
        try:
            for threads, cells in ((384, 1), (512, 3), (672, 2)):
                for Y in Ys:
                    Y.fill_(float("nan"))
                fk.fe_ks_batch_configure(b, [1, 1, 0], cells, 2, 2.0, False, threads=threads)
                fk.fe_ks_batch_apply(b, Xs, Ys, stream)
                fk.fe_ks_batch_status(b)
                for (_, _, _, pr), Y, R in zip(spec, Ys, refs):
                    err = parity_err(Y.double().cpu().numpy(), R.double().cpu().numpy())
                    assert err <= TOL[pr], err
            with pytest.raises(fk.FeKsError, match="ERR_ARG"):
                fk.fe_ks_batch_configure(b, [2, 0, 0], 1, 1, 2.0, False)    # tile configurations 0 / 1
            with pytest.raises(fk.FeKsError, match="ERR_ARG"):
                fk.fe_ks_batch_configure(b, [0, 0, 0], 1, 1, 2.0, False, threads=256)
        finally:
            fk.fe_ks_batch_destroy(b)
    finally:
        for c in ctxs:
            fk.fe_ks_destroy(c)


def test_batched_fp64_systems_match_oracle(batch_setup):
    wls, hps, ctxs, Xs, Ys, refs, b = batch_setup
    fk.fe_ks_batch_configure(b, [0] * 6, 1, 1, 2.0, False)
    fk.fe_ks_batch_apply(b, Xs, Ys, torch.cuda.current_stream().cuda_stream)
    fk.fe_ks_batch_status(b)
    for s in (0, 2, 4):
        Yref = Problem(wls[s]).apply(Xs[s].cpu().numpy())
        assert parity_err(Ys[s].cpu().numpy(), Yref) <= 1e-12


def test_batched_launch_in_cuda_graph(batch_setup):
    wls, hps, ctxs, Xs, Ys, refs, b = batch_setup
    fk.fe_ks_batch_configure(b, [1] * 6, 2, 2, 2.0, False)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fk.fe_ks_batch_apply(b, Xs, Ys, side.cuda_stream)      # warm-up outside capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        fk.fe_ks_batch_apply(b, Xs, Ys, torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        for Y in Ys:
            Y.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        fk.fe_ks_batch_status(b)
        _check(Ys, refs)


def test_bounded_wait_reports_timeout_and_recovers(batch_setup):
    wls, hps, ctxs, Xs, Ys, refs, b = batch_setup
    fk.fe_ks_batch_configure(b, [0] * 6, 1, 1, 0.02, True)   # one phase-0 item never arrives
    fk.fe_ks_batch_apply(b, Xs, Ys, torch.cuda.current_stream().cuda_stream)
    with pytest.raises(fk.FeKsError, match="TIMEOUT"):
        fk.fe_ks_batch_status(b)
    fk.fe_ks_batch_configure(b, [0] * 6, 1, 1, 2.0, False)
    fk.fe_ks_batch_apply(b, Xs, Ys, torch.cuda.current_stream().cuda_stream)
    fk.fe_ks_batch_status(b)
    _check(Ys, refs)


@pytest.mark.parametrize("t64,t32", [(256, 384), (384, 512), (512, 256)])
def test_split_batch_equals_individual_applications(batch_setup, t64, t32):
    """Split mode: FP64 and FP32 systems drained by two concurrent class objects."""
    wls, hps, ctxs, Xs, Ys, refs, b = batch_setup
    fk.fe_ks_batch_configure(b, [(s // 2) % 2 for s in range(6)], 2, 2, 2.0, False)
    fk.fe_ks_batch_set_split(b, t64, t32)
    try:
        for Y in Ys:
            Y.fill_(float("nan"))
        fk.fe_ks_batch_apply(b, Xs, Ys, torch.cuda.current_stream().cuda_stream)
        fk.fe_ks_batch_status(b)
        _check(Ys, refs)
    finally:
        fk.fe_ks_batch_set_split(b, 0, 0)


def test_split_batch_in_cuda_graph_and_timeout(batch_setup):
    """The forked pair of launches captures into one graph and replays; a never-published
    item of the FP64 class still ends in FE_KS_ERR_TIMEOUT, and the batch recovers."""
    wls, hps, ctxs, Xs, Ys, refs, b = batch_setup
    fk.fe_ks_batch_configure(b, [1] * 6, 2, 2, 2.0, False)
    fk.fe_ks_batch_set_split(b, 256, 384)
    try:
        stream = torch.cuda.current_stream()
        fk.fe_ks_batch_apply(b, Xs, Ys, stream.cuda_stream)      # warm-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fk.fe_ks_batch_apply(b, Xs, Ys, torch.cuda.current_stream().cuda_stream)
        for _ in range(2):
            for Y in Ys:
                Y.fill_(float("nan"))
            g.replay()
            torch.cuda.synchronize()
            fk.fe_ks_batch_status(b)
            _check(Ys, refs)
        del g
        fk.fe_ks_batch_configure(b, [1] * 6, 2, 2, 0.02, True)   # system 0 (FP64) misses one item
        fk.fe_ks_batch_apply(b, Xs, Ys, stream.cuda_stream)
        with pytest.raises(fk.FeKsError, match="TIMEOUT"):
            fk.fe_ks_batch_status(b)
        fk.fe_ks_batch_configure(b, [1] * 6, 2, 2, 2.0, False)
        fk.fe_ks_batch_apply(b, Xs, Ys, stream.cuda_stream)
        fk.fe_ks_batch_status(b)
        _check(Ys, refs)
    finally:
        fk.fe_ks_batch_set_split(b, 0, 0)
        fk.fe_ks_batch_configure(b, [0] * 6, 1, 1, 2.0, False)


def test_uncovered_systems_run_direct_in_the_batch():
    """Systems the persistent routines do not cover -- a complex (Bloch) operator, n_q = n_p + 2,
    degree 2, the pair-of-floats and 16-bit precisions -- are accepted and applied by their
    own kernels on side streams, next to queue systems; each equals its own fe_ks_apply,
    bit for bit (the same kernels on the same data), also inside a captured graph."""
    stream = torch.cuda.current_stream().cuda_stream
    spec = [  # (workload, precision)
        (Workload("cx", L=6.0, n=2, p=4, nq=5, n_v=3, kfrac=(0.2, 0, 0), complex=True, gga=True, n_atoms=1,
                  seed=11), fk.FE_KS_F64),
        (Workload("q2", L=6.0, n=2, p=5, nq=8, n_v=4, gga=True, n_atoms=1, seed=12), fk.FE_KS_F32),
        (Workload("d2", L=6.0, n=3, p=2, nq=3, n_v=5, gga=True, seed=13), fk.FE_KS_F64),
        (Workload("ff", L=6.0, n=2, p=6, nq=7, n_v=4, gga=True, n_atoms=2, seed=14), fk.FE_KS_F64E),
        (Workload("bf", L=6.0, n=2, p=8, nq=9, n_v=9, gga=True, n_atoms=2, seed=15), fk.FE_KS_BF16),
        (Workload("qq", L=6.0, n=2, p=6, nq=7, n_v=6, gga=True, n_atoms=1, seed=16), fk.FE_KS_F32),   # queue
        (Workload("q6", L=6.0, n=2, p=4, nq=5, n_v=3, gga=True, n_atoms=1, seed=17), fk.FE_KS_F64),   # queue
    ]
    hps = [HostProblem(wl) for wl, _ in spec]
    ctxs = [fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, stream) for hp, (wl, _) in zip(hps, spec)]
    b = None
    try:
        Xs, Ys, refs = [], [], []
        for (wl, pr), ctx in zip(spec, ctxs):
            X = torch.from_numpy(trial_vectors(wl)).cuda().to(torch_dtype(pr, wl.complex))
            R = torch.empty_like(X)
            fk.fe_ks_apply(ctx, X, R, wl.n_v, pr)
            Xs.append(X)
            Ys.append(torch.full_like(X, float("nan")))
            refs.append(R)
        b = fk.fe_ks_batch_create(ctxs, [wl.n_v for wl, _ in spec], [pr for _, pr in spec])
        fk.fe_ks_batch_apply(b, Xs, Ys, stream)
        fk.fe_ks_batch_status(b)
        torch.cuda.synchronize()
        for s, (Y, R) in enumerate(zip(Ys, refs)):
            if s < 5:
                assert torch.equal(Y, R), s
            else:
                err = parity_err(Y.double().cpu().numpy(), R.double().cpu().numpy())
                assert err <= TOL[spec[s][1]], (s, err)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fk.fe_ks_batch_apply(b, Xs, Ys, torch.cuda.current_stream().cuda_stream)
        for Y in Ys:
            Y.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        fk.fe_ks_batch_status(b)
        for s in range(5):
            assert torch.equal(Ys[s], refs[s]), s
        with pytest.raises(fk.FeKsError, match="ERR_ARG"):
            fk.fe_ks_batch_create(ctxs[:1], [3], [99])
        with pytest.raises(fk.FeKsError, match="n_q = n_p"):
            fk.fe_ks_batch_create(ctxs[1:2], [4], [fk.FE_KS_BF16])
    finally:
        if b is not None:
            fk.fe_ks_batch_destroy(b)
        for c in ctxs:
            fk.fe_ks_destroy(c)


@pytest.mark.parametrize("direct,split", [([1, 0, 0, 0, 0, 0], (0, 0)), ([0, 1, 0, 1, 0, 0], (0, 0)),
                                          ([1] * 6, (0, 0)), ([0, 0, 1, 0, 0, 1], (256, 384))])
def test_direct_systems_equal_individual_applications(batch_setup, direct, split):
    """Direct systems run their own kernels on side streams beside the persistent launch of
    the others (also with split mode, and with no system left in the queue)."""
    wls, hps, ctxs, Xs, Ys, refs, b = batch_setup
    fk.fe_ks_batch_configure(b, [(s // 2) % 2 for s in range(6)], 2, 2, 2.0, False)
    fk.fe_ks_batch_set_split(b, *split)
    fk.fe_ks_batch_set_direct(b, direct)
    try:
        for Y in Ys:
            Y.fill_(float("nan"))
        fk.fe_ks_batch_apply(b, Xs, Ys, torch.cuda.current_stream().cuda_stream)
        fk.fe_ks_batch_status(b)
        _check(Ys, refs)
    finally:
        fk.fe_ks_batch_set_direct(b, None)
        fk.fe_ks_batch_set_split(b, 0, 0)


def test_direct_systems_in_cuda_graph(batch_setup):
    """The forked per-system streams and the persistent launch capture as one graph."""
    wls, hps, ctxs, Xs, Ys, refs, b = batch_setup
    fk.fe_ks_batch_configure(b, [1] * 6, 2, 2, 2.0, False)
    fk.fe_ks_batch_set_direct(b, [1, 0, 1, 0, 0, 0])
    try:
        stream = torch.cuda.current_stream()
        fk.fe_ks_batch_apply(b, Xs, Ys, stream.cuda_stream)      # warm-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fk.fe_ks_batch_apply(b, Xs, Ys, torch.cuda.current_stream().cuda_stream)
        for _ in range(2):
            for Y in Ys:
                Y.fill_(float("nan"))
            g.replay()
            torch.cuda.synchronize()
            fk.fe_ks_batch_status(b)
            _check(Ys, refs)
    finally:
        fk.fe_ks_batch_set_direct(b, None)
