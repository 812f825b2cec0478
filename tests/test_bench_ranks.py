"""Multi-rank host logic of bench.py on the CPU (gloo, two ranks).

The operator does not shard: N GPUs run N replicas, with a barrier and the
slowest rank's time.  These tests cover that logic without a GPU: the MAX
all-reduce of the per-rank times, the whole-job value, and the reference arm
under a two-rank launch (rank 0 prints one JSON line, rank 1 exits quietly).
"""
import json
import os
import socket
import subprocess
import sys
import tempfile

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
        value = bench.whole_job_value(1000, world, ms)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"ms": ms, "value": value}, f)
    finally:
        dist.destroy_process_group()


def test_slowest_rank_time_and_whole_job_value():
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(2, _free_port(), d), nprocs=2, start_method="spawn")
        res = [json.load(open(os.path.join(d, f"rank{r}.json"))) for r in range(2)]
    for r in res:
        assert r["ms"] == 15.0                       # the slower rank's time on every rank
        assert r["value"] == pytest.approx(2 * 1000 / 0.015)


def test_single_rank_keeps_its_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, None) == 12.5
    assert bench.whole_job_value(10, 1, 2.0) == pytest.approx(5000.0)


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_under_two_ranks(rank):
    env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--workload", "C1",
                        "--steps", "1", "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    if rank == 1:
        assert lines == []
        return
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


@pytest.mark.parametrize("key", ["C2", "C3", "C4", "AE"])
def test_bench_flop_model_matches_the_oracle_model(key):
    """bench.alg_flops splits the oracle's closed form of eq. flopRealMF / flopComplexMF
    (n_s = 9 x (atom, cell) pairs, the vector count taken as real columns: 2 per complex
    vector) into the fused cell kernel's share (cell terms + half of the nonlocal term, the
    roofline's numerator) and the projection kernel's share (the other half)."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import flops
    from synth import CONFIGS
    wl = CONFIGS[key]
    n_pairs = 5 * wl.n_atoms
    local, proj = bench.alg_flops(wl, n_pairs, wl.n_v)
    cols = wl.n_v * (2 if wl.complex else 1)
    model = flops.mf_complex_total if wl.complex else flops.mf_real_total
    want = model(wl.p + 1, wl.nq, cols, wl.n_cells, 9 * n_pairs)
    assert local + proj == pytest.approx(want, rel=1e-12)
    assert proj == pytest.approx((want - model(wl.p + 1, wl.nq, cols, wl.n_cells, 0)) / 2, rel=1e-12)
