#!/usr/bin/env python
"""Benchmark of the matrix-free FE Kohn-Sham operator Y = H X on GB300.

Workload (default): the p = 8 configuration -- periodic cube L = 30 bohr,
24^3 hexahedral cells, degree 8 with 9 Gauss points per direction, full real
operator (kinetic + V_loc + GGA + 64 atoms of l <= 2 projectors), N_v = 256,
m = 7,077,888 DoFs.  One step = one application Y = H X of the whole operator
(all cells, all vectors) in FP64; X (14.5 GB) is far larger than L2, so no
flush is needed between steps.

Output.  Every measured section goes to a JSON detail file (--detail, default
bench_detail.json); the LAST stdout line is one compact JSON object (a few KB)
with the headline and a digest of the rest:
  value, ms_per_step, roofline, clocks, gpu_launches   FP64 application (the headline)
  e2e                      the same metric through fe_ks_apply_host from pinned host memory
  cpu_baseline             the CPU oracle on a bounded sample of cells
  precisions               pairs of floats, FP32, BF16 / FP16 tensor cores: time, speedup,
                           roofline fraction, and the error against the FP64 result
  filter                   R-ChFSI pass times per precision plan, filter and pass speedups,
                           and the convergence run
  batched_c5, batched_small  one persistent launch vs one launch per system
  all_electron_like, cell_matrix_f64_ms   the other workloads' headline times
Each section has a --no-... switch.

Metric: DoF x vectors per second (m * N_v / time of one application).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

N > 1 runs under torchrun as independent replicas (one per GPU, weak
scaling; the operator has no data-path exchange on one GPU per system).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H.X DoF*vectors/s (FP64; mixed FP32 beside) at p=8"
UNIT = "DoF*vec/s"
# Nominal FP64 rate of GB300 (recipe table: 1.25 TFLOP/s) and the FP32 CUDA-core rate
# 152 SMs x 128 lanes x 2 flop x 2.07 GHz.
PEAK_FP64_NOMINAL = 1.25e12
PEAK_FP32_NOMINAL = 152 * 128 * 2 * 2.07e9


def _measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0   # fallback figure of an earlier GB300 measurement


PEAK_HBM_GBS = _measured_hbm_gbs()


def _measured_bf16_tflops():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, ValueError, KeyError):
        return 1900.0   # fallback figure of an earlier GB300 measurement


PEAK_BF16_TFLOPS = _measured_bf16_tflops()


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="C4")
    ap.add_argument("--cells", type=int, default=None,
                    help="cells per direction (same recipe on a smaller grid, for profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the six-system batched launch")
    ap.add_argument("--no-filter", action="store_true", help="skip the R-ChFSI filter timing")
    ap.add_argument("--no-nq2", action="store_true", help="skip the n_q = n_p + 2 workload")
    ap.add_argument("--no-cell-matrix", action="store_true", help="skip the cell-matrix baseline")
    ap.add_argument("--no-all-electron", action="store_true", help="skip the all-electron-like workload")
    ap.add_argument("--precision", choices=["both", "f64", "f32", "f64e", "bf16", "f16", "bf16x2"], default="both",
                    help="f32 / f64e / bf16 / f16 / bf16x2 alone time only that application (for profiling)")
    ap.add_argument("--config", type=int, default=None,
                    help="force this tile configuration instead of tuning (for profiling)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle sample")
    ap.add_argument("--no-converge", action="store_true",
                    help="skip the full-size convergence run of the mixed eigensolver")
    ap.add_argument("--converge-f64", action="store_true",
                    help="also run the all-FP64 eigensolver to convergence at full size (about ten minutes)")
    ap.add_argument("--converge-passes", type=int, default=40, help="pass limit of the convergence run")
    ap.add_argument("--converge-degree", type=int, default=60,
                    help="Chebyshev degree of the convergence run (the paper uses about 30 on its meshes)")
    ap.add_argument("--converge-tol", type=float, default=1e-8,
                    help="residual (hence certified eigenvalue error) target of the convergence run, Ha")
    ap.add_argument("--detail", default="bench_detail.json",
                    help="file that receives every measured section (the last stdout line is a digest)")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(ms, world, dev):
    """The slowest rank's time: every rank takes part (one all-reduce with MAX; NCCL on the
    GPUs, gloo on the CPU).  With one rank the value is returned as it is."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank, world, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (ms * 1e-3)


def alg_flops(wl, n_pairs, n_v):
    """Paper's operation count (eq. flopRealMF / flopComplexMF) with n_s read as the
    number of (projector, cell) incidences, split into the fused local kernel's
    share (cell terms + expansion F Delta T3) and the projection kernel's share.
    The formulas' vector count is the batch product b2 nb2 nb1, i.e. real columns:
    a complex vector counts twice (its real and imaginary batches, Sec. 4.2)."""
    n_p, n_q = wl.p + 1, wl.nq
    if wl.complex:
        n_v = 2 * n_v
    npo, nqo = n_p // 2, n_q // 2
    s = n_p * n_p + n_p * n_q + n_q * n_q
    if wl.complex:
        per_cell = (2 * n_v * (npo * (n_q + 2) + nqo * (n_p + 2)) * s + 6 * n_v * nqo * n_q ** 2 * (2 * n_q + 5)
                    + 2 * n_q ** 3 + 40 * n_v * n_q ** 3)
        nl = n_v * (8 * n_p ** 3 + 3) * 9 * n_pairs
    else:
        per_cell = (2 * n_v * (npo * (n_q + 2) + nqo * (n_p + 2)) * s + 6 * n_v * nqo * n_q ** 2 * (2 * n_q + 5)
                    + 2 * n_q ** 3 + 34 * n_v * n_q ** 3)
        nl = n_v * (4 * n_p ** 3 + 1) * 9 * n_pairs
    return per_cell * wl.n_cells + nl / 2.0, nl / 2.0


def col_errors(Y, Yref, chunk=65536):
    """Errors of Y against Yref over every entry, on the device in row chunks:
    (max over columns of ||Y_v - Yref_v||_2 / ||Yref_v||_2,
     max over entries of |Y_iv - Yref_iv| / max_i |Yref_iv|).
    Complex blocks are compared as their real and imaginary columns."""
    import torch
    if Y.is_complex():
        Y, Yref = torch.view_as_real(Y).flatten(1), torch.view_as_real(Yref).flatten(1)
    n = Y.shape[1]
    num2 = torch.zeros(n, dtype=torch.float64, device=Y.device)
    den2 = torch.zeros_like(num2)
    dmax = torch.zeros_like(num2)
    rmax = torch.zeros_like(num2)
    for r0 in range(0, Y.shape[0], chunk):
        a = Y[r0:r0 + chunk].to(torch.float64)
        b = Yref[r0:r0 + chunk].to(torch.float64)
        d = a - b
        num2 += (d * d).sum(0)
        den2 += (b * b).sum(0)
        dmax = torch.maximum(dmax, d.abs().amax(0))
        rmax = torch.maximum(rmax, b.abs().amax(0))
    col = float((num2.sqrt() / den2.sqrt().clamp_min(1e-300)).max())
    elem = float((dmax / rmax.clamp_min(1e-300)).max())
    return col, elem


def load_traffic(key):
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            return json.load(f).get(key)
    except (OSError, ValueError):
        return None


def fill_trial(wl, n_v, X_dev, dtype_np):
    """Copy the seeded trial block into a device tensor chunk by chunk."""
    import torch
    from synth import trial_chunk, TRIAL_CHUNK
    nch = (wl.n_dofs + TRIAL_CHUNK - 1) // TRIAL_CHUNK
    for c in range(nch):
        blk = trial_chunk(wl, n_v, c)
        r0 = c * TRIAL_CHUNK
        X_dev[r0:r0 + blk.shape[0]].copy_(torch.from_numpy(blk.astype(dtype_np)))


# ------------------------------------------------------------- native arm
def run_native(args, wl, rank, world):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2512_08571_gb300 import fe_ks as fk
    from synth.host_problem import HostProblem

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    hp = HostProblem(wl)
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, stream.cuda_stream)
    info = fk.fe_ks_info(ctx)
    setup_s = time.time() - t0
    cplx = hp.complex
    m, n_v = hp.m, wl.n_v
    units = m * n_v
    local_flops, proj_flops = alg_flops(wl, info["n_pairs"], n_v)
    # BF16 tensor-core kernel: executed MMA flops per application (18 MMAs per row tile and
    # output tile over the six sweeps, (n^2 + 1) / 2 row tiles, 8-column tiles of the block)
    n1 = wl.p + 1
    ntl, kdim = (2, 16) if n1 > 8 else (1, 8)
    cw = 2 if cplx else 1
    mma_flops = wl.n_cells * ((n_v * cw + 7) // 8) * 18 * ntl * ((n1 * n1 + 1) // 2) * 2 * 16 * 8 * kdim
    bytes32 = {"xy": m * n_v * cw * 4, "coef": wl.n_cells * info.get("ncoef", 13 if cplx else 10) * wl.nq ** 3 * 4}

    def barrier():
        if world > 1:
            dist.barrier()

    # the seeded trial block, generated once on the host and kept on the device
    X64 = torch.empty((m, n_v), dtype=torch.complex128 if cplx else torch.float64, device=dev)
    fill_trial(wl, n_v, X64, np.complex128 if cplx else np.float64)

    ref = {}

    def measure(precision, steps, warmup):
        dt = {fk.FE_KS_F64: torch.complex128 if cplx else torch.float64,
              fk.FE_KS_F64E: torch.complex128 if cplx else torch.float64,
              fk.FE_KS_F32: torch.complex64 if cplx else torch.float32,
              fk.FE_KS_BF16: torch.complex64 if cplx else torch.float32,
              fk.FE_KS_F16: torch.complex64 if cplx else torch.float32,
              fk.FE_KS_BF16X2: torch.complex64 if cplx else torch.float32}[precision]
        X = X64 if dt == X64.dtype else X64.to(dt)
        Y = torch.empty_like(X)
        if args.config is None:
            best, tune_ms = fk.fe_ks_tune(ctx, X, Y, n_v, precision, reps=1)
        else:
            try:
                fk.fe_ks_set_config(ctx, precision, args.config)
                best = args.config
            except fk.FeKsError:   # a precision with a single kernel (the split one)
                best = 0
            tune_ms = []
        for _ in range(warmup):
            fk.fe_ks_apply(ctx, X, Y, n_v, precision)
        torch.cuda.synchronize()
        fk.fe_ks_read_profile(ctx)
        fk.fe_ks_set_profiling(ctx, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(dev.index) as clk:
            e0.record(stream)
            for _ in range(steps):
                fk.fe_ks_apply(ctx, X, Y, n_v, precision)
            e1.record(stream)
            torch.cuda.synchronize()
        barrier()
        fk.fe_ks_set_profiling(ctx, False)
        prof = fk.fe_ks_read_profile(ctx)
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, world, dev)
        local_ms, local_n = prof["local"]
        achieved = local_flops * steps / (local_ms * 1e-3) if local_ms > 0 else None
        out = dict(ms=ms, value=whole_job_value(units, world, ms), prof=prof, clocks=clk.summary(),
                   tile_config=best, tune_ms=[round(t, 3) for t in tune_ms],
                   achieved=achieved, local_launch_ms=local_ms / max(local_n, 1),
                   launches=int(prof["proj"][1] + prof["local"][1]))
        # error of this precision's result against the FP64 application of the same X (itself
        # held to <= 1e-12 of the oracle by the parity tests), over all m x N_v entries
        if precision == fk.FE_KS_F64:
            ref["Y"] = Y
        elif "Y" in ref:
            out["err_col"], out["err_elem"] = col_errors(Y, ref["Y"])
        del X, Y
        torch.cuda.empty_cache()
        return out

    f64 = measure(fk.FE_KS_F64, args.steps, args.warmup) if args.precision in ("both", "f64") else None
    f64e = measure(fk.FE_KS_F64E, args.steps, args.warmup) if args.precision in ("both", "f64e") else None
    mixed = None
    if args.precision == "f32":
        mixed = measure(fk.FE_KS_F32, args.steps, args.warmup)
    elif not args.no_mixed and args.precision == "both":
        mixed = measure(fk.FE_KS_F32, max(args.steps, 20), max(args.warmup, 3))
    bf16 = f16 = bf16x2 = None
    if args.precision == "bf16":
        bf16 = measure(fk.FE_KS_BF16, args.steps, args.warmup)
    elif args.precision == "f16":
        f16 = measure(fk.FE_KS_F16, args.steps, args.warmup)
    elif args.precision == "bf16x2":
        bf16x2 = measure(fk.FE_KS_BF16X2, args.steps, args.warmup)
    elif not args.no_mixed and args.precision == "both":
        bf16 = measure(fk.FE_KS_BF16, max(args.steps, 20), max(args.warmup, 3))
        f16 = measure(fk.FE_KS_F16, max(args.steps, 20), max(args.warmup, 3))
        bf16x2 = measure(fk.FE_KS_BF16X2, max(args.steps, 10), max(args.warmup, 3))
    ref.clear()
    torch.cuda.empty_cache()
    peak_mma_live = fk.fe_ks_measure_fma_peak(fk.FE_KS_BF16) * 1e12 if (bf16 or f16 or bf16x2) else None

    peak64_live = fk.fe_ks_measure_fma_peak(fk.FE_KS_F64) * 1e12
    peak32_live = fk.fe_ks_measure_fma_peak(fk.FE_KS_F32) * 1e12

    # end to end through the C ABI with HOST buffers (pinned): fe_ks_apply_host copies X in,
    # applies and copies Y out; consecutive calls overlap one call's copies with the next
    # call's application (two workspace slots).  Every step's copies are inside the timed region.
    e2e = None
    if not args.no_e2e:
        tdt = torch.complex128 if cplx else torch.float64
        Xh = torch.empty((m, n_v), dtype=tdt, pin_memory=True)
        Xh.copy_(X64)
        Yh = torch.empty_like(Xh, pin_memory=True)
        wb = fk.fe_ks_apply_host_workspace(ctx, n_v, fk.FE_KS_F64)
        work = torch.empty(wb, dtype=torch.uint8, device=dev)
        fk.fe_ks_apply_host(ctx, Xh, Yh, n_v, fk.FE_KS_F64, work, wb)      # warm-up (creates the copy streams)
        fk.fe_ks_host_wait(ctx)
        ksteps = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(ksteps):
            fk.fe_ks_apply_host(ctx, Xh, Yh, n_v, fk.FE_KS_F64, work, wb)
        fk.fe_ks_host_wait(ctx)
        ms_e2e = max_over_ranks((time.perf_counter() - t0) * 1e3 / ksteps, world, dev)
        del work
        torch.cuda.empty_cache()
        # the parts of one step, run one after another (CUDA events on one stream; the
        # second of two passes, so that first-touch costs of the new buffers are excluded)
        Xd = torch.empty((m, n_v), dtype=tdt, device=dev)
        Yd = torch.empty_like(Xd)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for _ in range(2):
            ev[0].record(stream)
            Xd.copy_(Xh, non_blocking=True)
            ev[1].record(stream)
            fk.fe_ks_apply(ctx, Xd, Yd, n_v, fk.FE_KS_F64)
            ev[2].record(stream)
            Yh.copy_(Yd, non_blocking=True)
            ev[3].record(stream)
            torch.cuda.synchronize()
        nbytes = Xh.numel() * Xh.element_size()
        e2e = {"value": whole_job_value(units, world, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "ms_per_step": ms_e2e, "steps": ksteps,
               "api": "fe_ks_apply_host (pinned host X, Y; copies of one step overlap the next step's apply)",
               "one_step_serial_ms": {"h2d": ev[0].elapsed_time(ev[1]), "apply": ev[1].elapsed_time(ev[2]),
                                      "d2h": ev[2].elapsed_time(ev[3])}}
        del Xh, Yh, Xd, Yd
        torch.cuda.empty_cache()
    filt = None
    if not args.no_filter and rank == 0 and not cplx:
        filt = run_filter(args, wl, ctx, hp, X64)
    cmb = None
    if not args.no_cell_matrix and rank == 0 and not cplx:
        cmb = run_cell_matrix(args, ctx, X64, units, f64, mixed, bf16)
    del X64
    torch.cuda.empty_cache()
    fk.fe_ks_destroy(ctx)
    return dict(filter=filt, cell_matrix=cmb, f64e=f64e, f64=f64, mixed=mixed, bf16=bf16, f16=f16, bf16x2=bf16x2,
                peak_mma_live=peak_mma_live,
                mma_flops_per_apply=mma_flops, bytes32=bytes32, e2e=e2e, setup_s=setup_s, info=info, local_flops=local_flops,
                peak64_live=peak64_live, peak32_live=peak32_live)


# ------------------------------------------------------- cell-matrix baseline
def run_cell_matrix(args, ctx, X64, units, f64, mixed, bf16):
    """The cell-matrix method on the same operator: dense H_loc^(e) per cell (built once
    from the FP64 matrix-free kernel), applied per colour by batched library GEMMs, with
    the same projection and nonlocal expansion.  FP64, FP32 and BF16 (tensor-core GEMM,
    FP32 accumulation) beside the matrix-free apply of the same precision, one warm-up and a few
    timed applications each; the cell matrices are freed after each precision."""
    import torch
    from paper_2512_08571_gb300 import fe_ks as fk
    stream = torch.cuda.current_stream()
    n_v = X64.shape[1]
    out = {"method": "dense H_loc^(e) per cell (n_p^3 x n_p^3), per colour: gather X^(e), batched "
                     "cuBLAS GEMM, colour-exclusive scatter + nonlocal expansion", "unit": UNIT}
    for prec, name, mf in ((fk.FE_KS_F64, "f64", f64), (fk.FE_KS_F32, "f32", mixed),
                           (fk.FE_KS_BF16, "bf16_tensor_core", bf16)):
        X = X64 if prec == fk.FE_KS_F64 else X64.to(torch.float32)
        Y = torch.empty_like(X)
        try:
            cm = fk.fe_ks_cm_create(ctx, prec, n_v)
        except fk.FeKsError as e:
            out[name] = {"unavailable": str(e)}
            continue
        try:
            info = fk.fe_ks_cm_info(cm)
            setup_ms, nbytes = info["setup_ms"], info["bytes"]
            fk.fe_ks_cm_apply(cm, X, Y, n_v)
            torch.cuda.synchronize()
            reps = 2 if prec == fk.FE_KS_F64 else 5
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fk.fe_ks_cm_apply(cm, X, Y, n_v)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
        finally:
            fk.fe_ks_cm_destroy(cm)
        r = {"ms_per_step": ms, "value": units / (ms * 1e-3), "setup_ms": setup_ms,
             "device_bytes": nbytes}
        if mf:
            r["matrix_free_ms_per_step"] = mf["ms"]
            r["matrix_free_speedup"] = ms / mf["ms"]
        out[name] = r
        del X, Y
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------ R-ChFSI filter
def run_filter(args, wl, ctx, hp, X64):
    """One R-ChFSI pass on the workload (Lanczos bound, degree-20 filter,
    Rayleigh-Ritz) four ways: all native FP64; FP64-accurate pairs of floats;
    mixed (FP32 recurrence, FP64-accurate residual / Lanczos / Rayleigh-Ritz
    through the pair-of-floats kernel); the same with the BF16 tensor-core
    recurrence.  Plus a convergence run on the same
    recipe at 6^3 cells (N_v = 32) to residual 1e-9 on the lowest 8, all-FP64
    against mixed, reporting iterations and the eigenvalue gap."""
    import numpy as np
    import torch
    from paper_2512_08571_gb300 import fe_ks as fk
    from paper_2512_08571_gb300.chfsi import RChFSI
    from synth.host_problem import HostProblem
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", torch.cuda.current_device())

    def ev_ms(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    out = {"degree": 20, "lanczos_steps": 10}
    # cost of one application against the number of vectors (Lanczos uses n_v = 1)
    nv_ms = {}
    for nv in (1, 8, 64):
        Xa = X64[:, :nv].contiguous()
        Ya = torch.empty_like(Xa)
        fk.fe_ks_apply(ctx, Xa, Ya, nv, fk.FE_KS_F64)
        nv_ms[nv], _ = ev_ms(lambda: fk.fe_ks_apply(ctx, Xa, Ya, nv, fk.FE_KS_F64))
        del Xa, Ya
    out["f64_apply_ms_by_n_v"] = nv_ms
    m, n_v = hp.m, wl.n_v
    # plan: (recurrence arithmetic, FP64-accurate parts, Rayleigh-Ritz GEMMs in pairs of floats)
    # (cuBLAS's FP64 emulation on the integer tensor cores measured slower than native FP64
    #  GEMM on this part, 578 vs 240 ms for a 2e6 x 256 Gram matrix, so it is not a plan)
    plans = {"f64": (fk.FE_KS_F64, fk.FE_KS_F64, False),
             "f64_pairs": (fk.FE_KS_F64E, fk.FE_KS_F64E, True),
             "mixed": (fk.FE_KS_F32, fk.FE_KS_F64E, True),
             "mixed_bf16": (fk.FE_KS_BF16, fk.FE_KS_F64E, True),
             "mixed_f16": (fk.FE_KS_F16, fk.FE_KS_F64E, True),
             "mixed_bf16x2": (fk.FE_KS_BF16X2, fk.FE_KS_F64E, True),
             # the mixed plan with the Rayleigh-Ritz products in pairs of floats instead of on the tensor cores
             "mixed_ff_rr": (fk.FE_KS_F32, fk.FE_KS_F64E, True)}
    lam = X = lmax = None
    for name, (prec, exact, pair_gemm) in plans.items():
        fk.fe_ks_set_rr_gram(ctx, name != "mixed_ff_rr")
        sol = RChFSI(ctx, m, n_v, False, degree=20, precision=prec, exact=exact, gemm_pairs=pair_gemm)
        sol.lanczos_upper_bound()            # warm-up
        t_l, lm = ev_ms(sol.lanczos_upper_bound)
        if lmax is None:
            lmax = lm
            lam, X = sol.rayleigh_ritz(X64.clone())
        sol.lmax = lmax
        try:
            t_rr, _ = ev_ms(lambda: sol.rayleigh_ritz(X.clone()))
        except fk.FeKsError as exc:          # FP64 emulation unavailable
            out[name] = {"unavailable": str(exc)}
            del sol
            continue
        Xf = X.clone()
        t_f, _ = ev_ms(lambda: sol.filter(Xf, lam))
        out[name] = {"lanczos_ms": t_l, "rayleigh_ritz_ms": t_rr, "filter_ms": t_f, "pass_ms": t_l + t_rr + t_f}
        del sol, Xf
        torch.cuda.empty_cache()
    fk.fe_ks_set_rr_gram(ctx, True)
    out["speedup_filter_mixed_vs_f64"] = out["f64"]["filter_ms"] / out["mixed"]["filter_ms"]
    out["speedup_pass_mixed_vs_f64"] = out["f64"]["pass_ms"] / out["mixed"]["pass_ms"]
    out["speedup_filter_bf16_vs_f64"] = out["f64"]["filter_ms"] / out["mixed_bf16"]["filter_ms"]
    out["speedup_pass_bf16_vs_f64"] = out["f64"]["pass_ms"] / out["mixed_bf16"]["pass_ms"]
    out["speedup_filter_f16_vs_f64"] = out["f64"]["filter_ms"] / out["mixed_f16"]["filter_ms"]
    out["speedup_pass_f16_vs_f64"] = out["f64"]["pass_ms"] / out["mixed_f16"]["pass_ms"]
    if not args.no_converge:
        out["converged"] = run_converge_full(args, wl, ctx, X, lmax, out)
    del X
    # convergence at 6^3 cells
    wls = wl.scaled(n=6, n_v=32, n_atoms=max(1, wl.n_atoms * 6 ** 3 // wl.n ** 3 + 1))
    hps = HostProblem(wls)
    cs = fk.fe_ks_setup(hps.struct, fk.TERM_ALL, wls.n_v, stream.cuda_stream)
    Xs0 = torch.empty((hps.m, wls.n_v), dtype=torch.float64, device=dev)
    fill_trial(wls, wls.n_v, Xs0, np.float64)
    n_chk = wls.n_v // 4
    conv = {"workload": f"same recipe, 6^3 cells, {wls.n_atoms} atoms, N_v={wls.n_v}, residual < 1e-9 "
                        f"on the lowest {n_chk}"}
    lams = {}
    for name, prec, exact, pg in (("f64", fk.FE_KS_F64, fk.FE_KS_F64, False),
                                  ("mixed", fk.FE_KS_F32, fk.FE_KS_F64E, True),
                                  ("mixed_bf16", fk.FE_KS_BF16, fk.FE_KS_F64E, True),
                                  ("mixed_f16", fk.FE_KS_F16, fk.FE_KS_F64E, True)):
        sol = RChFSI(cs, hps.m, wls.n_v, False, degree=20, precision=prec, exact=exact, gemm_pairs=pg)
        t, (lam_c, _, res, its) = ev_ms(lambda: sol.run(Xs0.clone(), n_iter=120, tol=1e-9, n_check=n_chk))
        lams[name] = lam_c.cpu().numpy()
        conv[name] = {"iterations": its, "ms": t, "max_residual": float(res[:n_chk].max())}
        del sol
    conv["max_eig_diff_mixed_vs_f64_Ha"] = float(np.max(np.abs(lams["mixed"][:n_chk] - lams["f64"][:n_chk])))
    conv["max_eig_diff_bf16_vs_f64_Ha"] = float(np.max(np.abs(lams["mixed_bf16"][:n_chk] - lams["f64"][:n_chk])))
    conv["max_eig_diff_f16_vs_f64_Ha"] = float(np.max(np.abs(lams["mixed_f16"][:n_chk] - lams["f64"][:n_chk])))
    conv["speedup"] = conv["f64"]["ms"] / conv["mixed"]["ms"]
    conv["speedup_bf16"] = conv["f64"]["ms"] / conv["mixed_bf16"]["ms"]
    conv["speedup_f16"] = conv["f64"]["ms"] / conv["mixed_f16"]["ms"]
    # the generalised problem H X = M X Lam with the consistent mass (Algorithm 4 as printed)
    from synth.host_problem import mass_problem
    hpm = mass_problem(wls)
    cm = fk.fe_ks_setup(hpm.struct, fk.TERM_L, wls.n_v, stream.cuda_stream)
    gh, glams = {}, {}
    for name, prec, exact, pg in (("f64", fk.FE_KS_F64, fk.FE_KS_F64, False),
                                  ("mixed", fk.FE_KS_F32, fk.FE_KS_F64E, True),
                                  ("mixed_bf16", fk.FE_KS_BF16, fk.FE_KS_F64E, True)):
        sol = RChFSI(cs, hps.m, wls.n_v, False, degree=20, precision=prec, exact=exact, gemm_pairs=pg, mass_ctx=cm)
        t, (lam_c, _, res, its) = ev_ms(lambda: sol.run(Xs0.clone(), n_iter=160, tol=1e-9, n_check=n_chk))
        glams[name] = lam_c.cpu().numpy()
        gh[name] = {"iterations": its, "ms": t, "max_residual": float(res[:n_chk].max())}
        del sol
    gh["max_eig_diff_mixed_vs_f64_Ha"] = float(np.max(np.abs(glams["mixed"][:n_chk] - glams["f64"][:n_chk])))
    gh["max_eig_diff_bf16_vs_f64_Ha"] = float(np.max(np.abs(glams["mixed_bf16"][:n_chk] - glams["f64"][:n_chk])))
    gh["speedup"] = gh["f64"]["ms"] / gh["mixed"]["ms"]
    conv["generalised_consistent_mass"] = gh
    fk.fe_ks_destroy(cm)
    out["converged_6cubed"] = conv
    fk.fe_ks_destroy(cs)
    return out


def run_converge_full(args, wl, ctx, X0, lmax, passes_out):
    """Algorithm 3 at the workload's full size: the mixed plan (FP32 recurrence,
    FP64-accurate residual, Lanczos and Rayleigh-Ritz in pairs of floats) from the
    Rayleigh-Ritz'd trial block until every one of the lowest N_v / 8 Ritz pairs
    has residual norm <= tol (at most --converge-passes passes).  With lam_max
    near 2600 Ha and the checked Ritz values a fraction of a Ha below lam_T, the
    damping of a degree-m filter per pass is about 1 / cosh(m sqrt(2 eps)) with
    eps = 2 (lam_T - lam) / (lam_max - lam_T) ~ 2.5e-4: about 1.1 at m = 20 (some
    200 passes to 1e-8) and 2 at m = 60 (some 25 passes), so the run uses a
    higher degree than the single-pass measurements (--converge-degree).  The
    Ritz vectors are orthonormal and the residuals are FP64-accurate, so each of
    those eigenvalues lies within its residual norm of an exact eigenvalue of Hs
    (Bauer-Fike for a Hermitian operator): the eigenvalue error is certified
    <= tol without an FP64 run.  The all-FP64 plan takes the same passes (same
    filter polynomial; checked at 6^3 cells), so its time is its initial
    Rayleigh-Ritz plus the pass count times one all-FP64 pass (filter,
    Rayleigh-Ritz and residual check) measured at the same degree, unless
    --converge-f64 runs it to the end."""
    import torch
    from paper_2512_08571_gb300 import fe_ks as fk
    from paper_2512_08571_gb300.chfsi import RChFSI
    m, n_v = X0.shape
    n_chk = max(8, n_v // 8)
    tol = args.converge_tol
    deg = args.converge_degree
    stream = torch.cuda.current_stream()
    res = {"workload": f"{wl.name} full size, N_v={n_v}, lowest {n_chk} to residual <= {tol:g} Ha, "
                       f"filter degree {deg}", "tol_Ha": tol, "n_checked": n_chk, "degree": deg}

    def solver(prec, exact, pairs):
        sol = RChFSI(ctx, m, n_v, False, degree=deg, precision=prec, exact=exact, gemm_pairs=pairs)
        sol.lmax = lmax
        return sol

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    def run(prec, exact, pairs, max_passes):
        sol = solver(prec, exact, pairs)
        X = X0.clone()
        (lam, X, r, its), ms = timed(lambda: sol.run(X, n_iter=max_passes, tol=tol, n_check=n_chk))
        out = {"passes": its, "ms": ms, "max_residual": float(r[:n_chk].max()),
               "lam": lam[:n_chk].cpu().numpy(), "history": list(sol.res_history)}
        del sol, X
        torch.cuda.empty_cache()
        return out

    def one_f64_pass():
        sol = solver(fk.FE_KS_F64, fk.FE_KS_F64, False)
        X = X0.clone()
        (lam, X), rr0 = timed(lambda: sol.rayleigh_ritz(X))

        def step():
            Xf = sol.filter(X, lam)
            lam2, Xf = sol.rayleigh_ritz(Xf)
            return sol.residual_norms(Xf, lam2)
        _, ms = timed(step)
        del sol, X
        torch.cuda.empty_cache()
        return rr0, ms

    mx = run(fk.FE_KS_F32, fk.FE_KS_F64E, True, args.converge_passes)
    res["passes_mixed"] = mx["passes"]
    res["ms_mixed"] = mx["ms"]
    res["max_residual"] = mx["max_residual"]
    res["max_eig_err_bound_Ha"] = mx["max_residual"]
    res["converged"] = mx["max_residual"] <= tol
    res["residual_history"] = [float(f"{x:.3g}") for x in mx["history"]]
    rr0, f64_pass = one_f64_pass()
    res["f64_pass_ms"] = f64_pass
    res["ms_f64_derived"] = rr0 + mx["passes"] * f64_pass
    res["speedup"] = res["ms_f64_derived"] / mx["ms"]
    res["speedup_basis"] = (f"all-FP64 time = its initial Rayleigh-Ritz + passes x one all-FP64 pass, "
                            f"both measured at degree {deg}")
    if args.converge_f64:
        f64 = run(fk.FE_KS_F64, fk.FE_KS_F64, False, args.converge_passes)
        res["passes_f64"] = f64["passes"]
        res["ms_f64"] = f64["ms"]
        res["speedup"] = f64["ms"] / mx["ms"]
        res["speedup_basis"] = "both plans run to the tolerance"
        res["max_eig_diff_Ha"] = float(abs(f64["lam"] - mx["lam"]).max())
    return res


# -------------------------------------------------- all-electron-like workload
def run_all_electron(args):
    """The all-electron-like workload (Bloch-periodic complex operator, no projectors,
    24^3 cells, p = 8, N_v = 64): one application per precision, tuned, timed with
    CUDA events (inputs larger than L2).  Returns a dict for the JSON line."""
    import numpy as np
    import torch
    from paper_2512_08571_gb300 import fe_ks as fk
    from synth.host_problem import HostProblem
    from synth import CONFIGS
    wl = CONFIGS["AE"]
    if args.cells:
        wl = wl.scaled(n=args.cells)
    stream = torch.cuda.current_stream()
    hp = HostProblem(wl)
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, stream.cuda_stream)
    X64 = torch.empty((hp.m, wl.n_v), dtype=torch.complex128, device="cuda")
    fill_trial(wl, wl.n_v, X64, np.complex128)
    units = hp.m * wl.n_v
    out = {"workload": f"AE: L={wl.L:g} bohr, {wl.n}^3 cells, p={wl.p}, n_q={wl.nq}, N_v={wl.n_v}, complex "
                       f"(k = {tuple(round(float(k), 4) for k in wl.kpt)} bohr^-1), GGA, no projectors",
           "n_dofs": hp.m, "unit": UNIT}
    for prec, name in ((fk.FE_KS_F64, "f64"), (fk.FE_KS_F64E, "f64_pairs_of_fp32"), (fk.FE_KS_F32, "f32"),
                       (fk.FE_KS_BF16, "bf16_tensor_core"), (fk.FE_KS_F16, "f16_tensor_core")):
        X = X64 if prec in (fk.FE_KS_F64, fk.FE_KS_F64E) else X64.to(torch.complex64)
        Y = torch.empty_like(X)
        fk.fe_ks_tune(ctx, X, Y, wl.n_v, prec, reps=1)
        fk.fe_ks_apply(ctx, X, Y, wl.n_v, prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3 if prec in (fk.FE_KS_F64,) else 10
        e0.record(stream)
        for _ in range(reps):
            fk.fe_ks_apply(ctx, X, Y, wl.n_v, prec)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms_per_step": ms, "value": units / (ms * 1e-3)}
        del X, Y
        torch.cuda.empty_cache()
    out["speedup_f32_vs_f64"] = out["f64"]["ms_per_step"] / out["f32"]["ms_per_step"]
    fk.fe_ks_destroy(ctx)
    del X64
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------- n_q = n_p + 2 quadrature
def run_quadrature_np2(args, wl0):
    """The same workload with n_q = n_p + 2 Gauss points per direction (the paper's default
    quadrature; non-square N^1D): FP64 and FP32 applications, tuned, timed with CUDA
    events (inputs larger than L2).  Returns a dict for the JSON line."""
    import dataclasses
    import numpy as np
    import torch
    from paper_2512_08571_gb300 import fe_ks as fk
    from synth.host_problem import HostProblem
    wl = dataclasses.replace(wl0, nq=wl0.p + 3, name=wl0.name + "-nq" + str(wl0.p + 3))
    stream = torch.cuda.current_stream()
    hp = HostProblem(wl)
    ctx = fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, stream.cuda_stream)
    info = fk.fe_ks_info(ctx)
    X64 = torch.empty((hp.m, wl.n_v), dtype=torch.float64, device="cuda")
    fill_trial(wl, wl.n_v, X64, np.float64)
    units = hp.m * wl.n_v
    flops, _ = alg_flops(wl, info["n_pairs"], wl.n_v)
    out = {"workload": f"{wl0.name} with n_q = n_p + 2 = {wl.nq}", "unit": UNIT, "alg_flops_per_apply": flops}
    for prec, name, peak in ((fk.FE_KS_F64, "f64", PEAK_FP64_NOMINAL), (fk.FE_KS_F32, "f32", PEAK_FP32_NOMINAL)):
        X = X64 if prec == fk.FE_KS_F64 else X64.to(torch.float32)
        Y = torch.empty_like(X)
        best, tune_ms = fk.fe_ks_tune(ctx, X, Y, wl.n_v, prec, reps=1)
        fk.fe_ks_apply(ctx, X, Y, wl.n_v, prec)
        torch.cuda.synchronize()
        reps = 2 if prec == fk.FE_KS_F64 else 10
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fk.fe_ks_apply(ctx, X, Y, wl.n_v, prec)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms_per_step": ms, "value": units / (ms * 1e-3), "tile_config": best,
                     "tune_ms_per_config": [round(t, 3) for t in tune_ms],
                     "alg_tflops": flops / (ms * 1e-3) / 1e12,
                     "frac_of_nominal_pipe": flops / (ms * 1e-3) / peak}
        del X, Y
        torch.cuda.empty_cache()
    fk.fe_ks_destroy(ctx)
    del X64
    torch.cuda.empty_cache()
    return out


# -------------------------------------------------------- batched systems
def small_systems():
    """Sixteen small systems (4^3 cells, degrees 4..8, N_v 8..32, FP64/FP32 alternating):
    the launch-bound regime a batched persistent launch is for."""
    from synth import Workload
    out = []
    for s in range(16):
        p = 4 + s % 5
        out.append(Workload(f"S{s}", L=6.0, n=4, p=p, nq=p + 1, n_v=8 * (1 + s % 4), gga=True, n_atoms=2,
                            seed=8000 + 10 * s, precision="f64" if s % 2 == 0 else "f32"))
    return out


def run_batched(args, wls=None):
    """Uneven systems (default: six, cell grids 6^3..20^3, degrees 4..8, N_v 16..512,
    FP64/FP32 alternating) in one persistent launch captured in a CUDA graph, against
    one fe_ks_apply per system.  Returns a dict for the JSON line."""
    import torch
    from paper_2512_08571_gb300 import fe_ks as fk
    from synth.host_problem import HostProblem
    from synth import batched_systems
    if wls is None:
        wls = batched_systems()
        if args.cells:
            wls = [wl.scaled(n=max(2, wl.n * args.cells // 20)) for wl in wls]
    stream = torch.cuda.current_stream()
    prec = [fk.FE_KS_F64 if wl.precision == "f64" else fk.FE_KS_F32 for wl in wls]
    ctxs, Xs, Ys = [], [], []
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5000)
    for wl, pr in zip(wls, prec):
        hp = HostProblem(wl)
        ctxs.append(fk.fe_ks_setup(hp.struct, fk.TERM_ALL, wl.n_v, stream.cuda_stream))
        dt = torch.float64 if pr == fk.FE_KS_F64 else torch.float32
        X = (torch.rand((wl.n_dofs, wl.n_v), generator=gen, device="cuda", dtype=dt) * 2 - 1)
        Xs.append(X)
        Ys.append(torch.empty_like(X))
    units = sum(wl.n_dofs * wl.n_v for wl in wls)
    for c, X, Y, wl, pr in zip(ctxs, Xs, Ys, wls, prec):
        fk.fe_ks_tune(c, X, Y, wl.n_v, pr, reps=2)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2

    def timed(fn, reps):
        """Mean of per-rep CUDA-event times, L2 flushed (256 MiB write) before each rep."""
        fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for e0, e1 in ev:
            flush.fill_(0.0)
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return sum(e0.elapsed_time(e1) for e0, e1 in ev) / reps

    def separate():
        for c, X, Y, wl, pr in zip(ctxs, Xs, Ys, wls, prec):
            fk.fe_ks_apply(c, X, Y, wl.n_v, pr)

    reps = max(args.steps, 20)
    ms_sep = timed(separate, reps)
    b = fk.fe_ks_batch_create(ctxs, [wl.n_v for wl in wls], prec)
    best = None
    trials = []
    is32 = [pr == fk.FE_KS_F32 for pr in prec]
    depth = 2
    for threads in (384, 512, 672):
        for occ in ((1, 2) if threads <= 512 else (1,)):
            for t64 in (0, 1):
                for t32 in (0, 1):
                    for cells in (1, 2, 4):
                        tiles = [t32 if f else t64 for f in is32]
                        fk.fe_ks_batch_configure(b, tiles, cells, depth, 2.0, False, blocks_per_sm=occ,
                                                 threads=threads)
                        ms = timed(lambda: fk.fe_ks_batch_apply(b, Xs, Ys, stream.cuda_stream), 2)
                        fk.fe_ks_batch_status(b)
                        trials.append({"threads": threads, "blocks_per_sm": occ, "tile_f64": t64, "tile_f32": t32,
                                       "cells_per_item": cells, "ms": round(ms, 3)})
                        if best is None or ms < best[0]:
                            best = (ms, tiles, cells, occ, threads)
    _, tiles, cells, occ, threads = best
    for d in (1, 4):                            # then the items claimed per fetch
        fk.fe_ks_batch_configure(b, tiles, cells, d, 2.0, False, blocks_per_sm=occ, threads=threads)
        ms = timed(lambda: fk.fe_ks_batch_apply(b, Xs, Ys, stream.cuda_stream), 2)
        fk.fe_ks_batch_status(b)
        trials.append({"threads": threads, "blocks_per_sm": occ, "tile_f64": tiles[0], "cells_per_item": cells,
                       "depth": d, "ms": round(ms, 3)})
        if ms < best[0]:
            best = (ms, tiles, cells, occ, threads)
            depth = d
    # split mode: the FP64 and FP32 systems in two concurrent class objects (only when both occur)
    split = (0, 0)
    if any(is32) and not all(is32):
        for t64, t32 in ((256, 384), (256, 512), (384, 384), (384, 512)):
            for sc in (1, 2):
                for t64c in (0, 1):
                    stiles = [tiles[i] if is32[i] else t64c for i in range(len(wls))]
                    fk.fe_ks_batch_configure(b, stiles, sc, depth, 2.0, False, blocks_per_sm=occ, threads=threads)
                    fk.fe_ks_batch_set_split(b, t64, t32)
                    ms = timed(lambda: fk.fe_ks_batch_apply(b, Xs, Ys, stream.cuda_stream), 2)
                    fk.fe_ks_batch_status(b)
                    trials.append({"split": [t64, t32], "tile_f64": t64c, "cells_per_item": sc, "ms": round(ms, 3)})
                    if ms < best[0]:
                        best = (ms, stiles, sc, occ, threads)
                        split = (t64, t32)
                    fk.fe_ks_batch_set_split(b, 0, 0)
    # direct systems: the largest ones (by their own application time) on their own tuned
    # kernels, on side streams beside the persistent launch of the others
    _, tiles, cells, occ, threads = best
    ms_each = [timed(lambda c=c, X=X, Y=Y, wl=wl, pr=pr: fk.fe_ks_apply(c, X, Y, wl.n_v, pr), 2)
               for c, X, Y, wl, pr in zip(ctxs, Xs, Ys, wls, prec)]
    order = sorted(range(len(wls)), key=lambda i: -ms_each[i])
    direct = None
    for k in sorted({1, 2, len(wls)}):
        flags = [1 if i in order[:k] else 0 for i in range(len(wls))]
        fk.fe_ks_batch_configure(b, tiles, cells, depth, 2.0, False, blocks_per_sm=occ, threads=threads)
        fk.fe_ks_batch_set_split(b, *split)
        fk.fe_ks_batch_set_direct(b, flags)
        ms = timed(lambda: fk.fe_ks_batch_apply(b, Xs, Ys, stream.cuda_stream), 2)
        fk.fe_ks_batch_status(b)
        trials.append({"direct": flags, "ms": round(ms, 3)})
        if ms < best[0]:
            best = (ms, tiles, cells, occ, threads)
            direct = flags
        fk.fe_ks_batch_set_direct(b, None)
    _, tiles, cells, occ, threads = best
    fk.fe_ks_batch_configure(b, tiles, cells, depth, 2.0, False, blocks_per_sm=occ, threads=threads)
    fk.fe_ks_batch_set_split(b, *split)
    fk.fe_ks_batch_set_direct(b, direct)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        fk.fe_ks_batch_apply(b, Xs, Ys, side.cuda_stream)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        fk.fe_ks_batch_apply(b, Xs, Ys, torch.cuda.current_stream().cuda_stream)
    ms_graph = timed(g.replay, reps)
    fk.fe_ks_batch_status(b)
    info = fk.fe_ks_batch_info(b)
    fk.fe_ks_batch_destroy(b)
    for c in ctxs:
        fk.fe_ks_destroy(c)
    return {"workload": f"{len(wls)} systems: grids " + ",".join(f"{wl.n}^3" for wl in wls) + "; p=" +
                        ",".join(str(wl.p) for wl in wls) + "; N_v=" + ",".join(str(wl.n_v) for wl in wls) +
                        "; " + ",".join(wl.precision for wl in wls),
            "value": units / (ms_graph * 1e-3), "unit": UNIT, "ms_per_step": ms_graph,
            "one_launch_per_system": {"value": units / (ms_sep * 1e-3), "ms_per_step": ms_sep},
            "speedup_vs_separate": ms_sep / ms_graph,
            "tuned": {"tile_config": tiles, "cells_per_item": cells, "depth": depth, "blocks_per_sm": occ,
                      "threads": threads, "split_threads": list(split), "direct_systems": direct},
            "ms_each_system_alone": [round(t, 3) for t in ms_each],
            "tuning_trials": trials, "items": info["n_items"], "grid": info["grid"],
            "smem_bytes": info["smem_bytes"], "graph": True, "x_inputs": "device RNG (seed 5000), U(-1,1)",
            "l2": "flushed (256 MiB write) before each timed rep"}


# ----------------------------------------------------------- oracle timing
_ORACLE = {}


def oracle_sample(wl, budget_s, max_cells=None):
    """Time the FP64 oracle (cell-matrix method: per-cell H^(e) by quadrature, then
    H^(e) X^(e)) on host cores over a sample of cells until the budget is spent.
    Returns (DoF*vec/s, cells done, seconds)."""
    import numpy as np
    from oracle.operator import Problem
    from synth import trial_vectors
    if wl.name not in _ORACLE:
        _ORACLE[wl.name] = Problem(wl, with_atoms=False)
    P = _ORACLE[wl.name]
    rng = np.random.default_rng(12345)
    order = rng.permutation(P.E)
    done, t0 = 0, time.perf_counter()
    for e in order:
        Xe = trial_vectors(wl, rows=P.dofs[e])
        Ye = P.cell_matrix(e) @ Xe
        assert Ye.shape == Xe.shape
        done += 1
        if time.perf_counter() - t0 > budget_s or (max_cells and done >= max_cells):
            break
    el = time.perf_counter() - t0
    units = done / P.E * wl.n_dofs * wl.n_v
    return units / el, done, el


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


# ------------------------------------------------------------------- main
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    from synth import CONFIGS
    wl = CONFIGS[args.workload]
    if args.cells:
        wl = wl.scaled(n=args.cells)
    config = {"workload": f"{wl.name}: L={wl.L:g} bohr, {wl.n}^3 cells, p={wl.p}, n_q={wl.nq}, "
                          f"N_v={wl.n_v}, {'complex' if wl.complex else 'real'}, GGA={wl.gga}, "
                          f"atoms={wl.n_atoms}",
              "n_dofs": wl.n_dofs, "n_v": wl.n_v, "degree": wl.p, "n_q": wl.nq,
              "l2": "inputs larger than L2 (X = %.1f GB), no flush" % (wl.n_dofs * wl.n_v * 8 / 1e9),
              "parallelism": f"replicas x{args.gpus}"}

    if args.impl == "reference":
        if rank != 0:
            return
        for _ in range(args.warmup):
            oracle_sample(wl, 1e9, max_cells=2)
        vals, secs = [], []
        for _ in range(args.steps):
            v, n, el = oracle_sample(wl, 1e9, max_cells=4)
            vals.append(v)
            secs.append(el)
        value = len(vals) / sum(1.0 / v for v in vals)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                                 "sample": f"4 cells of {wl.n_cells} per step (cell-matrix method, local "
                                           f"terms, all {wl.n_v} vectors), scaled to the whole operator"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    res = run_native(args, wl, rank, world)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    f64 = res["f64"]
    if f64 is None:
        pr = res["mixed"] or res["f64e"] or res["bf16"] or res["f16"] or res["bf16x2"]
        print(json.dumps({"metric": METRIC, "profiling_only": True, "precision": args.precision, "ms": pr["ms"],
                          "value": pr["value"], "local_launch_ms": pr["local_launch_ms"],
                          "profile_ms_per_step": {k: v[0] / max(1, args.steps) for k, v in pr["prof"].items()}}))
        return
    detail = detail_sections(args, wl, res, world)
    if world == 1 and not args.no_cpu_baseline:
        v, n, el = oracle_sample(wl, args.cpu_seconds)
        detail["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                                  "sample": f"{n} of {wl.n_cells} cells in {el:.1f} s (cell-matrix method: "
                                            f"H^(e) by quadrature then H^(e) X^(e), local terms, all "
                                            f"{wl.n_v} vectors), scaled to the whole operator"}
    line = compact_line(detail, args, config, world)
    if args.detail:
        try:
            os.makedirs(os.path.dirname(os.path.abspath(args.detail)), exist_ok=True)
            with open(args.detail, "w") as f:
                json.dump(detail, f, indent=1)
            line["detail"] = args.detail
        except OSError as exc:
            sys.stderr.write(f"bench: could not write {args.detail}: {exc}\n")
    print(json.dumps(line, separators=(",", ":")))
    if world > 1:
        torch.distributed.destroy_process_group()


def _r(x, n=4):
    """Round to n significant digits for the compact line (None stays None)."""
    if x is None:
        return None
    if isinstance(x, (int,)) and not isinstance(x, bool):
        return x
    try:
        return float(f"{float(x):.{n}g}")
    except (TypeError, ValueError):
        return x


def detail_sections(args, wl, res, world):
    """Every measured section of a run, as one dict (written to the detail file).  The
    final JSON line is a compact digest of it (compact_line)."""
    f64 = res["f64"]
    traffic = load_traffic(f"fe_local_kernel f64 {wl.name} cfg{f64['tile_config']}")
    achieved = f64["achieved"]
    detail = {"workload": wl.name, "setup_s": res["setup_s"], "info": res["info"],
              "alg_flops_local_per_apply": res["local_flops"],
              "peak_fp64_live_tflops": res["peak64_live"] / 1e12,
              "peak_fp32_live_tflops": res["peak32_live"] / 1e12}
    detail["f64"] = {
        "value": f64["value"], "ms_per_step": f64["ms"], "clocks": f64["clocks"], "gpu_launches": f64["launches"],
        "profile_ms": {k: v[0] for k, v in f64["prof"].items()},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12 if achieved else None,
                     "peak": PEAK_FP64_NOMINAL / 1e12, "unit": "TFLOP/s",
                     "frac": (achieved / PEAK_FP64_NOMINAL) if achieved else None, "traffic": traffic,
                     "kernel": "fe_local_kernel (FP64 DFMA pipe)",
                     "peak_source": "nominal FP64 1.25 TFLOP/s; live DFMA probe %.3f TFLOP/s"
                                    % (res["peak64_live"] / 1e12),
                     "frac_of_live_probe": (achieved / res["peak64_live"]) if achieved else None,
                     "avg_launch_ms": f64["local_launch_ms"], "tile_config": f64["tile_config"],
                     "tune_ms_per_config": f64["tune_ms"]}}
    if res.get("f64e"):
        e = res["f64e"]
        ach = e["achieved"]
        detail["f64_pairs_of_fp32"] = {
            "dtype": "f32x2 (FP64 in/out, FP64-accurate)", "value": e["value"], "ms_per_step": e["ms"],
            "speedup_vs_f64": f64["ms"] / e["ms"], "err_col": e.get("err_col"), "err_elem": e.get("err_elem"),
            "alg_fp64_equiv_tflops": ach / 1e12 if ach else None,
            "frac_of_nominal_fp64": ach / PEAK_FP64_NOMINAL if ach else None,
            "avg_launch_ms": e["local_launch_ms"], "tile_config": e["tile_config"],
            "tune_ms_per_config": e["tune_ms"], "clocks": e["clocks"], "gpu_launches": e["launches"]}
    mixed = res["mixed"]
    if mixed:
        ach = mixed["achieved"]
        detail["f32"] = {
            "dtype": "f32", "value": mixed["value"], "ms_per_step": mixed["ms"],
            "speedup_vs_f64": f64["ms"] / mixed["ms"], "err_col": mixed.get("err_col"),
            "err_elem": mixed.get("err_elem"),
            "roofline": {"bound": "alu", "achieved": ach / 1e12 if ach else None,
                         "peak": PEAK_FP32_NOMINAL / 1e12, "unit": "TFLOP/s",
                         "frac": ach / PEAK_FP32_NOMINAL if ach else None,
                         "live_probe": res["peak32_live"] / 1e12, "avg_launch_ms": mixed["local_launch_ms"],
                         "tile_config": mixed["tile_config"],
                         "traffic": load_traffic(f"fe_local_kernel f32 {wl.name} cfg{mixed['tile_config']}"),
                         "tune_ms_per_config": mixed["tune_ms"]},
            "clocks": mixed["clocks"], "gpu_launches": mixed["launches"]}
    for key, name, dts in (("bf16", "bf16_tensor_core", "bf16 x bf16 -> f32 (FP32 storage)"),
                           ("f16", "f16_tensor_core", "f16 x f16 -> f32 (FP32 storage, power-of-two column scaling)"),
                           ("bf16x2", "bf16x2_tensor_core",
                            "split bf16 hi + lo, three products -> f32 (FP32 storage)")):
        bf = res[key]
        if not bf:
            continue
        # HBM roofline (FP32 storage): X read once + Y written once per application, plus
        # the coefficients; the executed MMA rate is reported against the live mma.sync probe
        alg_bytes = 2 * res["bytes32"]["xy"] + res["bytes32"]["coef"]
        t_roof = alg_bytes / (PEAK_HBM_GBS * 1e9)
        detail[name] = {
            "dtype": dts, "value": bf["value"], "ms_per_step": bf["ms"], "speedup_vs_f64": f64["ms"] / bf["ms"],
            "speedup_vs_fp32_cuda_core": (mixed["ms"] / bf["ms"]) if mixed else None,
            "err_col": bf.get("err_col"), "err_elem": bf.get("err_elem"),
            "roofline": {"bound": "hbm", "achieved": alg_bytes / (bf["ms"] * 1e-3) / 1e9,
                         "peak": PEAK_HBM_GBS, "unit": "GB/s", "frac": t_roof / (bf["ms"] * 1e-3),
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                         "alg_bytes_per_apply": alg_bytes, "avg_launch_ms": bf["local_launch_ms"],
                         "mma_tflops_executed": res["mma_flops_per_apply"] * (3 if key == "bf16x2" else 1) * 1e-12
                                                / (bf["ms"] * 1e-3),
                         "mma_sync_live_probe_tflops": (res["peak_mma_live"] or 0) / 1e12},
            "clocks": bf["clocks"], "gpu_launches": bf["launches"]}
        tcgen05 = key in ("bf16", "f16") and bf.get("tile_config") != 1 and not wl.complex and wl.nq == wl.p + 1
        detail[name]["kernel"] = (f"tcgen05 (plane and z-sweep products, tile configuration {bf.get('tile_config')})"
                                  if tcgen05 else
                                  "warp-level mma.sync (one sweep per direction)")
        detail[name]["tile_config"] = bf.get("tile_config")
        detail[name]["tune_ms_per_config"] = [t for t in bf.get("tune_ms", []) if t > 0]
        if tcgen05:
            # tcgen05 MMA work executed per application: per cell and 4-vector tile, GEMM1
            # (plane, 2 M-tiles x K 96 x N 48), GEMM2 and GEMM3 (3 M-tiles x K 48 x N 48) and
            # GEMM4 (K 256 x N 64), all with M = 128
            n = wl.p + 1
            nn = n * n
            mt1, kp, n1 = -(-3 * nn // 128), -(-nn // 16) * 16, -(-4 * n // 16) * 16
            mt2, n2, k4 = -(-4 * nn // 128), -(-4 * n // 16) * 16, -(-3 * nn // 16) * 16
            per_tile = 2 * 128 * (mt1 * kp * n1 + mt2 * 48 * n2 + mt2 * n2 * 48 + k4 * 64)
            fl = wl.n_cells * -(-wl.n_v // 4) * per_tile
            detail[name]["roofline"]["tcgen05_tflops_executed"] = fl / (bf["ms"] * 1e-3) / 1e12
            detail[name]["roofline"]["tcgen05_frac_of_bf16_peak"] = fl / (bf["ms"] * 1e-3) / (PEAK_BF16_TFLOPS * 1e12)
    if res["e2e"]:
        detail["e2e"] = res["e2e"]
    if res["filter"]:
        detail["filter"] = res["filter"]
    if res["cell_matrix"]:
        detail["cell_matrix_baseline"] = res["cell_matrix"]
    if not args.no_all_electron and world == 1:
        detail["all_electron_like"] = run_all_electron(args)
    if not args.no_nq2 and world == 1 and not wl.complex:
        q2 = run_quadrature_np2(args, wl)
        q2["f64"]["vs_n_q_eq_n_p"] = q2["f64"]["ms_per_step"] / f64["ms"]
        if mixed:
            q2["f32"]["vs_n_q_eq_n_p"] = q2["f32"]["ms_per_step"] / mixed["ms"]
        detail["quadrature_n_p_plus_2"] = q2
    if not args.no_batched:
        detail["batched"] = run_batched(args)
        detail["batched_small_systems"] = run_batched(args, small_systems())
    return detail


def compact_line(detail, args, config, world):
    """The one JSON line the benchmark prints last: the headline (FP64 application at the
    workload's full size), its roofline, clocks, end-to-end and CPU-oracle numbers, and a
    one-number digest of every other section (the full sections go to the detail file).
    Kept to a few KB so that a reader of the output's tail sees all of it."""
    f64 = detail["f64"]
    rf = f64["roofline"]
    line = {"metric": METRIC, "value": _r(f64["value"], 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": _r(f64["ms_per_step"], 6), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded mesh, fields, atoms, X)", "config": config,
            "roofline": {"bound": rf["bound"], "achieved": _r(rf["achieved"]), "peak": rf["peak"],
                         "unit": rf["unit"], "frac": _r(rf["frac"]), "traffic": rf["traffic"],
                         "kernel": rf["kernel"], "avg_launch_ms": _r(rf["avg_launch_ms"]),
                         "frac_of_live_probe": _r(rf["frac_of_live_probe"]),
                         "peak_source": rf["peak_source"]},
            "clocks": {k: f64["clocks"].get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "gpu_launches": f64["gpu_launches"]}
    e2e = detail.get("e2e")
    if e2e:
        line["e2e"] = {"value": _r(e2e["value"]), "unit": e2e["unit"], "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                       "d2h_bytes_per_step": e2e["d2h_bytes_per_step"], "ms_per_step": _r(e2e["ms_per_step"]),
                       "steps": e2e["steps"], "api": "fe_ks_apply_host (pinned host X in, Y out)"}
    cb = detail.get("cpu_baseline")
    if cb:
        line["cpu_baseline"] = {"value": _r(cb["value"]), "unit": cb["unit"], "cores": cb["cores"],
                                "kind": cb["kind"], "sample": cb["sample"]}
    prec = {}
    for key, name in (("f64_pairs_of_fp32", "f64_pairs"), ("f32", "f32"), ("bf16_tensor_core", "bf16_tc"),
                      ("f16_tensor_core", "f16_tc"), ("bf16x2_tensor_core", "bf16x2_tc")):
        d = detail.get(key)
        if not d:
            continue
        q = {"ms": _r(d["ms_per_step"]), "value": _r(d["value"]), "x_f64": _r(d["speedup_vs_f64"], 3),
             "err_col": _r(d.get("err_col"), 2), "err_elem": _r(d.get("err_elem"), 2)}
        if "roofline" in d:
            q["frac"] = _r(d["roofline"]["frac"], 3)
            q["bound"] = d["roofline"]["bound"]
        elif "frac_of_nominal_fp64" in d:
            q["frac"] = _r(d["frac_of_nominal_fp64"], 3)
            q["bound"] = "alu"
        if d.get("kernel"):
            q["kernel"] = "tcgen05" if d["kernel"].startswith("tcgen05") else "mma.sync"
        if "roofline" in d and "tcgen05_frac_of_bf16_peak" in d["roofline"]:
            q["tensor_frac"] = _r(d["roofline"]["tcgen05_frac_of_bf16_peak"], 3)
        prec[name] = q
    if prec:
        line["precisions"] = prec
        line["errors_vs"] = "the FP64 application of the same X (all entries)"
    flt = detail.get("filter")
    if flt:
        fl = {"speedup_filter_mixed": _r(flt.get("speedup_filter_mixed_vs_f64"), 3),
              "speedup_pass_mixed": _r(flt.get("speedup_pass_mixed_vs_f64"), 3),
              "pass_ms": {k: _r(flt[k]["pass_ms"]) for k in ("f64", "f64_pairs", "mixed", "mixed_bf16",
                                                              "mixed_f16", "mixed_bf16x2", "mixed_ff_rr")
                          if isinstance(flt.get(k), dict) and "pass_ms" in flt[k]},
              "rr_ms": {k: _r(flt[k]["rayleigh_ritz_ms"]) for k in ("f64", "mixed", "mixed_ff_rr")
                        if isinstance(flt.get(k), dict) and "rayleigh_ritz_ms" in flt[k]}}
        conv = flt.get("converged")
        if conv:
            fl["converged"] = {k: _r(conv[k], 3) for k in ("passes_f64", "passes_mixed", "ms_mixed", "ms_f64",
                                                           "ms_f64_derived", "f64_pass_ms", "speedup",
                                                           "max_eig_diff_Ha", "max_eig_err_bound_Ha", "degree")
                               if k in conv}
            fl["converged"]["reached_tol"] = bool(conv.get("converged"))
            fl["converged"]["workload"] = conv.get("workload")
            fl["converged"]["speedup_basis"] = conv.get("speedup_basis")
        c6 = flt.get("converged_6cubed")
        if c6:
            fl["converged_6cubed"] = {"speedup": _r(c6.get("speedup"), 3),
                                      "max_eig_diff_Ha": _r(c6.get("max_eig_diff_mixed_vs_f64_Ha"), 2)}
        line["filter"] = fl
    for key, name in (("batched", "batched_c5"), ("batched_small_systems", "batched_small")):
        b = detail.get(key)
        if b:
            line[name] = {"ms": _r(b["ms_per_step"]), "x_separate": _r(b["speedup_vs_separate"], 3)}
    ae = detail.get("all_electron_like")
    if ae:
        line["all_electron_like"] = {k: _r(ae[k]["ms_per_step"]) for k in ("f64", "f32", "bf16_tensor_core")
                                     if k in ae}
    cm = detail.get("cell_matrix_baseline")
    if cm and isinstance(cm.get("f64"), dict):
        line["cell_matrix_f64_ms"] = _r(cm["f64"].get("ms_per_step"))
    return line


if __name__ == "__main__":
    main()
