"""Benchmark: reconstructions/sec to relative residual 1e-4 on the
128x128x64, k = 2..9, s = 2 synthetic workload (one step = one full MH3D
reconstruction: A^T d, CG on the normal equations to rel. residual 1e-4,
true-residual check), plus the HBM roofline of one CG iteration (the
unit that dominates a step) and of the forward operator A.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mh3d|reference]
       [--mode 0|1] [--workload NAME]
Under torchrun (N > 1) every rank solves its own volume (independent
replicas, no data-path collective); the timing barrier and the max over ranks
use the default process group.
Prints ONE JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "reconstructions/sec to rel. residual 1e-4"
PRECISION = ("FP32 operator and vectors; inner products: exact FP32 products summed in float pairs (hi + lo), "
             "FP64 totals; CG step lengths and stopping test FP64")
UNIT = "reconstructions/s"
WORKLOAD = "mh_128x128x64_k8_s2"
# DRAM bytes (read + write) of one CG iteration's three kernels, summed from
# one ncu capture with cold L2 (ncu's default cache flush between kernels).
TRAFFIC_PER_ITER_FUSED = 37891584   # 25.23 MB T_y + 12.66 MB fused T_z + X normal (mean of four iterations)
TRAFFIC_PER_ITER = 42103808   # 25.22 MB T_y + 4.24 MB T_z + 12.64 MB X normal (mean of two iterations), writes stay in L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mh3d", choices=["mh3d", "reference"])
    ap.add_argument("--mode", type=int, default=0, help="0 fused normal operator, 1 explicit A then A^T")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default launch variants instead of the autotuner's choice")
    ap.add_argument("--batched", action="store_true",
                    help="the 64-volume batched workload (one JSON line of its own)")
    ap.add_argument("--learned", action="store_true",
                    help="train the warm-start network and compare warm and zero starts (own JSON line)")
    ap.add_argument("--mhad", action="store_true",
                    help="MHAD image timing and the MHAD warm start against the zero start (own JSON line)")
    ap.add_argument("--mhad-lambda", type=float, default=1e-2)
    ap.add_argument("--general", action="store_true",
                    help="the general (three-component, non-separable PSF) operators' timing (own JSON line)")
    ap.add_argument("--train-n", type=int, default=2000)
    ap.add_argument("--test-n", type=int, default=200)
    ap.add_argument("--batch-n", type=int, default=32,
                    help="learned: volumes of the batched zero-start / warm-start comparison")
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--channels", type=int, nargs="+", default=[16, 32, 64, 128],
                    help="learned: channels per level of the warm-start network (2..5 levels; default the "
                         "four-level 16-128 network)")
    ap.add_argument("--count-iters", action="store_true",
                    help="reference arm: run the oracle's CG to the tolerance once and print its iteration count")
    return ap.parse_args()


def fused_zx(wl) -> bool:
    """Whether the library runs T_z together with the drive-axis pass (normal,
    forward and adjoint operators) as one cluster launch for this workload
    (its instantiated (nx, nz, s) pairs, unless MH3D_FUSE_ZX=0 or
    MH3D_GENERIC=1)."""
    if os.environ.get("MH3D_FUSE_ZX", "1").startswith("0") or os.environ.get("MH3D_GENERIC", "0") not in ("", "0"):
        return False
    nx, _, nz = wl.n
    return wl.ds_factor == 2 and (nx, nz) in ((128, 64), (64, 64), (96, 64))


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_throughput(local_total_s: float, steps: int, device):
    """Whole-job throughput of independent replicas (one volume per rank, no
    data-path collective): the job time is the slowest rank's (one MAX
    all-reduce of the timing only) and the value counts every rank's steps.
    Returns (value, job_seconds)."""
    import torch
    import torch.distributed as dist

    ws, total = 1, float(local_total_s)
    if dist.is_available() and dist.is_initialized():
        ws = dist.get_world_size()
        t = torch.tensor([total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    return ws * steps / total, total


def make_case(wl: W.Workload, seed: int, forward_fn):
    """Phantom, sensitivity and noisy portraits at the workload's SNR.
    forward_fn(rho) -> clean portraits (complex, numpy)."""
    rho = W.phantom(wl.n, wl.voxel_mm, seed, wl.n_blobs, wl.n_lines, wl.log_amplitudes)
    b = W.sensitivity(wl.n, wl.voxel_mm, kind=wl.sens)
    return rho, b


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mh3d_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.5)   # nvidia-smi's start-up, so that sampling covers the timed region
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            return self._summary()
        finally:
            try:
                os.remove(self.path)
            except OSError:
                pass

    def _summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def bench_mh3d(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    else:
        torch.cuda.set_device(0)
    from paper_2503_13802_gb300 import (Plan, make_opts, mh3d_adjoint, mh3d_forward, mh3d_plan_autotune,
                                        mh3d_plan_tuning, mh3d_solve, mh3d_solve_host)

    wl = W.WORKLOADS[args.workload]
    dev = torch.device("cuda", torch.cuda.current_device())
    seed = wl.seeds[rank % len(wl.seeds)]
    rho, b = make_case(wl, seed, None)
    nx, ny, nz = wl.n
    plan = Plan(wl.n, voxel_mm=wl.voxel_mm, ds_factor=wl.ds_factor, k_min=wl.k_min, k_max=wl.k_max,
                sensitivity=b)
    K = wl.k_max - wl.k_min + 1
    mx = nx // wl.ds_factor
    rho_t = torch.as_tensor(rho, dtype=torch.float32, device=dev).contiguous()
    d = torch.empty((K, nz, ny, mx), dtype=torch.complex64, device=dev)
    mh3d_forward(plan, rho_t, d)
    sig2 = float(torch.sum(torch.abs(d.to(torch.complex128)) ** 2)) / (d.numel() * 10 ** (wl.snr_db / 10))
    noise = torch.as_tensor(W.unit_complex_noise(tuple(d.shape), seed).astype(np.complex64), device=dev)
    d = (d + math.sqrt(sig2) * noise).contiguous()
    x = torch.empty((nz, ny, nx), dtype=torch.float32, device=dev)
    opts = make_opts(lam=wl.lam, lam_relative=True, rel_tol=wl.rel_tol, max_iter=wl.max_iter,
                     fixed_iters=wl.fixed_iters, normal_mode=args.mode)
    # the library's autotuner picks the launch variants for this size (set-up, untimed)
    tuning = None
    if not args.no_autotune:
        mh3d_plan_autotune(plan)
        tuning = mh3d_plan_tuning(plan)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        info = mh3d_solve(plan, d, opts, x)
    # timed region: K reconstructions, L2 flushed between steps (outside the events)
    times, iters = [], []
    with Clocks(torch.cuda.current_device()) as clk:
        barrier()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = mh3d_solve(plan, d, opts, x)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            iters.append(info["iters"])
        barrier()
    value, total = replica_throughput(sum(times), args.steps, dev)

    it_med = int(statistics.median(iters))
    N = nx * ny * nz
    M = K * mx * ny * nz

    # Roofline of one CG iteration, the unit that dominates a step: the loop
    # body's three kernels (T_y with the fused CG vector update, T_z, and the
    # drive-axis normal pass with b, lambda p and the two dot products).  The
    # loop runs inside a CUDA graph, so its per-iteration duration is measured
    # live with events on this stream as the difference of two solves with a
    # fixed iteration count (it_med and 2): set-up and exit work cancel.
    def fixed_solve_seconds(n_it, reps=5, fp32_div=False):
        of = make_opts(lam=wl.lam, lam_relative=True, max_iter=n_it, fixed_iters=1, normal_mode=args.mode,
                       fp32_scalar_div=fp32_div)
        mh3d_solve(plan, d, of, x)
        ts = []
        for _ in range(reps):
            flush.zero_()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            mh3d_solve(plan, d, of, x)
            a1.record(stream)
            a1.synchronize()
            ts.append(a0.elapsed_time(a1) / 1e3)
        return statistics.median(ts)

    it_lo = 2
    it_s = (fixed_solve_seconds(it_med) - fixed_solve_seconds(it_lo)) / (it_med - it_lo)
    # the same with CG's beta and alpha as FP32 quotients (fp32_scalar_div),
    # for the cost of the default FP64 quotients
    it_s_f32 = (fixed_solve_seconds(it_med, fp32_div=True) - fixed_solve_seconds(it_lo, fp32_div=True)) / (
        it_med - it_lo)
    # Algorithmic bytes of one CG iteration: the CG vectors x, r and p read
    # and written once each and b read once, 7 float32 vectors of N (28 N
    # bytes); the operator's intermediates stay on chip in this count.  The
    # single-reduction form this library runs also streams s and q (11
    # vectors, `design_alg_bytes`), and its passes move two intermediate
    # volumes and second reads of b and r (17 vectors, `design_bytes_per_iter`).
    it_alg = 7 * 4 * N if args.mode == 0 else 7 * 4 * N + 2 * 8 * M

    # Roofline of the forward operator A (T_y + T_z + X_fwd), L2 flushed
    # before each application so rho and b come from HBM and d goes to HBM.
    fwd_t, adj_t = [], []
    r_out = torch.empty_like(x)
    for i in range(10 + 3):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mh3d_forward(plan, rho_t, d)
        e1.record(stream)
        flush.zero_()
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        mh3d_adjoint(plan, d, r_out)
        e3.record(stream)
        torch.cuda.synchronize()
        if i >= 3:
            fwd_t.append(e0.elapsed_time(e1) / 1e3)
            adj_t.append(e2.elapsed_time(e3) / 1e3)
    # the same operators through cuFFT (torch.fft) and torch's elementwise kernels
    cf = CufftOperators(plan, torch.as_tensor(b, dtype=torch.float32, device=dev).contiguous())
    cf_f, cf_a = [], []
    d_cf = torch.empty_like(d)
    r_cf = torch.empty_like(x)
    for i in range(6 + 2):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cf.forward(rho_t, d_cf)
        e1.record(stream)
        flush.zero_()
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        cf.adjoint(d, r_cf)
        e3.record(stream)
        torch.cuda.synchronize()
        if i >= 2:
            cf_f.append(e0.elapsed_time(e1) / 1e3)
            cf_a.append(e2.elapsed_time(e3) / 1e3)
    alg_bytes = 4 * N + 4 * N + 8 * M          # rho + b + complex64 portraits
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    fwd_s = statistics.mean(fwd_t)
    adj_s = statistics.mean(adj_t)
    achieved = it_alg / it_s / 1e9

    # e2e: host portraits in, host image out, through the C ABI
    d_host = d.cpu().pin_memory()
    x_host = torch.empty((nz, ny, nx), dtype=torch.float32).pin_memory()
    mh3d_solve_host(plan, d_host, opts, x_host)
    e2e_t = []
    for _ in range(max(3, min(args.steps, 10))):
        t0 = time.perf_counter()
        mh3d_solve_host(plan, d_host, opts, x_host)
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = 1.0 / statistics.mean(e2e_t)

    # explicit A-then-A^T reconstructions for comparison (mode 1)
    other = None
    if args.mode == 0:
        o1 = make_opts(lam=wl.lam, lam_relative=True, rel_tol=wl.rel_tol, max_iter=wl.max_iter, normal_mode=1)
        mh3d_solve(plan, d, o1, x)
        tt = []
        for _ in range(5):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            inf1 = mh3d_solve(plan, d, o1, x)
            e1.record(stream)
            e1.synchronize()
            tt.append(e0.elapsed_time(e1) / 1e3)
        other = {"mode": "explicit A then A^T (portrait through L2/HBM)", "value": 5 / sum(tt),
                 "iters": inf1["iters"]}

    # the relative lambda sets the conditioning and so the iteration count:
    # the same reconstruction at lambda = 1e-4 ||A||_2^2 (kappa ~ 1e4), same rule
    lam_sens = None
    if args.mode == 0:
        o4 = make_opts(lam=wl.lam * 0.1, lam_relative=True, rel_tol=wl.rel_tol, max_iter=20 * wl.max_iter)
        inf4 = mh3d_solve(plan, d, o4, x)
        tt = []
        for _ in range(5):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            inf4 = mh3d_solve(plan, d, o4, x)
            e1.record(stream)
            e1.synchronize()
            tt.append(e0.elapsed_time(e1) / 1e3)
        lam_sens = {"lambda": wl.lam * 0.1, "value": 5 / sum(tt), "unit": UNIT, "iters": inf4["iters"],
                    "status": inf4["status"], "rel_res_true": inf4["rel_res_true"]}

    # kernels per solve: A^T d (3, or 2 with the fused adjoint pass), CG init
    # (1), s0 = N r0 (per_iter), the graph loop (two iterations per body,
    # every body launches all its kernels), the true residual (per_iter + 1)
    per_iter = (2 if fused_zx(wl) else 3) if args.mode == 0 else 6
    adj_launches = 2 if fused_zx(wl) else 3
    launches_per_step = adj_launches + 1 + per_iter + per_iter * 2 * ((it_med + 1) // 2) + per_iter + 1
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "precision": PRECISION, "data": "synthetic",
        "config": {"workload": wl.name, "grid": list(wl.n), "harmonics": [wl.k_min, wl.k_max],
                   "ds_factor": wl.ds_factor, "sensitivity": wl.sens, "phantom": f"{wl.n_blobs} blobs + {wl.n_lines} lines",
                   "snr_db": wl.snr_db, "lambda": wl.lam, "rel_tol": wl.rel_tol,
                   "normal_mode": "fused Fourier-block A^T A" if args.mode == 0 else "explicit A then A^T",
                   "cg_iters": it_med, "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{ws}", "autotune": tuning},
        "roofline": {"kernel": ("CG iteration = graph body (k_tpass_ct T_y + CG update, k_zxnrm_ct T_z + "
                                "drive-axis normal pass)" if fused_zx(wl) else
                                "CG iteration = graph body (k_tpass_ct T_y + CG update, k_tpass_ct T_z, k_xnrm_ct)")
                               if args.mode == 0 else "CG iteration, explicit A then A^T",
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": (TRAFFIC_PER_ITER_FUSED if fused_zx(wl) else TRAFFIC_PER_ITER)
                                if args.mode == 0 else None,
                     "alg_bytes_per_launch": it_alg, "us_per_launch": it_s * 1e6,
                     "alg_bytes_note": "per CG iteration: x, r, p read + written and b read (28 N bytes)",
                     "design_alg_bytes": 11 * 4 * N,
                     "design_bytes_per_iter": (15 if fused_zx(wl) else 17) * 4 * N,
                     "fp32_scalar_div_us_per_iter": it_s_f32 * 1e6,
                     "forward_A": {"us": fwd_s * 1e6, "alg_bytes": alg_bytes, "achieved_gbs": alg_bytes / fwd_s / 1e9,
                                   "frac": alg_bytes / fwd_s / 1e9 / peak},
                     "adjoint_AT": {"us": adj_s * 1e6, "alg_bytes": alg_bytes,
                                    "achieved_gbs": alg_bytes / adj_s / 1e9, "frac": alg_bytes / adj_s / 1e9 / peak},
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
        "cufft_comparison": {"what": "A and A^T with cuFFT (torch.fft) + torch elementwise kernels, same spectra",
                             "forward_us": 1e6 * statistics.mean(cf_f), "adjoint_us": 1e6 * statistics.mean(cf_a),
                             "forward_speedup_of_mh3d": statistics.mean(cf_f) / fwd_s,
                             "adjoint_speedup_of_mh3d": statistics.mean(cf_a) / adj_s},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(8 * M),
                "d2h_bytes_per_step": int(4 * N)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
    }
    if other:
        line["explicit_mode"] = other
    if lam_sens:
        line["lambda_sensitivity"] = lam_sens
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def oracle_case(wl: W.Workload):
    """The bench workload's first volume for the FP64 oracle: geometry,
    tables, sensitivity and noisy portraits (seed wl.seeds[0]); the relative
    lambda's ||A||_2^2 (the oracle's own Lanczos) is computed here, as set-up."""
    import oracle

    g = oracle.Geometry(n=wl.n, voxel_mm=wl.voxel_mm, ds_factor=wl.ds_factor, k_min=wl.k_min, k_max=wl.k_max)
    rho = W.phantom(wl.n, wl.voxel_mm, wl.seeds[0], wl.n_blobs, wl.n_lines, wl.log_amplitudes)
    b = W.sensitivity(wl.n, wl.voxel_mm, kind=wl.sens)
    tables = oracle.psf_tables(g)
    clean = oracle.forward(g, rho, b, tables)
    sig2 = np.sum(np.abs(clean) ** 2) / (clean.size * 10 ** (wl.snr_db / 10))
    d = clean + math.sqrt(sig2) * W.unit_complex_noise(clean.shape, wl.seeds[0])
    lam_abs = wl.lam * oracle.operator_norm2(g)
    opts = oracle.SolveOpts(lam=lam_abs, rel_tol=wl.rel_tol, max_iter=wl.max_iter)
    return g, tables, b, d, opts


def oracle_reconstruction(g, tables, b, d, opts):
    """One whole reconstruction by the oracle (A^T d, CG to the stopping
    rule); returns (seconds, iterations)."""
    import oracle

    t0 = time.perf_counter()
    _, it, _ = oracle.cg(g, d, b, opts, tables=tables)
    return time.perf_counter() - t0, int(it)


def cpu_baseline(wl: W.Workload):
    """The FP64 oracle as it stands on all host cores: one whole
    reconstruction of the bench workload (A^T d, CG to rel. residual 1e-4),
    timed, nothing scaled."""
    import oracle

    case = oracle_case(wl)
    t, it = oracle_reconstruction(*case)
    cores = oracle.num_threads()
    return {"value": 1.0 / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one whole reconstruction at {tuple(wl.n)} K={wl.k_max - wl.k_min + 1} s={wl.ds_factor}: "
                      f"oracle A^T d + CG to rel. residual {wl.rel_tol:g} ({it} iterations, {t:.1f} s on "
                      f"{cores} threads), not scaled"}


class CufftOperators:
    """The forward and adjoint operators written with cuFFT (torch.fft) and
    torch's elementwise kernels, from the plan's own spectra: the comparison
    arm for the hand-written passes (same model, same inputs, same GPU).
    Forward: U = DFT3(b rho) (nz Z)(ny Y); per harmonic, fold the drive-axis
    spectrum of U nx X_k by s (the row selector), inverse DFT on the portrait
    mesh, times e^{i theta_k}.  Adjoint: per harmonic, DFT3 of
    Re(e^{-i theta_k} y_k), periodised s times (zero insertion), times
    conj(nx X_k); the sum times conj((nz Z)(ny Y)), inverse DFT3, times b."""

    def __init__(self, plan, b_t):
        import torch

        from paper_2503_13802_gb300 import mh3d_plan_spectra

        X, Y, Z, ph = mh3d_plan_spectra(plan)
        self.nz, self.ny, self.nx = plan.shape
        self.K = plan.K
        self.mx = plan.portrait_shape[3]
        self.s = self.nx // self.mx
        self.Xt = X * self.nx
        self.Hyz = (Z * self.nz)[:, None, None] * (Y * self.ny)[None, :, None]
        self.ph = ph
        self.b = b_t
        self.torch = torch

    def forward(self, rho, d):
        torch = self.torch
        u = rho * self.b if self.b is not None else rho
        U = torch.fft.fftn(u.to(torch.complex64), dim=(0, 1, 2)) * self.Hyz
        for k in range(self.K):
            V = (U * self.Xt[k][None, None, :]).reshape(self.nz, self.ny, self.s, self.mx).sum(dim=2)
            d[k] = torch.fft.ifftn(V, dim=(0, 1, 2)).real * (self.ph[k] / self.s)

    def adjoint(self, d, rho):
        torch = self.torch
        acc = None
        for k in range(self.K):
            v = (d[k] * self.ph[k].conj()).real
            Vn = torch.fft.fftn(v.to(torch.complex64), dim=(0, 1, 2)).repeat(1, 1, self.s)
            t = Vn * self.Xt[k].conj()[None, None, :]
            acc = t if acc is None else acc + t
        r = torch.fft.ifftn(acc * self.Hyz.conj(), dim=(0, 1, 2)).real
        rho.copy_(r * self.b if self.b is not None else r)


def bench_batched(args):
    """The 64-volume workload: sizes drawn (seed 777) from 64^3, 96x96x64,
    128x128x64 and 192x192x96; volume i has phantom and noise seed 1000 + i;
    K = 8, s = 2, Gaussian b, 25 dB, CG to rel. residual 1e-4.  One step =
    one mh3d_solve_batched call over all 64 volumes (one CUDA graph);
    value = volumes / second.  The same volumes solved one after another by
    mh3d_solve are reported beside it."""
    import torch

    from paper_2503_13802_gb300 import (Plan, make_opts, mh3d_forward, mh3d_plan_autotune, mh3d_plan_tuning,
                                        mh3d_solve, mh3d_solve_batched)

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    wl = W.WORKLOADS[WORKLOAD]
    sizes = W.batch_sizes(64, 777)
    tuning = {}
    plans, ds, xs = [], [], []
    for i, n in enumerate(sizes):
        rho = W.phantom(n, (1.0, 1.0, 1.0), 1000 + i, wl.n_blobs, wl.n_lines)
        b = W.sensitivity(n, (1.0, 1.0, 1.0), kind="gaussian")
        pl = Plan(n, ds_factor=wl.ds_factor, k_min=wl.k_min, k_max=wl.k_max, sensitivity=b)
        d = torch.empty(pl.portrait_shape, dtype=torch.complex64, device=dev)
        mh3d_forward(pl, torch.as_tensor(rho, dtype=torch.float32, device=dev).contiguous(), d)
        sig2 = float(torch.sum(torch.abs(d.to(torch.complex128)) ** 2)) / (d.numel() * 10 ** (wl.snr_db / 10))
        noise = torch.as_tensor(W.unit_complex_noise(tuple(d.shape), 1000 + i).astype(np.complex64), device=dev)
        plans.append(pl)
        ds.append((d + math.sqrt(sig2) * noise).contiguous())
        xs.append(torch.empty(pl.shape, dtype=torch.float32, device=dev))
        if not args.no_autotune:
            # the autotuner times each size class once; later plans of a class take its choice
            mh3d_plan_autotune(pl)
            tuning["x".join(map(str, n))] = mh3d_plan_tuning(pl)
    opts = make_opts(lam=wl.lam, lam_relative=True, rel_tol=wl.rel_tol, max_iter=wl.max_iter)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        infos = mh3d_solve_batched(plans, ds, opts, xs)
    times = []
    with Clocks(0) as clk:
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos = mh3d_solve_batched(plans, ds, opts, xs)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
    total = sum(times)
    value = len(plans) * args.steps / total
    # one after another, for comparison
    seq = []
    for _ in range(2):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for pl, d, x in zip(plans, ds, xs):
            mh3d_solve(pl, d, opts, x)
        e1.record(stream)
        e1.synchronize()
        seq.append(e0.elapsed_time(e1) / 1e3)
    iters = [inf["iters"] for inf in infos]
    worst = max(inf["rel_res_true"] for inf in infos)
    cpu = None if args.no_cpu_baseline else batched_cpu_baseline(wl, sizes, iters)
    line = {
        "metric": "batched reconstructions/sec to rel. residual 1e-4", "value": value, "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "precision": PRECISION,
        "data": "synthetic",
        "config": {"workload": "batch64_mixed_k8_s2", "volumes": len(plans),
                   "size_classes": [list(c) for c in W.BATCH_SIZE_CLASSES],
                   "count_per_class": [sizes.count(c) for c in W.BATCH_SIZE_CLASSES],
                   "voxels_total": int(sum(p.N for p in plans)), "harmonics": [wl.k_min, wl.k_max],
                   "ds_factor": wl.ds_factor, "snr_db": wl.snr_db, "lambda": wl.lam, "rel_tol": wl.rel_tol,
                   "launch": "one CUDA graph, one branch per volume", "l2": "flushed between steps (256 MB write)",
                   "autotune": tuning or None},
        "cg_iters": {"min": min(iters), "max": max(iters), "mean": statistics.mean(iters)},
        "worst_rel_res_true": worst,
        "one_after_another": {"value": len(plans) / statistics.mean(seq), "unit": UNIT,
                              "ms": 1e3 * statistics.mean(seq)},
        "clocks": clk.summary(),
    }
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


def batched_cpu_baseline(wl, sizes, iters):
    """The FP64 oracle on the host cores for the 64-volume workload: one
    volume per size class (its first one), A^T d and one CG iteration,
    scaled to that class's mean GPU iteration count; the batch estimate sums
    the classes' per-volume times over their volume counts."""
    import oracle

    per_class, total = {}, 0.0
    for c in W.BATCH_SIZE_CLASSES:
        idx = [i for i, n in enumerate(sizes) if n == c]
        if not idx:
            continue
        i = idx[0]
        g = oracle.Geometry(n=c, voxel_mm=(1.0, 1.0, 1.0), ds_factor=wl.ds_factor, k_min=wl.k_min, k_max=wl.k_max)
        rho = W.phantom(c, (1.0, 1.0, 1.0), 1000 + i, wl.n_blobs, wl.n_lines)
        b = W.sensitivity(c, (1.0, 1.0, 1.0), kind="gaussian")
        tables = oracle.psf_tables(g)
        clean = oracle.forward(g, rho, b, tables)
        sig2 = np.sum(np.abs(clean) ** 2) / (clean.size * 10 ** (wl.snr_db / 10))
        d = clean + math.sqrt(sig2) * W.unit_complex_noise(clean.shape, 1000 + i)
        t0 = time.perf_counter()
        # one iteration's cost does not depend on lambda: an absolute weight
        # spares the Lanczos run of the relative one
        oracle.cg(g, d, b, oracle.SolveOpts(lam=wl.lam, rel_tol=0.0, max_iter=1), tables=tables)
        t = time.perf_counter() - t0
        it = statistics.mean(iters[j] for j in idx)
        vol_s = t / 2.5 * (it + 2.5)
        per_class["x".join(map(str, c))] = {"seconds_per_volume": vol_s, "volumes": len(idx), "sample_s": t}
        total += vol_s * len(idx)
    return {"value": len(sizes) / total, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "one volume per size class, A^T d + 1 CG iteration, scaled to the class's mean "
                      "GPU iteration count", "per_class": per_class}


def bench_learned(args):
    """Learned warm start on the 128x128x64, K = 8, s = 2 workload: phantoms
    with 5-200 blobs (log-uniform) + 3 lines, SNR U(15, 40) dB, Gaussian b.
    Trains the network on --train-n volumes (seeds 10000 + i; target: the
    zero-start CG solution to 1e-4), then on the 200 test volumes (seeds
    20000 + i) times zero-start CG against warm start (A^T d, network, CG
    from x0 with the device-side fallback), each with CUDA events on the
    stream.  Noise: torch's seeded CUDA generator (seed = volume seed)."""
    import torch

    from paper_2503_13802_gb300 import Plan, make_opts, mh3d_forward, mh3d_solve
    from paper_2503_13802_gb300.warmstart import WarmStart

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    wl = W.WORKLOADS[WORKLOAD]
    b = W.sensitivity(wl.n, wl.voxel_mm, kind="gaussian")
    plan = Plan(wl.n, voxel_mm=wl.voxel_mm, ds_factor=wl.ds_factor, k_min=wl.k_min, k_max=wl.k_max, sensitivity=b)
    opts = make_opts(lam=wl.lam, lam_relative=True, rel_tol=wl.rel_tol, max_iter=wl.max_iter)
    stream = torch.cuda.current_stream()

    def portraits(seed):
        rho, snr = W.learned_case(wl.n, wl.voxel_mm, seed)
        d = torch.empty(plan.portrait_shape, dtype=torch.complex64, device=dev)
        mh3d_forward(plan, torch.as_tensor(rho, dtype=torch.float32, device=dev).contiguous(), d)
        sig2 = float(torch.sum(torch.abs(d.to(torch.complex128)) ** 2)) / (d.numel() * 10 ** (snr / 10))
        gen = torch.Generator(device=dev).manual_seed(int(seed))
        noise = torch.randn(d.shape, generator=gen, dtype=torch.complex64, device=dev)
        return (d + math.sqrt(sig2) * noise).contiguous()

    ws = WarmStart(plan, channels=tuple(args.channels))
    ws.init_params(args.seed)
    t_gen = time.perf_counter()
    rhs_list, tgt_list = [], []
    x = torch.empty(plan.shape, dtype=torch.float32, device=dev)
    for seed in W.LEARNED_TRAIN_SEEDS[:args.train_n]:
        d = portraits(seed)
        rhs_list.append(ws.back_projection(d, torch.empty_like(x)))
        mh3d_solve(plan, d, opts, x)
        tgt_list.append(x.clone())
    t_gen = time.perf_counter() - t_gen
    t_fit = time.perf_counter()
    hist = ws.fit(rhs_list, tgt_list, epochs=args.epochs, lr_max=args.lr, lr_min=args.lr * 1e-2, seed=args.seed)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t_fit
    del rhs_list, tgt_list

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    test = W.LEARNED_TEST_SEEDS[:args.test_n]
    tests = [portraits(sd) for sd in test]
    for d in tests[:3]:   # warm-up
        mh3d_solve(plan, d, opts, x)
        ws.solve(d, x, lam=wl.lam, lam_relative=True, rel_tol=wl.rel_tol, max_iter=wl.max_iter)
    n0, n1, t0, t1, tinf, fb, r0 = [], [], [], [], [], 0, []
    for d in tests:
        i0, s0 = timed(lambda: mh3d_solve(plan, d, opts, x))
        i1, s1 = timed(lambda: ws.solve(d, x, lam=wl.lam, lam_relative=True, rel_tol=wl.rel_tol,
                                        max_iter=wl.max_iter))
        _, si = timed(lambda: ws.predict(d))
        n0.append(i0["iters"])
        n1.append(i1["iters"])
        t0.append(s0)
        t1.append(s1)
        tinf.append(si)
        fb += int(i1["x0_rejected"])
        r0.append(i1["history"][0])
    ratio = np.array(t0) / np.array(t1)
    m, sd = float(ratio.mean()), float(ratio.std(ddof=1)) if len(ratio) > 1 else 0.0
    half = 1.972 * sd / math.sqrt(len(ratio))

    # the learned + batched form: the first test volumes in one batched call,
    # zero start (mh3d_solve_batched) against the network's x0 per volume
    # (inference included) through mh3d_solve_batched_warm
    from paper_2503_13802_gb300 import mh3d_solve_batched

    nb = min(args.batch_n, len(tests))
    bplans = [Plan(wl.n, voxel_mm=wl.voxel_mm, ds_factor=wl.ds_factor, k_min=wl.k_min, k_max=wl.k_max,
                   sensitivity=b) for _ in range(nb)]
    bd = tests[:nb]
    bx = [torch.empty(plan.shape, dtype=torch.float32, device=dev) for _ in range(nb)]
    bx0 = [torch.empty(plan.shape, dtype=torch.float32, device=dev) for _ in range(nb)]
    bopts = make_opts(lam=wl.lam, lam_relative=True, rel_tol=wl.rel_tol, max_iter=wl.max_iter, x0_fallback=True)

    def batch_zero():
        return mh3d_solve_batched(bplans, bd, bopts, bx)

    def batch_warm():
        for i in range(nb):
            ws.predict(bd[i], bx0[i])
        return mh3d_solve_batched(bplans, bd, bopts, bx, x0s=bx0)

    for _ in range(2):   # warm-up (graph capture)
        batch_zero()
        batch_warm()
    tb0, tb1, ib0, ib1 = [], [], [], []
    for _ in range(3):
        inf0, s0 = timed(batch_zero)
        inf1, s1 = timed(batch_warm)
        tb0.append(s0)
        tb1.append(s1)
        ib0.extend(v["iters"] for v in inf0)
        ib1.extend(v["iters"] for v in inf1)
    batched = {"volumes": nb, "zero_start_value": nb / float(np.mean(tb0)), "warm_start_value": nb / float(np.mean(tb1)),
               "speedup": float(np.mean(tb0)) / float(np.mean(tb1)), "zero_mean_iters": float(np.mean(ib0)),
               "warm_mean_iters": float(np.mean(ib1)),
               "what": "one mh3d_solve_batched call over the first test volumes, zero start, against the "
                       "network's x0 per volume (inference timed in) through mh3d_solve_batched_warm"}
    line = {
        "metric": "reconstructions/sec to rel. residual 1e-4 with learned warm start", "value": len(t1) / sum(t1),
        "unit": UNIT, "n_gpus": 1, "steps": len(t1), "warmup": 3, "ms_per_step": 1e3 * float(np.mean(t1)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 solve, bf16 network (f32 accumulation)", "data": "synthetic",
        "config": {"workload": "learned_128x128x64_k8_s2", "train_volumes": args.train_n, "test_volumes": len(t1),
                   "epochs": args.epochs, "channels": list(args.channels), "params": ws.net.nparam,
                   "lr": args.lr, "seed": args.seed},
        "zero_start": {"value": len(t0) / sum(t0), "mean_iters": float(np.mean(n0))},
        "warm_start": {"mean_iters": float(np.mean(n1)), "inference_ms": 1e3 * float(np.mean(tinf)),
                       "fallback_rate": fb / len(t1),
                       "median_initial_rel_res": float(np.median(r0))},
        "speedup": {"mean": m, "ci95": [m - half, m + half], "per": "volume, zero-start time / warm-start time"},
        "batched": batched,
        "train": {"loss_per_epoch": hist, "data_s": t_gen, "fit_s": t_fit},
    }
    print(json.dumps(line), flush=True)


def bench_mhad(args):
    """MHAD (App. D, Eq. mhadM) on the 128x128x64, K = 8, s = 2 workload and
    the test volumes of the learned warm start (seeds 20000 + i, same phantom
    and noise recipe): (1) the native image alone, timed with CUDA events
    over repeated calls with the L2 flushed between them (algorithmic bytes:
    the K M complex64 portraits read, the N-float model-grid image written);
    (2) per volume, zero-start CG against CG from the MHAD warm start
    (image, / b, least-squares scale, then CG with the device-side
    fallback), both to rel. residual 1e-4."""
    import torch

    from paper_2503_13802_gb300 import Plan, make_opts, mh3d_forward, mh3d_mhad, mh3d_mhad_warm_start, mh3d_solve

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    wl = W.WORKLOADS[WORKLOAD]
    b = W.sensitivity(wl.n, wl.voxel_mm, kind="gaussian")
    plan = Plan(wl.n, voxel_mm=wl.voxel_mm, ds_factor=wl.ds_factor, k_min=wl.k_min, k_max=wl.k_max, sensitivity=b)
    opts = make_opts(lam=wl.lam, lam_relative=True, rel_tol=wl.rel_tol, max_iter=wl.max_iter)
    stream = torch.cuda.current_stream()
    lam_m = args.mhad_lambda

    def portraits(seed):
        rho, snr = W.learned_case(wl.n, wl.voxel_mm, seed)
        d = torch.empty(plan.portrait_shape, dtype=torch.complex64, device=dev)
        mh3d_forward(plan, torch.as_tensor(rho, dtype=torch.float32, device=dev).contiguous(), d)
        sig2 = float(torch.sum(torch.abs(d.to(torch.complex128)) ** 2)) / (d.numel() * 10 ** (snr / 10))
        gen = torch.Generator(device=dev).manual_seed(int(seed))
        noise = torch.randn(d.shape, generator=gen, dtype=torch.complex64, device=dev)
        return (d + math.sqrt(sig2) * noise).contiguous()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    test = W.LEARNED_TEST_SEEDS[:args.test_n]
    tests = [portraits(sd) for sd in test]
    x = torch.empty(plan.shape, dtype=torch.float32, device=dev)
    x0 = torch.empty_like(x)
    img = torch.empty(plan.N, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    for _ in range(5):
        mh3d_mhad(plan, tests[0], lam_m, img, upsample=True)
    us = []
    for i in range(50):
        flush.zero_()
        _, t = timed(lambda: mh3d_mhad(plan, tests[i % len(tests)], lam_m, img, upsample=True))
        us.append(1e6 * t)
    us_img = float(np.median(us))
    alg = plan.K * int(np.prod(plan.portrait_shape[1:])) * 8 + plan.N * 4
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0))
    except (OSError, ValueError):
        peak = 6800.0

    warm_opts = make_opts(lam=wl.lam, lam_relative=True, rel_tol=wl.rel_tol, max_iter=wl.max_iter, x0=x0,
                          x0_fallback=True)

    def warm(d):
        mh3d_mhad_warm_start(plan, d, lam_m, x0)
        return mh3d_solve(plan, d, warm_opts, x)

    for d in tests[:3]:   # warm-up
        mh3d_solve(plan, d, opts, x)
        warm(d)
    n0, n1, t0, t1, fb, r0 = [], [], [], [], 0, []
    for d in tests:
        i0, s0 = timed(lambda: mh3d_solve(plan, d, opts, x))
        i1, s1 = timed(lambda: warm(d))
        n0.append(i0["iters"])
        n1.append(i1["iters"])
        t0.append(s0)
        t1.append(s1)
        fb += int(i1["x0_rejected"])
        r0.append(i1["history"][0])
    ratio = np.array(t0) / np.array(t1)
    m, sd = float(ratio.mean()), float(ratio.std(ddof=1)) if len(ratio) > 1 else 0.0
    half = 1.972 * sd / math.sqrt(len(ratio))

    # the learned + batched form: the first test volumes in one batched call,
    # zero start (mh3d_solve_batched) against the network's x0 per volume
    # (inference included) through mh3d_solve_batched_warm
    from paper_2503_13802_gb300 import mh3d_solve_batched

    nb = min(args.batch_n, len(tests))
    bplans = [Plan(wl.n, voxel_mm=wl.voxel_mm, ds_factor=wl.ds_factor, k_min=wl.k_min, k_max=wl.k_max,
                   sensitivity=b) for _ in range(nb)]
    bd = tests[:nb]
    bx = [torch.empty(plan.shape, dtype=torch.float32, device=dev) for _ in range(nb)]
    bx0 = [torch.empty(plan.shape, dtype=torch.float32, device=dev) for _ in range(nb)]
    bopts = make_opts(lam=wl.lam, lam_relative=True, rel_tol=wl.rel_tol, max_iter=wl.max_iter, x0_fallback=True)

    def batch_zero():
        return mh3d_solve_batched(bplans, bd, bopts, bx)

    def batch_warm():
        for i in range(nb):
            ws.predict(bd[i], bx0[i])
        return mh3d_solve_batched(bplans, bd, bopts, bx, x0s=bx0)

    for _ in range(2):   # warm-up (graph capture)
        batch_zero()
        batch_warm()
    tb0, tb1, ib0, ib1 = [], [], [], []
    for _ in range(3):
        inf0, s0 = timed(batch_zero)
        inf1, s1 = timed(batch_warm)
        tb0.append(s0)
        tb1.append(s1)
        ib0.extend(v["iters"] for v in inf0)
        ib1.extend(v["iters"] for v in inf1)
    batched = {"volumes": nb, "zero_start_value": nb / float(np.mean(tb0)), "warm_start_value": nb / float(np.mean(tb1)),
               "speedup": float(np.mean(tb0)) / float(np.mean(tb1)), "zero_mean_iters": float(np.mean(ib0)),
               "warm_mean_iters": float(np.mean(ib1)),
               "what": "one mh3d_solve_batched call over the first test volumes, zero start, against the "
                       "network's x0 per volume (inference timed in) through mh3d_solve_batched_warm"}
    line = {
        "metric": "reconstructions/sec to rel. residual 1e-4 with MHAD warm start", "value": len(t1) / sum(t1),
        "unit": UNIT, "n_gpus": 1, "steps": len(t1), "warmup": 3, "ms_per_step": 1e3 * float(np.mean(t1)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 tables, FP64 sums)",
        "data": "synthetic", "config": {"workload": "learned_128x128x64_k8_s2 test volumes", "test_volumes": len(t1),
                                        "mhad_lambda": lam_m},
        "mhad_image": {"us": us_img, "alg_bytes": alg, "achieved_gbs": alg / us_img / 1e3,
                       "frac": alg / us_img / 1e3 / peak, "l2": "flushed before each call"},
        "zero_start": {"value": len(t0) / sum(t0), "mean_iters": float(np.mean(n0))},
        "warm_start": {"mean_iters": float(np.mean(n1)), "fallback_rate": fb / len(t1),
                       "median_initial_rel_res": float(np.median(r0))},
        "speedup": {"mean": m, "ci95": [m - half, m + half], "per": "volume, zero-start time / warm-start time"},
    }
    print(json.dumps(line), flush=True)


def bench_general(args):
    """The general model's forward and adjoint (mh3d_general_*) at the
    128x128x64, K = 8, s = 2 size with three sensitivity components.  The PSF
    samples are random (this leg times the operators; their parity with the
    tensor PSF is tests/test_gpu_general.py).  CUDA events around each call,
    L2 flushed before it; the K*3 spectra (201 MB) exceed the L2 as well.
    Algorithmic bytes: forward = rho + b (3 components) + the spectra read
    and the portraits written; adjoint = the portraits + spectra + b read and
    the image written."""
    import torch

    from paper_2503_13802_gb300 import Plan, mh3d_general_adjoint, mh3d_general_forward, mh3d_general_set_psf

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    wl = W.WORKLOADS[WORKLOAD]
    plan = Plan(wl.n, voxel_mm=wl.voxel_mm, ds_factor=wl.ds_factor, k_min=wl.k_min, k_max=wl.k_max)
    K, N = plan.K, plan.N
    M = int(np.prod(plan.portrait_shape[1:]))
    rng = np.random.default_rng(3)
    mh3d_general_set_psf(plan, (1e-2 * rng.standard_normal(K * 3 * N)).astype(np.float32))
    rho = torch.randn(plan.shape, dtype=torch.float32, device=dev)
    bvec = (0.5 + torch.rand((3,) + tuple(plan.shape), dtype=torch.float32, device=dev)).contiguous()
    d = torch.empty(plan.portrait_shape, dtype=torch.complex64, device=dev)
    out = torch.empty(plan.shape, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()

    def timed(fn):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return 1e3 * e0.elapsed_time(e1)

    fwd = lambda: mh3d_general_forward(plan, rho, d, bvec)   # noqa: E731
    adj = lambda: mh3d_general_adjoint(plan, d, out, bvec)   # noqa: E731
    for _ in range(max(3, args.warmup)):
        fwd()
        adj()
    steps = max(1, args.steps)
    us_f = float(np.median([timed(fwd) for _ in range(steps)]))
    us_a = float(np.median([timed(adj) for _ in range(steps)]))
    spectra = K * 3 * N * 8
    alg_f = N * 4 + 3 * N * 4 + spectra + K * M * 8
    alg_a = K * M * 8 + spectra + 3 * N * 4 + N * 4
    # the general model's CG (mh3d_general_solve), a fixed number of
    # iterations on the portraits of rho: time per solve / iterations
    from paper_2503_13802_gb300 import make_opts, mh3d_general_solve
    fwd()
    x = torch.empty(plan.shape, dtype=torch.float32, device=dev)
    it = 20
    go = make_opts(lam=1e-3, max_iter=it, fixed_iters=True)
    mh3d_general_solve(plan, d, go, x, bvec)
    sol_us = float(np.median([timed(lambda: mh3d_general_solve(plan, d, go, x, bvec)) for _ in range(3)]))
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0))
    except (OSError, ValueError):
        peak = 6800.0
    line = {
        "metric": "general-model forward + adjoint pairs/s", "value": 1e6 / (us_f + us_a), "unit": "pairs/s",
        "n_gpus": 1, "steps": steps, "warmup": max(3, args.warmup), "ms_per_step": (us_f + us_a) / 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "general_128x128x64_k8_s2", "psf": "random samples (timing only)",
                   "sensitivity": "three components", "l2": "flushed before each call"},
        "forward": {"us": us_f, "alg_bytes": alg_f, "achieved_gbs": alg_f / us_f / 1e3,
                    "frac": alg_f / us_f / 1e3 / peak, "launches": 7},
        "adjoint": {"us": us_a, "alg_bytes": alg_a, "achieved_gbs": alg_a / us_a / 1e3,
                    "frac": alg_a / us_a / 1e3 / peak, "launches": 8},
        "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
        "general_cg": {"iterations": it, "us_per_solve": sol_us, "us_per_iteration": sol_us / it,
                       "what": "mh3d_general_solve, lambda 1e-3, fixed iterations (A^T d, the CG set-up and "
                               "one forward + adjoint per iteration through the portrait buffer)"},
    }
    print(json.dumps(line), flush=True)


def bench_reference(args):
    """The FP64 oracle as the reference arm, rank 0 only: every timed step is
    one whole reconstruction of the bench workload (A^T d and CG to rel.
    residual 1e-4, about 17 s on 16 Arm cores), timed as it runs.  A warm-up
    step is one application of the oracle's normal operator (it brings the
    thread pool and the tables in; a whole reconstruction would only repeat a
    timed step)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    wl = W.WORKLOADS[args.workload]
    g, tables, b, d, opts = oracle_case(wl)
    if args.count_iters:
        t, it = oracle_reconstruction(g, tables, b, d, opts)
        print(json.dumps({"oracle_cg_iters": it, "seconds": t, "cores": oracle.num_threads()}), flush=True)
        return
    for _ in range(args.warmup):
        oracle.normal_apply(g, np.ones(g.shape), b, opts, tables)
    times, iters = [], []
    for _ in range(args.steps):
        t, it = oracle_reconstruction(g, tables, b, d, opts)
        times.append(t)
        iters.append(it)
    total = sum(times)
    value = args.steps / total
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "grid": list(wl.n), "harmonics": [wl.k_min, wl.k_max],
                       "ds_factor": wl.ds_factor, "rel_tol": wl.rel_tol, "cg_iters": int(statistics.median(iters))},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"every step one whole oracle reconstruction (A^T d + CG to rel. residual "
                                       f"{wl.rel_tol:g}, {int(statistics.median(iters))} iterations) on {cores} "
                                       f"threads, timed, not scaled; warm-up steps: one normal-operator "
                                       f"application each"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        bench_reference(args)
    elif args.batched:
        bench_batched(args)
    elif args.learned:
        bench_learned(args)
    elif args.mhad:
        bench_mhad(args)
    elif args.general:
        bench_general(args)
    else:
        bench_mh3d(args)


if __name__ == "__main__":
    main()
