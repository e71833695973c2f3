#!/usr/bin/env python
"""Benchmark of the SARA/SDMM imaging hot path on GB300.

Workload (default): the largest single-GPU configuration, a 1024 x 1024 sky
(500 point sources, 40 blobs, diffuse component), M = 10,485,760
visibilities (Gaussian (u, v) density plus 10% uniform), Kaiser-Bessel width
J = 6, oversampling 2, Psi = Dirac + db1..db8 at 5 levels (q = 9), R = 64
uneven blocks, FP32 operators with FP64 reductions, 20 dB input SNR,
synthetic seeded data. One step = one SDMM iteration (Psi^dagger + prox,
Phi + block projections, positivity, Psi, Phi^dagger and CG_ITERS
conjugate-gradient steps of Phi^dagger Phi) on the plan's resident state,
launched as one captured CUDA graph.

Passes (all in one run):
  A  timed pass: W warm-up steps, then K steps each bracketed by CUDA events
     on the launching stream; a 512 MiB buffer is rewritten between steps to
     flush L2 (outside the events).                      -> value, ms_per_step
  B  roofline pass: the same K steps launched eagerly with per-kernel CUDA
     events; the dominant kernel's algorithmic flops (or bytes) / mean
     duration.                                            -> roofline
  C  end-to-end pass: K calls of purify_sdmm_solve with pinned host buffers
     (y in, x in/out), one iteration each, wall-clock timed.  -> e2e
  D  Phi, Phi^dagger, Psi, Psi^dagger through the C ABI: algorithmic GB/s
     and the fraction of the HBM peak; Phi + Phi^dagger Gvis/s.
                                             -> roofline.operators, Gvis/s
  E  the 256 x 256 (M = 655,360, R = 8) and 64 x 64 FP64 workloads by the
     same rules (rank 0, N = 1).                         -> other_workloads
  F  CPU baseline: the FP64 oracle, one SDMM iteration on the host cores
     (whole, or on a stated visibility sample; rank 0, N = 1 only).

With torchrun (N > 1) every rank solves its own independent problem (replicas,
weak scaling); the max over ranks of the timed region sets the time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CG_ITERS = 8
FLUSH_BYTES = 512 << 20
HBM_FALLBACK_GBS = 6800.0


# --------------------------------------------------------------- helpers
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}


def algorithmic_bytes(name: str, info, dtype_bytes: int = 4) -> float | None:
    """Bytes a kernel launch must move at minimum (FP32, internal order):
    visibility kernels 8 B per (u, v) pair and 8 B per complex visibility,
    the oversampled grid 8 B per cell read or written once, images 4 B per
    pixel, coefficients 4 B per entry."""
    N, M, Kx, Ky, D = info.N, info.M, info.Kx, info.Ky, info.D
    ny = int(round(np.sqrt(N * Ky / Kx)))
    c = 2 * dtype_bytes
    table = {
        "degrid": 8 * M + c * M + c * Kx * Ky,
        "grid": 8 * M + c * M + c * Kx * Ky,
        # G^H G of the forward grid: coordinates once, the grid read once and
        # the output grid written once (no visibility vector)
        "normal_gg": 8 * M + 2 * c * Kx * Ky,
        "fft_rows_fwd": dtype_bytes * N + c * ny * Kx,
        "fft_cols_fwd": c * ny * Kx + c * Kx * Ky,
        "fft_cols_inv": c * Kx * Ky + c * ny * Kx,
        "fft_rows_inv": c * ny * Kx + 2 * dtype_bytes * N,
        "prox_l1": 4 * dtype_bytes * D,
        "proj_norms": 3 * c * M,
        "proj_apply": 5 * c * M,
        "positivity": 5 * dtype_bytes * N,
        "relchange": 10 * dtype_bytes * N,   # with the last CG update: x, xprev, r, p, u, s in; x, p, s, r out
    }
    return float(table[name]) if name in table else None


def algorithmic_flops(name: str, info) -> float | None:
    """FP32 operations a launch must perform (kernel weights evaluated from
    J per-tap polynomials of degree 8-10 per axis, J*J taps of a real weight
    times a complex value; FFT passes 5 n log2 n per length-n transform)."""
    import math
    J, M = info.J, info.M
    deg = 10 if J <= 3 else (9 if J == 4 else 8)
    weights = 2 * J * (deg + 1) * 2          # Horner: one FMA (2 flops) per coefficient
    taps = J * J * (1 + 4)                    # weight product + complex multiply-accumulate
    ny = int(round(np.sqrt(info.N * info.Ky / info.Kx)))
    table = {
        "grid": M * (weights + taps),
        "normal_gg": M * (weights + 2 * taps),
        "degrid": M * (weights + taps),
        "fft_rows_fwd": ny * 5 * info.Kx * math.log2(info.Kx),
        "fft_rows_inv": ny * 5 * info.Kx * math.log2(info.Kx),
        "fft_cols_fwd": info.Kx * 5 * info.Ky * math.log2(info.Ky),
        "fft_cols_inv": info.Kx * 5 * info.Ky * math.log2(info.Ky),
    }
    return float(table[name]) if name in table else None


def fp32_peak_tflops(sm_mhz: float | None) -> float:
    """Non-tensor FP32 peak from unit counts: 152 SMs x 128 FP32 lanes x 2
    flops (FMA) x clock (the sampled maximum SM clock, else 2070 MHz)."""
    return 152 * 128 * 2 * (sm_mhz or 2070.0) * 1e6 / 1e12


def source_sha1(relpath: str) -> str:
    return hashlib.sha1(open(os.path.join(ROOT, relpath), "rb").read()).hexdigest()


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current source of that kernel and for this workload; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        e = d.get(f"{kernel}@{workload}")
        if not e:
            return None
        if e.get("source_sha1") != source_sha1(e["source"]):
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


KERNEL_SOURCE = {"degrid": "paper_1502_05037_gb300/csrc/nufft.cu", "grid": "paper_1502_05037_gb300/csrc/nufft.cu",
                 "normal_gg": "paper_1502_05037_gb300/csrc/nufft.cu"}


# ------------------------------------------------------ ranks (replicas)
def replica_workload(wl, rank: int):
    """The workload rank `rank` solves: rank 0 the named one, every other rank
    an independent problem of the same shape (its seeds shifted by 1000 per
    rank)."""
    from paper_1502_05037_gb300 import synth
    if rank == 0:
        return wl
    return synth.Workload(**{**wl.__dict__, "index": wl.index + 1000 * rank})


def max_over_ranks(value: float, dist, device) -> float:
    """The largest `value` over all ranks (the value itself without a
    process group)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, steps: int, total_ms: float) -> float:
    """Whole-job throughput: every rank runs `steps` steps; the slowest
    rank's time sets the job's."""
    return world * steps / (total_ms / 1e3)


# -------------------------------------------------------- problem set-up
def setup_problem(wl_name: str, replica: int, dev, grid_mode: int = 0):
    import torch

    import paper_1502_05037_gb300 as pk
    from paper_1502_05037_gb300 import problem, synth

    wl = synth.WORKLOADS[wl_name] if isinstance(wl_name, str) else wl_name
    wl = replica_workload(wl, replica)
    x_true, u, v, offs, nz = wl.draw()
    f64 = wl.dtype == "f64"
    rt, ct = (torch.float64, torch.complex128) if f64 else (torch.float32, torch.complex64)
    plan = pk.Plan(wl.nx, wl.ny, torch.from_numpy(u).to(dev), torch.from_numpy(v).to(dev), kb_width=wl.J,
                   levels=wl.levels, block_offsets=offs, stream=torch.cuda.current_stream(dev),
                   dtype=pk.PURIFY_F64 if f64 else pk.PURIFY_F32, grid_mode=grid_mode)
    xt = torch.from_numpy(x_true).to(rt).to(dev)
    y0 = torch.empty(wl.M, dtype=ct, device=dev)
    pk.purify_phi(plan, xt, y0)
    sigma = problem.noise_sigma_from_norm(float(torch.linalg.vector_norm(y0.to(torch.complex128)).item()), wl.M,
                                          wl.snr_db)
    y = y0 + torch.from_numpy(sigma * nz).to(ct).to(dev)
    eps = problem.chi2_epsilon(sigma, np.diff(offs))
    return wl, plan, y, eps, x_true


# ------------------------------------------------------------------ ours
def operator_bytes(wl, info) -> dict:
    """Algorithmic bytes of one application of each operator (FP32, the
    minimum traffic with the Kaiser-Bessel weights computed on the fly):
    Phi and Phi^dagger move the image (4 B per pixel), the oversampled grid
    written once and read once after F (16 B per cell), the coordinates and
    the visibilities (8 + 8 B each): 4N + 16 K^2 + 16 M; Psi^dagger and Psi
    read or write the image once and every coefficient once: 4N + 4qN."""
    N, M, K2, q = info.N, info.M, info.Kx * info.Ky, info.q
    vis = 4 * N + 16 * K2 + 16 * M
    wav = 4 * N + 4 * q * N
    return {"phi": vis, "phi_adj": vis, "psi": wav, "psi_adj": wav}


def time_operators(pk, plan, wl, dev, stream, flush, reps, peak):
    """Each operator through the C ABI (caller order for the visibilities),
    `reps` timed calls after 3 untimed ones, L2 flushed before each call;
    mean milliseconds, algorithmic GB/s and the fraction of the HBM peak."""
    import torch
    rdt = torch.float64 if wl.dtype == "f64" else torch.float32
    cdt = torch.complex128 if wl.dtype == "f64" else torch.complex64
    info = plan.info
    x_true = synth_sky(wl)
    xin = torch.from_numpy(x_true).to(rdt).to(dev)
    yv = torch.empty(wl.M, dtype=cdt, device=dev)
    xa = torch.empty((wl.ny, wl.nx), dtype=cdt, device=dev)
    c = torch.empty((info.q, wl.ny, wl.nx), dtype=rdt, device=dev)
    xo = torch.empty_like(xin)
    calls = {"phi": lambda: pk.purify_phi(plan, xin, yv), "phi_adj": lambda: pk.purify_phi_adj(plan, yv, xa),
             "psi_adj": lambda: pk.purify_psi_adj(plan, xin, c), "psi": lambda: pk.purify_psi(plan, c, xo)}
    ab = operator_bytes(wl, info)
    out = {}
    for name, fn in calls.items():
        for _ in range(3):
            fn()
        evs = []
        for k in range(reps):
            flush.fill_(k & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize(dev)
        ms = sum(a.elapsed_time(b) for a, b in evs) / reps
        gbs = ab[name] / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "algorithmic_bytes": ab[name], "gbs": gbs, "frac_of_hbm": gbs / peak}
    return out


def synth_sky(wl):
    return wl.draw()[0]


def timed_iterations(pk, plan, dev, stream, flush, steps, warmup, clocks=None):
    """`warmup` untimed then `steps` timed SDMM iterations (graph replays),
    each bracketed by CUDA events on the launching stream, the L2 flushed
    before each (outside the events). Returns the per-step milliseconds."""
    import torch
    for i in range(warmup):
        flush.fill_(i & 0xFF)
        pk.purify_sdmm_iterate(plan, 1)
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_((k + 7) & 0xFF)
        evs[k][0].record(stream)
        pk.purify_sdmm_iterate(plan, 1)
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    return [a.elapsed_time(b) for a, b in evs]


def other_workload(pk, name, dev, steps, warmup, cg_iters, flush):
    """SDMM iterations/s and Phi + Phi^dagger Gvis/s on another workload
    (same timing rules as the headline; reported beside it)."""
    import torch
    wl, plan, y, eps, x_true = setup_problem(name, 0, dev)
    stream = torch.cuda.current_stream(dev)
    rdt = torch.float64 if wl.dtype == "f64" else torch.float32
    x = torch.zeros((wl.ny, wl.nx), dtype=rdt, device=dev)
    pk.purify_sdmm_solve(plan, y, eps, x, max_iter=0, cg_iters=cg_iters)
    ms = timed_iterations(pk, plan, dev, stream, flush, steps, warmup)
    peak, _ = peaks()
    ops = time_operators(pk, plan, wl, dev, stream, flush, max(5, steps // 2), peak)
    out = {"workload": describe(wl), "value": steps / (sum(ms) / 1e3), "unit": "iters/s",
           "ms_per_step": sum(ms) / steps, "steps": steps, "dtype": wl.dtype,
           "phi_phiadj_gvis_s": wl.M / ((ops["phi"]["ms"] + ops["phi_adj"]["ms"]) * 1e-3) / 1e9,
           "operators": ops}
    plan.close()
    return out


def describe(wl) -> str:
    return (f"{wl.name}: {wl.nx}x{wl.ny} sky, M={wl.M}, J={wl.J}, alpha=2, q=9, L={wl.levels}, R={wl.R}, "
            f"{wl.snr_db:g} dB, {wl.dtype}")


def run_ours(args):
    import torch

    import paper_1502_05037_gb300 as pk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_1502_05037_gb300 import build as pbuild
    pbuild.build()
    pk.load()

    wl, plan, y, eps, x_true = setup_problem(args.workload, rank, dev, args.grid_mode)
    stream = torch.cuda.current_stream(dev)
    rdt = torch.float64 if wl.dtype == "f64" else torch.float32
    cdt = torch.complex128 if wl.dtype == "f64" else torch.complex64
    x = torch.zeros((wl.ny, wl.nx), dtype=rdt, device=dev)
    # initialise the solver state: nu by power iteration, default gamma
    st0 = pk.purify_sdmm_solve(plan, y, eps, x, max_iter=0, cg_iters=args.cg_iters)
    nu, gamma = st0.nu, st0.gamma
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    # ---- pass A: timed steps (graph replays)
    for i in range(args.warmup):
        flush.fill_(i & 0xFF)
        pk.purify_sdmm_iterate(plan, 1)
    barrier()
    xs_probe = torch.empty_like(x)
    cg0 = pk.purify_sdmm_solve(plan, None, None, xs_probe, max_iter=0, resume=True,
                               cg_iters=args.cg_iters).cg_iters_total
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = pk.purify_launch_count()
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_((k + 7) & 0xFF)
            evs[k][0].record(stream)
            pk.purify_sdmm_iterate(plan, 1)
            evs[k][1].record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall0
    launches = pk.purify_launch_count() - launches0
    # CG updates actually applied per timed iteration (work is not skipped)
    cg_per_step = (pk.purify_sdmm_solve(plan, None, None, xs_probe, max_iter=0, resume=True,
                                        cg_iters=args.cg_iters).cg_iters_total - cg0) / args.steps
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, dist, dev)
    clocks = clk.summary()
    value = job_rate(world, args.steps, total_ms)

    # ---- pass B: per-kernel timing of the same steps (eager launches)
    pk.purify_timing_enable(plan, True)
    pk.purify_timing_read(plan, reset=True)
    for k in range(args.steps):
        flush.fill_((k + 3) & 0xFF)
        pk.purify_sdmm_iterate(plan, 1)
    torch.cuda.synchronize(dev)
    ktimes = pk.purify_timing_read(plan, reset=True)
    pk.purify_timing_enable(plan, False)
    dom = max(ktimes.items(), key=lambda kv: kv[1][1]) if ktimes else None
    peak, peak_src = peaks()
    dtb = 8 if wl.dtype == "f64" else 4
    roofline = None
    if dom:
        name, (nl, tms) = dom
        per = tms / nl
        ab = algorithmic_bytes(name, plan.info, dtb)
        af = algorithmic_flops(name, plan.info)
        tr = ncu_traffic(name, wl.name)
        alu_peak = fp32_peak_tflops(clocks.get("sm_max_mhz"))
        # the binding resource by arithmetic intensity against the ridge point
        ai = (af / ab) if (af and ab) else 0.0
        ridge = alu_peak * 1e12 / (peak * 1e9)
        common = {"kernel": name, "traffic": tr, "algorithmic_bytes_per_launch": ab,
                  "algorithmic_flops_per_launch": af, "mean_launch_us": per * 1e3,
                  "launches_per_step": nl / args.steps, "arithmetic_intensity": ai, "ridge_flop_per_byte": ridge,
                  "share_of_kernel_time": tms / sum(t for _, t in ktimes.values()),
                  "hbm_gbs": ab / (per * 1e-3) / 1e9 if ab else None, "hbm_peak": peak, "hbm_peak_source": peak_src}
        if af and ai > ridge:
            achieved = af / (per * 1e-3) / 1e12
            roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                        "frac": achieved / alu_peak, "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x clock",
                        **common}
        else:
            achieved = ab / (per * 1e-3) / 1e9 if ab else None
            roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": (achieved / peak if achieved else None), "peak_source": peak_src, **common}
    kernel_table = kernel_rates(ktimes, plan.info, args.steps, dtb, wl.levels)
    inf = plan.info
    decomposition = {"grid": inf.grid_mode, "degrid": inf.degrid_mode, "normal": inf.normal_mode,
                     "lane_tile": inf.lane_tile, "legend": "1 tile subproblems, 2 run sets, 3 a lane per run, 4 a lane pair per run, "
                               "5 a lane pair per run with runs grouped by grid tile, 6 a lane pair per run with "
                               "stored patches summed per cell in a fixed order (deterministic)",
                     "fft": {"rows_per_block": inf.fft_rows_per_block, "cols_per_block": inf.fft_cols_per_block,
                             "cols_per_thread": inf.fft_cols_per_thread}}

    # ---- pass C: end to end through the public API with pinned host buffers
    y_host = torch.empty(wl.M, dtype=cdt, pin_memory=True)
    y_host.copy_(y.cpu())
    x_host = torch.zeros((wl.ny, wl.nx), dtype=rdt, pin_memory=True)
    e2e_times = []
    for k in range(args.warmup + args.steps):
        x_host.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        pk.purify_sdmm_solve(plan, y_host.numpy(), eps, x_host.numpy(), max_iter=1, cg_iters=args.cg_iters,
                             gamma=gamma, nu=nu)
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_total = sum(e2e_times)
    e2e_total = max_over_ranks(e2e_total, dist, dev)
    rb = dtb
    e2e = {"value": job_rate(world, args.steps, e2e_total * 1e3), "unit": "iters/s",
           "h2d_bytes_per_step": wl.M * 2 * rb + wl.nx * wl.ny * rb, "d2h_bytes_per_step": wl.nx * wl.ny * rb,
           "call": "purify_sdmm_solve(host y, host x, max_iter=1)"}

    # ---- pass A': the same timed steps with the circulant-embedded CG normal operator
    toep = None
    if args.toeplitz_pass:
        xt0 = torch.zeros((wl.ny, wl.nx), dtype=rdt, device=dev)
        pk.purify_sdmm_solve(plan, y, eps, xt0, max_iter=0, cg_iters=args.cg_iters, gamma=gamma, nu=nu, toeplitz=True)
        tms_l = timed_iterations(pk, plan, dev, stream, flush, args.steps, args.warmup)
        tms = sum(tms_l)
        toep = {"value": args.steps / (tms / 1e3), "unit": "iters/s", "ms_per_step": tms / args.steps,
                "note": "CG normal operator by circulant embedding of the exact model (separate parity class)"}

    # ---- pass A'': primal-dual (Chambolle-Pock) iterations on the same problem,
    # timed as the difference of two synchronous solves (setup and statistics
    # cancel)
    pdl = None
    if args.pd_pass:
        xp = torch.zeros((wl.ny, wl.nx), dtype=rdt, device=dev)
        pk.purify_pd_solve(plan, y, eps, xp, iters=5, nu=nu)   # captures the iteration graph
        reps = 4 * args.steps
        walls = []
        for n_it in (5, 5 + reps):
            xp.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            pk.purify_pd_solve(plan, y, eps, xp, iters=n_it, nu=nu)
            walls.append(time.perf_counter() - t0)
        per = (walls[1] - walls[0]) / reps
        pdl = {"value": 1.0 / per, "unit": "iters/s", "ms_per_step": per * 1e3,
               "note": "Chambolle-Pock primal-dual iterations (no inner CG; a different solver of problem (3), "
                       "parity-tested against its FP64 oracle), back to back without an L2 flush, from the "
                       "wall-clock difference of two synchronous solves"}

    # ---- pass D: each operator through the C ABI (caller order), Phi + Phi^dagger Gvis/s
    ops = time_operators(pk, plan, wl, dev, stream, flush, args.steps, peak)
    gvis = wl.M / ((ops["phi"]["ms"] + ops["phi_adj"]["ms"]) * 1e-3) / 1e9
    if roofline is not None:
        roofline["operators"] = {k: {**v, "target_frac": 0.6} for k, v in ops.items()}
        roofline["operators_note"] = ("whole operators through the C ABI, algorithmic bytes (4N + 16K^2 + 16M for "
                                      "Phi and Phi^dagger, 4N + 4qN for Psi and Psi^dagger) over CUDA-event "
                                      "time, against the measured HBM copy bandwidth")
    plan.close()
    del y

    # ---- pass E: the other single-GPU workloads, reported beside the headline
    others = {}
    if rank == 0 and world == 1 and not args.no_other_workloads:
        for name in ("sara256_r8", "sara64_fp64"):
            if name != wl.name:
                others[name] = other_workload(pk, name, dev, max(args.steps, 20), args.warmup, args.cg_iters,
                                              flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, args.cg_iters, args.cpu_vis_fraction)

    if rank == 0:
        line = {
            "metric": "SDMM iters/s", "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": wl.dtype, "data": "synthetic",
            "config": {"workload": describe(wl),
                       "cg_iters": args.cg_iters, "cg_steps_applied_per_iteration": cg_per_step,
                       "decomposition": decomposition,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2, and a 512 MiB buffer rewritten between timed steps"},
            "phi_phiadj_gvis_s": gvis, "phi_ms": ops["phi"]["ms"], "phi_adj_ms": ops["phi_adj"]["ms"],
            "e2e": e2e, "gpu_launches": int(launches), "gpu_launches_per_step": launches / args.steps,
            "wall_s_timed": t_wall, "clocks": clocks, "roofline": roofline, "cpu_baseline": cpu,
            "toeplitz_cg": toep,
            "primal_dual": pdl,
            "other_workloads": others,
            "kernels": kernel_table,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def kernel_rates(ktimes, info, steps, dtb, levels):
    """Per-kernel-kind launches and milliseconds per step, with the
    algorithmic GB/s where the kind has a fixed per-launch byte count; the
    wavelet kinds are rated per transform (all levels of one Psi^dagger are
    dwt_level launches, all levels of one Psi are idwt_level launches plus
    one idwt_final), at 4N + 4qN bytes per transform."""
    table = {}
    for k, (n, t) in sorted(ktimes.items(), key=lambda kv: -kv[1][1]):
        ab = algorithmic_bytes(k, info, dtb)
        table[k] = {"launches_per_step": n / steps, "ms_per_step": t / steps,
                    "gbs": ab / (t / n * 1e-3) / 1e9 if ab else None}
    wav = dtb * (info.N + info.q * info.N)
    if "dwt_level" in ktimes:
        n, t = ktimes["dwt_level"]
        table["dwt_level"]["gbs_per_transform"] = (n / levels) * wav / (t * 1e-3) / 1e9
    if "idwt_final" in ktimes:
        nf_, tf = ktimes["idwt_final"]
        tl = ktimes.get("idwt_level", (0, 0.0))[1]
        table["idwt_final"]["gbs_per_transform_with_idwt_level"] = nf_ * wav / ((tf + tl) * 1e-3) / 1e9
    return table


# ------------------------------------------------------------- oracle arm
# The FP64 oracle timed on the host cores. Its gridding and degridding are
# sums and maps over visibilities, so they run in spawned worker processes
# on contiguous visibility chunks (each worker calls the oracle's own
# degrid/grid on its chunk; the chunk grids are added in chunk order), and
# its FFTs use scipy.fft with one worker thread per core. Nothing of the
# oracle's arithmetic changes.
_W = {}


def _pool_init(spec):
    from multiprocessing import shared_memory
    _W["shm"] = []
    for key, (name, shape, dt) in spec["arrays"].items():
        h = shared_memory.SharedMemory(name=name)
        _W["shm"].append(h)
        _W[key] = np.ndarray(shape, dtype=dt, buffer=h.buf)
    _W["spec"] = spec
    _W["plans"] = {}


def _pool_plan(k):
    from oracle import nufft as onf
    if k not in _W["plans"]:
        sp = _W["spec"]
        a, b = sp["chunks"][k]
        _W["plans"][k] = onf.NufftPlan(sp["nx"], sp["ny"], _W["u"][a:b], _W["v"][a:b], sp["J"])
    return _W["plans"][k]


def _pool_degrid(k):
    from oracle import nufft as onf
    a, b = _W["spec"]["chunks"][k]
    _W["y_out"][a:b] = onf.degrid(_pool_plan(k), _W["X"])
    return k


def _pool_grid(k):
    from oracle import nufft as onf
    a, b = _W["spec"]["chunks"][k]
    _W["grids"][k] = onf.grid(_pool_plan(k), _W["y_in"][a:b])
    return k


class OracleVisPool:
    """G and G^H of the oracle over `workers` visibility chunks in spawned
    processes, the arrays in shared memory."""

    def __init__(self, nx, ny, J, u, v, workers):
        import concurrent.futures as cf
        import multiprocessing as mp
        from multiprocessing import shared_memory
        M = u.size
        Kx, Ky = 2 * nx, 2 * ny
        self.P = max(1, min(workers, M))
        edges = np.linspace(0, M, self.P + 1).astype(np.int64)
        shapes = {"u": ((M,), np.float64), "v": ((M,), np.float64), "X": ((Ky, Kx), np.complex128),
                  "y_in": ((M,), np.complex128), "y_out": ((M,), np.complex128),
                  "grids": ((self.P, Ky, Kx), np.complex128)}
        self.shm, self.a, arrays = [], {}, {}
        for key, (shape, dt) in shapes.items():
            nbytes = int(np.prod(shape)) * np.dtype(dt).itemsize
            h = shared_memory.SharedMemory(create=True, size=max(nbytes, 1))
            self.shm.append(h)
            self.a[key] = np.ndarray(shape, dtype=dt, buffer=h.buf)
            arrays[key] = (h.name, shape, np.dtype(dt).str)
        self.a["u"][:] = u
        self.a["v"][:] = v
        spec = {"arrays": arrays, "chunks": [(int(edges[k]), int(edges[k + 1])) for k in range(self.P)],
                "nx": nx, "ny": ny, "J": J}
        self.ex = cf.ProcessPoolExecutor(max_workers=self.P, mp_context=mp.get_context("spawn"),
                                         initializer=_pool_init, initargs=(spec,))

    def degrid(self, X):
        self.a["X"][:] = X
        list(self.ex.map(_pool_degrid, range(self.P)))
        return self.a["y_out"].copy()

    def grid(self, y):
        self.a["y_in"][:] = y
        list(self.ex.map(_pool_grid, range(self.P)))
        g = self.a["grids"]
        out = g[0].copy()
        for k in range(1, self.P):
            out += g[k]
        return out

    def close(self):
        self.ex.shutdown(wait=True)
        for h in self.shm:
            h.close()
            h.unlink()


class OracleRun:
    """The FP64 oracle's SDMM iterations (k_CG = cg_iters) on the workload, or
    on a random visibility sample of it (vis_fraction < 1: the same blocks,
    each cut to its sampled visibilities), with the visibility pool above.
    step() runs one iteration and returns its wall seconds and the seconds of
    it spent in gridding and degridding."""

    def __init__(self, wl_name: str, cg_iters: int, vis_fraction: float, cores: int, seed: int = 0):
        import scipy.fft

        from oracle import nufft as onf
        from oracle import sdmm as osd
        from paper_1502_05037_gb300 import synth

        self.osd, self.cg_iters, self.cores = osd, cg_iters, cores
        self.wl = wl = synth.WORKLOADS[wl_name]
        x_true, u, v, offs, nz = wl.draw()
        if vis_fraction < 1.0:
            g = np.random.default_rng(seed)
            Ms = int(max(1024, min(wl.M, round(vis_fraction * wl.M))))
            idx = np.sort(g.choice(wl.M, Ms, replace=False))
            blk = np.searchsorted(offs, idx, side="right") - 1
            counts = np.bincount(blk, minlength=wl.R)
            counts = counts[counts > 0]
            offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
            u, v, nz = u[idx], v[idx], nz[idx]
        self.Ms = u.size
        self.pool = OracleVisPool(wl.nx, wl.ny, wl.J, u.astype(np.float64), v.astype(np.float64), cores)
        self.t_vis = 0.0
        run = self

        def degrid(X):
            t0 = time.perf_counter()
            r = run.pool.degrid(X)
            run.t_vis += time.perf_counter() - t0
            return r

        def grid(y):
            t0 = time.perf_counter()
            r = run.pool.grid(y)
            run.t_vis += time.perf_counter() - t0
            return r

        class PooledProblem(osd.Problem):
            def phi_n(self, x):
                return degrid(onf.fft2(onf.scale_pad(self.plan, x))) / self.nu

            def phi_n_adj_re(self, y):
                return np.real(onf.crop_scale(self.plan, onf.ifft2_unnormalised(grid(y)))) / self.nu

        with scipy.fft.set_workers(cores):
            op = onf.NufftPlan(wl.nx, wl.ny, u.astype(np.float64), v.astype(np.float64), wl.J)
            y0 = degrid(onf.fft2(onf.scale_pad(op, x_true)))
            sig = osd.noise_sigma(y0, wl.snr_db)
            eps = osd.epsilon_chi2(sig, np.diff(offs))
            # fixed constants: nu and gamma change no step count of the oracle's work
            self.prob = PooledProblem(op, wl.levels, y0 + sig * nz, offs, eps, nu=1.0, gamma=1e-4)
            self.state = osd.init_state(self.prob, np.zeros((wl.ny, wl.nx)))

    def step(self):
        import scipy.fft
        self.t_vis = 0.0
        with scipy.fft.set_workers(self.cores):
            t0 = time.perf_counter()
            self.osd.sdmm_iteration(self.prob, self.state, self.cg_iters)
            wall = time.perf_counter() - t0
        return wall, self.t_vis

    def scaled(self, wall, t_vis):
        """The iteration's seconds with its visibility work scaled to all M."""
        return wall + t_vis * (self.wl.M / self.Ms - 1.0)

    def close(self):
        self.pool.close()


def cpu_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(wl, cg_iters, vis_fraction=0.0):
    cores = cpu_threads()
    if vis_fraction <= 0.0:
        vis_fraction = min(1.0, 1.5e6 / wl.M)
    run = OracleRun(wl.name, cg_iters, vis_fraction, cores)
    try:
        wall, t_vis = run.step()
    finally:
        run.close()
    if run.Ms == wl.M:
        value, how = 1.0 / wall, "one whole FP64 oracle SDMM iteration on the full workload"
    else:
        value = 1.0 / run.scaled(wall, t_vis)
        how = (f"one FP64 oracle SDMM iteration on {run.Ms} of {wl.M} visibilities, its gridding time scaled "
               f"to all M")
    return {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
            "sample": f"{how} (k_CG={cg_iters}; {wall:.1f} s wall, {t_vis:.1f} s of it gridding and degridding "
                      f"in {cores} spawned processes over visibility chunks; scipy.fft with {cores} workers)"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = cpu_threads()
    run = OracleRun(args.workload, args.cg_iters, args.ref_vis_fraction, cores)
    wl = run.wl
    walls, scaled = [], []
    try:
        for k in range(args.warmup + args.steps):
            wall, t_vis = run.step()
            if k >= args.warmup:
                walls.append(wall)
                scaled.append(run.scaled(wall, t_vis))
    finally:
        run.close()
    value = args.steps / sum(scaled)
    whole = run.Ms == wl.M
    line = {
        "impl": "reference", "metric": "SDMM iters/s", "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": describe(wl), "cg_iters": args.cg_iters},
        "value_scaled_from_sample": not whole,
        "cpu_baseline": {"value": value, "unit": "iters/s", "kind": "oracle", "cores": cores,
                         "sample": (f"each step: one FP64 oracle SDMM iteration (k_CG={args.cg_iters}) on a fixed "
                                    f"random sample of {run.Ms} of {wl.M} visibilities (ms_per_step is its wall "
                                    f"time); value scales the gridding and degridding time to all M"
                                    if not whole else
                                    f"each step: one whole FP64 oracle SDMM iteration (k_CG={args.cg_iters})")
                         + f"; gridding in {cores} spawned processes, scipy.fft with {cores} workers"},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_profile_op(args):
    """Launch one operator W + K times on the workload (for ncu captures)."""
    import torch

    import paper_1502_05037_gb300 as pk
    from paper_1502_05037_gb300 import build as pbuild
    pbuild.build()
    dev = torch.device("cuda", 0)
    wl, plan, y, eps, x_true = setup_problem(args.workload, 0, dev, args.grid_mode)
    x = torch.from_numpy(x_true.astype(np.float32)).to(dev)
    yv = torch.empty(wl.M, dtype=torch.complex64, device=dev)
    xa = torch.empty((wl.ny, wl.nx), dtype=torch.complex64, device=dev)
    c = torch.empty((plan.info.q, wl.ny, wl.nx), dtype=torch.float32, device=dev)
    xo = torch.empty_like(x)
    if args.profile_op == "iteration":
        xs = torch.zeros_like(x)
        pk.purify_sdmm_solve(plan, y, eps, xs, max_iter=0, cg_iters=args.cg_iters, nu=1.0, gamma=1e-4)
    torch.cuda.synchronize(dev)
    # the profiled range (ncu --profile-from-start off): the W + K calls only,
    # not the plan's autotuning or the solver's set-up
    torch.cuda.profiler.start()
    t0 = time.perf_counter()
    for k in range(args.warmup + args.steps):
        if args.profile_op == "phi":
            pk.purify_phi(plan, x, yv)
        elif args.profile_op == "phi_adj":
            pk.purify_phi_adj(plan, y, xa)
        elif args.profile_op == "psi_adj":
            pk.purify_psi_adj(plan, x, c)
        elif args.profile_op == "psi":
            pk.purify_psi(plan, c, x)
        elif args.profile_op == "normal":
            pk.purify_phi_normal(plan, x, xo)
        else:
            pk.purify_sdmm_iterate(plan, 1)
    torch.cuda.synchronize(dev)
    torch.cuda.profiler.stop()
    print(json.dumps({"profile_op": args.profile_op, "calls": args.warmup + args.steps,
                      "wall_s": time.perf_counter() - t0, "launches": pk.purify_launch_count()}))


def run_channels(args):
    """Batched channels: 32 independent 512 x 512 problems (M ~ U(0.5N, 5N),
    R ~ U{4..16}) advanced together by one captured graph per iteration."""
    import torch

    import paper_1502_05037_gb300 as pk
    from paper_1502_05037_gb300 import build as pbuild
    from paper_1502_05037_gb300 import synth
    pbuild.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    chans = []
    for ch in range(args.channels):
        wl = synth.channel_workload(ch)
        _, plan, y, eps, _ = setup_problem(wl, 0, dev)
        x = torch.zeros((wl.ny, wl.nx), dtype=torch.float32, device=dev)
        pk.purify_sdmm_solve(plan, y, eps, x, max_iter=0, cg_iters=args.cg_iters)
        chans.append((wl, plan, y, eps))
    torch.cuda.synchronize(dev)
    stream = torch.cuda.Stream(dev)
    batch = pk.Batch([c[1] for c in chans], stream)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for i in range(args.warmup):
        pk.purify_batch_iterate(batch, 1)
    stream.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = pk.purify_launch_count()
    with ClockSampler(0) as clk:
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            torch.cuda.synchronize(dev)
            evs[k][0].record(stream)
            pk.purify_batch_iterate(batch, 1)
            evs[k][1].record(stream)
        stream.synchronize()
    launches = pk.purify_launch_count() - launches0
    tms = sum(a.elapsed_time(b) for a, b in evs)
    # the same iterations one channel after another (each plan's own graph)
    for c in chans:
        pk.purify_sdmm_iterate(c[1], 1)
    torch.cuda.synchronize(dev)
    seq = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for c in chans:
            pk.purify_sdmm_iterate(c[1], 1)
        b.record()
        seq.append((a, b))
    torch.cuda.synchronize(dev)
    tseq = sum(a.elapsed_time(b) for a, b in seq)
    M_tot = sum(c[0].M for c in chans)
    line = {
        "metric": "SDMM iters/s (channel-iterations, batched)", "value": len(chans) * args.steps / (tms / 1e3),
        "unit": "channel-iters/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tms / args.steps, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{len(chans)} channels of 512x512, M in [0.5N, 5N] (total {M_tot}), J=6, q=9, L=4, "
                               f"R in 4..16, 30 dB", "cg_iters": args.cg_iters},
        "sequential_ms_per_step": tseq / args.steps, "batched_speedup": tseq / tms,
        "gpu_launches": int(launches), "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_sharded(args):
    """Block-sharded SDMM (strong scaling): under torchrun each rank holds the
    blocks i = rank mod N of the workload on its GPU; x and the wavelet state
    are replicated; the two N-pixel exchanges per iteration and per CG step
    are NCCL all-reduces. Timed like the headline: W warm-up then K
    iterations bracketed by CUDA events, the max over ranks."""
    import torch

    import paper_1502_05037_gb300 as pk
    from paper_1502_05037_gb300 import build as pbuild
    from paper_1502_05037_gb300 import sharded, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    pbuild.build()
    wl = synth.WORKLOADS[args.workload]
    x_true, u, v, offs, nz = wl.draw()
    stream = torch.cuda.current_stream(dev)
    # the unsharded constants: nu by power iteration over all shards, gamma
    # from the summed dirty image (both through the exchange)
    blocks = sharded.shard_blocks(wl.R, world, rank)
    idx, loffs = sharded.shard_visibilities(offs, blocks)
    plan = pk.Plan(wl.nx, wl.ny, torch.from_numpy(u[idx]).to(dev), torch.from_numpy(v[idx]).to(dev), kb_width=wl.J,
                   levels=wl.levels, block_offsets=loffs, stream=stream)
    allreduce = sharded.all_reduce_images if dist is not None else sharded.sum_in_place
    xt = torch.from_numpy(x_true.astype(np.float32)).to(dev)
    y0 = torch.empty(idx.size, dtype=torch.complex64, device=dev)
    pk.purify_phi(plan, xt, y0)
    ysq = torch.tensor([float(torch.linalg.vector_norm(y0.to(torch.complex128)) ** 2)], dtype=torch.float64,
                       device=dev)
    if dist is not None:
        dist.all_reduce(ysq)
    from paper_1502_05037_gb300 import problem
    sigma = problem.noise_sigma_from_norm(float(ysq.sqrt().item()), wl.M, wl.snr_db)
    y = y0 + torch.from_numpy((sigma * nz[idx]).astype(np.complex64)).to(dev)
    eps = problem.chi2_epsilon(sigma, np.diff(offs))[blocks]
    # nu: power iteration on the summed normal operator
    g = torch.Generator(device="cpu").manual_seed(7)
    w = torch.randn((wl.ny, wl.nx), generator=g, dtype=torch.float32).to(dev)
    w /= torch.linalg.vector_norm(w)
    out = torch.empty_like(w)
    lam = 0.0
    for _ in range(30):
        pk.purify_phi_normal(plan, w, out)
        allreduce([out])
        lam = float(torch.linalg.vector_norm(out.double()).item())
        w = out / lam
    nu = float(np.sqrt(lam))
    dirty = torch.empty((wl.ny, wl.nx), dtype=torch.complex64, device=dev)
    pk.purify_phi_adj(plan, y, dirty)
    dr = dirty.real.contiguous()
    allreduce([dr])
    c = torch.empty((plan.info.q, wl.ny, wl.nx), dtype=torch.float32, device=dev)
    pk.purify_psi_adj(plan, dr, c)
    gamma = 1e-3 * float(c.abs().max().item()) / nu ** 2
    x0 = torch.zeros((wl.ny, wl.nx), dtype=torch.float32, device=dev)
    pk.purify_sdmm_solve(plan, y, eps, x0, max_iter=0, cg_iters=args.cg_iters, gamma=gamma, nu=nu)
    drv = sharded.ShardedSdmm([sharded.LibraryShard(plan, dev, torch.float32)], allreduce, args.cg_iters)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for i in range(args.warmup):
        drv.iterate(1)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    evs = []
    with ClockSampler(dev.index or 0) as clk:
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            drv.iterate(1)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize(dev)
    total = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dist, dev)
    if rank == 0:
        line = {"metric": "SDMM iters/s (block-sharded)", "value": args.steps / (total / 1e3), "unit": "iters/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
                "higher_is_better": True, "scaling": "strong", "dtype": "f32", "data": "synthetic",
                "config": {"workload": describe(wl), "cg_iters": args.cg_iters,
                           "parallelism": f"blocks round-robin over {world} shards, NCCL all-reduce of N-pixel "
                                          f"images ({1 + args.cg_iters} per iteration)"},
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_groups(args):
    """Time to tolerance of the stochastic block-subset SDMM (G groups, one
    drawn per iteration) against plain SDMM on the same problem: wall time
    until the objective is within 1e-3 of the plain solve's converged
    objective and every block meets its bound to 1e-3, checked every 10
    iterations through the C ABI (the checks are timed in every arm)."""
    import torch

    import paper_1502_05037_gb300 as pk
    from paper_1502_05037_gb300 import build as pbuild
    from paper_1502_05037_gb300 import synth
    pbuild.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    wl, plan, y, eps, x_true = setup_problem(args.workload, 0, dev)
    rdt = torch.float32
    cg = args.cg_iters
    # the plain converged objective
    x = torch.zeros((wl.ny, wl.nx), dtype=rdt, device=dev)
    st0 = pk.purify_sdmm_solve(plan, y, eps, x, max_iter=0, cg_iters=cg)
    nu, gamma = st0.nu, st0.gamma
    ref = pk.purify_sdmm_solve(plan, y, eps, x, max_iter=args.groups_cap * 2, cg_iters=cg, gamma=gamma, nu=nu,
                               rel_obj_tol=1e-6, eps_tol=1e-4, check_every=10, raise_on_error=False)
    f_star = ref.objective
    snr = lambda t: float(20 * np.log10(np.linalg.norm(x_true) / np.linalg.norm(x_true - t.cpu().numpy())))
    snr_star = snr(x)
    arms = []
    for G in [0] + [g for g in args.groups_list if 1 < g <= wl.R]:
        seq = synth.group_sequence(args.groups_cap, G, 7000 + G) if G else None
        x = torch.zeros((wl.ny, wl.nx), dtype=rdt, device=dev)
        # graph capture and group set-up outside the timed solve
        pk.purify_sdmm_solve(plan, y, eps, x, max_iter=G if G else 1, cg_iters=cg, gamma=gamma, nu=nu,
                             block_groups=G, group_seq=np.arange(G, dtype=np.int32) if G else None)
        x.zero_()
        torch.cuda.synchronize(dev)
        t, it, reached, st = 0.0, 0, False, None
        while it < args.groups_cap:
            t0 = time.perf_counter()
            st = pk.purify_sdmm_solve(plan, y, eps, x, max_iter=10, cg_iters=cg, gamma=gamma, nu=nu,
                                      resume=it > 0, block_groups=G,
                                      group_seq=seq[it:it + 10] if G else None)
            t += time.perf_counter() - t0
            it += 10
            if st.objective <= (1 + 1e-3) * f_star and st.max_resid_over_eps <= 1 + 1e-3:
                reached = True
                break
        arms.append({"groups": G, "seconds": t, "iterations": it, "reached": reached,
                     "objective_over_plain_converged": st.objective / f_star,
                     "max_resid_over_eps": st.max_resid_over_eps, "snr_db": snr(x)})
        print(f"[groups] G={G}: {t:.3f} s, {it} iterations, reached {reached}", file=sys.stderr, flush=True)
    plain = arms[0]
    line = {
        "metric": "time-to-tolerance, block-subset SDMM vs plain", "unit": "x (plain seconds / block-subset seconds)",
        "higher_is_better": True, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
        "config": {"workload": describe(wl), "cg_iters": cg,
                   "tolerance": "objective <= (1 + 1e-3) x plain converged objective and every "
                                "||y_i - Phi_i x|| / eps_i <= 1 + 1e-3, checked every 10 iterations",
                   "groups": "block i in group i mod G, one group per iteration drawn uniformly (seeded)"},
        "plain_converged": {"objective": f_star, "iterations": ref.iters, "snr_db": snr_star},
        "arms": arms,
        "speedup": {str(a["groups"]): (plain["seconds"] / a["seconds"] if a["reached"] and plain["reached"] else None)
                    for a in arms[1:]},
    }
    print(json.dumps(line), flush=True)


def run_warmstart(args):
    """Time to tolerance of SARA from the learned warm start versus the plain
    SARA solve on held-out problems (all GPU work through the C ABI; the
    protocol is in paper_1502_05037_gb300/warmstart.py)."""
    import torch

    import paper_1502_05037_gb300 as pk
    from paper_1502_05037_gb300 import build as pbuild
    from paper_1502_05037_gb300 import warmstart as ws
    pbuild.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t_all = time.perf_counter()
    net = pk.Unet(ws.N_SIDE, ws.N_SIDE, 4, 32, max_batch=args.batch, seed=1)
    t_data = t_train = 0.0
    losses = []
    if args.unet_params and os.path.exists(args.unet_params):
        net.set_params(torch.from_numpy(np.load(args.unet_params)).to(dev))
    else:
        t0 = time.perf_counter()
        inputs, targets = ws.build_training_set(dev, ws.BENCH, args.train_samples, args.target_iters, args.pass_iters)
        t_data = time.perf_counter() - t0
        print(f"[warmstart] {inputs.shape[0]} SARA targets in {t_data:.1f} s", file=sys.stderr, flush=True)
        t0 = time.perf_counter()
        losses = ws.train(net, inputs, targets, args.epochs, args.batch, args.lr)
        torch.cuda.synchronize(dev)
        t_train = time.perf_counter() - t0
        print(f"[warmstart] trained {args.epochs} epochs in {t_train:.1f} s, losses {losses}", file=sys.stderr,
              flush=True)
        del inputs, targets
        if args.unet_params:
            prm = torch.empty(net.num_params, dtype=torch.float32, device=dev)
            net.get_params(prm)
            np.save(args.unet_params, prm.cpu().numpy())
    rows = []
    for s in range(args.eval_samples):
        p = ws.make_problem(ws.EVAL_SEED0 + s, dev)
        ws.start(p, torch.zeros((ws.N_SIDE, ws.N_SIDE), dtype=torch.float32, device=dev))   # nu, gamma
        if s == 0:   # first use of the solver graphs outside the timed arms
            ws.sara_plain(p, dev)
            ws.sara_learned(p, net, dev)
        row = ws.compare(p, ws.sara_plain(p, dev), ws.sara_learned(p, net, dev, args.learned_passes))
        rows.append(row)
        print(f"[warmstart] eval {s}: plain {row['t_plain']:.3f} s / {row['it_plain']} it, learned "
              f"{row['t_learned']:.3f} s / {row['it_learned']} it, reached {row['reached']}, objective excess "
              f"{row['obj_excess']:.2e}, SNR plain {row['snr_plain']:.3f} learned {row['snr_learned']:.3f} "
              f"prediction {row['snr_prediction']:.3f} dB", file=sys.stderr, flush=True)
        p.plan.close()
    tp = np.array([r["t_plain"] for r in rows])
    tl = np.array([r["t_learned"] for r in rows])
    ok = np.array([r["reached"] for r in rows], dtype=float)
    # a miss costs its learned attempt plus the plain solve (the fallback)
    cost = tl + (1.0 - ok) * tp
    speedup = tp.sum() / cost.sum()
    g = np.random.default_rng(0)
    boot = []
    for _ in range(2000):
        i = g.integers(0, len(rows), len(rows))
        boot.append(tp[i].sum() / cost[i].sum())
    lo, hi = np.percentile(boot, [2.5, 97.5])
    line = {
        "metric": "time-to-tolerance learned vs plain", "value": speedup,
        "unit": "x (plain seconds / learned seconds, misses counted with the plain solve as fallback)",
        "higher_is_better": True, "n_gpus": 1, "dtype": "f32 SDMM, bf16 U-Net", "data": "synthetic",
        "config": {"workload": f"SARA ({ws.PASSES} reweighted passes) on {ws.N_SIDE}x{ws.N_SIDE} skies, M={ws.M_VIS}, "
                               f"J={ws.J}, L={ws.LEVELS}, R=1, {ws.SNR_DB:g} dB; U-Net 4 levels base 32",
                   "train_samples": args.train_samples, "eval_samples": len(rows), "eval_seeds":
                   f"{ws.EVAL_SEED0}..{ws.EVAL_SEED0 + len(rows) - 1}", "target_iters": args.target_iters,
                   "pass_iters": args.pass_iters, "epochs": args.epochs, "batch": args.batch, "lr": args.lr,
                   "pass_rule": f"relative objective change < {ws.PASS_REL_TOL:g} over 10 iterations and every "
                                f"||y_i - Phi_i x||/eps_i <= 1+{ws.PASS_EPS_TOL:g} (both arms, no true sky)",
                   "plain": f"W = I pass from x = 0, then {ws.PASSES} reweighted passes (rho = std(Psi^dagger x) "
                            f"halved per pass)",
                   "learned": f"U-Net prediction (inference timed), then {args.learned_passes} reweighted passes "
                              f"from it",
                   "reached": f"objective under the plain final weights <= (1 + {ws.OBJ_TOL:g}) x plain, "
                              f"constraint ratios <= 1 + {ws.PASS_EPS_TOL:g}, SNR >= plain SNR - {ws.SNR_TOL:g} dB"},
        "speedup_ci95": [float(lo), float(hi)],
        "speedup_without_fallback": float(tp.sum() / tl.sum()),
        "reached_fraction": float(ok.mean()),
        "plain": {"seconds_mean": float(tp.mean()), "iters_mean": float(np.mean([r["it_plain"] for r in rows]))},
        "learned": {"seconds_mean": float(tl.mean()), "iters_mean": float(np.mean([r["it_learned"] for r in rows]))},
        "snr_db": {"plain": float(np.mean([r["snr_plain"] for r in rows])),
                   "learned": float(np.mean([r["snr_learned"] for r in rows])),
                   "prediction": float(np.mean([r["snr_prediction"] for r in rows]))},
        "objective_excess": {"mean": float(np.mean([r["obj_excess"] for r in rows])),
                             "max": float(np.max([r["obj_excess"] for r in rows]))},
        "constraint_ratio_max": {"plain": float(max(r["ratio_plain"] for r in rows)),
                                 "learned": float(max(r["ratio_learned"] for r in rows))},
        "train_loss": {"first_epoch": losses[0] if losses else None, "last_epoch": losses[-1] if losses else None},
        "seconds": {"data": t_data, "train": t_train, "total": time.perf_counter() - t_all},
        "gpu_launches": pk.purify_launch_count(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=250)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="sara1024_r64")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the extra timed passes on the 256x256 and 64x64 workloads")
    ap.add_argument("--cg-iters", type=int, default=CG_ITERS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-vis-fraction", type=float, default=0.0,
                    help="visibility fraction of the timed oracle iteration of cpu_baseline (1 = whole iteration; "
                         "0 = whole up to 1.5 M visibilities, else a 1.5 M sample)")
    ap.add_argument("--ref-vis-fraction", type=float, default=1.0 / 64,
                    help="visibility sample of each oracle step of --impl reference")
    ap.add_argument("--no-pd-pass", dest="pd_pass", action="store_false",
                    help="skip timing the primal-dual solver")
    ap.add_argument("--no-toeplitz-pass", dest="toeplitz_pass", action="store_false",
                    help="skip the extra timed pass with the circulant-embedded CG normal operator")
    ap.add_argument("--channels32", action="store_true",
                    help="batched independent 512x512 channel problems (one graph per iteration)")
    ap.add_argument("--channels", type=int, default=32)
    ap.add_argument("--shard-blocks", action="store_true",
                    help="block-sharded SDMM over the ranks (strong scaling; NCCL all-reduce of images)")
    ap.add_argument("--groups", action="store_true",
                    help="time-to-tolerance of the stochastic block-subset SDMM versus plain SDMM")
    ap.add_argument("--groups-list", type=int, nargs="*", default=[2, 4, 8])
    ap.add_argument("--groups-cap", type=int, default=3000)
    ap.add_argument("--warmstart", action="store_true",
                    help="time-to-tolerance of the learned warm start versus zero start (trains the U-Net)")
    ap.add_argument("--train-samples", type=int, default=2000)
    ap.add_argument("--eval-samples", type=int, default=200)
    ap.add_argument("--learned-passes", type=int, default=2)
    ap.add_argument("--unet-params", default=None,
                    help="U-Net parameter file (.npy): loaded if it exists (no training), else written after training")
    ap.add_argument("--target-iters", type=int, default=300)
    ap.add_argument("--pass-iters", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--grid-mode", type=int, default=0,
                    help="gridding decomposition of the timed plan (0 autotuned; 6 deterministic: stored run "
                         "patches summed per cell in a fixed order)")
    ap.add_argument("--profile-op", choices=["phi", "phi_adj", "psi", "psi_adj", "normal", "iteration"], default=None,
                    help="only launch this operator W + K times (for ncu captures); prints no bench line")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.channels32:
        run_channels(args)
    elif args.groups:
        run_groups(args)
    elif args.shard_blocks:
        run_sharded(args)
    elif args.warmstart:
        run_warmstart(args)
    elif args.profile_op:
        run_profile_op(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
