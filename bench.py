#!/usr/bin/env python
"""Benchmark of the SARA/SDMM imaging hot path on GB300.

Workload (default): 256 x 256 sky, M = 655,360 visibilities (Gaussian (u, v)
density), Kaiser-Bessel width J = 6, oversampling 2, Psi = Dirac + db1..db8 at
4 levels (q = 9), R = 8 uneven blocks, FP32 operators with FP64 reductions,
30 dB input SNR, synthetic seeded data. One step = one SDMM iteration
(Psi^dagger + prox, Phi + block projections, positivity, Psi, Phi^dagger and
CG_ITERS conjugate-gradient steps of Phi^dagger Phi) on the plan's resident
state, launched as one captured CUDA graph.

Passes (all in one run):
  A  timed pass: W warm-up steps, then K steps each bracketed by CUDA events
     on the launching stream; a 512 MiB buffer is rewritten between steps to
     flush L2 (outside the events).                      -> value, ms_per_step
  B  roofline pass: the same K steps launched eagerly with per-kernel CUDA
     events; the dominant kernel's algorithmic bytes / mean duration.
  C  end-to-end pass: K calls of purify_sdmm_solve with pinned host buffers
     (y in, x in/out), one iteration each, wall-clock timed.  -> e2e
  D  Phi + Phi^dagger through the C ABI (caller order).      -> Gvis/s
  E  CPU baseline: the FP64 oracle, one SDMM iteration on a visibility
     sample, scaled to the full workload (rank 0, N = 1 only).

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


def ncu_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current source of that kernel; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        e = d.get(kernel)
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
def setup_problem(wl_name: str, replica: int, dev):
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
                   dtype=pk.PURIFY_F64 if f64 else pk.PURIFY_F32)
    xt = torch.from_numpy(x_true).to(rt).to(dev)
    y0 = torch.empty(wl.M, dtype=ct, device=dev)
    pk.purify_phi(plan, xt, y0)
    sigma = problem.noise_sigma_from_norm(float(torch.linalg.vector_norm(y0.to(torch.complex128)).item()), wl.M,
                                          wl.snr_db)
    y = y0 + torch.from_numpy(sigma * nz).to(ct).to(dev)
    eps = problem.chi2_epsilon(sigma, np.diff(offs))
    return wl, plan, y, eps, x_true


# ------------------------------------------------------------------ ours
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

    wl, plan, y, eps, x_true = setup_problem(args.workload, rank, dev)
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
    roofline = None
    if dom:
        name, (nl, tms) = dom
        per = tms / nl
        ab = algorithmic_bytes(name, plan.info, 8 if wl.dtype == "f64" else 4)
        af = algorithmic_flops(name, plan.info)
        tr = ncu_traffic(name)
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
    kernel_table = {k: {"launches_per_step": n / args.steps, "ms_per_step": t / args.steps,
                        "gbs": (algorithmic_bytes(k, plan.info, 8 if wl.dtype == "f64" else 4) / (t / n * 1e-3) / 1e9
                                if algorithmic_bytes(k, plan.info) else None)}
                    for k, (n, t) in sorted(ktimes.items(), key=lambda kv: -kv[1][1])}

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
    rb = 8 if wl.dtype == "f64" else 4
    e2e = {"value": job_rate(world, args.steps, e2e_total * 1e3), "unit": "iters/s",
           "h2d_bytes_per_step": wl.M * 2 * rb + wl.nx * wl.ny * rb, "d2h_bytes_per_step": wl.nx * wl.ny * rb,
           "call": "purify_sdmm_solve(host y, host x, max_iter=1)"}

    # ---- pass A': the same timed steps with the circulant-embedded CG normal operator
    toep = None
    if args.toeplitz_pass:
        xt0 = torch.zeros((wl.ny, wl.nx), dtype=rdt, device=dev)
        pk.purify_sdmm_solve(plan, y, eps, xt0, max_iter=0, cg_iters=args.cg_iters, gamma=gamma, nu=nu, toeplitz=True)
        for i in range(args.warmup):
            flush.fill_(i & 0xFF)
            pk.purify_sdmm_iterate(plan, 1)
        torch.cuda.synchronize(dev)
        tev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_((k + 11) & 0xFF)
            tev[k][0].record(stream)
            pk.purify_sdmm_iterate(plan, 1)
            tev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        tms = sum(a.elapsed_time(b) for a, b in tev)
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

    # ---- pass D: Phi + Phi^dagger Gvis/s (caller order, device buffers)
    xin = torch.from_numpy(x_true).to(rdt).to(dev)
    yv = torch.empty(wl.M, dtype=cdt, device=dev)
    xa = torch.empty((wl.ny, wl.nx), dtype=cdt, device=dev)
    for _ in range(3):
        pk.purify_phi(plan, xin, yv)
        pk.purify_phi_adj(plan, yv, xa)
    ph = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        pk.purify_phi(plan, xin, yv)
        b.record(stream)
        pk.purify_phi_adj(plan, yv, xa)
        c.record(stream)
        ph.append((a, b, c))
    torch.cuda.synchronize(dev)
    t_phi = sum(a.elapsed_time(b) for a, b, _ in ph) / args.steps
    t_adj = sum(b.elapsed_time(c) for _, b, c in ph) / args.steps
    gvis = wl.M / ((t_phi + t_adj) * 1e-3) / 1e9

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, args.cg_iters, budget_s=args.cpu_budget)

    if rank == 0:
        line = {
            "metric": "SDMM iters/s", "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": wl.dtype, "data": "synthetic",
            "config": {"workload": f"{wl.name}: {wl.nx}x{wl.ny} sky, M={wl.M}, J={wl.J}, alpha=2, q=9, "
                                   f"L={wl.levels}, R={wl.R}, {wl.snr_db:g} dB",
                       "cg_iters": args.cg_iters, "cg_steps_applied_per_iteration": cg_per_step,
                       "parallelism": f"replicas x{world}",
                       "l2": "512 MiB buffer rewritten between timed steps"},
            "phi_phiadj_gvis_s": gvis, "phi_ms": t_phi, "phi_adj_ms": t_adj,
            "e2e": e2e, "gpu_launches": int(launches), "gpu_launches_per_step": launches / args.steps,
            "wall_s_timed": t_wall, "clocks": clocks, "roofline": roofline, "cpu_baseline": cpu,
            "toeplitz_cg": toep,
            "primal_dual": pdl,
            "kernels": kernel_table,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------- oracle arm
def oracle_iteration_seconds(wl_name: str, cg_iters: int, vis_sample: int, seed=0):
    """Seconds of one FP64 oracle SDMM iteration on the workload, measured on
    a visibility sample and scaled: the sampled iteration is timed whole,
    then the visibility-proportional steps (gridding and degridding, once per
    Phi and Phi^dagger: cg_iters + 1 of each) are timed alone on the sample and
    extrapolated linearly to all M visibilities."""
    from oracle import nufft as onf
    from oracle import sdmm as osd
    from paper_1502_05037_gb300 import problem, synth

    wl = synth.WORKLOADS[wl_name]
    x_true, u, v, offs, nz = wl.draw()
    g = np.random.default_rng(seed)
    Ms = int(min(wl.M, max(1024, vis_sample)))
    idx = np.sort(g.choice(wl.M, Ms, replace=False))
    blk = np.searchsorted(offs, idx, side="right") - 1
    offs_s = np.concatenate([[0], np.cumsum(np.bincount(blk, minlength=wl.R))])
    keep = np.diff(offs_s) > 0
    offs_s = np.concatenate([[0], np.cumsum(np.diff(offs_s)[keep])])
    op = onf.NufftPlan(wl.nx, wl.ny, u[idx].astype(np.float64), v[idx].astype(np.float64), wl.J)
    y0 = onf.phi(op, x_true)
    sig = problem.noise_sigma_from_norm(float(np.linalg.norm(y0)), Ms, wl.snr_db)
    y = y0 + sig * nz[idx]
    eps = problem.chi2_epsilon(sig, np.diff(offs_s))
    # fixed constants: nu and gamma change no step count of the oracle's work
    prob = osd.Problem(op, wl.levels, y, offs_s, eps, nu=1.0, gamma=1e-4)
    st = osd.init_state(prob, np.zeros((wl.ny, wl.nx)))
    t0 = time.perf_counter()
    osd.sdmm_iteration(prob, st, cg_iters)
    t_iter = time.perf_counter() - t0
    X = onf.fft2(onf.scale_pad(op, x_true))
    t0 = time.perf_counter()
    onf.degrid(op, X)
    onf.grid(op, y)
    t_vis = time.perf_counter() - t0
    total = t_iter + (cg_iters + 1) * t_vis * (wl.M / Ms - 1.0)
    return total, Ms, t_iter, t_vis


def cpu_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(wl, cg_iters, budget_s=20.0):
    Ms = int(65536 * max(0.25, budget_s / 20.0))
    total, Ms, t_iter, t_vis = oracle_iteration_seconds(wl.name, cg_iters, Ms)
    return {"value": 1.0 / total, "unit": "iters/s", "cores": 1, "kind": "oracle",
            "threads_available": cpu_threads(),
            "sample": f"one FP64 oracle SDMM iteration (k_CG={cg_iters}) on {Ms} of {wl.M} visibilities "
                      f"({t_iter:.1f} s), gridding+degridding timed alone on the sample ({t_vis:.2f} s) "
                      f"and scaled to all visibilities; NumPy/SciPy single-threaded"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1502_05037_gb300 import synth
    wl = synth.WORKLOADS[args.workload]
    per_step_budget = max(1.0, 150.0 / max(1, args.steps + args.warmup))
    Ms = int(65536 * per_step_budget / 6.0)
    secs = []
    for k in range(args.warmup + args.steps):
        total, Ms_used, t_iter, t_vis = oracle_iteration_seconds(args.workload, args.cg_iters, Ms, seed=k)
        if k >= args.warmup:
            secs.append(total)
    value = args.steps / sum(secs)
    line = {
        "impl": "reference", "metric": "SDMM iters/s", "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{wl.name}: {wl.nx}x{wl.ny} sky, M={wl.M}, J={wl.J}, alpha=2, q=9, "
                               f"L={wl.levels}, R={wl.R}, {wl.snr_db:g} dB", "cg_iters": args.cg_iters},
        "cpu_baseline": {"value": value, "unit": "iters/s", "kind": "oracle", "cores": 1,
                         "sample": f"each step: one oracle SDMM iteration on {Ms_used} of {wl.M} visibilities, "
                                   f"visibility-proportional steps scaled to all M"},
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
    wl, plan, y, eps, x_true = setup_problem(args.workload, 0, dev)
    x = torch.from_numpy(x_true.astype(np.float32)).to(dev)
    yv = torch.empty(wl.M, dtype=torch.complex64, device=dev)
    xa = torch.empty((wl.ny, wl.nx), dtype=torch.complex64, device=dev)
    c = torch.empty((plan.info.q, wl.ny, wl.nx), dtype=torch.float32, device=dev)
    if args.profile_op == "iteration":
        xs = torch.zeros_like(x)
        pk.purify_sdmm_solve(plan, y, eps, xs, max_iter=0, cg_iters=args.cg_iters, nu=1.0, gamma=1e-4)
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
        else:
            pk.purify_sdmm_iterate(plan, 1)
    torch.cuda.synchronize(dev)
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


def run_warmstart(args):
    """Time-to-tolerance of SARA from the learned warm start versus the plain
    SARA solve on held-out problems (all GPU work through the C ABI)."""
    import torch

    import paper_1502_05037_gb300 as pk
    from paper_1502_05037_gb300 import build as pbuild
    from paper_1502_05037_gb300 import warmstart as ws
    pbuild.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t_all = time.perf_counter()
    # training data: SARA solutions of seeded problems
    dirty, target = [], []
    t0 = time.perf_counter()
    for i in range(0, args.train_samples, 32):
        probs = [ws.make_problem(ws.TRAIN_SEED0 + s, dev) for s in range(i, min(i + 32, args.train_samples))]
        sols = ws.sara_targets(probs, dev, args.target_iters, args.pass_iters)
        for p, x in zip(probs, sols):
            dirty.append(p.dirty)
            target.append(x)
        for p in probs:
            p.plan.close()
    inputs = torch.stack(dirty).contiguous()
    targets = torch.stack(target).contiguous()
    t_data = time.perf_counter() - t0
    print(f"[warmstart] {len(dirty)} SARA targets in {t_data:.1f} s", file=sys.stderr, flush=True)
    net = pk.Unet(ws.N_SIDE, ws.N_SIDE, 4, 32, max_batch=args.batch, seed=1)
    t0 = time.perf_counter()
    losses = ws.train(net, inputs, targets, args.epochs, args.batch, args.lr)
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0
    print(f"[warmstart] trained {args.epochs} epochs in {t_train:.1f} s, losses {losses}", file=sys.stderr, flush=True)
    del inputs, targets
    # evaluation on held-out seeds
    rows = []
    for s in range(args.eval_samples):
        p = ws.make_problem(ws.EVAL_SEED0 + s, dev)
        ws.start(p, torch.zeros((ws.N_SIDE, ws.N_SIDE), dtype=torch.float32, device=dev))   # nu, gamma
        if s == 0:   # first use of the solver graphs outside the timed arms
            ws.sara_plain(p, dev)
        t_plain, it_plain, x_plain, w_plain, st_plain = ws.sara_plain(p, dev)
        snr = lambda x: float(20 * np.log10(np.linalg.norm(p.x_true) / np.linalg.norm(p.x_true - x.cpu().numpy())))
        snr_plain = snr(x_plain)
        t_warm, it_warm, x_warm, st_warm, reached, pred_snr, passes = ws.sara_learned(p, net, dev, snr_plain - 0.05)
        obj_plain, ratio_plain = ws.objective_at(p, x_plain, w_plain)
        obj_warm, ratio_warm = ws.objective_at(p, x_warm, w_plain)
        rows.append((t_plain, it_plain, t_warm, it_warm, snr_plain, snr(x_warm), obj_warm / obj_plain - 1.0,
                     ratio_plain, ratio_warm, float(reached), pred_snr, passes))
        print(f"[warmstart] eval {s}: plain {t_plain:.3f} s / {it_plain} it, learned {t_warm:.3f} s / {it_warm} it "
              f"(reached {reached}, {passes} passes), SNR plain {rows[-1][4]:.3f} learned {rows[-1][5]:.3f} prediction {pred_snr:.3f} dB",
              file=sys.stderr, flush=True)
        p.plan.close()
    arr = np.array(rows)
    speedup = arr[:, 0].sum() / arr[:, 2].sum()
    # with the plain solve as fallback: a problem whose learned solve does not
    # reach the plain quality costs its learned attempt plus the plain solve
    fallback = arr[:, 0].sum() / (arr[:, 2] + (1.0 - arr[:, 9]) * arr[:, 0]).sum()
    line = {
        "metric": "time-to-tolerance learned vs plain", "value": speedup, "unit": "x (plain seconds / learned seconds)",
        "higher_is_better": True, "n_gpus": 1, "dtype": "f32 SDMM, bf16 U-Net", "data": "synthetic",
        "config": {"workload": f"SARA ({ws.PASSES} reweighted passes) on {ws.N_SIDE}x{ws.N_SIDE} skies, M={ws.M_VIS}, "
                               f"J={ws.J}, L={ws.LEVELS}, R=1, {ws.SNR_DB:g} dB; U-Net 4 levels base 32",
                   "train_samples": args.train_samples, "eval_samples": args.eval_samples,
                   "target_iters": args.target_iters, "pass_iters": args.pass_iters, "epochs": args.epochs,
                   "batch": args.batch, "lr": args.lr,
                   "pass_tolerance": f"relative objective change < {ws.PASS_REL_TOL:g} over 10 iterations and every "
                                     f"||y_i - Phi_i x||/eps_i <= 1+{ws.PASS_EPS_TOL:g}",
                   "plain": "W = I pass from x = 0, then the reweighted passes (rho = std(Psi^dagger x) halved per pass)",
                   "learned": "U-Net prediction, weights from it, reweighted passes from it until SNR >= plain SNR "
                              "- 0.05 dB and constraints hold (checked every 10 iterations; a stagnating pass is "
                              "followed by one more with weights from its result; at most 2 passes, 3000 iterations; "
                              "inference and checks timed)"},
        "plain": {"seconds_mean": float(arr[:, 0].mean()), "iters_mean": float(arr[:, 1].mean())},
        "learned": {"seconds_mean": float(arr[:, 2].mean()), "iters_mean": float(arr[:, 3].mean())},
        "value_with_plain_fallback": fallback,
        "reached_plain_quality": float(arr[:, 9].mean()),
        "learned_passes_mean": float(arr[:, 11].mean()),
        "snr_db": {"plain": float(arr[:, 4].mean()), "learned": float(arr[:, 5].mean()),
                   "prediction": float(arr[:, 10].mean()),
                   "min_learned_minus_plain": float((arr[:, 5] - arr[:, 4]).min())},
        "objective_excess_under_plain_weights": {"mean": float(arr[:, 6].mean()), "max": float(arr[:, 6].max())},
        "constraint_ratio_max": {"plain": float(arr[:, 7].max()), "learned": float(arr[:, 8].max())},
        "train_loss": {"first_epoch": losses[0], "last_epoch": losses[-1]},
        "seconds": {"data": t_data, "train": t_train, "total": time.perf_counter() - t_all},
        "gpu_launches": pk.purify_launch_count(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="sara256_r8")
    ap.add_argument("--cg-iters", type=int, default=CG_ITERS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-pd-pass", dest="pd_pass", action="store_false",
                    help="skip timing the primal-dual solver")
    ap.add_argument("--no-toeplitz-pass", dest="toeplitz_pass", action="store_false",
                    help="skip the extra timed pass with the circulant-embedded CG normal operator")
    ap.add_argument("--channels32", action="store_true",
                    help="batched independent 512x512 channel problems (one graph per iteration)")
    ap.add_argument("--channels", type=int, default=32)
    ap.add_argument("--warmstart", action="store_true",
                    help="time-to-tolerance of the learned warm start versus zero start (trains the U-Net)")
    ap.add_argument("--train-samples", type=int, default=2000)
    ap.add_argument("--eval-samples", type=int, default=24)
    ap.add_argument("--target-iters", type=int, default=300)
    ap.add_argument("--pass-iters", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--profile-op", choices=["phi", "phi_adj", "psi", "psi_adj", "iteration"], default=None,
                    help="only launch this operator W + K times (for ncu captures); prints no bench line")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.channels32:
        run_channels(args)
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
