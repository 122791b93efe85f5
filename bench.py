"""Throughput benchmark of the LLG hot path on GB300.

Metric: LLG cell-steps/s (cells x accepted integrator steps per second).
Headline workload (the largest single-GPU case): 512x512x64 cells of 3 nm
cubes (16.7 M cells), Ms 8e5, A 1.3e-11, alpha 0.02, seeded random vortex,
FP32 Dormand-Prince RK45 (rtol 1e-6, device-side controller) with the FP64
Newell tensor setup and exact FFT demag on the 1024x1024x128 padded grid.
One step = one accepted RK45 step (6 field evaluations, each
exchange + demag, plus the stage, error and controller kernels).

Multi-GPU: replicas only (independent runs of the same workload per rank,
no data-path collective); value = sum of cell-steps over ranks / max time.

--impl reference times the FP64 CPU oracle (the only reference available:
the paper ships no code) on samples of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "LLG cell-steps/s: plain FP32 vs batched/surrogate, at stated error vs FP64 oracle"
UNIT = "cell-steps/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 7 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 7 and r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for q, n in enumerate(names):
                if len(r) >= 7 and r[3 + q].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _traffic_for(kernel: str, workload: str):
    """ncu DRAM bytes per launch recorded in profiles/traffic.json for this
    kernel on this workload, used only while the source files that define
    the kernel still hash to the values recorded with the capture (any change
    to them makes it null)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            ent = json.load(f)["kernels"][f"{kernel}@{workload}"]
        h = hashlib.sha256()
        for rel in ent["sources"]:
            with open(os.path.join(ROOT, rel), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != ent["sources_sha256"]:
            return None
        return ent["dram_bytes_per_launch"]
    except Exception:
        return None


# Sample grids of the headline workload (same material, 3 nm cubes, vortex
# start, RK45, exact demag), largest first: the oracle steps the largest one
# that fits its time budget.
REFERENCE_SAMPLES = [(512, 512, 64), (256, 256, 64), (256, 256, 32), (128, 128, 32), (128, 128, 16),
                     (64, 64, 16), (32, 32, 16), (16, 16, 16), (16, 16, 8), (8, 8, 8), (4, 4, 4)]
REFERENCE_BUDGET_S = 240.0


def _host_cores() -> int:
    return os.cpu_count() or 1


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def _vortex_sample(shape):
    from dataclasses import replace
    w = W.vortex_512x512x64()
    g = W.Grid(shape[0], shape[1], shape[2], w.grid.dx, w.grid.dy, w.grid.dz)
    return replace(w, grid=g)


def _oracle_solver(shape):
    from oracle.demag import demag_spectrum
    from oracle.fields import Problem
    from oracle.llg import Solver
    w = _vortex_sample(shape)
    p = Problem.from_workload(w.grid, w.mat)
    s = Solver(p, W.m_vortex(w.grid, seed=w.seed), K_hat=demag_spectrum(p.shape, p.d), dt=1e-14, rtol=w.rtol)
    s.k1 = s.slope(s.m)
    return s, w.grid.n


def _oracle_run(args):
    """One oracle process: W untimed and K timed fixed-dt RK45 steps of a
    sample grid; returns (cells, seconds of the K steps)."""
    shape, warmup, steps = args
    s, n = _oracle_solver(shape)
    for _ in range(warmup):
        s.rk45_step_fixed(1e-14)
    t0 = time.perf_counter()
    for _ in range(steps):
        s.rk45_step_fixed(1e-14)
    return n, time.perf_counter() - t0


def _oracle_pool(shape, warmup, steps, procs):
    """The oracle as it stands in `procs` processes at once (one per host
    core, spawned so that no CUDA state is inherited), each stepping its own
    copy of the sample; returns total cell-steps / the slowest process's
    time, and that time."""
    import multiprocessing as mp
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_oracle_run, [(shape, warmup, steps)] * procs)
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    t = max(r[1] for r in res)
    return sum(r[0] for r in res) * steps / t, t


def _per_cell_step_probe():
    probe, n = _oracle_solver((32, 32, 16))
    probe.rk45_step_fixed(1e-14)
    t0 = time.perf_counter()
    for _ in range(2):
        probe.rk45_step_fixed(1e-14)
    return (time.perf_counter() - t0) / (2 * n)


def _pick_sample(per_cell_step, steps, budget_s):
    for cand in REFERENCE_SAMPLES:
        if per_cell_step * cand[0] * cand[1] * cand[2] * steps <= budget_s:
            return cand
    return REFERENCE_SAMPLES[-1]


def cpu_baseline(seconds_budget=12.0, steps=3):
    """The FP64 oracle as it stands on this host: fixed-dt RK45 steps of a
    sample of the headline workload sized to about `seconds_budget` of
    stepping, once in one process (one core) and once in one process per
    host core (each stepping its own copy); Newell/FFT setup excluded."""
    per = _per_cell_step_probe()
    shape = _pick_sample(per, steps, seconds_budget)
    _, t1 = _oracle_run((shape, 0, steps))
    n = shape[0] * shape[1] * shape[2]
    one = n * steps / t1
    cores = _host_cores()
    allv, tall = _oracle_pool(shape, 0, steps, cores)
    return {"value": allv, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": _cpu_model(),
            "single_core": {"value": one, "cores": 1, "seconds": round(t1, 2)},
            "sample": f"{steps} fixed-dt RK45 step(s) of a {shape[0]}x{shape[1]}x{shape[2]} sample of the "
                      f"512x512x64 workload (same material, 3 nm cubes, vortex start, exact demag; numpy FP64), "
                      f"in each of {cores} processes at once ({tall:.1f} s); one process alone: {one:.3g} "
                      f"cell-steps/s ({t1:.1f} s)"}


def run_reference(args):
    """The FP64 CPU oracle on this host's cores, W warm-up and exactly K
    timed RK45 steps.  Each step is a bounded sample of the headline
    workload: one process per host core, each stepping its own copy of the
    largest sample grid (same material, cell size, integrator, exact demag)
    whose K + W steps fit in about REFERENCE_BUDGET_S seconds (cost per
    cell-step probed on 32x32x16, doubled for the shared memory system)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    w = W.vortex_512x512x64()
    per = _per_cell_step_probe()
    total = args.steps + args.warmup
    shape = _pick_sample(2.0 * per, total, REFERENCE_BUDGET_S)
    cores = _host_cores()
    val, el = _oracle_pool(shape, args.warmup, args.steps, cores)
    sample = (f"each step one RK45 step (dt 1e-14 s) of a {shape[0]}x{shape[1]}x{shape[2]} sample of the "
              f"workload (same material, 3 nm cubes, vortex start, exact demag; numpy FP64) in each of "
              f"{cores} processes at once, {args.steps} timed after {args.warmup} warm-up, {el:.1f} s")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "cells": w.grid.n, "grid": [w.grid.nx, w.grid.ny, w.grid.nz],
                   "cell_nm": [3, 3, 3], "integrator": "rk45-dopri5", "rtol": w.rtol,
                   "demag": f"exact-fft {2*shape[0]}x{2*shape[1]}x{2*shape[2]} (sample grid)",
                   "precision": "fp64-cpu-oracle", "parallelism": f"{cores} oracle processes (rank 0)",
                   "sample_grid": list(shape)},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu_model": _cpu_model()},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def aggregate_ranks(ms: float, cell_steps: float, ws: int, device: str):
    """Whole-job numbers of a replicas-only run: the slowest rank's time and
    the cell-steps of all ranks (one all-reduce each; no data-path
    collective exists)."""
    if ws <= 1:
        return ms, float(cell_steps)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(cell_steps)], dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return float(t.item()), float(c.item())


def _timed(stream, fn):
    """Device time (ms) of fn() on `stream`, synchronised on both sides."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _material(mm, w):
    return mm.Material(w.mat.Ms, w.mat.A, w.mat.alpha, w.mat.Ku1, w.mat.u, w.mat.D)


def _ctx(mm, stream, w, prec=32, dt=1e-14):
    g = w.grid
    cfg = mm.make_config(precision=prec, integrator=mm.MM_RK45, demag=mm.MM_DEMAG_EXACT, dt=dt, rtol=w.rtol)
    c = mm.mm_create(mm.make_grid(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), _material(mm, w).s, cfg)
    mm.mm_set_stream(c, stream.cuda_stream)
    if any(w.B_ext):
        mm.mm_set_field(c, 0, w.B_ext)
    return c


def fp32_vs_fp64(mm, stream, w, m0, n_steps=20, dt=2e-14):
    """The same n fixed RK45 steps from the same state in FP32 and in FP64:
    max|m_fp32 - m_fp64| and each precision's device throughput on those
    steps (the FP64 GPU path is held to the FP64 oracle within 1e-11 by the
    parity tests)."""
    g = w.grid
    out, rate = {}, {}
    for prec in (32, 64):
        c = _ctx(mm, stream, w, prec, dt)
        mm.mm_set_m(c, 0, m0)
        mm.mm_step_dt(c, np.full(3, dt))          # warm-up (graph capture, first slope)
        mm.mm_set_m(c, 0, m0)
        ms = _timed(stream, lambda: mm.mm_step_dt(c, np.full(n_steps, dt)))
        rate[prec] = g.n * n_steps / (ms * 1e-3)
        out[prec] = mm.mm_get_m(c, 0, m0.shape)
        mm.mm_destroy(c)
    return float(np.abs(out[32] - out[64]).max()), rate


def error_vs_oracle(mm, stream, shape=(64, 64, 16), n_steps=10):
    """Trajectory error against the FP64 oracle on a sample of the headline
    workload (same material, 3 nm cubes, vortex start): the oracle's own
    accepted RK45 steps, replayed by the GPU in FP32 and in FP64."""
    from oracle.demag import demag_spectrum
    from oracle.fields import Problem
    from oracle.llg import Solver
    w = _vortex_sample(shape)
    g = w.grid
    m0 = W.m_vortex(g, seed=w.seed)
    p = Problem.from_workload(g, w.mat)
    o = Solver(p, m0, K_hat=demag_spectrum(p.shape, p.d), dt=1e-14, rtol=w.rtol)
    dts = [o.rk45_step() for _ in range(n_steps)]
    out = {}
    for prec in (32, 64):
        c = _ctx(mm, stream, w, prec)
        mm.mm_set_m(c, 0, m0)
        mm.mm_step_dt(c, np.asarray(dts))
        out[f"fp{prec}_max_abs_dm"] = float(np.abs(mm.mm_get_m(c, 0, m0.shape) - o.m).max())
        mm.mm_destroy(c)
    out.update({"after_steps": n_steps, "t_sim_s": float(sum(dts)),
                "sample": f"{shape[0]}x{shape[1]}x{shape[2]} of the workload's material and cells, vortex start; "
                          "the oracle's accepted RK45 steps replayed", "bars": {"fp32": 1e-5, "fp64": 1e-11}})
    return out


def profile_kernels(mm, ctx, steps):
    """Per-kernel CUDA-event timing of `steps` more steps (graphs bypassed):
    {name: launches, share, avg_us, GB/s} and the dominant kernel's entry."""
    mm.mm_set_profiling(ctx, True)
    mm.mm_step(ctx, steps)
    prof = mm.mm_get_profile(ctx)
    mm.mm_set_profiling(ctx, False)
    tot = sum(p["total_ms"] for p in prof) or 1.0
    kernels = {p["name"]: {"launches": p["launches"], "share": round(p["total_ms"] / tot, 4),
                           "avg_us": round(1e3 * p["total_ms"] / max(1, p["launches"]), 2),
                           "GBps": round(p["bytes_per_launch"] / (p["total_ms"] / max(1, p["launches"]) * 1e-3) / 1e9, 1)
                           if p["bytes_per_launch"] > 0 else None}
               for p in sorted(prof, key=lambda p: -p["total_ms"])}
    return kernels, max(prof, key=lambda p: p["total_ms"])


def roofline_of(dom, workload):
    avg_ms = dom["total_ms"] / max(1, dom["launches"])
    achieved = dom["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    return {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1), "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": _traffic_for(dom["name"], workload), "algorithmic_bytes_per_launch": dom["bytes_per_launch"],
            "avg_launch_us": round(1e3 * avg_ms, 2)}


def variant_single(mm, stream, w, m0, steps, warmup=5):
    """A single-instance RK45 workload timed like the headline: K accepted
    steps on the library stream, per-kernel shares and the dominant kernel's
    roofline."""
    g = w.grid
    c = _ctx(mm, stream, w)
    mm.mm_set_m(c, 0, m0)
    mm.mm_step(c, warmup)
    s0 = mm.mm_get_stats(c)
    ms = _timed(stream, lambda: mm.mm_step(c, steps))
    s1 = mm.mm_get_stats(c)
    n = s1["accepted"] - s0["accepted"]
    kernels, dom = profile_kernels(mm, c, 2)
    mm.mm_destroy(c)
    return {"workload": w.name, "grid": [g.nx, g.ny, g.nz], "cells": g.n, "value": g.n * n / (ms * 1e-3),
            "unit": UNIT, "steps": n, "ms_per_step": ms / max(1, n), "kernel_launches_per_step":
            (s1["kernel_launches"] - s0["kernel_launches"]) / max(1, n),
            "roofline": roofline_of(dom, w.name), "kernels": kernels}


def variant_film_fp64(mm, stream):
    """The 128x32x1 permalloy film of 3.90625x3.90625x3 nm cells (FP64 RK45,
    rtol 1e-6, exchange + demag + Zeeman, field (-24.6, 4.3, 0) mT, seeded
    perturbed (1,1,1) start) over its whole 0.5 ns: a launch- and
    latency-bound case, reported as microseconds and kernel launches per
    accepted step (the attempts run as CUDA graphs of 8)."""
    w = W.film_128x32()
    g = w.grid
    m0 = W.m_uniform_perturbed(g, seed=w.seed)
    c = _ctx(mm, stream, w, prec=64)
    mm.mm_set_m(c, 0, m0)
    blob = mm.mm_get_state(c)
    mm.mm_run(c, 0.05e-9)                 # warm-up (first slope, graph capture)
    mm.mm_set_state(c, blob)
    mm.mm_step(c, 1)                      # graphs again after the restore
    s0 = mm.mm_get_stats(c)
    ms = _timed(stream, lambda: mm.mm_run(c, w.t_end))
    s1 = mm.mm_get_stats(c)
    n = s1["accepted"] - s0["accepted"]
    att = s1["attempts"] - s0["attempts"]
    mm.mm_destroy(c)
    return {"workload": w.name, "grid": [g.nx, g.ny, g.nz], "cells": g.n, "precision": "fp64",
            "t_sim_ns": w.t_end * 1e9, "accepted_steps": n, "attempts": att, "wall_ms": ms,
            "us_per_step": 1e3 * ms / max(1, n), "value": g.n * n / (ms * 1e-3), "unit": UNIT,
            "kernel_launches_per_step": (s1["kernel_launches"] - s0["kernel_launches"]) / max(1, n),
            "graph_launches_per_step": round(att / 8.0 / max(1, n), 3),
            "note": "timed from the second step to t_end (the first re-captures the graphs)"}


def variant_cufft(mm, stream, reps=5):
    """The same zero-padded demag convolution through cuFFT (torch.fft R2C /
    C2R on the library's stream) with the full tensor spectrum expanded from
    the library's stored half range, against the library's pruned passes on
    the headline grid and the 256x256x16 film: ms per evaluation and the
    largest difference of the fields relative to the largest field."""
    import torch
    out = []
    cases = ((W.vortex_512x512x64(), lambda g: W.m_vortex(g, seed=5)),
             (W.dmi_256x256x16(), lambda g: W.m_random_sphere(g, seed=2)))
    demag_kernels = ("fft_x_r2c", "fft_y_fwd", "fft_conv", "fft_y_inv", "fft_x_c2r")
    for w, mk in cases:
        g = w.grid
        m0 = mk(g)
        c = _ctx(mm, stream, w)
        mm.mm_set_m(c, 0, m0)
        mm.mm_get_heff(c, 0, m0.shape, 16)            # warm-up
        mm.mm_set_profiling(c, True)
        for _ in range(reps):
            H_ours = mm.mm_get_heff(c, 0, m0.shape, 16)
        prof = {p["name"]: p for p in mm.mm_get_profile(c)}
        mm.mm_set_profiling(c, False)
        ours_ms = sum(prof[k]["total_ms"] / prof[k]["launches"] for k in demag_kernels if k in prof)
        K, (Px, Py, Pz) = mm.mm_get_demag_kernel(c)
        m_dev = mm.mm_get_m(c, 0, m0.shape)
        mm.mm_destroy(c)
        dev = torch.device("cuda")
        with torch.cuda.stream(stream):
            Kt = torch.tensor(K, dtype=torch.float32, device=dev)          # [6][Pz/2+1][Py/2+1][Kx]
            ky = torch.arange(Py, device=dev)
            kz = torch.arange(Pz, device=dev)
            kyf = torch.where(ky <= Py // 2, ky, Py - ky)
            kzf = torch.where(kz <= Pz // 2, kz, Pz - kz)
            sy = torch.where(ky <= Py // 2, 1.0, -1.0).to(torch.float32)
            sz = torch.where(kz <= Pz // 2, 1.0, -1.0).to(torch.float32)
            Kf = Kt[:, kzf][:, :, kyf]                                      # [6][Pz][Py][Kx]
            syz = (sy[None, :, None] * sz[:, None, None])
            Kf[3] *= sy[None, :, None]
            Kf[4] *= sz[:, None, None]
            Kf[5] *= syz
            x = torch.tensor(w.mat.Ms * m_dev, dtype=torch.float32, device=dev)
            comp = ((0, 3, 4), (3, 1, 5), (4, 5, 2))

            def conv():
                M = torch.fft.rfftn(x, s=(Pz, Py, Px), dim=(1, 2, 3))
                Hh = torch.stack([Kf[a] * M[0] + Kf[b] * M[1] + Kf[d] * M[2] for a, b, d in comp])
                return torch.fft.irfftn(Hh, s=(Pz, Py, Px), dim=(1, 2, 3), norm="forward")[:, :g.nz, :g.ny, :g.nx]

            def ffts():
                M = torch.fft.rfftn(x, s=(Pz, Py, Px), dim=(1, 2, 3))
                return torch.fft.irfftn(M, s=(Pz, Py, Px), dim=(1, 2, 3), norm="forward")

            H_cu = conv()
            ffts()
            t_all = _timed(stream, lambda: [conv() for _ in range(reps)]) / reps
            t_fft = _timed(stream, lambda: [ffts() for _ in range(reps)]) / reps
            Hc = H_cu.double().cpu().numpy()
        del Kt, Kf, x, H_cu
        torch.cuda.empty_cache()
        out.append({"workload": w.name, "grid": [g.nx, g.ny, g.nz], "padded": [Px, Py, Pz],
                    "ours_ms_per_eval": round(ours_ms, 4), "cufft_ms_per_eval": round(t_all, 4),
                    "cufft_ffts_only_ms": round(t_fft, 4), "speedup_vs_cufft": round(t_all / ours_ms, 3),
                    "max_rel_diff": float(np.abs(H_ours - Hc).max() / np.abs(Hc).max())})
    return {"what": "ours: sum of the five demag kernels' CUDA-event times per evaluation (profiling pass); "
                    "cuFFT: rfftn of 3 padded components + tensor multiply (torch elementwise) + irfftn, "
                    "CUDA events, FP32", "cases": out}


def variant_drift(mm, stream, steps=200, every=20, dt=2e-14):
    """FP32 against FP64 on the 256x256x16 DMI film from its random state:
    the same fixed RK45 steps replayed in both precisions, max|m32 - m64|
    after every `every` steps up to `steps`."""
    w = W.dmi_256x256x16()
    m0 = W.m_random_sphere(w.grid, seed=w.seed)
    ctx = {p: _ctx(mm, stream, w, p, dt) for p in (32, 64)}
    curve = []
    try:
        for p in (32, 64):
            mm.mm_set_m(ctx[p], 0, m0)
        done = 0
        while done < steps:
            for p in (32, 64):
                mm.mm_step_dt(ctx[p], np.full(every, dt))
            done += every
            d = np.abs(mm.mm_get_m(ctx[32], 0, m0.shape) - mm.mm_get_m(ctx[64], 0, m0.shape)).max()
            curve.append([done, float(d)])
    finally:
        for c in ctx.values():
            mm.mm_destroy(c)
    return {"workload": w.name, "dt_s": dt, "max_abs_dm_fp32_vs_fp64": curve,
            "note": "fixed RK45 steps replayed in both precisions from the same seeded random state"}


def variant_cnn(mm, reps=5):
    """The surrogate network on the tensor cores: the forward pass on the
    512x512 film and one training step's backward pass (batch of 16 128x128
    windows), per kernel from the library's CUDA-event profile, with
    throughput on the network's algorithmic FLOPs (real channels:
    2 x 25 x (3*32 + 32*32 + 32*32 + 32*3) per pixel per contraction)
    against the measured BF16 peak."""
    w = W.skyrmion_512()
    g = w.grid
    M = mm.Material(w.mat.Ms, w.mat.A, w.mat.alpha, w.mat.Ku1, w.mat.u, w.mat.D)
    c = mm.mm_create(mm.make_grid(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), M.s,
                     mm.make_config(precision=32, integrator=mm.MM_RK45, demag=mm.MM_DEMAG_EXACT, dt=1e-13))
    per_px = 2.0 * 25 * (3 * 32 + 32 * 32 + 32 * 32 + 32 * 3)
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        peak = 1900.0
    try:
        rng = np.random.default_rng(4)
        mm.mm_surrogate_weights(c, rng.normal(0.0, 0.05, mm.SURROGATE_NPARAMS), c_in=1.0)
        x = rng.normal(size=(1, 3, g.ny, g.nx))
        mm.mm_surrogate_forward(c, x)
        mm.mm_set_profiling(c, True)
        for _ in range(reps):
            mm.mm_surrogate_forward(c, x)
        fwd = [p for p in mm.mm_get_profile(c) if p["name"].startswith("cnn_conv")]
        mm.mm_set_profiling(c, False)
        xb = rng.normal(size=(16, 3, 128, 128))
        tb = rng.normal(size=(16, 3, 128, 128))
        mm.mm_surrogate_grad(c, xb, tb)
        mm.mm_set_profiling(c, True)
        for _ in range(reps):
            mm.mm_surrogate_grad(c, xb, tb)
        bwd = [p for p in mm.mm_get_profile(c) if p["name"] in ("cnn_dweight", "cnn_dgrad")]
        mm.mm_set_profiling(c, False)
    finally:
        mm.mm_destroy(c)
    fwd_us = 1e3 * sum(p["total_ms"] for p in fwd) / reps
    tf = per_px * g.nx * g.ny / (fwd_us * 1e-6) / 1e12
    bw = {p["name"]: {"per_step_us": round(1e3 * p["total_ms"] / reps, 2),
                      "per_launch_us": round(1e3 * p["total_ms"] / p["launches"], 2)} for p in bwd}
    dw_us = bw.get("cnn_dweight", {}).get("per_step_us")
    out = {"forward": {"grid": [g.nx, g.ny], "us": round(fwd_us, 2),
                       "layers_us": {p["name"]: round(1e3 * p["total_ms"] / p["launches"], 2) for p in fwd},
                       "algorithmic_gflop": round(per_px * g.nx * g.ny / 1e9, 3), "tflops": round(tf, 1),
                       "frac_of_bf16_peak": round(tf / peak, 4)},
           "backward": {"batch": [16, 128, 128], "kernels": bw},
           "bf16_peak_tflops": peak}
    if dw_us:
        # weight gradients of all four layers: the same FLOPs as one forward pass
        tfw = per_px * 16 * 128 * 128 / (dw_us * 1e-6) / 1e12
        out["backward"]["weight_grad_tflops"] = round(tfw, 1)
        out["backward"]["weight_grad_frac_of_bf16_peak"] = round(tfw / peak, 4)
    return out


def variant_peaks(mm):
    """Measured FMA throughput (FP32, FP64) of this GPU, the denominators of
    the ALU-bound lines."""
    f32 = max(mm.mm_measure_peak(32) for _ in range(3))
    f64 = max(mm.mm_measure_peak(64) for _ in range(3))
    return {"fp32_tflops": round(f32 / 1e12, 2), "fp64_tflops": round(f64 / 1e12, 3),
            "how": "grid of 8 independent FMA chains per thread (8 CTAs of 256 per SM), CUDA events"}


def variant_batched(mm, stream, steps):
    """1024 finite-temperature replicas of uneven sizes, FP32 Heun, one
    persistent launch per stage, graph-captured, autotuned launch shape."""
    import torch
    R = 1024
    sizes = W.replica_sizes(R, seed=3)
    J = W.replica_currents(R)
    mat = W.Material(Ms=1.1e6, A=2e-11, alpha=0.01, Ku1=9e5, u=(0.0, 0.0, 1.0))
    M = mm.Material(mat.Ms, mat.A, mat.alpha, mat.Ku1, mat.u, mat.D)
    grids = [mm.make_grid(n, n, 1, 2e-9, 2e-9, 1e-9) for n in sizes]
    base_seed = 3
    cfg = mm.make_config(precision=32, integrator=mm.MM_HEUN, demag=mm.MM_DEMAG_EXACT, dt=1e-14, T=300.0,
                         seed=base_seed)
    ctx = mm.mm_create_batch(grids, M.s, cfg, None)
    mm.mm_set_stream(ctx, stream.cuda_stream)
    tq = mm.make_torque(mm.MM_TORQUE_SOT, p=(0, 1, 0), theta_SH=0.1)
    mm.mm_set_torque(ctx, tq, J)
    m0 = []
    for r, n in enumerate(sizes):
        m = W.m_perp(W.Grid(n, n, 1, 2e-9, 2e-9, 1e-9), seed=1000 + r, tilt=0.05)
        mm.mm_set_m(ctx, r, m)
        m0.append(m)
    t_tune = time.perf_counter()
    nt, blocks = mm.mm_batch_autotune(ctx, None)
    t_tune = time.perf_counter() - t_tune
    mm.mm_step(ctx, 3)
    s0 = mm.mm_get_stats(ctx)
    ms = _timed(stream, lambda: mm.mm_step(ctx, steps))
    s1 = mm.mm_get_stats(ctx)
    n_acc = s1["accepted"] - s0["accepted"]
    cells = int(sum(n * n for n in sizes))
    # FP32 batch vs FP64 single-instance runs of three replicas (same Philox key,
    # same current) over the 3 + steps steps the batch has taken
    n_total = 3 + steps
    checks = sorted({0, int(np.argmin(sizes)), int(np.argmax(sizes))})
    errs = []
    for r in checks:
        n = sizes[r]
        c64 = mm.make_config(precision=64, integrator=mm.MM_HEUN, demag=mm.MM_DEMAG_EXACT, dt=1e-14, T=300.0,
                             seed=base_seed + r)
        s = mm.mm_create(mm.make_grid(n, n, 1, 2e-9, 2e-9, 1e-9), M.s, c64)
        mm.mm_set_m(s, 0, m0[r])
        mm.mm_set_torque(s, tq, J[r:r + 1])
        mm.mm_step(s, n_total)
        shape = m0[r].shape
        errs.append(float(np.abs(mm.mm_get_m(ctx, r, shape) - mm.mm_get_m(s, 0, shape)).max()))
        mm.mm_destroy(s)
    # the smallest replica against the FP64 oracle over the same steps (same
    # Philox key and current; the oracle steps it alone)
    from oracle.fields import Problem
    from oracle.llg import Solver, Torque, replica_seed
    r = int(np.argmin(sizes))
    n = sizes[r]
    o = Solver(Problem.from_workload(W.Grid(n, n, 1, 2e-9, 2e-9, 1e-9), mat), m0[r],
               terms=("exchange", "anisotropy", "zeeman", "demag"), T=300.0, seed=replica_seed(base_seed, r),
               dt=1e-14, torque=Torque(kind="sot", J=J[r], p=(0, 1, 0), theta_SH=0.1))
    for _ in range(n_total):
        o.heun_step()
    err_oracle = float(np.abs(mm.mm_get_m(ctx, r, m0[r].shape) - o.m).max())
    mm.mm_destroy(ctx)
    torch.cuda.synchronize()
    return {"workload": "1024 perpendicular free layers, sizes {32,48,64,96,128}^2 x 1 of 2x2x1 nm, T=300 K, "
                        "damping-like SOT J in [1e11,3e11] A/m^2, exact demag, FP32 Heun dt=1e-14 s",
            "value": cells * n_acc / (ms * 1e-3), "unit": UNIT, "cells": cells, "replicas": R,
            "steps": n_acc, "ms_per_step": ms / max(1, n_acc),
            "launch_shape": {"threads": nt, "ctas": blocks, "stacked": nt == 0},
            "autotune_s": round(t_tune, 2),
            "error_vs_fp64": {"max_abs_dm": max(errs), "after_steps": n_total, "replicas_checked": checks,
                              "against": "FP64 single-instance GPU runs with the same Philox key"},
            "error_vs_oracle": {"max_abs_dm": err_oracle, "after_steps": n_total, "replica": r, "size": n,
                                "against": "the FP64 CPU oracle stepping that replica alone (same key, current)"}}


def variant_trials_films(mm, stream, steps=200, R=512, n=64, n_trials=16384):
    """Retire/refill over thermal switching trials of 64x64 films with exact
    demag (Results, "Replica batching"): 512 slots, 16384 trials with their
    own current and Philox key, FP32 Depondt-Mertens, stop test after every
    step; the same run timed on the persistent launch shape and on the
    stacked shape."""
    mat = W.Material(Ms=1.1e6, A=2e-11, alpha=0.02, Ku1=9e5, u=(0.0, 0.0, 1.0))
    M = mm.Material(mat.Ms, mat.A, mat.alpha, mat.Ku1, mat.u, mat.D)
    g = mm.make_grid(n, n, 1, 2e-9, 2e-9, 1e-9)
    J = np.linspace(2e11, 2e12, n_trials)
    m_init = np.zeros((3, 1, n, n))
    m_init[2] = 1.0
    out = {"workload": f"{R} slots of {n}x{n}x1 films of 2x2x1 nm, {n_trials} trials (STT J in [2e11, 2e12] A/m^2, "
                       "300 K), exact demag, FP32 Depondt-Mertens dt=1e-13 s, retire at m_z <= 0",
           "unit": "cell-steps/s", "steps": steps}
    for shape in ("persistent", "stacked"):
        cfg = mm.make_config(precision=32, integrator=mm.MM_DM, demag=mm.MM_DEMAG_EXACT, dt=1e-13, T=0.0,
                             terms=1 | 4 | 8 | 16 | 32)
        ctx = mm.mm_create_batch([g] * R, M.s, cfg, None)
        try:
            mm.mm_set_stream(ctx, stream.cuda_stream)
            mm.mm_set_torque(ctx, mm.make_torque(mm.MM_TORQUE_STT, p=(0, 0, -1), P=0.6, Lambda=1.0), np.zeros(R))
            if shape == "stacked":
                mm.mm_batch_set_shape(ctx, 0)
            else:
                mm.mm_batch_set_shape(ctx, 256, min(R, 304))
            mm.mm_trials_start(ctx, J, np.full(n_trials, 300.0), m_init, axis=(0, 0, 1), threshold=0.0,
                               max_steps=4000, base_seed=5, refill=True)
            mm.mm_step(ctx, 5)
            ms = _timed(stream, lambda: mm.mm_step(ctx, steps))
            done = mm.mm_trials_result(ctx)[2]
        finally:
            mm.mm_destroy(ctx)
        out[shape] = {"ms_per_step": ms / steps, "value": R * n * n * steps / (ms * 1e-3), "trials_done": int(done)}
    out["stacked_over_persistent"] = out["persistent"]["ms_per_step"] / out["stacked"]["ms_per_step"]
    return out


# The paper's replica-batching table (Results, "Replica batching"): physics,
# replica grid, replica count R, and its published throughput (on its own
# hardware, an RTX 5060 Ti).  Materials are not printed there; the
# perpendicular Co-like film used here is stated in the output.
BATCH_TABLE = [
    ("macrospin: anisotropy + STT + thermal", (1, 1), 1024, 4 | 8 | 32, False, "replica-steps/s", 3.7e7),
    ("8x8x1: exchange + uniaxial + Zeeman", (8, 8), 256, 1 | 4 | 8, False, "cell-steps/s", 1.4e8),
    ("16x16x1: exchange + uniaxial + Zeeman + demag", (16, 16), 256, 1 | 4 | 8 | 16, True, "cell-steps/s", 8.9e7),
]


def variant_batching_table(mm, stream, steps=2048):
    """The three rows of the paper's batching table with the
    Depondt-Mertens engine: FP32, 4 nm cells, Ms 1e6, A 1.5e-11, alpha 0.05,
    Ku 1.1e6 along z, Bz 50 mT, STT (p = z, P 0.6) at 1e12 A/m^2 and 300 K
    on the macrospin row."""
    out = []
    M = mm.Material(1.0e6, 1.5e-11, 0.05, 1.1e6, (0.0, 0.0, 1.0), 0.0)
    for name, (nx, ny), R, terms, demag, unit, paper in BATCH_TABLE:
        cfg = mm.make_config(precision=32, integrator=mm.MM_DM,
                             demag=mm.MM_DEMAG_EXACT if demag else mm.MM_DEMAG_OFF, dt=1e-13, terms=terms)
        grids = [mm.make_grid(nx, ny, 1, 4e-9, 4e-9, 4e-9)] * R
        ctx = mm.mm_create_batch(grids, M.s, cfg, None)
        mm.mm_set_stream(ctx, stream.cuda_stream)
        mm.mm_set_field(ctx, 0, (0.0, 0.0, 0.05))
        if terms & 32:
            mm.mm_set_temperature(ctx, np.full(R, 300.0))
            mm.mm_set_torque(ctx, mm.make_torque(mm.MM_TORQUE_STT, p=(0, 0, 1), P=0.6, Lambda=1.0),
                             np.full(R, 1e12))
        for r in range(R):
            mm.mm_set_m(ctx, r, W.m_perp(W.Grid(nx, ny, 1, 4e-9, 4e-9, 4e-9), seed=r, tilt=0.1))
        shape = mm.mm_batch_autotune(ctx, None) if demag else None
        mm.mm_step(ctx, 64)
        ms = _timed(stream, lambda: mm.mm_step(ctx, steps))
        per = R * (nx * ny if unit == "cell-steps/s" else 1)
        value = per * steps / (ms * 1e-3)
        st = mm.mm_get_stats(ctx)
        out.append({"row": name, "grid": [nx, ny, 1], "R": R, "value": value, "unit": unit,
                    "paper_value": paper, "ratio_vs_paper": value / paper, "steps": steps,
                    "ms_per_step": ms / steps, "kernel_launches_total": st["kernel_launches"],
                    "launch_shape": None if shape is None else {"threads": shape[0], "ctas": shape[1],
                                                                "stacked": shape[0] == 0}})
        mm.mm_destroy(ctx)
    return {"integrator": "Depondt-Mertens (MM_DM), FP32", "rows": out,
            "paper_hardware": "RTX 5060 Ti (the paper's); this run: one GB300"}


# The paper's thermally assisted STT switching sweep (Results, "Replica
# batching"): a Pt/Co-like macrospin with a 10 nm cell, thermal stability
# Delta = K V / kB T = 121 at 300 K and T = 0 threshold Jc0 = 2.60e12 A/m^2;
# 25 currents x 400 trials = 10,000 replicas, 20,000 steps.  Ms and alpha are
# not printed: Ms = 1e6 A/m and alpha = 0.0513 give that Delta and, with
# P = 0.6, Lambda = 1 (epsilon = 0.3) and t_F = 10 nm, that Jc0
# (Jc0 = alpha H_K e mu0 Ms t_F / (hbar epsilon), H_K = 2 K / (mu0 Ms)).
def variant_stt_sweep(mm, stream, steps=20000, n_points=25, trials=400, dt=1e-12):
    import torch
    kB, T = 1.380649e-23, 300.0
    d = 10e-9
    V = d ** 3
    Ms, alpha = 1.0e6, 0.0513
    K = 121.0 * kB * T / V
    mu0, e, hbar = 4e-7 * np.pi, 1.602176634e-19, 1.054571817e-34
    HK = 2 * K / (mu0 * Ms)
    eps = 0.3
    Jc0 = alpha * HK * e * mu0 * Ms * d / (hbar * eps)
    ratios = np.linspace(0.6, 1.2, n_points)
    J = np.repeat(ratios * Jc0, trials)
    R = J.size
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    M = mm.Material(Ms, 1e-11, alpha, K, (0.0, 0.0, 1.0), 0.0)
    cfg = mm.make_config(precision=32, integrator=mm.MM_DM, demag=mm.MM_DEMAG_OFF, dt=dt, terms=4 | 8 | 32)
    ctx = mm.mm_create_batch([mm.make_grid(1, 1, 1, d, d, d)] * R, M.s, cfg, None)
    mm.mm_set_stream(ctx, stream.cuda_stream)
    mm.mm_set_torque(ctx, mm.make_torque(mm.MM_TORQUE_STT, p=(0, 0, 1), P=0.6, Lambda=1.0, t_F=d), np.zeros(R))
    m0 = np.array([0.0, 0.0, -1.0]).reshape(3, 1, 1, 1)
    mm.mm_trials_start(ctx, J, np.full(R, T), m0, axis=(0, 0, -1), threshold=0.0, max_steps=steps, base_seed=17,
                       refill=False)
    t_setup = time.perf_counter() - t0
    ms = _timed(stream, lambda: mm.mm_step(ctx, steps))
    st, sw, done = mm.mm_trials_result(ctx)
    mm.mm_destroy(ctx)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    p_sw = sw.reshape(n_points, trials).mean(axis=1)
    k = int(np.argmax(p_sw >= 0.5)) if (p_sw >= 0.5).any() else -1
    return {"workload": f"{R} Pt/Co-like macrospin trials ({n_points} currents x {trials}), {steps} steps of "
                        f"{dt * 1e12:.1f} ps, 300 K, FP32 Depondt-Mertens, retire at m_z >= 0",
            "wall_s_end_to_end": wall, "setup_s": t_setup, "stepping_ms": ms,
            "replica_steps_per_s_upper": R * steps / (ms * 1e-3),
            "replica_steps_taken": int(st[st > 0].sum()),
            "paper_wall_s": 0.6, "paper_naive_loop_wall_s": 2.5 * 3600,
            "trials_done": done, "Jc0": Jc0, "J_over_Jc0": [round(float(x), 4) for x in ratios],
            "P_sw": [round(float(x), 4) for x in p_sw],
            "J_over_Jc0_at_P_half": float(ratios[k]) if k >= 0 else None,
            "paper_J_over_Jc0_at_P_half": 0.97}


# The muMAG standard problem 4 (Results, "Validation against the muMAG
# standard problems"): a 500 x 125 x 3 nm permalloy strip (128 x 32 x 1 cells,
# Ms 8e5, A 1.3e-11, alpha 0.02) switched by field A, mu0 H = (-24.6, 4.3, 0) mT,
# from the s-state.  Reading of the s-state protocol (the paper cites it, does
# not restate it): relax from the uniform [1, 1, 1] state in zero field with
# alpha = 1 for 5 ns.  The paper reports <m_x>(1 ns) = -0.980 for its code
# against the muMAG reference -0.986, and a switching time of ~175 ps.
def variant_sp4(mm, stream, relax_ns=5.0, t_end=1e-9, sample_ps=5.0):
    g = W.film_128x32().grid
    out = {"geometry": "128x32x1 cells of 3.90625x3.90625x3 nm (500x125x3 nm), RK45 rtol 1e-6",
           "s_state": f"uniform [1,1,1] relaxed {relax_ns} ns in zero field with alpha = 1",
           "paper_mx_1ns": -0.980, "mumag_reference_mx_1ns": -0.986, "paper_t_switch_ps": 175.0}
    G = mm.make_grid(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz)
    traj = {}
    for prec in (64, 32):
        Mr = mm.Material(8.0e5, 1.3e-11, 1.0)
        cr = mm.mm_create(G, Mr.s, mm.make_config(precision=prec, integrator=mm.MM_RK45, demag=mm.MM_DEMAG_EXACT,
                                                  dt=1e-13, rtol=1e-6))
        mm.mm_set_stream(cr, stream.cuda_stream)
        m0 = np.zeros((3,) + g.shape)
        m0[:] = (1 / np.sqrt(3.0))
        mm.mm_set_m(cr, 0, m0)
        mm.mm_run(cr, relax_ns * 1e-9)
        ms = mm.mm_get_m(cr, 0, m0.shape)
        mm.mm_destroy(cr)
        Md = mm.Material(8.0e5, 1.3e-11, 0.02)
        cd = mm.mm_create(G, Md.s, mm.make_config(precision=prec, integrator=mm.MM_RK45, demag=mm.MM_DEMAG_EXACT,
                                                  dt=1e-13, rtol=1e-6))
        mm.mm_set_stream(cd, stream.cuda_stream)
        mm.mm_set_m(cd, 0, ms)
        mm.mm_set_field(cd, 0, (-24.6e-3, 4.3e-3, 0.0))
        ts, mx = [0.0], [float(ms[0].mean())]
        t0 = time.perf_counter()
        n = int(round(t_end / (sample_ps * 1e-12)))
        for k in range(1, n + 1):
            mm.mm_run(cd, k * sample_ps * 1e-12)
            ts.append(k * sample_ps)
            mx.append(float(mm.mm_get_m(cd, 0, m0.shape)[0].mean()))
        wall = time.perf_counter() - t0
        st = mm.mm_get_stats(cd)
        mm.mm_destroy(cd)
        tsw = next((ts[i - 1] + (ts[i] - ts[i - 1]) * mx[i - 1] / (mx[i - 1] - mx[i])
                    for i in range(1, len(mx)) if mx[i - 1] > 0 >= mx[i]), None)
        traj[prec] = np.array(mx)
        out[f"fp{prec}"] = {"s_state_mx": float(ms[0].mean()), "s_state_my": float(ms[1].mean()),
                            "mx_1ns": mx[-1], "t_switch_ps": tsw, "accepted_steps": st["accepted"],
                            "rejected_steps": st["rejected"], "wall_s": round(wall, 2)}
    out["max_abs_mx_diff_fp32_vs_fp64_pp"] = float(100 * np.abs(traj[32] - traj[64]).max())
    return out


# The paper's throughput scenarios (ms per field evaluation, FP32) and its
# published numbers on its own hardware (an RTX 5060 Ti): this code's cuFFT
# build and the best solver of its comparison.  Grid shapes are not printed
# there beyond the cell counts; the ones used here are stated per scenario.
PAPER_SCENARIOS = [
    ("SP#4-like 2-D film, T = 0", (200, 50, 1), (2.5e-9, 2.5e-9, 3e-9), 0.042, 0.042),
    ("power-of-two 3-D", (64, 64, 16), (3e-9, 3e-9, 3e-9), 0.155, 0.155),
    ("medium 3-D", (150, 150, 24), (3e-9, 3e-9, 3e-9), 2.610, 1.663),
    ("large 3-D", (250, 250, 40), (3e-9, 3e-9, 3e-9), 12.72, 11.13),
]


def variant_scenarios(mm, stream, steps=60):
    """ms per field evaluation on the paper's four throughput scenarios:
    permalloy (Ms 8e5, A 1.3e-11, alpha 0.02), exchange + exact demag,
    FP32 RK45 (six evaluations per step) from a seeded perturbed state."""
    out = []
    M = mm.Material(8.0e5, 1.3e-11, 0.02)
    for name, (nx, ny, nz), (dx, dy, dz), paper_cs, paper_best in PAPER_SCENARIOS:
        g = W.Grid(nx, ny, nz, dx, dy, dz)
        cfg = mm.make_config(precision=32, integrator=mm.MM_RK45, demag=mm.MM_DEMAG_EXACT, dt=1e-14, rtol=1e-6)
        ctx = mm.mm_create(mm.make_grid(nx, ny, nz, dx, dy, dz), M.s, cfg)
        mm.mm_set_stream(ctx, stream.cuda_stream)
        mm.mm_set_m(ctx, 0, W.m_uniform_perturbed(g, seed=1))
        mm.mm_step(ctx, 10)
        s0 = mm.mm_get_stats(ctx)
        ms = _timed(stream, lambda: mm.mm_step(ctx, steps))
        s1 = mm.mm_get_stats(ctx)
        attempts = max(1, s1["attempts"] - s0["attempts"])
        per_eval = ms / (6 * attempts)
        out.append({"scenario": name, "grid": [nx, ny, nz], "cell_nm": [dx * 1e9, dy * 1e9, dz * 1e9],
                    "cells": g.n, "ms_per_field_eval": round(per_eval, 5),
                    "paper_ms_per_field_eval": {"this_code_cufft": paper_cs, "best_in_paper": paper_best,
                                                "hardware": "RTX 5060 Ti"},
                    "attempts": attempts})
        mm.mm_destroy(ctx)
    return {"metric": "ms per field evaluation (RK45: 6 per attempted step)", "scenarios": out}


def variant_surrogate(mm, stream, steps, train_steps=1500):
    """512x512x1 skyrmion-lattice film, FP32 RK45: exact FFT demag against the
    BF16 CNN surrogate refreshed exactly every k attempted steps."""
    import torch
    w = W.skyrmion_512()
    g = w.grid
    M = mm.Material(w.mat.Ms, w.mat.A, w.mat.alpha, w.mat.Ku1, w.mat.u, w.mat.D)
    cfg = mm.make_config(precision=32, integrator=mm.MM_RK45, demag=mm.MM_DEMAG_EXACT, dt=1e-13, rtol=w.rtol)
    ctx = mm.mm_create(mm.make_grid(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), M.s, cfg)
    mm.mm_set_stream(ctx, stream.cuda_stream)
    mm.mm_set_field(ctx, 0, w.B_ext)
    m0 = W.m_skyrmion_lattice(g, seed=w.seed, spacing=40e-9, radius=8e-9)
    mm.mm_set_m(ctx, 0, m0)
    mm.mm_step(ctx, 30)                          # leave the initial transient
    tcfg = mm.make_train_cfg(n_snapshots=24, snap_every=4, max_gap=6, crop=128, batch=16, steps=train_steps,
                             lr=1e-3, seed=4)
    t_train = time.perf_counter()
    loss = mm.mm_surrogate_train(ctx, tcfg)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_train
    blob = mm.mm_get_state(ctx)
    t0 = mm.mm_get_time(ctx)[0]

    def run(k, tol):
        mm.mm_set_state(ctx, blob)
        mm.mm_surrogate_set(ctx, k, tol)
        s0 = mm.mm_get_stats(ctx)
        ms = _timed(stream, lambda: mm.mm_step(ctx, steps))
        s1 = mm.mm_get_stats(ctx)
        n_acc = s1["accepted"] - s0["accepted"]
        t1 = mm.mm_get_time(ctx)[0]
        st = mm.mm_surrogate_get_stats(ctx) if k else None
        m1 = mm.mm_get_m(ctx, 0, m0.shape)
        mm.mm_surrogate_set(ctx, 0, tol)
        return {"value": g.n * n_acc / (ms * 1e-3), "steps": n_acc, "ms_per_step": ms / max(1, n_acc),
                "t_sim": t1 - t0, "stats": st, "m": m1}

    exact = run(0, 1e-3)
    # exact reference at each surrogate run's end time (RK45 step sizes differ)
    out = {"workload": "512x512x1 skyrmion-lattice film of 2x2x1 nm, Ms 5.8e5, A 1.5e-11, Ku 8e5, D 3.5e-3, "
                       "alpha 0.3, Bz 0.2 T, FP32 RK45 rtol 1e-6",
           "exact": {k: v for k, v in exact.items() if k not in ("m", "stats")},
           "train": {"pairs_from_snapshots": 24, "optimiser_steps": train_steps, "final_loss": loss,
                     "seconds": round(t_train, 2)}, "tol": 1e-3, "k": {}}
    for k in (5, 10, 20):
        r = run(k, 1e-3)
        mm.mm_set_state(ctx, blob)
        mm.mm_run(ctx, t0 + r["t_sim"])
        m_ref = mm.mm_get_m(ctx, 0, m0.shape)
        st = r["stats"]
        out["k"][str(k)] = {"value": r["value"], "speedup_vs_exact": r["value"] / exact["value"],
                            "steps": r["steps"], "ms_per_step": r["ms_per_step"],
                            "max_abs_dm_vs_exact_run": float(np.abs(r["m"] - m_ref).max()),
                            "fallback": bool(st["fallback"]), "field_error_last": st["last_error"],
                            "field_error_max": st["max_error"], "exact_evals": st["exact_evals"],
                            "surrogate_evals": st["surrogate_evals"]}
    out["unit"] = UNIT
    mm.mm_destroy(ctx)
    torch.cuda.synchronize()
    return out


def run_gpu(args):
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    import paper_2608_15253_gb300 as mm
    if not os.path.exists(mm.lib_path):
        from paper_2608_15253_gb300 import build as B
        B.build()
    w = W.vortex_512x512x64()
    if args.grid:
        w = _vortex_sample(tuple(int(v) for v in args.grid.split(",")))
        from dataclasses import replace
        w = replace(w, name=f"vortex_{w.grid.nx}x{w.grid.ny}x{w.grid.nz}_rk45")
    g = w.grid
    stream = torch.cuda.current_stream()
    ctx = _ctx(mm, stream, w)
    m0 = W.m_vortex(g, seed=w.seed + rank)
    mm.mm_set_m(ctx, 0, m0)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    mm.mm_step(ctx, args.warmup)
    torch.cuda.synchronize()
    s0 = mm.mm_get_stats(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        mm.mm_step(ctx, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1)
    s1 = mm.mm_get_stats(ctx)
    steps = s1["accepted"] - s0["accepted"]
    attempts = s1["attempts"] - s0["attempts"]
    launches = s1["kernel_launches"] - s0["kernel_launches"]
    t_max, total_cells_steps = aggregate_ranks(ms, g.n * steps, ws, "cuda")
    value = total_cells_steps / (t_max * 1e-3)

    # per-kernel CUDA-event timing of the same kind of steps (graphs bypassed)
    kernels, dom = profile_kernels(mm, ctx, max(2, min(args.steps, 3)))

    # end to end through the C ABI with host buffers: every step uploads the
    # state (float64, 3N) from page-locked host memory and reads the new
    # state back into it
    k_e2e = max(1, min(args.steps, 10))
    pinned = torch.empty(m0.size, dtype=torch.float64, pin_memory=True)
    mh = pinned.numpy().reshape(m0.shape)
    mm.mm_get_m(ctx, 0, m0.shape, out=mh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        mm.mm_set_m(ctx, 0, mh)
        mm.mm_step(ctx, 1)
        mm.mm_get_m(ctx, 0, m0.shape, out=mh)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = g.n * k_e2e / e2e_s * ws
    mm.mm_destroy(ctx)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / max(1, steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "cells": g.n, "grid": [g.nx, g.ny, g.nz], "cell_nm": [3, 3, 3],
                   "integrator": "rk45-dopri5", "rtol": w.rtol,
                   "demag": f"exact-fft {2*g.nx}x{2*g.ny}x{2*g.nz} (pruned passes, FP64 Newell setup)",
                   "precision": "fp32 (fp64 Newell setup and reductions)", "parallelism": f"replicas x{ws}",
                   "accepted_steps": steps, "attempts": attempts,
                   "l2": "inputs larger than L2: working set ~3 GB (state, 7 slopes, spectrum, tensor) > 126 MB"},
        "gpu_launches": launches,
        "roofline": roofline_of(dom, w.name),
        "kernels": kernels,
        "clocks": clk.summary(),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 3 * g.n * 8,
                "d2h_bytes_per_step": 3 * g.n * 8, "steps": k_e2e,
                "host_buffers": "page-locked float64 [3][z][y][x]"},
    }
    if not args.no_variants and rank == 0:
        try:
            line["error_vs_oracle"] = error_vs_oracle(mm, stream)
        except Exception as e:
            line["error_vs_oracle"] = {"error": f"{type(e).__name__}: {e}"}
        err, rate = fp32_vs_fp64(mm, stream, w, W.m_vortex(g, seed=w.seed), n_steps=5)
        line["fp64"] = {"value": rate[64], "unit": UNIT, "fp32_same_steps": rate[32],
                        "max_abs_dm_fp32_vs_fp64": err,
                        "note": "the headline grid, 5 replayed RK45 steps of dt 2e-14 s from the same state, "
                                "all-FP64 GPU run against the FP32 one"}
        line["variants"] = {}
        wanted = [v for v in args.variants.split(",") if v]
        dmi = W.dmi_256x256x16()
        for name, fn in (("peaks", lambda: variant_peaks(mm)),
                         ("dmi_256x256x16", lambda: variant_single(mm, stream, dmi, W.m_random_sphere(dmi.grid, 2),
                                                                   args.steps)),
                         ("film_128x32_fp64", lambda: variant_film_fp64(mm, stream)),
                         ("drift", lambda: variant_drift(mm, stream)),
                         ("cnn", lambda: variant_cnn(mm)),
                         ("trials_films", lambda: variant_trials_films(mm, stream)),
                         ("cufft", lambda: variant_cufft(mm, stream)),
                         ("batched", lambda: variant_batched(mm, stream, args.batch_steps)),
                         ("surrogate", lambda: variant_surrogate(mm, stream, args.surrogate_steps)),
                         ("paper_scenarios", lambda: variant_scenarios(mm, stream)),
                         ("batching_table", lambda: variant_batching_table(mm, stream)),
                         ("stt_sweep", lambda: variant_stt_sweep(mm, stream)),
                         ("sp4", lambda: variant_sp4(mm, stream))):
            if name not in wanted:
                continue
            try:
                line["variants"][name] = fn()
            except Exception as e:  # a failed variant is reported, the headline line still prints
                line["variants"][name] = {"error": f"{type(e).__name__}: {e}"}
        pk = line["variants"].get("peaks", {})
        if "fp64_tflops" in pk:
            line["fp64"]["fp64_peak_tflops"] = pk["fp64_tflops"]
    if rank == 0:
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", default="", help="nx,ny,nz: a smaller case of the same workload (profiling)")
    ap.add_argument("--no-variants", action="store_true", help="skip the error, FP64 and variant lines")
    ap.add_argument("--variants", default="peaks,dmi_256x256x16,film_128x32_fp64,drift,cufft,cnn,batched,trials_films,"
                                          "surrogate,"
                                          "paper_scenarios,batching_table,stt_sweep,sp4",
                    help="comma list of variant lines to run")
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--surrogate-steps", type=int, default=100)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
