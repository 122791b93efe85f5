"""Throughput benchmark of the LLG hot path on GB300.

Metric: LLG cell-steps/s (cells x accepted integrator steps per second).
Workload (single GPU): 256x256x16 cells of 2 nm, Ms 5.8e5, A 1.5e-11,
Ku 8e5 along z, interfacial DMI 3e-3, alpha 0.1, seeded random unit
vectors, FP32 Dormand-Prince RK45 (rtol 1e-6, device-side controller) with
exact FFT demag on the 512x512x32 padded grid.  One step = one accepted
RK45 step (6 field evaluations, each exchange+DMI+anisotropy+demag, plus
the stage, error and controller kernels).

Multi-GPU: replicas only (independent runs of the same workload per rank,
no data-path collective); value = sum of cell-steps over ranks / max time.

--impl reference times the FP64 CPU oracle (the only reference available:
the paper ships no code) on the same workload on the host cores.
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


def _traffic_for(kernel: str):
    """ncu DRAM bytes per launch recorded in profiles/traffic.json, used only
    while the source files that define the kernel still hash to the values
    recorded with the capture (any change to them makes it null)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            ent = json.load(f)["kernels"][kernel]
        h = hashlib.sha256()
        for rel in ent["sources"]:
            with open(os.path.join(ROOT, rel), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != ent["sources_sha256"]:
            return None
        return ent["dram_bytes_per_launch"]
    except Exception:
        return None


def cpu_baseline(seconds_budget=60.0):
    """The FP64 oracle as it stands on this host's cores: RK45 steps of the
    same 256x256x16 workload (setup excluded), bounded to about a minute."""
    from oracle.demag import demag_spectrum
    from oracle.fields import Problem
    from oracle.llg import Solver
    w = W.dmi_256x256x16()
    p = Problem.from_workload(w.grid, w.mat)
    K = demag_spectrum(p.shape, p.d)
    s = Solver(p, W.m_random_sphere(w.grid, seed=2), K_hat=K, dt=1e-14, rtol=1e-6)
    s.k1 = s.slope(s.m)
    done = 0
    t0 = time.perf_counter()
    while True:
        s.rk45_step_fixed(1e-14)
        done += 1
        el = time.perf_counter() - t0
        if el > seconds_budget / 3 or done >= 3:
            break
    return {"value": w.grid.n * done / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} RK45 step(s) of the 256x256x16 workload (numpy FP64, single-threaded "
                      f"FFT and array ops; Newell/FFT setup excluded), {el:.1f} s"}


REFERENCE_BUDGET_S = 240.0
# sample grids of the 256x256x16 workload (same material, 2 nm cells, RK45), largest first
REFERENCE_SAMPLES = [(256, 256, 16), (128, 128, 16), (64, 64, 16), (32, 32, 16), (16, 16, 16),
                     (16, 16, 8), (8, 8, 8), (4, 4, 4)]


def _oracle_solver(w, nx, ny, nz):
    from dataclasses import replace

    from oracle.demag import demag_spectrum
    from oracle.fields import Problem
    from oracle.llg import Solver
    g = W.Grid(nx, ny, nz, w.grid.dx, w.grid.dy, w.grid.dz)
    ws = replace(w, grid=g)
    p = Problem.from_workload(g, ws.mat)
    s = Solver(p, W.m_random_sphere(g, seed=2), K_hat=demag_spectrum(p.shape, p.d), dt=1e-14, rtol=w.rtol)
    s.k1 = s.slope(s.m)
    return s, g.n


def run_reference(args):
    """The FP64 CPU oracle timed on this host, W warm-up and exactly K timed
    RK45 steps.  Each step is a bounded sample of the 256x256x16 workload: the
    largest grid of the same material, cell size and integrator whose K + W
    steps fit in about REFERENCE_BUDGET_S seconds (cost per cell-step taken
    from two steps of a 32x32x16 probe)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    w = W.dmi_256x256x16()
    probe, n_probe = _oracle_solver(w, 32, 32, 16)
    probe.rk45_step_fixed(1e-14)
    t0 = time.perf_counter()
    for _ in range(2):
        probe.rk45_step_fixed(1e-14)
    per_cell_step = (time.perf_counter() - t0) / (2 * n_probe)
    total = args.steps + args.warmup
    shape = REFERENCE_SAMPLES[-1]
    for cand in REFERENCE_SAMPLES:
        if per_cell_step * cand[0] * cand[1] * cand[2] * total <= REFERENCE_BUDGET_S:
            shape = cand
            break
    s, n = _oracle_solver(w, *shape)
    for _ in range(args.warmup):
        s.rk45_step_fixed(1e-14)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.rk45_step_fixed(1e-14)
    el = time.perf_counter() - t0
    val = n * args.steps / el
    sample = (f"each step one RK45 step (dt 1e-14 s) of a {shape[0]}x{shape[1]}x{shape[2]} sample of the "
              f"workload (same material, 2 nm cells, exact demag; numpy FP64, single-threaded), "
              f"{args.steps} timed after {args.warmup} warm-up, {el:.1f} s")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "cells": w.grid.n, "grid": [w.grid.nx, w.grid.ny, w.grid.nz],
                   "cell_nm": [2, 2, 2], "integrator": "rk45-dopri5", "rtol": w.rtol,
                   "demag": f"exact-fft {2*shape[0]}x{2*shape[1]}x{2*shape[2]} (sample grid)",
                   "precision": "fp64-cpu-oracle", "parallelism": "one CPU thread (rank 0)",
                   "sample_grid": list(shape)},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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


def fp32_vs_fp64(mm, stream, w, m0, n_steps=20, dt=2e-14):
    """The same n fixed RK45 steps from the same state in FP32 and in FP64:
    max|m_fp32 - m_fp64| (the FP64 GPU path stands in for the FP64 oracle
    here; the parity tests hold it to the oracle within 1e-11) and each
    precision's device throughput on those steps."""
    g = w.grid
    M = mm.Material(w.mat.Ms, w.mat.A, w.mat.alpha, w.mat.Ku1, w.mat.u, w.mat.D)
    out, rate = {}, {}
    for prec in (32, 64):
        cfg = mm.make_config(precision=prec, integrator=mm.MM_RK45, demag=mm.MM_DEMAG_EXACT, dt=dt, rtol=w.rtol)
        c = mm.mm_create(mm.make_grid(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), M.s, cfg)
        mm.mm_set_stream(c, stream.cuda_stream)
        mm.mm_set_m(c, 0, m0)
        mm.mm_step_dt(c, np.full(3, dt))          # warm-up (graph capture, first slope)
        mm.mm_set_m(c, 0, m0)
        ms = _timed(stream, lambda: mm.mm_step_dt(c, np.full(n_steps, dt)))
        rate[prec] = g.n * n_steps / (ms * 1e-3)
        out[prec] = mm.mm_get_m(c, 0, m0.shape)
        mm.mm_destroy(c)
    return float(np.abs(out[32] - out[64]).max()), rate


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
    mm.mm_destroy(ctx)
    torch.cuda.synchronize()
    return {"workload": "1024 perpendicular free layers, sizes {32,48,64,96,128}^2 x 1 of 2x2x1 nm, T=300 K, "
                        "damping-like SOT J in [1e11,3e11] A/m^2, exact demag, FP32 Heun dt=1e-14 s",
            "value": cells * n_acc / (ms * 1e-3), "unit": UNIT, "cells": cells, "replicas": R,
            "steps": n_acc, "ms_per_step": ms / max(1, n_acc),
            "launch_shape": {"threads": nt, "ctas": blocks, "stacked": nt == 0},
            "autotune_s": round(t_tune, 2),
            "error_vs_fp64": {"max_abs_dm": max(errs), "after_steps": n_total, "replicas_checked": checks,
                              "against": "FP64 single-instance GPU runs with the same Philox key"}}


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
    w = W.dmi_256x256x16()
    if args.grid:
        nx, ny, nz = (int(v) for v in args.grid.split(","))
        from dataclasses import replace
        w = replace(w, name=f"dmi_{nx}x{ny}x{nz}_rk45", grid=W.Grid(nx, ny, nz, 2e-9, 2e-9, 2e-9))
    g = w.grid
    M = mm.Material(w.mat.Ms, w.mat.A, w.mat.alpha, w.mat.Ku1, w.mat.u, w.mat.D)
    cfg = mm.make_config(precision=32, integrator=mm.MM_RK45, demag=mm.MM_DEMAG_EXACT, dt=1e-14, rtol=w.rtol)
    ctx = mm.mm_create(mm.make_grid(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), M.s, cfg)
    stream = torch.cuda.current_stream()
    mm.mm_set_stream(ctx, stream.cuda_stream)
    m0 = W.m_random_sphere(g, seed=2 + rank)
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
    mm.mm_set_profiling(ctx, True)
    mm.mm_step(ctx, max(2, min(args.steps, 5)))
    prof = mm.mm_get_profile(ctx)
    mm.mm_set_profiling(ctx, False)
    tot = sum(p["total_ms"] for p in prof) or 1.0
    dom = max(prof, key=lambda p: p["total_ms"])
    avg_ms = dom["total_ms"] / max(1, dom["launches"])
    achieved = dom["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    kernels = {p["name"]: {"launches": p["launches"], "share": round(p["total_ms"] / tot, 4),
                           "avg_us": round(1e3 * p["total_ms"] / max(1, p["launches"]), 2),
                           "GBps": round(p["bytes_per_launch"] / (p["total_ms"] / max(1, p["launches"]) * 1e-3) / 1e9, 1)
                           if p["bytes_per_launch"] > 0 else None}
               for p in sorted(prof, key=lambda p: -p["total_ms"])}

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

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / max(1, steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "cells": g.n, "grid": [g.nx, g.ny, g.nz], "cell_nm": [2, 2, 2],
                   "integrator": "rk45-dopri5", "rtol": w.rtol, "demag": f"exact-fft {2*g.nx}x{2*g.ny}x{2*g.nz}",
                   "precision": "fp32 (fp64 Newell setup)", "parallelism": f"replicas x{ws}",
                   "accepted_steps": steps, "attempts": attempts,
                   "l2": "working set ~220 MB > 126 MB L2 (state, 7 slopes, spectrum, tensor)"},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": _traffic_for(dom["name"]), "algorithmic_bytes_per_launch": dom["bytes_per_launch"],
                     "avg_launch_us": round(1e3 * avg_ms, 2)},
        "kernels": kernels,
        "clocks": clk.summary(),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 3 * g.n * 8,
                "d2h_bytes_per_step": 3 * g.n * 8, "steps": k_e2e,
                "host_buffers": "page-locked float64 [3][z][y][x]"},
    }
    mm.mm_destroy(ctx)
    if not args.no_variants and rank == 0:
        m0_err = W.m_random_sphere(g, seed=2)
        err, rate = fp32_vs_fp64(mm, stream, w, m0_err)
        line["error_vs_fp64"] = {"max_abs_dm": err, "after_steps": 20, "dt_s": 2e-14,
                                 "against": "FP64 GPU path on the same steps (held to the FP64 oracle "
                                            "within 1e-11 by the parity tests)"}
        line["fp64"] = {"value": rate[64], "unit": UNIT, "fp32_same_steps": rate[32],
                        "note": "20 replayed RK45 steps of dt 2e-14 s from the same random state"}
        line["variants"] = {}
        wanted = [v for v in args.variants.split(",") if v]
        for name, fn in (("batched", lambda: variant_batched(mm, stream, args.batch_steps)),
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
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", default="", help="nx,ny,nz: a smaller case of the same workload (profiling)")
    ap.add_argument("--no-variants", action="store_true", help="skip the FP64, batched and surrogate lines")
    ap.add_argument("--variants", default="batched,surrogate,paper_scenarios,batching_table,stt_sweep,sp4",
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
