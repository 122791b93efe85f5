"""Ensembles of independent trials with retire/refill (ORACLE, test
infrastructure).

Results, "Replica batching": each trial carries its own current density J
and temperature T and its own Philox stream; an optional retire/refill
mechanism freezes a trial at the step where it crosses a stop condition and
restarts its slot with the next trial and a fresh noise stream.

Readings (the paper names the mechanism, not its rules):
 * trial q uses the key splitmix64(base_seed + q) (the replica key of slot q
   when nothing is refilled) and its own step counter, starting at 0, for
   the noise; it starts from m_init;
 * the stop condition is checked after every step: the mean over present
   cells of m . axis at or below `threshold` (e.g. a switched film);
 * a trial that reaches `max_steps` without stopping retires as not stopped;
 * a retiring slot takes the lowest trial index not yet started, so every
   trial's trajectory depends on q alone, never on the slot or on when it
   started.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from .fields import Problem
from .llg import Solver, Torque, dot, replica_seed


@dataclass
class TrialSpec:
    p: Problem
    m_init: np.ndarray
    J: np.ndarray                 # per trial, A/m^2
    T: np.ndarray                 # per trial, K
    terms: tuple = ("anisotropy", "zeeman")
    torque: Torque = field(default_factory=Torque)
    base_seed: int = 0
    dt: float = 1e-13
    axis: tuple = (0.0, 0.0, 1.0)
    threshold: float = 0.0
    max_steps: int = 1000
    integrator: str = "dm"        # "dm" or "heun"


def _solver(spec: TrialSpec, q: int) -> Solver:
    tq = replace(spec.torque, J=float(spec.J[q]))
    return Solver(spec.p, spec.m_init, terms=spec.terms, torque=tq, T=float(spec.T[q]),
                  seed=replica_seed(spec.base_seed, q), dt=spec.dt)


def _advance(s: Solver, spec: TrialSpec):
    if spec.integrator == "dm":
        s.dm_step(spec.dt)
    else:
        s.heun_step(spec.dt)


def _stopped(s: Solver, spec: TrialSpec) -> bool:
    a = np.asarray(spec.axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    proj = dot(s.m, np.broadcast_to(a[:, None, None, None], s.m.shape))
    return float(proj[s.p.present].mean()) <= spec.threshold


def run_trial(spec: TrialSpec, q: int):
    """Trial q alone: (steps taken, stopped flag, final m)."""
    s = _solver(spec, q)
    for n in range(1, spec.max_steps + 1):
        _advance(s, spec)
        if _stopped(s, spec):
            return n, True, s.m
    return spec.max_steps, False, s.m


def run_ensemble(spec: TrialSpec, n_trials: int, R: int, refill: bool = True):
    """R slots over n_trials trials.  Returns (results, starts, global_steps):
    results[q] = (steps, stopped) for every trial that ran, starts[q] =
    (slot, global step at which the trial took its first step)."""
    slots = [None] * R
    results, starts = {}, {}
    next_q = 0
    for r in range(R):
        if next_q < n_trials:
            slots[r] = [next_q, _solver(spec, next_q), 0]
            starts[next_q] = (r, 0)
            next_q += 1
    g = 0
    while any(sl is not None for sl in slots):
        for r in range(R):
            sl = slots[r]
            if sl is None:
                continue
            q, s, _ = sl
            _advance(s, spec)
            sl[2] += 1
            stop = _stopped(s, spec)
            if stop or sl[2] == spec.max_steps:
                results[q] = (sl[2], stop)
                slots[r] = None
                if refill and next_q < n_trials:
                    slots[r] = [next_q, _solver(spec, next_q), 0]
                    starts[next_q] = (r, g + 1)
                    next_q += 1
        g += 1
    return results, starts, g
