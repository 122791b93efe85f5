"""End-to-end pin of the oracle (exchange + Newell FFT demag + Zeeman +
Dormand-Prince RK45 with its step controller) against the muMAG Standard
Problem #4 result the paper prints (tests/golden/mumag_sp4_field_a.txt):
<m_x> one nanosecond into the field-A reversal of the 500 x 125 x 3 nm film
on 128 x 32 x 1 cells.  The s-state is the uniform [1,1,1] state relaxed in
zero field with alpha = 1 (2.5 ns here: about 80 s of CPU for the whole
test)."""
import math
import os

import numpy as np

import workloads as W
from oracle.demag import demag_spectrum
from oracle.fields import Problem
from oracle.llg import Solver

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mumag_sp4_field_a.txt")


def _fixture():
    out = {}
    for ln in open(GOLDEN):
        if ln.strip() and not ln.startswith("#"):
            k, v = ln.split("=")
            out[k.strip()] = float(v)
    return out


def _run_to(s, t_end):
    while s.t < t_end:
        s.dt = min(s.dt, t_end - s.t)
        s.rk45_step()


def test_standard_problem_4_field_a():
    fx = _fixture()
    g = W.Grid(128, 32, 1, 500e-9 / 128, 125e-9 / 32, 3e-9)
    relax = Problem.from_workload(g, W.Material(Ms=fx["Ms"], A=fx["A"], alpha=1.0))
    K = demag_spectrum(relax.shape, relax.d)
    s = Solver(relax, np.full((3,) + relax.shape, 1 / math.sqrt(3)), terms=("exchange", "demag"),
               K_hat=K, dt=1e-13, rtol=1e-6)
    _run_to(s, 2.5e-9)
    mx0, my0 = s.m[0].mean(), s.m[1].mean()
    assert 0.95 < mx0 < 0.98 and 0.1 < my0 < 0.15          # the s-state: mostly along +x
    B = (fx["B_mT_x"] * 1e-3, fx["B_mT_y"] * 1e-3, 0.0)
    drive = Problem.from_workload(g, W.Material(Ms=fx["Ms"], A=fx["A"], alpha=fx["alpha"]), B_ext=B)
    d = Solver(drive, s.m, terms=("exchange", "demag", "zeeman"), K_hat=K, dt=1e-13, rtol=1e-6)
    _run_to(d, 1e-9)
    mx = float(d.m[0].mean())
    ref = fx["mx_1ns_mumag_reference"]
    assert abs(mx - ref) < fx["band"] * abs(ref), mx
    # as close to the reference as the paper's own solver and OOMMF
    assert abs(mx - ref) <= abs(fx["mx_1ns_paper"] - ref) + 1e-3, mx
