"""Pin of the oracle's exchange + Zeeman + LLG dynamics against the lattice
spin-wave dispersion the paper prints for its 1-D permalloy chain (Results,
"Exchange spin-wave dispersion"; parameters in tests/golden/spin_wave_chain.txt).

On a periodic chain with the static field along z and alpha = 0, the cone
m = (sin t cos(kx + wt), sin t sin(kx + wt), cos t) is an exact solution of
Eq. 1: the lattice Laplacian maps the transverse part to -(4/dx^2) sin^2(k dx/2)
times itself and leaves m_z, so the cone precesses rigidly at
    w = gamma0 [B0 + (2A/Ms)(4/dx^2) sin^2(k dx/2) cos t],
which at small cone angle is the paper's lattice dispersion.  The oracle's
DOPRI5 integration of the chain must reproduce that frequency for modes from
the longest wavelength to the zone edge, and the continuum parabola must not
fit it there."""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle.constants import GAMMA0, MU0
from oracle.fields import Problem
from oracle.llg import Solver

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "spin_wave_chain.txt")


def _chain_params():
    out = {}
    with open(GOLDEN) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                key, val = ln.split("=")
                out[key.strip()] = float(val)
    return out


P = _chain_params()
NX, DX, B0 = int(P["nx"]), P["dx_m"], P["B0_T"]
MS, A = P["Ms_A_per_m"], P["A_J_per_m"]


def _lattice_omega(k, cos_t=1.0):
    return GAMMA0 * (B0 + (2 * A / MS) * (4 / DX ** 2) * math.sin(k * DX / 2) ** 2 * cos_t)


def _continuum_omega(k):
    return GAMMA0 * (B0 + (2 * A / MS) * k * k)


def _measured_omega(mode, sin_t, periods=1.25, steps_per_period=200):
    grid = W.Grid(NX, 1, 1, DX, DX, DX, (1, 0, 0))
    p = Problem.from_workload(grid, W.Material(Ms=MS, A=A, alpha=0.0), B_ext=(0.0, 0.0, B0))
    k = 2 * math.pi * mode / (NX * DX)
    x = np.arange(NX) * DX
    cos_t = math.sqrt(1 - sin_t * sin_t)
    m0 = np.zeros((3, 1, 1, NX))
    m0[0, 0, 0] = sin_t * np.cos(k * x)
    m0[1, 0, 0] = sin_t * np.sin(k * x)
    m0[2] = cos_t
    s = Solver(p, m0, terms=("exchange", "zeeman"))
    w_est = _lattice_omega(k, cos_t)
    dt = 2 * math.pi / w_est / steps_per_period
    z0 = s.m[0, 0, 0] + 1j * s.m[1, 0, 0]
    phase = 0.0
    prev = np.zeros(NX)
    for _ in range(int(periods * steps_per_period)):
        s.rk45_step_fixed(dt)
        z = (s.m[0, 0, 0] + 1j * s.m[1, 0, 0]) / z0
        ang = np.angle(z)
        phase_all = ang + 2 * math.pi * np.round((prev - ang) / (2 * math.pi))
        prev = phase_all
    # the cone stays rigid: every cell has advanced by the same angle
    assert np.ptp(prev) < 1e-9
    assert np.abs(np.hypot(s.m[0, 0, 0], s.m[1, 0, 0]) - sin_t).max() < 1e-10
    return float(prev.mean()) / s.t, k, cos_t


def test_chain_parameters_match_the_printed_exchange_length():
    l_ex = math.sqrt(2 * A / (MU0 * MS ** 2))
    assert round(l_ex * 1e9, 1) == P["l_ex_nm"]


@pytest.mark.parametrize("mode", [1, 17, 50, 100])
def test_small_cone_follows_the_lattice_dispersion(mode):
    """Small amplitude: the paper's printed lattice dispersion (up to the
    cone factor, here 1 - 5e-7)."""
    w, k, _ = _measured_omega(mode, sin_t=1e-3)
    assert w > 0                         # counter-clockwise about +B (Eq. 1)
    assert abs(w / _lattice_omega(k) - 1) < 1e-6
    if mode >= 50:
        # near the zone edge the continuum parabola is far off
        assert abs(w / _continuum_omega(k) - 1) > 0.05


@pytest.mark.parametrize("mode", [17, 100])
def test_large_cone_precesses_at_the_exact_cone_frequency(mode):
    """Finite amplitude: the exchange part scales with cos(cone angle)."""
    w, k, cos_t = _measured_omega(mode, sin_t=0.6)
    assert abs(w / _lattice_omega(k, cos_t) - 1) < 1e-9
    assert abs(w / _lattice_omega(k) - 1) > 1e-2
