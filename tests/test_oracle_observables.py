"""Pins of the oracle's energy, topological charge and mean magnetisation:
exact energies of uniform states (including the cube demag factor 1/3 by
symmetry), the charge of a Neel skyrmion against the lattice solid-angle
charge, invariances, and the present-cell average."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.constants import MU0
from oracle.demag import demag_spectrum
from oracle.fields import Problem
from oracle.observables import energy, topological_charge, topological_charge_bl


def test_uniform_state_energies():
    n = 5
    grid = W.Grid(n, n, n, 2e-9, 2e-9, 2e-9)
    Ms, Ku = 7e5, 3e5
    u = np.array([0.0, 0.6, 0.8])
    B = np.array([0.01, -0.02, 0.03])
    p = Problem.from_workload(grid, W.Material(Ms=Ms, A=1.3e-11, alpha=0.1, Ku1=Ku, u=tuple(u), D=2e-3), B_ext=tuple(B))
    mv = np.array([1.0, 0.0, 0.0])
    m = np.broadcast_to(mv[:, None, None, None], (3, n, n, n)).copy()
    E = energy(m, p, demag_spectrum(p.shape, p.d))
    V = grid.dx * grid.dy * grid.dz
    N = n ** 3
    assert E["exchange"] == 0.0
    assert abs(E["anisotropy"] - (-Ku * np.dot(mv, u) ** 2 * V * N)) < 1e-12 * Ku * V * N
    assert abs(E["zeeman"] - (-Ms * np.dot(mv, B) * V * N)) < 1e-12 * Ms * V * N
    # cube: body-averaged demag factor is exactly 1/3 along any axis
    assert abs(E["demag"] - 0.5 * MU0 * Ms ** 2 * V * N / 3) < 1e-10 * MU0 * Ms ** 2 * V * N
    assert abs(E["total"] - sum(v for k, v in E.items() if k != "total")) < 1e-20


def _neel_skyrmion(grid, R, w, pol=-1):
    x = (np.arange(grid.nx) - grid.nx / 2 + 0.5) * grid.dx
    y = (np.arange(grid.ny) - grid.ny / 2 + 0.5) * grid.dy
    X, Y = np.meshgrid(x, y)
    r = np.hypot(X, Y)
    # theta(r): pi at the centre, 0 far away (domain-wall profile at radius R)
    th = 2 * np.arctan(np.exp(-(r - R) / w))
    ph = np.arctan2(Y, X)
    m = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    if pol > 0:
        m[2] *= -1
        m[:2] *= 1
    return m[:, None, :, :]


def test_skyrmion_charge_is_minus_one():
    for n in (64, 128):
        grid = W.Grid(n, n, 1, 1e-9 * 64 / n, 1e-9 * 64 / n, 1e-9)
        p = Problem.from_workload(grid, W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.1))
        m = _neel_skyrmion(grid, R=12e-9, w=3e-9)
        Q = topological_charge(m, p)
        Qbl = topological_charge_bl(m, p)
        assert abs(Qbl - round(Qbl)) < 1e-3 and round(Qbl) == -1
        assert abs(Q + 1) < (0.02 if n == 64 else 0.006)
    # O(h^2) convergence of the finite-difference density


def test_charge_zero_for_uniform_and_rotation_invariant():
    grid = W.Grid(48, 48, 2, 1e-9, 1e-9, 1e-9)
    p = Problem.from_workload(grid, W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.1))
    m = np.zeros((3,) + p.shape)
    m[2] = 1
    assert topological_charge(m, p) == 0.0
    sk = _neel_skyrmion(W.Grid(48, 48, 1, 1e-9, 1e-9, 1e-9), R=8e-9, w=2e-9)
    m = np.concatenate([sk, sk], axis=1)
    Q = topological_charge(m, p)
    a = 0.7
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    mr = np.einsum("ab,bkji->akji", Rz, m)
    assert abs(topological_charge(mr, p) - Q) < 1e-12


def test_mean_magnetisation_counts_present_cells_only():
    """<m> is the average over present cells: a uniform state gives itself,
    values stored in absent cells do not enter, and two layers magnetised
    oppositely average to zero while each layer keeps its own direction."""
    from oracle.observables import mean_magnetisation
    grid = W.Grid(6, 5, 2, 1e-9, 1e-9, 1e-9)
    mat = W.Material(Ms=8e5, A=1.3e-11, alpha=0.1)
    Ms = np.full((2, 5, 6), 8e5)
    Ms[:, 1, 2] = 0.0                    # a hole through both layers
    Ms[1, 3, 4] = 0.0                    # and one in the top layer
    p = Problem.from_workload(grid, W.with_cells(mat, {"Ms": Ms}))
    m = np.zeros((3, 2, 5, 6))
    m[0, 0] = 1.0
    m[0, 1] = -1.0
    m[:, :, 1, 2] = 0.0
    m[2, :, 1, 2] = 1.0                  # garbage in the absent cells
    m[0, 1, 3, 4] = 0.0
    m[2, 1, 3, 4] = 1.0
    n0, n1 = 29, 28
    assert np.allclose(mean_magnetisation(m, p, 0), (1, 0, 0), atol=1e-15)
    assert np.allclose(mean_magnetisation(m, p, 1), (-1, 0, 0), atol=1e-15)
    assert np.allclose(mean_magnetisation(m, p), ((n0 - n1) / (n0 + n1), 0, 0), atol=1e-15)
    q = np.zeros_like(m)
    q[1] = 1.0
    assert np.allclose(mean_magnetisation(q, p), (0, 1, 0), atol=1e-15)
    none = Problem.from_workload(grid, W.with_cells(mat, {"Ms": np.zeros((2, 5, 6))}))
    assert np.all(mean_magnetisation(m, none) == 0)


def _two_wall_chain(dx, n, D, sense):
    """Periodic chain holding two Neel walls of the same rotation sense
    (m = (sin t, 0, cos t), t winding by 2 pi * sense), and the uniform
    state, on a grid periodic in y too (no free face where the interfacial
    DMI condition would act)."""
    A, K = 1.5e-11, 8e5
    grid = W.Grid(n, 1, 1, dx, 1e-9, 1e-9, (1, 1, 0))
    p = Problem.from_workload(grid, W.Material(Ms=5.8e5, A=A, alpha=0.1, Ku1=K, u=(0, 0, 1), D=D))
    delta = math.sqrt(A / K)
    x = (np.arange(n) + 0.5) * dx
    L = n * dx
    t = sense * (2 * np.arctan(np.exp((x - L / 4) / delta)) + 2 * np.arctan(np.exp((x - 3 * L / 4) / delta)))
    m = np.zeros((3, 1, 1, n))
    m[0, 0, 0] = np.sin(t)
    m[2, 0, 0] = np.cos(t)
    u = np.zeros_like(m)
    u[2] = 1.0
    terms = ("exchange", "dmi", "anisotropy")
    area = grid.dy * grid.dz
    return (energy(m, p, terms=terms)["total"] - energy(u, p, terms=terms)["total"]) / area / 2


@pytest.mark.parametrize("D", [0.0, 1e-3, 3e-3])
def test_neel_wall_energy_and_the_critical_dmi(D):
    """The wall energy per area behind the paper's analytic critical DMI
    D_c = 4 sqrt(AK)/pi (Results, skyrmion D-K phase diagram): a Neel wall of
    the sense the interfacial DMI favours costs 4 sqrt(AK) - pi|D|, the other
    sense 4 sqrt(AK) + pi|D|; on the lattice the profile's energy converges
    to these at second order in the cell size."""
    A, K = 1.5e-11, 8e5
    s0 = 4 * math.sqrt(A * K)
    scale = s0 + math.pi * abs(D)
    errs = []
    for dx, n, tol in [(0.5e-9, 400, 1.2e-3), (0.25e-9, 800, 3e-4)]:
        fav = _two_wall_chain(dx, n, D, sense=-1)       # t decreasing: favoured for D > 0
        unfav = _two_wall_chain(dx, n, D, sense=+1)
        errs.append(max(abs(fav - (s0 - math.pi * D)), abs(unfav - (s0 + math.pi * D))))
        assert errs[-1] < tol * scale
    assert errs[1] < 0.3 * errs[0]                      # second order in the cell size
    Dc = s0 / math.pi
    assert abs(_two_wall_chain(0.25e-9, 800, Dc, sense=-1)) < 2.5e-4 * s0
    assert _two_wall_chain(0.25e-9, 800, 1.1 * Dc, sense=-1) < 0
