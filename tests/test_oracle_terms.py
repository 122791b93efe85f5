"""Pins of the oracle's further local terms (Methods, "Physics and
discretization": cubic and surface anisotropy, RKKY interlayer exchange,
magnetoelastic anisotropy): each field is -(1/mu0 Ms V) dE/dm of the energy
written independently from its definition (oracle.observables), plus closed
forms and reductions to the pinned uniaxial term."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.constants import MU0
from oracle.fields import (Problem, h_anisotropy, h_cubic, h_magnetoelastic, h_rkky, h_surface)
from oracle.observables import energy


def _grid_problem(seed=0, holes=True, **kw):
    grid = W.Grid(4, 3, 3, 2e-9, 3e-9, 1.5e-9)
    mat = W.Material(Ms=7e5, A=1.2e-11, alpha=0.1, **kw)
    if holes:
        h = np.zeros(grid.shape, bool)
        h[1, 1, 2] = h[2, 0, 0] = True
        mat = W.with_cells(mat, {"Ms": np.where(h, 0.0, 7e5)})
    return grid, Problem.from_workload(grid, mat)


def _numeric_field(p, m, term):
    V = p.d[0] * p.d[1] * p.d[2]
    eps = 1e-6
    num = np.zeros_like(m)
    for c in range(3):
        for idx in np.ndindex(p.shape):
            if p.Ms[idx] <= 0:
                continue
            mp = m.copy(); mp[(c,) + idx] += eps
            mm = m.copy(); mm[(c,) + idx] -= eps
            dE = energy(mp, p, terms=(term,))[term] - energy(mm, p, terms=(term,))[term]
            num[(c,) + idx] = -dE / (2 * eps) / (MU0 * p.Ms[idx] * V)
    return num


def _check_gradient(p, m, term, fn):
    H = np.where(p.present, fn(m, p), 0.0)
    num = _numeric_field(p, m, term)
    assert np.abs(H).max() > 0
    assert np.abs(num - H).max() < 1e-6 * np.abs(H).max(), np.abs(num - H).max() / np.abs(H).max()


def test_cubic_field_is_energy_gradient():
    grid, p = _grid_problem(Kc1=4.8e4, Kc2=-1.5e4, c1=(1.0, 0.3, -0.2), c2=(0.1, 1.0, 0.4))
    m = W.random_m(grid, seed=1)
    _check_gradient(p, m, "cubic", h_cubic)


def test_surface_field_is_energy_gradient():
    grid, p = _grid_problem(Ks=1.1e-3)
    m = W.random_m(grid, seed=2)
    _check_gradient(p, m, "surface", h_surface)


def test_rkky_field_is_energy_gradient():
    grid, p = _grid_problem()
    p.rkky = (0, 2, -7.5e-4)
    m = W.random_m(grid, seed=3)
    _check_gradient(p, m, "rkky", h_rkky)


def test_magnetoelastic_field_is_energy_gradient():
    grid, p = _grid_problem(B1=-8.0e6, B2=5.5e6)
    p.strain = np.random.default_rng(4).normal(scale=1e-3, size=(6,) + p.shape)
    m = W.random_m(grid, seed=5)
    _check_gradient(p, m, "magnetoelastic", h_magnetoelastic)


@pytest.mark.parametrize("axes", [((1, 0, 0), (0, 1, 0)), ((1, 1, 0), (-1, 1, 0.5))])
def test_cubic_closed_forms(axes):
    """Easy and hard directions are stationary (no torque); the energy
    density is 0 along an axis, Kc1/4 along a face diagonal and
    Kc1/3 + Kc2/27 along a body diagonal of the cubic frame."""
    Kc1, Kc2 = 4.8e4, 2.0e4
    grid = W.Grid(1, 1, 1, 2e-9, 2e-9, 2e-9)
    p = Problem.from_workload(grid, W.Material(Ms=7e5, A=1e-11, alpha=0.1, Kc1=Kc1, Kc2=Kc2,
                                               c1=axes[0], c2=axes[1]))
    from oracle.fields import cubic_axes
    c1, c2, c3 = (c[:, 0, 0, 0] for c in cubic_axes(p))
    V = 8e-27
    for v, e_exp in ((c1, 0.0), (c2, 0.0), ((c1 + c2) / math.sqrt(2), Kc1 / 4),
                     ((c1 + c2 + c3) / math.sqrt(3), Kc1 / 3 + Kc2 / 27)):
        m = v.reshape(3, 1, 1, 1)
        H = h_cubic(m, p)[:, 0, 0, 0]
        assert np.linalg.norm(np.cross(v, H)) < 1e-9 * (2 * (Kc1 + Kc2) / (MU0 * 7e5))
        assert abs(energy(m, p, terms=("cubic",))["cubic"] / V - e_exp) < 1e-9 * Kc1


def test_magnetoelastic_uniaxial_strain_is_uniaxial_anisotropy():
    """Strain e_zz alone: B1 e_zz m_z^2 is a uniaxial anisotropy with
    Ku = -B1 e_zz along z (up to a constant), so the fields coincide."""
    grid = W.Grid(3, 2, 2, 2e-9, 2e-9, 2e-9)
    B1, ezz = -9e6, 4e-3
    p = Problem.from_workload(grid, W.Material(Ms=6e5, A=1e-11, alpha=0.1, B1=B1))
    p.strain[2] = ezz
    q = Problem.from_workload(grid, W.Material(Ms=6e5, A=1e-11, alpha=0.1, Ku1=-B1 * ezz, u=(0, 0, 1)))
    m = W.random_m(grid, seed=7)
    assert np.allclose(h_magnetoelastic(m, p), h_anisotropy(m, q), rtol=1e-13, atol=1e-9)


def test_surface_anisotropy_of_a_monolayer_is_uniaxial():
    """A single-layer film has two free z faces per cell: the surface term is
    the uniaxial anisotropy Ku = 2 Ks / dz along z."""
    grid = W.Grid(5, 4, 1, 2e-9, 2e-9, 1e-9)
    Ks = 8e-4
    p = Problem.from_workload(grid, W.Material(Ms=1e6, A=1e-11, alpha=0.1, Ks=Ks))
    q = Problem.from_workload(grid, W.Material(Ms=1e6, A=1e-11, alpha=0.1, Ku1=2 * Ks / 1e-9, u=(0, 0, 1)))
    m = W.random_m(grid, seed=8)
    assert np.allclose(h_surface(m, p), h_anisotropy(m, q), rtol=1e-13, atol=1e-9)


def test_rkky_parallel_and_antiparallel_energies():
    grid = W.Grid(3, 2, 3, 2e-9, 2e-9, 1e-9)
    J = 6e-4
    p = Problem.from_workload(grid, W.Material(Ms=8e5, A=1e-11, alpha=0.1))
    p.rkky = (0, 2, J)
    area = 6 * 2e-9 * 2e-9
    m = np.zeros((3,) + p.shape)
    m[2] = 1.0
    assert abs(energy(m, p, terms=("rkky",))["rkky"] + J * area) < 1e-12 * J * area
    m[2, 2] = -1.0
    assert abs(energy(m, p, terms=("rkky",))["rkky"] - J * area) < 1e-12 * J * area
    H = h_rkky(m, p)
    assert np.allclose(H[2, 0], -J / (MU0 * 8e5 * 1e-9)) and np.allclose(H[:, 1], 0.0)
