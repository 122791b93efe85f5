"""Pins of the oracle's local field terms: lattice eigen-relations of the
exchange and DMI stencils, and H = -dE/dm against an independently written
bond-sum energy (which fixes the sign of the free-edge DMI condition)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.constants import MU0
from oracle.fields import Problem, h_anisotropy, h_dmi, h_exchange, h_zeeman


def _prob(grid, Ms=8e5, A=1.3e-11, D=0.0, Ku=0.0, u=(0, 0, 1), cells=None):
    mat = W.Material(Ms=Ms, A=A, alpha=0.1, Ku1=Ku, u=u, D=D)
    if cells:
        mat = W.with_cells(mat, cells)
    return Problem.from_workload(grid, mat)


def test_exchange_uniform_is_zero():
    for pbc in [(0, 0, 0), (1, 1, 1)]:
        grid = W.Grid(5, 4, 3, 2e-9, 2e-9, 2e-9, pbc)
        p = _prob(grid)
        m = np.zeros((3,) + p.shape)
        m[1] = 1
        assert np.abs(h_exchange(m, p)).max() == 0.0


@pytest.mark.parametrize("q", [1, 3, 7])
def test_exchange_lattice_dispersion(q):
    """Periodic chain: the discrete Laplacian of a spiral of wavenumber k is
    -(4/dx^2) sin^2(k dx / 2) times the spiral (the lattice dispersion the
    paper's spin-wave test compares against)."""
    n, dx = 32, 5e-9
    grid = W.Grid(n, 1, 1, dx, 1e-9, 1e-9, (1, 0, 0))
    p = _prob(grid)
    k = 2 * math.pi * q / (n * dx)
    x = np.arange(n) * dx
    m = np.zeros((3,) + p.shape)
    m[0, 0, 0] = np.cos(k * x)
    m[1, 0, 0] = np.sin(k * x)
    H = h_exchange(m, p)
    lam = -(4 / dx ** 2) * math.sin(k * dx / 2) ** 2
    assert np.allclose(H, 2 * 1.3e-11 / (MU0 * 8e5) * lam * m, rtol=1e-12, atol=1e-6)


@pytest.mark.parametrize("q", [1, 5])
def test_dmi_spiral_closed_form(q):
    """Periodic cycloid m = (sin kx, 0, cos kx): central differences give
    H_DMI = -(2D/mu0 Ms)(sin(k dx)/dx) m."""
    n, dx, D = 40, 2e-9, 3e-3
    grid = W.Grid(n, 3, 1, dx, 2e-9, 1e-9, (1, 1, 0))
    p = _prob(grid, D=D)
    k = 2 * math.pi * q / (n * dx)
    x = np.arange(n) * dx
    m = np.zeros((3,) + p.shape)
    m[0] = np.sin(k * x)[None, None, :]
    m[2] = np.cos(k * x)[None, None, :]
    H = h_dmi(m, p)
    exp = -(2 * D / (MU0 * 8e5)) * (math.sin(k * dx) / dx) * m
    assert np.allclose(H, exp, rtol=1e-12, atol=1e-6)


def test_dmi_uniform_periodic_is_zero():
    grid = W.Grid(6, 5, 2, 2e-9, 2e-9, 1e-9, (1, 1, 0))
    p = _prob(grid, D=3e-3)
    m = np.zeros((3,) + p.shape)
    m[:] = np.array([0.3, -0.5, 0.8])[:, None, None, None]
    assert np.abs(h_dmi(m, p)).max() < 1e-9


def _bond_energy(m, p, D, A, Ms):
    """Independent discrete energy of the ghost-cell scheme (uniform A, D,
    Ms; free edges and Ms = 0 holes):
      exchange  A V/dx^2 |m_i - m_j|^2 per bond,
      DMI       D V/dx  d_ij.(m_i x m_j) per bond, d_ij = z x r_ij,
      edge      -(D^2 V / 4A)(|m|^2 - (a.m)^2) per missing neighbour in the
                plane, a = z x n (the second-order part of the ghost value).
    """
    nz, ny, nx = p.shape
    dx, dy, dz = p.d
    V = dx * dy * dz
    pres = p.Ms > 0
    E = 0.0
    axes = [(0, dx, np.array([0.0, 1.0, 0.0])), (1, dy, np.array([-1.0, 0.0, 0.0])), (2, dz, np.zeros(3))]
    for (d, h, dvec) in axes:
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    if not pres[k, j, i]:
                        continue
                    idx = [i, j, k]
                    for sgn in (+1, -1):
                        nb = list(idx)
                        nb[d] += sgn
                        inside = 0 <= nb[0] < nx and 0 <= nb[1] < ny and 0 <= nb[2] < nz
                        if inside and pres[nb[2], nb[1], nb[0]]:
                            if sgn > 0:
                                mi = m[:, k, j, i]
                                mj = m[:, nb[2], nb[1], nb[0]]
                                E += A * V / h ** 2 * np.dot(mi - mj, mi - mj)
                                E += D * V / h * np.dot(dvec, np.cross(mi, mj))
                        elif d < 2:
                            a = dvec if d == 0 else np.array([1.0, 0.0, 0.0])
                            mi = m[:, k, j, i]
                            E += -(D ** 2 * V / (4 * A)) * (np.dot(mi, mi) - np.dot(a, mi) ** 2)
    return E


def test_edge_field_is_energy_gradient():
    """H_ex + H_DMI = -(1/(mu0 Ms V)) dE/dm of the independent bond energy,
    on a film with free edges and holes.  With the edge condition's printed
    sign the ghost field would carry an extra antisymmetric first-order term
    and this identity would fail."""
    grid = W.Grid(5, 4, 2, 2e-9, 3e-9, 1e-9)
    D, A, Ms = 2.5e-3, 1.2e-11, 7e5
    holes = np.zeros(grid.shape, bool)
    holes[0, 1, 2] = holes[1, 3, 0] = True
    cells = {"Ms": np.where(holes, 0.0, Ms)}
    p = _prob(grid, Ms=Ms, A=A, D=D, cells=cells)
    m = W.random_m(grid, seed=11)
    m[:, holes] = 0.0
    H = h_exchange(m, p) + h_dmi(m, p)
    V = grid.dx * grid.dy * grid.dz
    eps = 1e-6
    num = np.zeros_like(m)
    for c in range(3):
        for k in range(grid.nz):
            for j in range(grid.ny):
                for i in range(grid.nx):
                    if holes[k, j, i]:
                        continue
                    mp = m.copy(); mp[c, k, j, i] += eps
                    mm = m.copy(); mm[c, k, j, i] -= eps
                    dE = (_bond_energy(mp, p, D, A, Ms) - _bond_energy(mm, p, D, A, Ms)) / (2 * eps)
                    num[c, k, j, i] = -dE / (MU0 * Ms * V)
    scale = np.abs(H).max()
    assert np.max(np.abs(num - H)) < 1e-6 * scale


def test_edge_ghost_sign_alternative_fails_the_gradient_identity():
    """The same check with the opposite ghost sign (the printed formula read
    literally) breaks the identity: the pin discriminates the two readings."""
    from oracle import fields as F
    grid = W.Grid(4, 3, 1, 2e-9, 2e-9, 1e-9)
    D, A, Ms = 3e-3, 1.5e-11, 6e5
    p = _prob(grid, Ms=Ms, A=A, D=D)
    m = W.random_m(grid, seed=5)
    orig = F._z_cross_n_cross_m
    try:
        F._z_cross_n_cross_m = lambda mm, d, s: -orig(mm, d, s)
        H_alt = h_exchange(m, p) + h_dmi(m, p)
    finally:
        F._z_cross_n_cross_m = orig
    H = h_exchange(m, p) + h_dmi(m, p)
    V = grid.dx * grid.dy * grid.dz
    eps = 1e-6
    i, j, k = 0, 1, 0           # an edge cell
    num = np.zeros(3)
    for c in range(3):
        mp = m.copy(); mp[c, k, j, i] += eps
        mm = m.copy(); mm[c, k, j, i] -= eps
        num[c] = -(_bond_energy(mp, p, D, A, Ms) - _bond_energy(mm, p, D, A, Ms)) / (2 * eps) / (MU0 * Ms * V)
    assert np.max(np.abs(num - H[:, k, j, i])) < 1e-6 * np.abs(H).max()
    assert np.max(np.abs(num - H_alt[:, k, j, i])) > 1e-2 * np.abs(H).max()


def test_anisotropy_and_zeeman_closed_forms():
    grid = W.Grid(3, 2, 1, 2e-9, 2e-9, 1e-9)
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    p = _prob(grid, Ms=5e5, Ku=4e5, u=tuple(u))
    m = np.broadcast_to(u[:, None, None, None], (3,) + p.shape).copy()
    H = h_anisotropy(m, p)
    assert np.allclose(H, 2 * 4e5 / (MU0 * 5e5) * m, rtol=1e-14)
    m2 = np.zeros_like(m)
    m2[0] = 2 / 3.0 * 0 + 1.0  # m = x: m.u = 1/3
    H2 = h_anisotropy(m2, p)
    assert np.allclose(H2, 2 * 4e5 / (MU0 * 5e5) * (1 / 3.0) * m, rtol=1e-14)
    p2 = Problem.from_workload(grid, W.Material(Ms=5e5, A=1e-11, alpha=0.1), B_ext=(0.01, 0.0, -0.2))
    Hz = h_zeeman(p2)
    assert np.allclose(Hz[:, 0, 0, 0], np.array([0.01, 0, -0.2]) / MU0)


# -- bulk DMI -------------------------------------------------------------------
def _bond_energy_general(m, p, Di, Db, A, Ms):
    """Independent discrete energy with interfacial (Di) and bulk (Db) DMI
    (uniform A, Ms; free faces and Ms = 0 holes):
      exchange  A V/h^2 |m_i - m_j|^2 per bond,
      DMI       (V/h) d_ij.(m_i x m_j) per bond, d_ij = Di z x r_ij - Db r_ij
                (bulk: Db m.(curl m) = -Db sum_d e_d.(m x d_d m)),
      face      -A V |c x m_i|^2 per missing neighbour, c = (Di z x n - Db n)/2A
                (the first-order part of the ghost value, squared).
    """
    nz, ny, nx = p.shape
    V = p.d[0] * p.d[1] * p.d[2]
    pres = p.Ms > 0
    E = 0.0
    unit = np.eye(3)
    zhat = unit[2]
    for d in range(3):
        h = p.d[d]
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    if not pres[k, j, i]:
                        continue
                    mi = m[:, k, j, i]
                    for sgn in (+1, -1):
                        nb = [i, j, k]
                        nb[d] += sgn
                        inside = 0 <= nb[0] < nx and 0 <= nb[1] < ny and 0 <= nb[2] < nz
                        n = sgn * unit[d]
                        if inside and pres[nb[2], nb[1], nb[0]]:
                            if sgn > 0:
                                mj = m[:, nb[2], nb[1], nb[0]]
                                E += A * V / h ** 2 * np.dot(mi - mj, mi - mj)
                                dvec = Di * np.cross(zhat, n) - Db * n
                                E += V / h * np.dot(dvec, np.cross(mi, mj))
                        else:
                            c = (Di * np.cross(zhat, n) - Db * n) / (2 * A)
                            w = np.cross(c, mi)
                            E += -A * V * np.dot(w, w)
    return E


@pytest.mark.parametrize("Di,Db", [(0.0, 2.2e-3), (1.5e-3, -2.0e-3)])
def test_bulk_edge_field_is_energy_gradient(Di, Db):
    """H_ex + H_DMI = -(1/(mu0 Ms V)) dE/dm of the independent bond energy on
    a two-layer block with free faces (top and bottom included) and holes,
    for bulk DMI alone and together with interfacial DMI."""
    from oracle.fields import h_dmi_bulk  # noqa: F401  (part of h_dmi when Db != 0)
    grid = W.Grid(4, 3, 2, 2e-9, 3e-9, 1.5e-9)
    A, Ms = 1.2e-11, 7e5
    holes = np.zeros(grid.shape, bool)
    holes[0, 1, 2] = holes[1, 2, 0] = True
    mat = W.with_cells(W.Material(Ms=Ms, A=A, alpha=0.1, D=Di, Db=Db), {"Ms": np.where(holes, 0.0, Ms)})
    p = Problem.from_workload(grid, mat)
    m = W.random_m(grid, seed=13)
    m[:, holes] = 0.0
    H = h_exchange(m, p) + h_dmi(m, p)
    V = grid.dx * grid.dy * grid.dz
    eps = 1e-6
    num = np.zeros_like(m)
    for c in range(3):
        for k in range(grid.nz):
            for j in range(grid.ny):
                for i in range(grid.nx):
                    if holes[k, j, i]:
                        continue
                    mp = m.copy(); mp[c, k, j, i] += eps
                    mm = m.copy(); mm[c, k, j, i] -= eps
                    dE = (_bond_energy_general(mp, p, Di, Db, A, Ms) - _bond_energy_general(mm, p, Di, Db, A, Ms))
                    num[c, k, j, i] = -dE / (2 * eps) / (MU0 * Ms * V)
    assert np.max(np.abs(num - H)) < 1e-6 * np.abs(H).max()


@pytest.mark.parametrize("q,hand", [(1, 1), (4, 1), (3, -1)])
def test_bulk_dmi_helix_closed_form(q, hand):
    """Periodic chain, Bloch helix m = (0, cos kx, hand sin kx): curl m =
    -hand (sin(k dx)/dx) m by central differences, so H_bulk =
    hand (2 Db/mu0 Ms)(sin(k dx)/dx) m; the exchange and DMI torques vanish
    (the helix of either hand is a stationary state of the local terms)."""
    n, dx, Db, Ms = 36, 2e-9, 2.5e-3, 8e5
    grid = W.Grid(n, 1, 1, dx, 2e-9, 2e-9, (1, 1, 1))
    p = Problem.from_workload(grid, W.Material(Ms=Ms, A=1.3e-11, alpha=0.1, Db=Db))
    k = 2 * math.pi * q / (n * dx)
    x = np.arange(n) * dx
    m = np.zeros((3,) + p.shape)
    m[1, 0, 0] = np.cos(k * x)
    m[2, 0, 0] = hand * np.sin(k * x)
    H = h_dmi(m, p)
    exp = hand * (2 * Db / (MU0 * Ms)) * (math.sin(k * dx) / dx) * m
    assert np.allclose(H, exp, rtol=1e-12, atol=1e-6)
    # the right-handed helix lowers the DMI energy for Db > 0
    assert hand * np.sum(m * H) > 0


def test_bulk_ghost_sign_alternative_fails_the_gradient_identity():
    """The bulk face condition with the opposite sign breaks the identity at
    a face cell: the pin discriminates the two signs."""
    from oracle import fields as F
    grid = W.Grid(3, 3, 2, 2e-9, 2e-9, 1e-9)
    A, Ms, Db = 1.5e-11, 6e5, 3e-3
    p = Problem.from_workload(grid, W.Material(Ms=Ms, A=A, alpha=0.1, Db=Db))
    m = W.random_m(grid, seed=6)
    orig = F._n_cross_m
    try:
        F._n_cross_m = lambda mm, d, s: -orig(mm, d, s)
        H_alt = h_exchange(m, p) + h_dmi(m, p)
    finally:
        F._n_cross_m = orig
    H = h_exchange(m, p) + h_dmi(m, p)
    V = grid.dx * grid.dy * grid.dz
    eps = 1e-6
    i, j, k = 0, 1, 0
    num = np.zeros(3)
    for c in range(3):
        mp = m.copy(); mp[c, k, j, i] += eps
        mm = m.copy(); mm[c, k, j, i] -= eps
        num[c] = -(_bond_energy_general(mp, p, 0.0, Db, A, Ms) - _bond_energy_general(mm, p, 0.0, Db, A, Ms)) \
            / (2 * eps) / (MU0 * Ms * V)
    assert np.max(np.abs(num - H[:, k, j, i])) < 1e-6 * np.abs(H).max()
    assert np.max(np.abs(num - H_alt[:, k, j, i])) > 1e-2 * np.abs(H).max()
