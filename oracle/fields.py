"""Local effective-field terms of the oracle (FP64, numpy).

Methods, "Physics and discretization": each contribution adds to H;
six-point Laplacian exchange with Neumann or periodic boundaries, uniaxial
anisotropy, Zeeman, interfacial DMI with the free boundary condition at grid
and geometry-mask edges.  Arrays are (3, nz, ny, nx) for vectors and
(nz, ny, nx) for scalars.

Readings taken where the paper is silent:
 * a neighbour is absent when it is outside a non-periodic grid or has
   Ms = 0 (the geometry mask);
 * exchange between two present cells uses the harmonic mean
   A_ij = 2 A_i A_j / (A_i + A_j) (mumax3's convention);
 * DMI uses the strength D_i of the cell where the field is evaluated;
 * the uniaxial axis u is a direction and is normalised;
 * free-edge ghost value.  The paper prints the edge condition as
   dm/dn = (D/2A)(z x n) x m.  Written with the field sign the paper also
   uses (H_DMI = (2D/mu0 Ms)(dmz/dx, dmz/dy, -dmx/dx - dmy/dy)), the natural
   boundary condition of that energy is dm/dn = -(D/2A)(z x n) x m; with the
   printed sign the ghost-cell field is not the gradient of any energy and
   energy is not dissipated at the edges.  The oracle takes the
   energy-consistent sign:  m_ghost = m_i - Delta (D_i/2A_i)(z x n) x m_i,
   used in both the exchange and the DMI sums, not renormalised.  The pin
   is tests/test_oracle_fields.py::test_edge_field_is_energy_gradient.
 * bulk DMI (named, not written out, in the paper): energy density
   Db m.(curl m), field H = -(2 Db/mu0 Ms) curl m, central differences in
   x, y and z.  Its natural boundary condition, dm/dn = (Db/2A) n x m, adds
   + Delta (Db_i/2A_i) n x m_i to the ghost value on every free face (the
   top and bottom of a film included).  Pinned the same way
   (test_bulk_edge_field_is_energy_gradient) and by the closed-form helix.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .constants import MU0


@dataclass
class Problem:
    """Per-cell description of one instance.

    Ms, A, alpha, Ku1, D (interfacial DMI), Db (bulk DMI): (nz, ny, nx);
    u: (3, nz, ny, nx); B_ext: (3, nz, ny, nx) tesla; d = (dx, dy, dz);
    pbc = (px, py, pz): nonzero makes the axis periodic, and the demag field
    then sums that many images of the sample on each side.
    """
    Ms: np.ndarray
    A: np.ndarray
    alpha: np.ndarray
    Ku1: np.ndarray
    u: np.ndarray
    D: np.ndarray
    B_ext: np.ndarray
    d: tuple
    pbc: tuple = (0, 0, 0)
    Db: np.ndarray = None

    def __post_init__(self):
        if self.Db is None:
            self.Db = np.zeros_like(self.Ms)

    @property
    def shape(self):
        return self.Ms.shape

    @property
    def present(self):
        return self.Ms > 0

    @staticmethod
    def from_workload(grid, mat, B_ext=(0.0, 0.0, 0.0)):
        shape = (grid.nz, grid.ny, grid.nx)

        def scal(name, default):
            v = mat.cell.get(name)
            return np.broadcast_to(np.asarray(default if v is None else v, dtype=np.float64), shape).copy()

        u = mat.cell.get("u")
        if u is None:
            u = np.broadcast_to(np.asarray(mat.u, dtype=np.float64)[:, None, None, None], (3,) + shape).copy()
        # the anisotropy axis is a direction: normalised per cell
        un = np.sqrt((np.asarray(u, dtype=np.float64) ** 2).sum(axis=0, keepdims=True))
        u = np.asarray(u, dtype=np.float64) / np.where(un > 0, un, 1.0)
        B = np.asarray(B_ext, dtype=np.float64)
        if B.ndim == 1:
            B = np.broadcast_to(B[:, None, None, None], (3,) + shape).copy()
        return Problem(Ms=scal("Ms", mat.Ms), A=scal("A", mat.A), alpha=scal("alpha", mat.alpha),
                       Ku1=scal("Ku1", mat.Ku1), u=np.asarray(u, dtype=np.float64), D=scal("D", mat.D),
                       B_ext=B, d=(grid.dx, grid.dy, grid.dz), pbc=tuple(grid.pbc),
                       Db=scal("Db", getattr(mat, "Db", 0.0)))


# array axis of each spatial direction in (nz, ny, nx) arrays
_AXIS = {0: 2, 1: 1, 2: 0}


def _shift(a: np.ndarray, direction: int, sign: int, periodic: bool, fill=0.0):
    """Value at the neighbour i + sign*e_direction (last three axes are z,y,x)."""
    ax = a.ndim - 3 + _AXIS[direction]
    if periodic:
        return np.roll(a, -sign, axis=ax)
    out = np.full_like(a, fill)
    n = a.shape[ax]
    src = [slice(None)] * a.ndim
    dst = [slice(None)] * a.ndim
    if sign > 0:
        src[ax] = slice(1, n)
        dst[ax] = slice(0, n - 1)
    else:
        src[ax] = slice(0, n - 1)
        dst[ax] = slice(1, n)
    out[tuple(dst)] = a[tuple(src)]
    return out


def _z_cross_n_cross_m(m: np.ndarray, direction: int, sign: int) -> np.ndarray:
    """(z x n) x m for the outward normal n = sign * e_direction."""
    out = np.zeros_like(m)
    if direction == 0:          # z x (+x) = +y ;  y x m = (mz, 0, -mx)
        out[0] = sign * m[2]
        out[2] = -sign * m[0]
    elif direction == 1:        # z x (+y) = -x ; -x x m = (0, mz, -my)
        out[1] = sign * m[2]
        out[2] = -sign * m[1]
    return out                  # z x (+-z) = 0


def _n_cross_m(m: np.ndarray, direction: int, sign: int) -> np.ndarray:
    """n x m for the outward normal n = sign * e_direction."""
    out = np.zeros_like(m)
    a, b = {0: (1, 2), 1: (2, 0), 2: (0, 1)}[direction]
    # for the cyclic triple (d, a, b): e_d x m = -m_b e_a + m_a e_b
    out[a] = -sign * m[b]
    out[b] = sign * m[a]
    return out


def neighbour_values(m: np.ndarray, p: Problem, direction: int, sign: int):
    """Neighbour magnetisation in direction sign*e_direction, the ghost value
    where the neighbour is absent, and the exchange coupling A_ij.

    Returns (m_nb, A_ij, present_nb).
    """
    periodic = bool(p.pbc[direction])
    Ms_nb = _shift(p.Ms, direction, sign, periodic, fill=0.0)
    A_nb = _shift(p.A, direction, sign, periodic, fill=0.0)
    m_nb = _shift(m, direction, sign, periodic, fill=0.0)
    present_nb = Ms_nb > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(p.A > 0, p.D / (2.0 * p.A), 0.0)
        ratio_b = np.where(p.A > 0, p.Db / (2.0 * p.A), 0.0)
        A_ij = np.where(present_nb & (p.A + A_nb > 0), 2.0 * p.A * A_nb / (p.A + A_nb), 0.0)
    ghost = m - p.d[direction] * ratio * _z_cross_n_cross_m(m, direction, sign)
    ghost = ghost + p.d[direction] * ratio_b * _n_cross_m(m, direction, sign)
    m_nb = np.where(present_nb, m_nb, ghost)
    A_ij = np.where(present_nb, A_ij, p.A)
    return m_nb, A_ij, present_nb


def _inv_mu0_Ms(p: Problem):
    with np.errstate(divide="ignore"):
        return np.where(p.Ms > 0, 1.0 / (MU0 * np.where(p.Ms > 0, p.Ms, 1.0)), 0.0)


def h_exchange(m: np.ndarray, p: Problem) -> np.ndarray:
    """H_ex,i = 2/(mu0 Ms_i) sum_j A_ij (m_j - m_i)/Delta_d^2 (six-point Laplacian)."""
    H = np.zeros_like(m)
    for direction in range(3):
        for sign in (+1, -1):
            m_nb, A_ij, _ = neighbour_values(m, p, direction, sign)
            H += A_ij * (m_nb - m) / p.d[direction] ** 2
    return 2.0 * _inv_mu0_Ms(p) * H


def h_dmi(m: np.ndarray, p: Problem) -> np.ndarray:
    """Interfacial DMI: H = 2D/(mu0 Ms) (dmz/dx, dmz/dy, -dmx/dx - dmy/dy),
    central differences over neighbour-or-ghost values."""
    grads = []
    for direction in (0, 1):
        mp, _, _ = neighbour_values(m, p, direction, +1)
        mm, _, _ = neighbour_values(m, p, direction, -1)
        grads.append((mp - mm) / (2.0 * p.d[direction]))
    gx, gy = grads
    H = np.stack([gx[2], gy[2], -gx[0] - gy[1]])
    H = 2.0 * p.D * _inv_mu0_Ms(p) * H
    if np.any(p.Db != 0):
        H = H + h_dmi_bulk(m, p)
    return H


def h_dmi_bulk(m: np.ndarray, p: Problem) -> np.ndarray:
    """Bulk DMI (Methods, "Physics and discretization"; energy density
    Db m.(curl m)): H = -2Db/(mu0 Ms) curl m, central differences over
    neighbour-or-ghost values along x, y and z."""
    curl = np.zeros_like(m)
    g = []
    for direction in range(3):
        mp, _, _ = neighbour_values(m, p, direction, +1)
        mm, _, _ = neighbour_values(m, p, direction, -1)
        g.append((mp - mm) / (2.0 * p.d[direction]))
    gx, gy, gz = g
    curl[0] = gy[2] - gz[1]
    curl[1] = gz[0] - gx[2]
    curl[2] = gx[1] - gy[0]
    return -2.0 * p.Db * _inv_mu0_Ms(p) * curl


def h_anisotropy(m: np.ndarray, p: Problem) -> np.ndarray:
    """Uniaxial: H = 2 Ku1/(mu0 Ms) (m.u) u."""
    mu = (m * p.u).sum(axis=0)
    return 2.0 * p.Ku1 * _inv_mu0_Ms(p) * mu * p.u


def h_zeeman(p: Problem) -> np.ndarray:
    """Zeeman: H = B_ext / mu0 (zero in absent cells)."""
    return np.where(p.present, p.B_ext / MU0, 0.0)


def h_local(m, p: Problem, terms=("exchange", "dmi", "anisotropy", "zeeman")) -> dict:
    out = {}
    if "exchange" in terms:
        out["exchange"] = h_exchange(m, p)
    if "dmi" in terms:
        out["dmi"] = h_dmi(m, p)
    if "anisotropy" in terms:
        out["anisotropy"] = h_anisotropy(m, p)
    if "zeeman" in terms:
        out["zeeman"] = h_zeeman(p)
    return out


def h_eff(m, p: Problem, demag_hat=None, h_thermal=None,
          terms=("exchange", "dmi", "anisotropy", "zeeman", "demag")) -> np.ndarray:
    """Total effective field (A/m) of the terms listed."""
    from .demag import h_demag
    H = np.zeros_like(m)
    for v in h_local(m, p, terms).values():
        H += v
    if "demag" in terms and demag_hat is not None:
        H += h_demag(m, p, demag_hat)
    if h_thermal is not None:
        H += h_thermal
    return np.where(p.present, H, 0.0)
