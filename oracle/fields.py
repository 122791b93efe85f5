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
    # further local terms (Methods: cubic and surface anisotropy, RKKY
    # interlayer exchange, magnetoelastic anisotropy)
    Kc1: np.ndarray = None
    Kc2: np.ndarray = None
    c1: np.ndarray = None       # (3, nz, ny, nx)
    c2: np.ndarray = None
    Ks: np.ndarray = None
    B1: np.ndarray = None
    B2: np.ndarray = None
    strain: np.ndarray = None   # (6, nz, ny, nx): xx, yy, zz, xy, xz, yz
    rkky: tuple = None          # (layer k1, layer k2, J in J/m^2)

    def __post_init__(self):
        for name in ("Db", "Kc1", "Kc2", "Ks", "B1", "B2"):
            if getattr(self, name) is None:
                setattr(self, name, np.zeros_like(self.Ms))
        if self.c1 is None:
            self.c1 = np.zeros((3,) + self.Ms.shape)
            self.c1[0] = 1.0
        if self.c2 is None:
            self.c2 = np.zeros((3,) + self.Ms.shape)
            self.c2[1] = 1.0
        if self.strain is None:
            self.strain = np.zeros((6,) + self.Ms.shape)

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
        def vec(name, default):
            v = mat.cell.get(name)
            if v is None:
                v = np.broadcast_to(np.asarray(default, dtype=np.float64)[:, None, None, None], (3,) + shape)
            return np.asarray(v, dtype=np.float64).copy()

        return Problem(Ms=scal("Ms", mat.Ms), A=scal("A", mat.A), alpha=scal("alpha", mat.alpha),
                       Ku1=scal("Ku1", mat.Ku1), u=np.asarray(u, dtype=np.float64), D=scal("D", mat.D),
                       B_ext=B, d=(grid.dx, grid.dy, grid.dz), pbc=tuple(grid.pbc),
                       Db=scal("Db", mat.Db), Kc1=scal("Kc1", mat.Kc1), Kc2=scal("Kc2", mat.Kc2),
                       c1=vec("c1", mat.c1), c2=vec("c2", mat.c2), Ks=scal("Ks", mat.Ks),
                       B1=scal("B1", mat.B1), B2=scal("B2", mat.B2))


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


def cubic_axes(p: Problem):
    """Unit cubic axes per cell: c1, c2 with its c1 component removed, and
    c3 = c1 x c2."""
    c1 = p.c1 / np.sqrt((p.c1 ** 2).sum(axis=0, keepdims=True))
    c2 = p.c2 - (p.c2 * c1).sum(axis=0, keepdims=True) * c1
    c2 = c2 / np.sqrt((c2 ** 2).sum(axis=0, keepdims=True))
    c3 = np.stack([c1[1] * c2[2] - c1[2] * c2[1], c1[2] * c2[0] - c1[0] * c2[2], c1[0] * c2[1] - c1[1] * c2[0]])
    return c1, c2, c3


def h_cubic(m: np.ndarray, p: Problem) -> np.ndarray:
    """Cubic anisotropy (Methods, "Physics and discretization"; the paper
    names the term): energy density Kc1 (a^2 b^2 + b^2 c^2 + c^2 a^2) +
    Kc2 a^2 b^2 c^2 with a, b, c the components of m on the cubic axes;
    H = -(1/mu0 Ms) dE/dm."""
    c1, c2, c3 = cubic_axes(p)
    a, b, c = (m * c1).sum(axis=0), (m * c2).sum(axis=0), (m * c3).sum(axis=0)
    g1 = p.Kc1 * 2 * a * (b * b + c * c) + p.Kc2 * 2 * a * b * b * c * c
    g2 = p.Kc1 * 2 * b * (a * a + c * c) + p.Kc2 * 2 * a * a * b * c * c
    g3 = p.Kc1 * 2 * c * (a * a + b * b) + p.Kc2 * 2 * a * a * b * b * c
    return -_inv_mu0_Ms(p) * (g1 * c1 + g2 * c2 + g3 * c3)


def _free_z_faces(p: Problem) -> np.ndarray:
    """Number (0, 1, 2) of absent z neighbours of every cell."""
    per = bool(p.pbc[2])
    up = _shift(p.Ms, 2, +1, per, fill=0.0) > 0
    dn = _shift(p.Ms, 2, -1, per, fill=0.0) > 0
    return (~up).astype(float) + (~dn).astype(float)


def h_surface(m: np.ndarray, p: Problem) -> np.ndarray:
    """Surface anisotropy (the paper names it): every free z face of a cell
    (an absent neighbour above or below) adds an anisotropy energy
    -Ks (m.z)^2 per face area, i.e. the uniaxial field
    (2 Ks / (mu0 Ms dz)) m_z z per face."""
    H = np.zeros_like(m)
    H[2] = 2.0 * p.Ks * _inv_mu0_Ms(p) / p.d[2] * _free_z_faces(p) * m[2]
    return H


def h_rkky(m: np.ndarray, p: Problem) -> np.ndarray:
    """RKKY interlayer exchange between layers k1 and k2 (the paper names
    it): energy -J m(k1).m(k2) per column area, so each coupled cell sees
    (J / (mu0 Ms dz)) times the moment of its partner across the spacer
    (where both cells are present)."""
    H = np.zeros_like(m)
    if p.rkky is None:
        return H
    k1, k2, J = p.rkky
    both = (p.Ms[k1] > 0) & (p.Ms[k2] > 0)
    inv = _inv_mu0_Ms(p)
    H[:, k1] += np.where(both, J * inv[k1] / p.d[2] * m[:, k2], 0.0)
    H[:, k2] += np.where(both, J * inv[k2] / p.d[2] * m[:, k1], 0.0)
    return H


def h_magnetoelastic(m: np.ndarray, p: Problem) -> np.ndarray:
    """Magnetoelastic anisotropy (the paper names it) for a given strain:
    energy density B1 (e_xx m_x^2 + e_yy m_y^2 + e_zz m_z^2) +
    2 B2 (e_xy m_x m_y + e_xz m_x m_z + e_yz m_y m_z); H = -(1/mu0 Ms) dE/dm."""
    e = p.strain
    g = np.stack([2 * p.B1 * e[0] * m[0] + 2 * p.B2 * (e[3] * m[1] + e[4] * m[2]),
                  2 * p.B1 * e[1] * m[1] + 2 * p.B2 * (e[3] * m[0] + e[5] * m[2]),
                  2 * p.B1 * e[2] * m[2] + 2 * p.B2 * (e[4] * m[0] + e[5] * m[1])])
    return -_inv_mu0_Ms(p) * g


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
    if "cubic" in terms:
        out["cubic"] = h_cubic(m, p)
    if "surface" in terms:
        out["surface"] = h_surface(m, p)
    if "rkky" in terms:
        out["rkky"] = h_rkky(m, p)
    if "magnetoelastic" in terms:
        out["magnetoelastic"] = h_magnetoelastic(m, p)
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
