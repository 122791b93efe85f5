"""Energy, topological charge and mean magnetisation of the oracle.

Energy (the quantity behind the energy-balance results, e.g. the
flower/vortex crossover and the skyrmion phase diagram): per cell
    e_ex  = -1/2 mu0 Ms m.H_ex,  e_dmi = -1/2 mu0 Ms m.H_dmi,
    e_dem = -1/2 mu0 Ms m.H_demag, e_anis = -Ku1 (m.u)^2,
    e_Z   = -mu0 Ms m.H_ext,
and, written from their definitions (``oracle.fields``): cubic
Kc1 (a^2 b^2 + b^2 c^2 + c^2 a^2) + Kc2 a^2 b^2 c^2, surface -(Ks/dz) m_z^2
per free z face, RKKY -(J/dz) m(k1).m(k2) per coupled cell pair,
magnetoelastic B1 sum e_ii m_i^2 + 2 B2 sum_{i<j} e_ij m_i m_j;
E_term = V sum_cells e, summed exactly-rounded (math.fsum).

Topological charge (the skyrmion-classification observable): per layer
    Q = (1/4pi) sum_cells m . (dm/dx x dm/dy) dx dy
with central differences inside and one-sided differences at edges and
next to absent cells (a reading: the paper does not give the stencil); for
nz > 1 the mean over layers.  ``topological_charge_bl`` is the lattice
(Berg-Luescher) solid-angle form, used as an independent check.

Mean magnetisation <m> (the averaged magnetisation the standard-problem and
relaxation results report): the average of the unit vectors over the present
cells (Ms > 0), of the whole grid or of one z-layer.
"""
from __future__ import annotations

import math

import numpy as np

from .constants import MU0
from .demag import h_demag
from .fields import Problem, _free_z_faces, _shift, cubic_axes, h_anisotropy, h_dmi, h_exchange, h_zeeman
from .llg import cross, dot

TERMS = ("exchange", "dmi", "anisotropy", "zeeman", "demag")


def energy(m, p: Problem, K_hat=None, terms=TERMS) -> dict:
    V = p.d[0] * p.d[1] * p.d[2]
    out = {}
    if "exchange" in terms:
        out["exchange"] = math.fsum((-0.5 * MU0 * p.Ms * dot(m, h_exchange(m, p)) * V).ravel())
    if "dmi" in terms:
        out["dmi"] = math.fsum((-0.5 * MU0 * p.Ms * dot(m, h_dmi(m, p)) * V).ravel())
    if "anisotropy" in terms:
        out["anisotropy"] = math.fsum((-p.Ku1 * dot(m, p.u) ** 2 * p.present * V).ravel())
    if "zeeman" in terms:
        out["zeeman"] = math.fsum((-MU0 * p.Ms * dot(m, h_zeeman(p)) * V).ravel())
    if "demag" in terms and K_hat is not None:
        out["demag"] = math.fsum((-0.5 * MU0 * p.Ms * dot(m, h_demag(m, p, K_hat)) * V).ravel())
    pres = p.present
    if "cubic" in terms:
        c1, c2, c3 = cubic_axes(p)
        a, b, c = dot(m, c1), dot(m, c2), dot(m, c3)
        e = p.Kc1 * (a * a * b * b + b * b * c * c + c * c * a * a) + p.Kc2 * a * a * b * b * c * c
        out["cubic"] = math.fsum((e * pres * V).ravel())
    if "surface" in terms:
        out["surface"] = math.fsum((-p.Ks / p.d[2] * _free_z_faces(p) * m[2] ** 2 * pres * V).ravel())
    if "rkky" in terms and p.rkky is not None:
        k1, k2, J = p.rkky
        both = (p.Ms[k1] > 0) & (p.Ms[k2] > 0)
        out["rkky"] = math.fsum((-J / p.d[2] * np.where(both, dot(m[:, k1], m[:, k2]), 0.0) * V).ravel())
    if "magnetoelastic" in terms:
        s = p.strain
        e = p.B1 * (s[0] * m[0] ** 2 + s[1] * m[1] ** 2 + s[2] * m[2] ** 2) + \
            2 * p.B2 * (s[3] * m[0] * m[1] + s[4] * m[0] * m[2] + s[5] * m[1] * m[2])
        out["magnetoelastic"] = math.fsum((e * pres * V).ravel())
    out["total"] = math.fsum(out.values())
    return out


def _derivative(m, p: Problem, direction: int):
    per = bool(p.pbc[direction])
    h = p.d[direction]
    Ms_p = _shift(p.Ms, direction, +1, per)
    Ms_m = _shift(p.Ms, direction, -1, per)
    mp = _shift(m, direction, +1, per)
    mm = _shift(m, direction, -1, per)
    has_p, has_m = Ms_p > 0, Ms_m > 0
    both = has_p & has_m
    g = np.where(both, (mp - mm) / (2 * h),
                 np.where(has_p, (mp - m) / h, np.where(has_m, (m - mm) / h, 0.0)))
    return g


def topological_charge(m, p: Problem) -> float:
    gx = _derivative(m, p, 0)
    gy = _derivative(m, p, 1)
    q = dot(m, cross(gx, gy)) * p.d[0] * p.d[1] / (4 * math.pi)
    q = np.where(p.present, q, 0.0)
    per_layer = [math.fsum(q[k].ravel()) for k in range(q.shape[0])]
    return math.fsum(per_layer) / len(per_layer)


def topological_charge_bl(m, p: Problem) -> float:
    """Berg-Luescher: sum of signed solid angles of the two triangles of every
    plaquette of four present cells, / 4 pi, averaged over layers."""
    nz, ny, nx = p.shape
    tot = []
    for k in range(nz):
        s = []
        for j in range(ny - 1):
            for i in range(nx - 1):
                cells = [(j, i), (j, i + 1), (j + 1, i + 1), (j + 1, i)]
                if not all(p.Ms[k, a, b] > 0 for a, b in cells):
                    continue
                v = [m[:, k, a, b] for a, b in cells]
                for tri in ((v[0], v[1], v[2]), (v[0], v[2], v[3])):
                    a, b, c = tri
                    num = np.dot(a, np.cross(b, c))
                    den = 1.0 + np.dot(a, b) + np.dot(b, c) + np.dot(c, a)
                    s.append(2.0 * math.atan2(num, den))
        tot.append(math.fsum(s) / (4 * math.pi))
    return sum(tot) / len(tot)


def mean_magnetisation(m, p: Problem, layer=None) -> np.ndarray:
    """<m> over the present cells (of z-layer ``layer`` when given)."""
    pres = p.present if layer is None else p.present[layer:layer + 1]
    mm = m if layer is None else m[:, layer:layer + 1]
    n = int(pres.sum())
    if n == 0:
        return np.zeros(3)
    return np.array([math.fsum(mm[c][pres].ravel()) / n for c in range(3)])
