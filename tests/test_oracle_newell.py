"""Pins of the oracle's Newell demagnetising tensor against facts that do not
depend on the oracle: closed-form special values, the Laplace identity,
the point-dipole limit, parity, and an independent quadrature."""
import math

import numpy as np
import pytest

import oracle
from oracle.demag import newell_analytic, newell_at, newell_octant, newell_quadrature
from prism import prism_factor as _aharoni_prism_factor

CELLS = [(1.0, 1.0, 1.0), (2.0, 2.0, 1.0), (3.90625, 3.90625, 3.0), (1.0, 1.0, 2.0), (1.0, 3.0, 0.5)]


@pytest.mark.parametrize("cell", CELLS)
def test_self_term_trace_is_one(cell):
    N = newell_at([(0, 0, 0)], cell)[0]
    assert abs(N[0] + N[1] + N[2] - 1.0) < 1e-13
    assert np.all(np.abs(N[3:]) < 1e-14)
    assert np.all(N[:3] > 0)


def test_cube_self_term_is_one_third():
    N = newell_at([(0, 0, 0)], (1.0, 1.0, 1.0))[0]
    assert np.allclose(N[:3], 1.0 / 3.0, atol=1e-14, rtol=0)


def test_flat_cell_self_term_ordering():
    # a flat cell has its largest factor along its shortest edge
    N = newell_at([(0, 0, 0)], (2.0, 2.0, 1.0))[0]
    assert N[2] > N[0] and abs(N[0] - N[1]) < 1e-14


@pytest.mark.parametrize("cell", CELLS)
def test_trace_vanishes_away_from_the_source(cell):
    # Laplace: the cell-averaged tensor of a distinct cell is traceless
    rng = np.random.default_rng(0)
    ijk = np.concatenate([
        [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 1, 1), (2, 0, 0), (2, 1, 0)],
        rng.integers(-40, 41, size=(60, 3)),
    ])
    ijk = ijk[np.any(ijk != 0, axis=1)]
    N = newell_at(ijk, cell)
    # relative to the largest element (diagonals all vanish along (1,1,1))
    scale = np.abs(N).max(axis=1)
    assert np.all(np.abs(N[:, 0] + N[:, 1] + N[:, 2]) <= 1e-11 * scale + 1e-15)


@pytest.mark.parametrize("cell", CELLS)
def test_closed_form_agrees_with_independent_quadrature(cell):
    """Two independent evaluations of the same integral: Newell's closed form
    and tent-weighted Gauss-Legendre of the point-dipole kernel."""
    s = max(cell)
    for dirv in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0.3, 0.7, 0.2), (1, 1, 1)]:
        for R in (2.0, 2.2):
            v = np.array(dirv, float) / np.linalg.norm(dirv) * R * s
            a = newell_analytic(*v, cell)
            q = newell_quadrature(*v, cell, 24)
            assert np.max(np.abs(a - q)) <= 1e-10 * np.max(np.abs(q)), (cell, dirv, R)


@pytest.mark.parametrize("band,nq", [(2.0, 16), (3.0, 12), (8.0, 6), (32.0, 4), (128.0, 3)])
def test_quadrature_converged_at_each_band_edge(band, nq):
    cell = (2.0, 2.0, 1.0)
    for dirv in [(1, 0, 0), (1, 1, 0), (0.3, 0.7, 0.2)]:
        v = np.array(dirv, float) / np.linalg.norm(dirv) * (band * 1.0001) * max(cell)
        lo = newell_quadrature(*v, cell, nq)
        hi = newell_quadrature(*v, cell, 24)
        assert np.max(np.abs(lo - hi)) <= 8e-14 * np.max(np.abs(hi))


def test_point_dipole_limit():
    """|R| >> cell: N_ab -> -(V/4pi|R|^3)(3 r_a r_b - delta_ab), error O((h/R)^2)."""
    cell = (1.0, 1.0, 1.0)
    V = 1.0
    for dirv in [(1, 0, 0), (1, 2, 0), (3, -1, 2)]:
        errs = []
        for R in (20, 40, 80):
            ijk = np.round(np.array(dirv, float) / np.linalg.norm(dirv) * R).astype(int)
            r = ijk.astype(float)
            rn = np.linalg.norm(r)
            u = r / rn
            dip = -(V / (4 * math.pi * rn ** 3)) * np.array(
                [3 * u[0] * u[0] - 1, 3 * u[1] * u[1] - 1, 3 * u[2] * u[2] - 1,
                 3 * u[0] * u[1], 3 * u[0] * u[2], 3 * u[1] * u[2]])
            N = newell_at([ijk], cell)[0]
            errs.append(np.max(np.abs(N - dip)) / np.max(np.abs(dip)))
        assert errs[0] < 5e-3
        # second-order decay: halving h/R divides the error by ~4
        assert errs[1] < errs[0] / 3.0 and errs[2] < errs[1] / 3.0


def test_parity_of_components():
    cell = (2.0, 2.0, 1.0)
    base = np.array([(1, 2, 1), (3, 1, 2), (5, 7, 0), (12, 3, 4)])
    N0 = newell_at(base, cell)
    for sx in (1, -1):
        for sy in (1, -1):
            for sz in (1, -1):
                Nm = newell_at(base * np.array([sx, sy, sz]), cell)
                exp = N0.copy()
                exp[:, 3] *= sx * sy
                exp[:, 4] *= sx * sz
                exp[:, 5] *= sy * sz
                assert np.allclose(Nm, exp, rtol=1e-13, atol=1e-18)


def test_octant_matches_pointwise():
    shape = (3, 5, 6)
    cell = (2.0, 1.5, 1.0)
    O = newell_octant(shape, cell)
    ijk = [(i, j, k) for k in range(3) for j in range(5) for i in range(6)]
    P = newell_at(ijk, cell)
    assert np.allclose(O.reshape(6, -1).T, P, rtol=0, atol=0)


def test_newell_auxiliary_symmetries():
    # f is even in every argument, g odd in x and y and even in z; on the
    # x axis f reduces to x^3/3 (its asinh/atan terms vanish there)
    assert abs(oracle.newell_f(2.0, 0.0, 0.0) - 8.0 / 3.0) < 1e-14
    for x, y, z in [(0.3, 1.2, 0.7), (2.0, 0.5, 1.5)]:
        f = oracle.newell_f(x, y, z)
        g = oracle.newell_g(x, y, z)
        assert oracle.newell_f(-x, y, -z) == f
        assert oracle.newell_g(-x, y, z) == -g and oracle.newell_g(x, -y, z) == -g
        assert oracle.newell_g(x, y, -z) == g


@pytest.mark.parametrize("cell", CELLS + [(4e-9, 2e-9, 1e-9)])
def test_self_term_equals_the_prism_demagnetising_factors(cell):
    N = newell_at([(0, 0, 0)], cell)[0]
    a, b, c = (v / 2 for v in cell)
    ref = [_aharoni_prism_factor(b, c, a), _aharoni_prism_factor(c, a, b), _aharoni_prism_factor(a, b, c)]
    assert np.allclose(N[:3], ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("shape,cell", [((2, 8, 12), (1.0, 1.0, 1.0)),
                                        ((3, 5, 40), (2.0, 3.0, 1.5)),
                                        ((1, 64, 64), (2e-9, 2e-9, 1e-9))])
def test_block_average_equals_the_prism_demagnetising_factors(shape, cell):
    """A block of cells magnetised uniformly is one prism: the mean over all
    cell pairs of the tensor at their displacement is the prism's factor.
    The sum runs over displacements up to 63 cells, so the closed form and
    every quadrature band of the far field below 128 cells enter."""
    nz, ny, nx = shape
    N = newell_octant(shape, cell)

    def mult(n):                       # ordered pairs at displacement |u| along one axis
        m = 2.0 * (n - np.arange(n))
        m[0] = n
        return m

    w = mult(nz)[:, None, None] * mult(ny)[None, :, None] * mult(nx)[None, None, :]
    mean = [float((N[comp] * w).sum()) / (nx * ny * nz) for comp in range(3)]
    a, b, c = nx * cell[0] / 2, ny * cell[1] / 2, nz * cell[2] / 2
    ref = [_aharoni_prism_factor(b, c, a), _aharoni_prism_factor(c, a, b), _aharoni_prism_factor(a, b, c)]
    assert np.allclose(mean, ref, rtol=1e-12, atol=1e-14)


def _asymptotic_newell():
    """Far-field expansion of the cell-averaged tensor, written from the
    mathematics alone: N_ab(R) = -(V / 4 pi) < d_a d_b 1/|R + w| >, with w the
    difference of two independent uniform points of the cell (per axis a
    triangular variable: <w^2> = h^2 / 6, <w^4> = h^4 / 15), expanded to
    fourth order:
      f + sum_d h_d^2 / 12 d_d^2 f + sum_d h_d^4 / 360 d_d^4 f
        + sum_{d<e} h_d^2 h_e^2 / 144 d_d^2 d_e^2 f,   f = d_a d_b 1/R.
    The omitted sixth-order terms are O((h / R)^6) relative."""
    sp = pytest.importorskip("sympy")
    X, Y, Z = sp.symbols("X Y Z", real=True)
    g = 1 / sp.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    ax = [X, Y, Z]
    fns = []
    for a, b in [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]:
        f = sp.diff(g, ax[a], ax[b])
        exprs = [f] + [sp.diff(f, ax[d], 2) for d in range(3)] + [sp.diff(f, ax[d], 4) for d in range(3)] + \
                [sp.diff(f, ax[d], 2, ax[e], 2) for d, e in [(0, 1), (0, 2), (1, 2)]]
        fns.append(sp.lambdify((X, Y, Z), exprs, "numpy"))

    def at(ijk, h):
        R = np.asarray(ijk, float) * np.asarray(h, float)
        V = h[0] * h[1] * h[2]
        out = []
        for fn in fns:
            v = fn(*R)
            s = v[0] + sum(h[d] ** 2 / 12 * v[1 + d] for d in range(3)) + \
                sum(h[d] ** 4 / 360 * v[4 + d] for d in range(3))
            s += h[0] ** 2 * h[1] ** 2 / 144 * v[7] + h[0] ** 2 * h[2] ** 2 / 144 * v[8] + \
                h[1] ** 2 * h[2] ** 2 / 144 * v[9]
            out.append(-V / (4 * math.pi) * s)
        return np.array(out)
    return at


@pytest.mark.parametrize("cell", [(2.0, 2.0, 1.0), (3.0, 3.0, 3.0), (3.90625, 3.90625, 3.0)])
def test_every_band_agrees_with_the_fourth_order_far_field_expansion(cell):
    """Every distance band of the tensor evaluation -- the closed form near
    the source and each Gauss quadrature order further out, the 3-point band
    beyond 128 cells included -- against the fourth-order expansion of the
    cell average of the point-dipole kernel: the difference must shrink like
    (h / R)^6 down to rounding, at the displacements the demag grids use
    (up to 511 x 511 x 63 cells)."""
    asym = _asymptotic_newell()
    hmax = max(cell)
    dirs = [(1, 0, 0), (1, 1, 0), (0.3, 0.7, 0.2), (2, -1, 3), (-5, 4, 1)]
    for R in (10, 16, 24, 40, 64, 100, 130, 200, 400, 700):
        for dv in dirs:
            u = np.array(dv, float) / np.linalg.norm(dv)
            ijk = np.round(u * R).astype(int)
            ijk = np.clip(ijk, -511, 511)
            N = newell_at([ijk], cell)[0]
            A = asym(ijk, cell)
            rel = np.max(np.abs(N - A)) / np.max(np.abs(A))
            dist = np.linalg.norm(ijk * np.asarray(cell)) / hmax
            assert rel <= (1.0 / dist) ** 6 + 1e-13, (cell, tuple(ijk), rel)
