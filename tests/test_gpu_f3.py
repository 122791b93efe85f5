"""GPU parity of bulk DMI and the periodic (image-sum) demag field against
the FP64 oracle (Methods, "Physics and discretization").

Tolerances as for the other field terms: FP64 1e-11, FP32 2e-6 (local) and
5e-6 (demag) relative to the largest |H|; whole steps 1e-11 / 1e-5."""
import numpy as np
import pytest

import workloads as W
from gpu_util import TERMS, make_ctx, need_gpu, oracle_problem, rel_err

pytestmark = pytest.mark.gpu

BULK_GRIDS = [
    W.Grid(17, 9, 2, 2e-9, 3e-9, 1.5e-9),
    W.Grid(8, 8, 1, 2e-9, 2e-9, 1e-9),
    W.Grid(16, 12, 3, 2e-9, 2e-9, 2e-9),
    W.Grid(1, 1, 1, 2e-9, 2e-9, 2e-9),
    W.Grid(12, 7, 3, 2e-9, 2e-9, 2e-9, (1, 1, 1)),
]


def _mat(grid, seed, cells, D=1.5e-3, Db=-2.5e-3):
    mat = W.Material(Ms=6e5, A=1.3e-11, alpha=0.1, Ku1=4e5, u=(0.3, 0.2, 0.9), D=D, Db=Db)
    if cells:
        mat = W.with_cells(mat, W.random_material_cells(grid, seed))
    return mat


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("gi", range(len(BULK_GRIDS)))
@pytest.mark.parametrize("cells", [False, True])
@pytest.mark.parametrize("D", [0.0, 1.5e-3])
def test_bulk_dmi_matches_oracle(prec, gi, cells, D):
    """Exchange and DMI fields with bulk DMI (alone and with interfacial
    DMI): the bulk face condition enters both through the ghost values."""
    mm = need_gpu()
    from oracle.constants import MU0
    from oracle.fields import h_dmi, h_exchange
    grid = BULK_GRIDS[gi]
    mat = _mat(grid, gi, cells, D=D)
    ctx = make_ctx(mm, grid, mat, precision=prec, demag=False)
    try:
        m = W.random_m(grid, seed=gi + 21)
        mm.mm_set_m(ctx, 0, m)
        m_dev = mm.mm_get_m(ctx, 0, m.shape)
        p = oracle_problem(grid, mat)
        tol = 1e-11 if prec == 64 else 2e-6
        hmin = min(grid.dx, grid.dy, grid.dz)
        coef = {"exchange": 2 * mat.A / (MU0 * mat.Ms * hmin ** 2),
                "dmi": 2 * (abs(mat.D) + abs(mat.Db)) / (MU0 * mat.Ms * hmin)}
        for name, fn in (("exchange", lambda: h_exchange(m_dev, p)), ("dmi", lambda: h_dmi(m_dev, p))):
            H = mm.mm_get_heff(ctx, 0, m.shape, TERMS[name])
            ref = np.where(p.present, fn(), 0.0)
            scale = max(np.abs(ref).max(), coef[name])
            assert np.abs(H - ref).max() <= tol * scale, (name, np.abs(H - ref).max() / scale)
    finally:
        mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", [64, 32])
def test_bulk_dmi_steps_match_oracle(prec):
    """RK45 replay with bulk DMI, exchange, anisotropy and demag on a film
    whose width is a multiple of four (the vectorised FP32 field kernel)."""
    mm = need_gpu()
    from oracle.llg import Solver
    grid = W.Grid(24, 16, 2, 2e-9, 2e-9, 2e-9)
    mat = W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.1, Ku1=6e5, u=(0, 0, 1), Db=3e-3)
    m0 = W.random_m(grid, seed=31)
    o = Solver(oracle_problem(grid, mat), m0, dt=1e-14, rtol=1e-6)
    dts = [o.rk45_step() for _ in range(20)]
    ctx = make_ctx(mm, grid, mat, precision=prec, demag=True, dt=1e-14)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_step_dt(ctx, dts)
        err = np.abs(mm.mm_get_m(ctx, 0, m0.shape) - o.m).max()
        assert err <= (1e-11 if prec == 64 else 1e-5), err
    finally:
        mm.mm_destroy(ctx)


PBC_GRIDS = [
    W.Grid(32, 16, 1, 2e-9, 2e-9, 1e-9, (3, 2, 0)),
    W.Grid(12, 10, 4, 2e-9, 3e-9, 2e-9, (1, 0, 2)),
    W.Grid(64, 64, 1, 3e-9, 3e-9, 2e-9, (6, 6, 0)),
    W.Grid(20, 6, 3, 2e-9, 2e-9, 2e-9, (0, 5, 0)),
    W.Grid(48, 40, 8, 2e-9, 2e-9, 2e-9, (2, 2, 0)),
]


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("gi", range(len(PBC_GRIDS)))
def test_periodic_demag_matches_oracle(prec, gi):
    mm = need_gpu()
    from oracle.demag import demag_spectrum, h_demag
    grid = PBC_GRIDS[gi]
    mat = _mat(grid, gi, cells=(gi % 2 == 1), D=0.0, Db=0.0)
    ctx = make_ctx(mm, grid, mat, precision=prec, demag=True)
    try:
        m = W.random_m(grid, seed=40 + gi)
        mm.mm_set_m(ctx, 0, m)
        m_dev = mm.mm_get_m(ctx, 0, m.shape)
        p = oracle_problem(grid, mat)
        ref = np.where(p.present, h_demag(m_dev, p, demag_spectrum(p.shape, p.d, images=grid.pbc)), 0.0)
        H = mm.mm_get_heff(ctx, 0, m.shape, TERMS["demag"])
        tol = 1e-11 if prec == 64 else 5e-6
        assert rel_err(H, ref) < tol, rel_err(H, ref)
    finally:
        mm.mm_destroy(ctx)


def test_periodic_film_approaches_the_slab():
    """128 x 128 film periodic in x and y with 32 images per side: uniform
    m_z gives H_z within 2e-3 of -Ms (the infinite slab)."""
    mm = need_gpu()
    grid = W.Grid(128, 128, 1, 4e-9, 4e-9, 1e-9, (32, 32, 0))
    mat = W.Material(Ms=8e5, A=1.3e-11, alpha=0.02)
    ctx = make_ctx(mm, grid, mat, precision=32, demag=True)
    try:
        m = np.zeros((3,) + grid.shape)
        m[2] = 1.0
        mm.mm_set_m(ctx, 0, m)
        H = mm.mm_get_heff(ctx, 0, m.shape, TERMS["demag"])
        assert np.abs(H[2] / 8e5 + 1).max() < 2e-3
        assert np.abs(H[:2] / 8e5).max() < 2e-3
    finally:
        mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", [64, 32])
def test_periodic_dm_steps_match_oracle(prec):
    """Depondt-Mertens steps of a periodic film with exchange, interfacial and
    bulk DMI, anisotropy and image-sum demag."""
    mm = need_gpu()
    from oracle.llg import Solver
    grid = W.Grid(24, 20, 1, 2e-9, 2e-9, 1e-9, (2, 3, 0))
    mat = W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.1, Ku1=8e5, u=(0, 0, 1), D=2e-3, Db=1e-3)
    m0 = W.random_m(grid, seed=33)
    o = Solver(oracle_problem(grid, mat), m0, dt=1e-14)
    for _ in range(25):
        o.dm_step()
    ctx = make_ctx(mm, grid, mat, precision=prec, integrator="dm", demag=True, dt=1e-14)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_step(ctx, 25)
        err = np.abs(mm.mm_get_m(ctx, 0, m0.shape) - o.m).max()
        assert err <= (1e-11 if prec == 64 else 1e-5), err
    finally:
        mm.mm_destroy(ctx)


def test_surrogate_refuses_periodic_grids():
    mm = need_gpu()
    grid = W.Grid(64, 64, 1, 2e-9, 2e-9, 1e-9, (2, 2, 0))
    ctx = make_ctx(mm, grid, W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.3), precision=32, demag=True)
    try:
        with pytest.raises(mm.MMError):
            mm.mm_surrogate_set(ctx, 5, 1e-3)
    finally:
        mm.mm_destroy(ctx)
