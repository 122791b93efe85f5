"""GPU parity of the further local terms (Methods, "Physics and
discretization": cubic and surface anisotropy, RKKY interlayer exchange,
magnetoelastic anisotropy) against the FP64 oracle: fields, energies, whole
steps in the single-instance and replica-batched engines.

Tolerances: fields FP64 1e-11, FP32 2e-6 relative to the term's scale;
energies FP64 1e-12, FP32 2e-6 relative; steps 1e-11 / 1e-5."""
import numpy as np
import pytest

import workloads as W
from gpu_util import TERMS, make_ctx, need_gpu, oracle_problem

pytestmark = pytest.mark.gpu

GRIDS = [
    W.Grid(16, 9, 3, 2e-9, 3e-9, 1.5e-9),
    W.Grid(8, 8, 1, 2e-9, 2e-9, 1e-9),
    W.Grid(24, 12, 4, 2e-9, 2e-9, 2e-9),
]

MAT = dict(Ms=6e5, A=1.3e-11, alpha=0.1, Ku1=2e5, u=(0.0, 0.0, 1.0), Kc1=4.5e4, Kc2=-2e4, c1=(1.0, 0.4, -0.2),
           c2=(-0.3, 1.0, 0.5), Ks=6e-4, B1=-7e6, B2=4e6)
STRAIN = (1.2e-3, -0.8e-3, 2.0e-3, 0.5e-3, -0.3e-3, 0.7e-3)


def _setup(mm, grid, prec, cells, per_cell_strain, integrator=None, demag=False, dt=1e-14):
    mat = W.Material(**MAT)
    if cells:
        mat = W.with_cells(mat, W.random_material_cells(grid, 5))
    ctx = make_ctx(mm, grid, mat, precision=prec, demag=demag, integrator=integrator, dt=dt)
    p = oracle_problem(grid, mat)
    if per_cell_strain:
        eps = np.random.default_rng(3).normal(scale=1e-3, size=(6,) + grid.shape)
        mm.mm_set_strain(ctx, eps_cell=eps)
        p.strain = eps
    else:
        mm.mm_set_strain(ctx, STRAIN)
        p.strain = np.broadcast_to(np.asarray(STRAIN)[:, None, None, None], (6,) + grid.shape).copy()
    if grid.nz >= 3:
        mm.mm_set_rkky(ctx, 0, grid.nz - 1, -8e-4)
        p.rkky = (0, grid.nz - 1, -8e-4)
    return ctx, mat, p


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("gi", range(len(GRIDS)))
@pytest.mark.parametrize("cells,per_cell", [(False, False), (True, True)])
def test_further_terms_match_oracle(prec, gi, cells, per_cell):
    mm = need_gpu()
    from oracle.constants import MU0
    from oracle.fields import h_cubic, h_magnetoelastic, h_rkky, h_surface
    grid = GRIDS[gi]
    ctx, mat, p = _setup(mm, grid, prec, cells, per_cell)
    try:
        m = W.random_m(grid, seed=gi + 50)
        mm.mm_set_m(ctx, 0, m)
        m_dev = mm.mm_get_m(ctx, 0, m.shape)
        tol = 1e-11 if prec == 64 else 2e-6
        scale = {"cubic": 2 * (abs(mat.Kc1) + abs(mat.Kc2)) / (MU0 * mat.Ms),
                 "surface": 4 * mat.Ks / (MU0 * mat.Ms * grid.dz),
                 "rkky": 8e-4 / (MU0 * mat.Ms * grid.dz),
                 "magnetoelastic": 2 * (abs(mat.B1) + abs(mat.B2)) * 3e-3 / (MU0 * mat.Ms)}
        fns = {"cubic": h_cubic, "surface": h_surface, "rkky": h_rkky, "magnetoelastic": h_magnetoelastic}
        for name, fn in fns.items():
            if name == "rkky" and grid.nz < 3:
                continue
            H = mm.mm_get_heff(ctx, 0, m.shape, TERMS[name])
            ref = np.where(p.present, fn(m_dev, p), 0.0)
            assert np.abs(ref).max() > 0, name
            assert np.abs(H - ref).max() <= tol * scale[name], (name, np.abs(H - ref).max() / scale[name])
    finally:
        mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", [64, 32])
def test_further_term_energies_match_oracle(prec):
    mm = need_gpu()
    from oracle.observables import energy
    grid = GRIDS[0]
    ctx, mat, p = _setup(mm, grid, prec, True, True)
    try:
        m = W.random_m(grid, seed=61)
        mm.mm_set_m(ctx, 0, m)
        m_dev = mm.mm_get_m(ctx, 0, m.shape)
        E = mm.mm_energy(ctx)
        ref = energy(m_dev, p, terms=("exchange", "anisotropy", "cubic", "surface", "rkky", "magnetoelastic"))
        tol = 1e-12 if prec == 64 else 2e-6
        for name, idx in (("cubic", mm.MM_E_CUBIC), ("surface", mm.MM_E_SURFACE), ("rkky", mm.MM_E_RKKY),
                          ("magnetoelastic", mm.MM_E_MEL)):
            assert abs(E[idx] - ref[name]) <= tol * abs(ref[name]), (name, E[idx], ref[name])
        parts = [E[i] for i in range(mm.MM_NENERGY) if i != mm.MM_E_TOTAL]
        assert abs(E[mm.MM_E_TOTAL] - sum(parts)) <= 1e-12 * sum(abs(v) for v in parts)
    finally:
        mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("integ", ["rk45", "dm"])
def test_steps_with_further_terms_match_oracle(prec, integ):
    """Whole steps with every term (exchange, anisotropies, RKKY across a
    spacer layer, magnetoelastic, demag)."""
    mm = need_gpu()
    from oracle.llg import Solver
    grid = W.Grid(20, 12, 4, 2e-9, 2e-9, 2e-9)
    ctx, mat, p = _setup(mm, grid, prec, False, False, integrator=integ, demag=True)
    terms = ("exchange", "anisotropy", "zeeman", "cubic", "surface", "rkky", "magnetoelastic", "demag")
    try:
        m0 = W.random_m(grid, seed=62)
        o = Solver(p, m0, terms=terms, dt=1e-14, rtol=1e-6)
        mm.mm_set_m(ctx, 0, m0)
        if integ == "rk45":
            dts = [o.rk45_step() for _ in range(15)]
            mm.mm_step_dt(ctx, dts)
        else:
            for _ in range(25):
                o.dm_step()
            mm.mm_step(ctx, 25)
        err = np.abs(mm.mm_get_m(ctx, 0, m0.shape) - o.m).max()
        assert err <= (1e-11 if prec == 64 else 1e-5), err
    finally:
        mm.mm_destroy(ctx)


def test_batched_replicas_with_further_terms():
    """Replica-batched Depondt-Mertens films with cubic, surface and
    magnetoelastic anisotropy (uniform strain) against the oracle."""
    mm = need_gpu()
    from oracle.llg import Solver
    sizes = [(16, 16), (24, 8), (8, 8)]
    cell = (2e-9, 2e-9, 1e-9)
    M = mm.Material(**{k: v for k, v in MAT.items()})
    cfg = mm.make_config(precision=32, integrator=mm.MM_DM, demag=mm.MM_DEMAG_EXACT, dt=1e-14)
    ctx = mm.mm_create_batch([mm.make_grid(nx, ny, 1, *cell) for nx, ny in sizes], M.s, cfg, None)
    ctx._mat = M
    try:
        mm.mm_set_strain(ctx, STRAIN)
        m0 = []
        for r, (nx, ny) in enumerate(sizes):
            m0.append(W.random_m(W.Grid(nx, ny, 1, *cell), seed=70 + r))
            mm.mm_set_m(ctx, r, m0[-1])
        mm.mm_step(ctx, 20)
        terms = ("exchange", "anisotropy", "zeeman", "cubic", "surface", "magnetoelastic", "demag")
        for r, (nx, ny) in enumerate(sizes):
            g = W.Grid(nx, ny, 1, *cell)
            p = oracle_problem(g, W.Material(**MAT))
            p.strain = np.broadcast_to(np.asarray(STRAIN)[:, None, None, None], (6,) + g.shape).copy()
            o = Solver(p, m0[r], terms=terms, dt=1e-14)
            for _ in range(20):
                o.dm_step()
            err = np.abs(mm.mm_get_m(ctx, r, m0[r].shape) - o.m).max()
            assert err <= 1e-5, (r, err)
    finally:
        mm.mm_destroy(ctx)


def test_unused_terms_cost_nothing():
    """With all their parameters zero the further terms are dropped from the
    field kernels: the field equals the classic terms' field exactly."""
    mm = need_gpu()
    grid = GRIDS[0]
    mat = W.Material(Ms=6e5, A=1.3e-11, alpha=0.1, Ku1=2e5)
    ctx = make_ctx(mm, grid, mat, precision=64, demag=False)
    try:
        m = W.random_m(grid, seed=63)
        mm.mm_set_m(ctx, 0, m)
        for name in ("cubic", "surface", "rkky", "magnetoelastic"):
            assert np.abs(mm.mm_get_heff(ctx, 0, m.shape, TERMS[name])).max() == 0.0
        E = mm.mm_energy(ctx)
        assert E[mm.MM_E_CUBIC] == E[mm.MM_E_SURFACE] == E[mm.MM_E_RKKY] == E[mm.MM_E_MEL] == 0.0
    finally:
        mm.mm_destroy(ctx)
