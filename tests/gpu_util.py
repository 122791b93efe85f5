"""Helpers shared by the GPU parity tests: build a libmm context and the
oracle problem for the same seeded workload."""
import numpy as np
import pytest

import workloads as W

TERMS = {"exchange": 1, "dmi": 2, "anisotropy": 4, "zeeman": 8, "demag": 16, "thermal": 32, "cubic": 64,
         "surface": 128, "rkky": 256, "magnetoelastic": 512}


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_15253_gb300 as mm
    mm.load()
    return mm


def make_ctx(mm, grid: W.Grid, mat: W.Material, precision=64, integrator=None, demag=True, terms=0,
             dt=1e-14, rtol=1e-6, T=0.0, seed=0, B=(0.0, 0.0, 0.0), B_cell=None):
    integ = {None: mm.MM_RK45, "rk45": mm.MM_RK45, "rk4": mm.MM_RK4, "heun": mm.MM_HEUN, "dm": mm.MM_DM,
             "dma": mm.MM_DM_ADAPTIVE}[integrator]
    g = mm.make_grid(grid.nx, grid.ny, grid.nz, grid.dx, grid.dy, grid.dz, grid.pbc)
    m = mm.Material(mat.Ms, mat.A, mat.alpha, mat.Ku1, mat.u, mat.D, cells=mat.cell, Db=mat.Db, Kc1=mat.Kc1,
                    Kc2=mat.Kc2, c1=mat.c1, c2=mat.c2, Ks=mat.Ks, B1=mat.B1, B2=mat.B2)
    cfg = mm.make_config(precision=precision, integrator=integ,
                         demag=mm.MM_DEMAG_EXACT if demag else mm.MM_DEMAG_OFF,
                         terms=terms, dt=dt, rtol=rtol, T=T, seed=seed)
    ctx = mm.mm_create(g, m.s, cfg)
    ctx._mat = m  # keep per-cell arrays alive
    if any(B) or B_cell is not None:
        mm.mm_set_field(ctx, 0, B, B_cell)
    return ctx


def oracle_problem(grid, mat, B=(0.0, 0.0, 0.0)):
    from oracle.fields import Problem
    return Problem.from_workload(grid, mat, B_ext=B)


def rel_err(a, b):
    scale = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / scale)
