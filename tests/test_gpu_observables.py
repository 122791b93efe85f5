"""GPU parity of the FP64-compensated observables (energy per term and
topological charge) and of the library's bookkeeping: checkpoint/resume,
determinism, host-side fault injection."""
import math

import numpy as np
import pytest

import workloads as W
from gpu_util import make_ctx, need_gpu, oracle_problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [64, 32])
def test_energy_matches_oracle(prec):
    mm = need_gpu()
    from oracle.demag import demag_spectrum
    from oracle.observables import energy
    grid = W.Grid(24, 16, 3, 2e-9, 2e-9, 2e-9)
    mat = W.with_cells(W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.1, Ku1=8e5, u=(0, 0, 1), D=3e-3),
                       W.random_material_cells(grid, 2))
    B = (0.01, 0.0, 0.1)
    ctx = make_ctx(mm, grid, mat, precision=prec, demag=True, B=B)
    try:
        m = W.random_m(grid, seed=4)
        mm.mm_set_m(ctx, 0, m)
        m_dev = mm.mm_get_m(ctx, 0, m.shape)
        p = oracle_problem(grid, mat, B)
        E = mm.mm_energy(ctx)
        ref = energy(m_dev, p, demag_spectrum(p.shape, p.d))
        names = ["exchange", "dmi", "anisotropy", "zeeman", "demag"]
        scale = max(abs(v) for v in ref.values())
        tol = 1e-12 if prec == 64 else 2e-6
        for q, nmn in enumerate(names):
            assert abs(E[q] - ref[nmn]) <= tol * scale, (nmn, E[q], ref[nmn])
        assert abs(E[5] - ref["total"]) <= tol * scale
    finally:
        mm.mm_destroy(ctx)


def _skyrmion(grid, R, w):
    x = (np.arange(grid.nx) - grid.nx / 2 + 0.5) * grid.dx
    y = (np.arange(grid.ny) - grid.ny / 2 + 0.5) * grid.dy
    X, Y = np.meshgrid(x, y)
    r = np.hypot(X, Y)
    th = 2 * np.arctan(np.exp(-(r - R) / w))
    ph = np.arctan2(Y, X)
    m = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    return np.broadcast_to(m[:, None], (3, grid.nz, grid.ny, grid.nx)).copy()


@pytest.mark.parametrize("prec", [64, 32])
def test_topological_charge_matches_oracle(prec):
    mm = need_gpu()
    from oracle.observables import topological_charge
    grid = W.Grid(96, 80, 2, 1e-9, 1e-9, 1e-9)
    mat = W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.1)
    ctx = make_ctx(mm, grid, mat, precision=prec, demag=False)
    try:
        m = _skyrmion(grid, 12e-9, 3e-9)
        mm.mm_set_m(ctx, 0, m)
        m_dev = mm.mm_get_m(ctx, 0, m.shape)
        p = oracle_problem(grid, mat)
        Q = mm.mm_topo_charge(ctx, 0, -1)
        Qo = topological_charge(m_dev, p)
        assert abs(Q - Qo) < (1e-12 if prec == 64 else 1e-6)
        assert abs(Q + 1) < 0.02
        assert abs(mm.mm_topo_charge(ctx, 0, 1) - Qo) < (1e-12 if prec == 64 else 1e-6)
    finally:
        mm.mm_destroy(ctx)


def test_checkpoint_resume_is_bit_exact():
    mm = need_gpu()
    grid = W.Grid(32, 16, 2, 2e-9, 2e-9, 2e-9)
    mat = W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.1, Ku1=8e5, u=(0, 0, 1), D=3e-3)
    m0 = W.random_m(grid, seed=1)
    a = make_ctx(mm, grid, mat, precision=32, demag=True)
    b = make_ctx(mm, grid, mat, precision=32, demag=True)
    try:
        mm.mm_set_m(a, 0, m0)
        mm.mm_step(a, 20)
        blob = mm.mm_get_state(a)
        mm.mm_step(a, 20)
        ma = mm.mm_get_m(a, 0, m0.shape)
        mm.mm_set_state(b, blob)
        mm.mm_step(b, 20)
        mb = mm.mm_get_m(b, 0, m0.shape)
        assert np.array_equal(ma, mb)
        assert mm.mm_get_time(a) == mm.mm_get_time(b)
    finally:
        mm.mm_destroy(a)
        mm.mm_destroy(b)


def test_two_identical_runs_are_bit_identical():
    """Catches shared-memory races that show up as nondeterminism."""
    mm = need_gpu()
    grid = W.Grid(48, 40, 4, 2e-9, 2e-9, 2e-9)
    mat = W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.1, Ku1=8e5, u=(0, 0, 1), D=3e-3)
    outs = []
    for _ in range(2):
        c = make_ctx(mm, grid, mat, precision=32, demag=True)
        try:
            mm.mm_set_m(c, 0, W.random_m(grid, seed=8))
            mm.mm_step(c, 15)
            outs.append(mm.mm_get_m(c, 0, (3, grid.nz, grid.ny, grid.nx)))
        finally:
            mm.mm_destroy(c)
    assert np.array_equal(outs[0], outs[1])


def test_fault_injection_leaves_context_usable():
    mm = need_gpu()
    grid = W.Grid(16, 8, 1, 2e-9, 2e-9, 1e-9)
    mat = W.Material(Ms=8e5, A=1.3e-11, alpha=0.02)
    c = make_ctx(mm, grid, mat, precision=32, demag=True)
    try:
        m0 = W.random_m(grid, seed=2)
        mm.mm_set_m(c, 0, m0)
        mm.mm_debug_inject(c, 2)            # NaN in the state
        with pytest.raises(mm.MMError) as e:
            mm.mm_step(c, 5)
        assert e.value.status in (mm.MM_ERR_NONFINITE, mm.MM_ERR_DT_UNDERFLOW)
        mm.mm_set_m(c, 0, m0)               # recover
        mm.mm_step(c, 5)
        mm.mm_debug_inject(c, 3)            # forced underflow
        with pytest.raises(mm.MMError) as e:
            mm.mm_step(c, 5)
        assert e.value.status == mm.MM_ERR_DT_UNDERFLOW
        mm.mm_debug_inject(c, 1)            # allocation failure on the next allocation
        with pytest.raises(mm.MMError) as e:
            mm.mm_set_field(c, 0, (0, 0, 0.1), np.zeros(3 * grid.n))
        assert e.value.status == mm.MM_ERR_OOM
    finally:
        mm.mm_destroy(c)


@pytest.mark.parametrize("prec", [64, 32])
def test_mean_magnetisation_matches_oracle(prec):
    """<m> over the present cells, whole grid and per layer, on a grid with
    holes; the oracle averages the host input normalised in FP64."""
    mm = need_gpu()
    from oracle.observables import mean_magnetisation
    grid = W.Grid(37, 21, 3, 2e-9, 2e-9, 2e-9)
    mat = W.with_cells(W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.1, Ku1=8e5, u=(0, 0, 1), D=3e-3),
                       W.random_material_cells(grid, 5))
    ctx = make_ctx(mm, grid, mat, precision=prec, demag=False)
    try:
        m = W.random_m(grid, seed=6)
        m = m + np.array([0.3, -0.2, 0.5])[:, None, None, None]
        mm.mm_set_m(ctx, 0, m)
        m_unit = m / np.linalg.norm(m, axis=0, keepdims=True)
        p = oracle_problem(grid, mat)
        tol = 1e-13 if prec == 64 else 1e-6
        got = mm.mm_mean_m(ctx, 0, -1)
        assert np.abs(got - mean_magnetisation(m_unit, p)).max() < tol
        for k in range(grid.nz):
            assert np.abs(mm.mm_mean_m(ctx, 0, k) - mean_magnetisation(m_unit, p, k)).max() < tol
        with pytest.raises(mm.MMError):
            mm.mm_mean_m(ctx, 0, grid.nz)
    finally:
        mm.mm_destroy(ctx)


def test_mean_magnetisation_of_batched_replicas():
    mm = need_gpu()
    from oracle.observables import mean_magnetisation
    sizes = [(32, 32), (17, 9), (48, 48), (32, 32)]
    mat = W.Material(Ms=1.1e6, A=2e-11, alpha=0.01, Ku1=9e5, u=(0.0, 0.0, 1.0))
    M = mm.Material(mat.Ms, mat.A, mat.alpha, mat.Ku1, mat.u, mat.D)
    cfg = mm.make_config(precision=32, integrator=mm.MM_HEUN, demag=mm.MM_DEMAG_OFF, dt=1e-14)
    ctx = mm.mm_create_batch([mm.make_grid(nx, ny, 1, 2e-9, 2e-9, 1e-9) for nx, ny in sizes], M.s, cfg, None)
    try:
        want = []
        for r, (nx, ny) in enumerate(sizes):
            grid = W.Grid(nx, ny, 1, 2e-9, 2e-9, 1e-9)
            m = W.random_m(grid, seed=10 + r) + np.array([0.1 * r, 0.4, -0.3])[:, None, None, None]
            mm.mm_set_m(ctx, r, m)
            m_unit = m / np.linalg.norm(m, axis=0, keepdims=True)
            want.append(mean_magnetisation(m_unit, oracle_problem(grid, mat)))
        for r in range(len(sizes)):
            assert np.abs(mm.mm_mean_m(ctx, r, -1) - want[r]).max() < 1e-6
            assert np.abs(mm.mm_mean_m(ctx, r, 0) - want[r]).max() < 1e-6
    finally:
        mm.mm_destroy(ctx)
