"""GPU parity of the Depondt-Mertens rotation scheme (Methods, "Integrators"
and "Replica batching"): the single-instance integrator in FP64 and FP32
with every field term, spin torques and the thermal field, and the
replica-batched engine, against the oracle's dm_step.

Bar: max over cells of |m_gpu - m_oracle| <= 1e-11 (FP64), <= 1e-5 (FP32)
after the stated number of steps."""
import numpy as np
import pytest

import workloads as W
from gpu_util import make_ctx, need_gpu, oracle_problem
from test_gpu_integrate import CASES

pytestmark = pytest.mark.gpu


def _oracle(grid, mat, m, B=(0, 0, 0), **kw):
    from oracle.llg import Solver
    return Solver(oracle_problem(grid, mat, B), m, **kw)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_dm_matches_oracle(prec, ci):
    mm = need_gpu()
    name, grid, mat, B = CASES[ci]
    m0 = W.random_m(grid, seed=60 + ci)
    dt, n = 1e-14, 30
    o = _oracle(grid, mat, m0, B, dt=dt)
    for _ in range(n):
        o.dm_step(dt)
    ctx = make_ctx(mm, grid, mat, precision=prec, integrator="dm", demag=True, B=B, dt=dt)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_step(ctx, n)
        t, _, steps = mm.mm_get_time(ctx)
        assert steps == n and abs(t - n * dt) < 1e-25
        err = np.abs(mm.mm_get_m(ctx, 0, m0.shape) - o.m).max()
        assert err <= (1e-11 if prec == 64 else 1e-5), err
    finally:
        mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("torque", ["sot", "stt", "zl"])
def test_dm_thermal_with_torque_matches_oracle(prec, torque):
    mm = need_gpu()
    from oracle.llg import Torque, replica_seed
    grid = W.Grid(20, 12, 1, 2e-9, 2e-9, 1e-9)
    mat = W.Material(Ms=1.1e6, A=2e-11, alpha=0.01, Ku1=9e5, u=(0, 0, 1), D=1e-3)
    J = 2.0e11
    if torque == "sot":
        tq_o = Torque(kind="sot", J=J, p=(0, 1, 0), theta_SH=0.1, fl_ratio=0.2)
        tq_g = mm.make_torque(mm.MM_TORQUE_SOT, p=(0, 1, 0), theta_SH=0.1, fl_ratio=0.2)
    elif torque == "stt":
        tq_o = Torque(kind="stt", J=J, p=(0.2, 0, 1), P=0.6, Lambda=1.5, eps_prime=0.05)
        tq_g = mm.make_torque(mm.MM_TORQUE_STT, p=(0.2, 0, 1), P=0.6, Lambda=1.5, eps_prime=0.05)
    else:
        J = 5e12
        tq_o = Torque(kind="zl", J=J, P=0.5, xi=0.05, direction=(1, 0.5, 0))
        tq_g = mm.make_torque(mm.MM_TORQUE_ZL, P=0.5, xi=0.05, direction=(1, 0.5, 0))
    m0 = W.m_perp(grid, seed=3, tilt=0.3)
    seed = 11
    o = _oracle(grid, mat, m0, terms=("exchange", "dmi", "anisotropy", "demag"), torque=tq_o, T=300.0,
                seed=replica_seed(seed, 0), dt=1e-14)
    ctx = make_ctx(mm, grid, mat, precision=prec, integrator="dm", demag=True, dt=1e-14, T=300.0, seed=seed,
                   terms=1 | 2 | 4 | 16 | 32)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_set_torque(ctx, tq_g, [J])
        n = 60
        for _ in range(n):
            o.dm_step()
        mm.mm_step(ctx, n)
        err = np.abs(mm.mm_get_m(ctx, 0, m0.shape) - o.m).max()
        assert err <= (1e-11 if prec == 64 else 1e-5), err
    finally:
        mm.mm_destroy(ctx)


def test_dm_exact_rotation_at_large_steps_fp64():
    """alpha = 0, uniform applied field, no exchange: the rotation vector is
    constant and 0.7 rad steps are exact (the closed form is the rotation
    by the accumulated angle about the field)."""
    mm = need_gpu()
    from oracle.constants import GAMMA0, MU0
    grid = W.Grid(8, 4, 1, 2e-9, 2e-9, 2e-9)
    mat = W.Material(Ms=8e5, A=1e-11, alpha=0.0)
    b = np.array([0.3, -0.5, 0.8])
    b /= np.linalg.norm(b)
    H0 = 4e5
    w = GAMMA0 * MU0 * H0
    dt = 0.7 / w
    ctx = make_ctx(mm, grid, mat, precision=64, integrator="dm", demag=False, terms=8, B=tuple(MU0 * H0 * b), dt=dt)
    try:
        m0 = W.random_m(grid, seed=2)
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_step(ctx, 9)
        m = mm.mm_get_m(ctx, 0, m0.shape)
        a = 9 * 0.7
        bb = b[:, None, None, None]
        par = (m0 * bb).sum(axis=0, keepdims=True) * bb
        perp = m0 - par
        bxp = np.stack([bb[1] * perp[2] - bb[2] * perp[1], bb[2] * perp[0] - bb[0] * perp[2],
                        bb[0] * perp[1] - bb[1] * perp[0]])
        exp = par + np.cos(a) * perp + np.sin(a) * bxp
        assert np.abs(m - exp).max() < 1e-12
    finally:
        mm.mm_destroy(ctx)


def test_dm_fp32_keeps_unit_norm_over_long_runs():
    mm = need_gpu()
    name, grid, mat, B = CASES[0]
    ctx = make_ctx(mm, grid, mat, precision=32, integrator="dm", demag=True, B=B, dt=2e-14, T=300.0, seed=4,
                   terms=1 | 2 | 4 | 8 | 16 | 32)
    try:
        m0 = W.random_m(grid, seed=5)
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_step(ctx, 3000)
        m = mm.mm_get_m(ctx, 0, m0.shape)
        assert np.isfinite(m).all()
        assert np.abs(np.sqrt((m ** 2).sum(axis=0)) - 1).max() < 1e-6
    finally:
        mm.mm_destroy(ctx)


# -- replica-batched engine -----------------------------------------------------
MAT = W.Material(Ms=1.1e6, A=2e-11, alpha=0.01, Ku1=9e5, u=(0.0, 0.0, 1.0))
CELL = (2e-9, 2e-9, 1e-9)


def _batch(mm, sizes, seeds, T, J, demag=True, dt=1e-14, terms=0):
    grids = [mm.make_grid(nx, ny, 1, *CELL) for nx, ny in sizes]
    M = mm.Material(MAT.Ms, MAT.A, MAT.alpha, MAT.Ku1, MAT.u, MAT.D)
    cfg = mm.make_config(precision=32, integrator=mm.MM_DM,
                         demag=mm.MM_DEMAG_EXACT if demag else mm.MM_DEMAG_OFF, dt=dt, T=0.0, terms=terms)
    ctx = mm.mm_create_batch(grids, M.s, cfg, seeds)
    ctx._mat = M
    mm.mm_set_temperature(ctx, T)
    mm.mm_set_torque(ctx, mm.make_torque(mm.MM_TORQUE_STT, p=(0, 0, 1), P=0.5, Lambda=1.3), J)
    return ctx


@pytest.mark.parametrize("demag", [True, False])
def test_batched_dm_matches_oracle(demag):
    mm = need_gpu()
    from oracle.llg import Solver, Torque
    sizes = [(32, 32), (16, 16), (17, 9), (64, 64), (8, 8), (96, 96), (24, 40)]
    R = len(sizes)
    seeds = np.arange(1, R + 1, dtype=np.uint64) * np.uint64(7919)
    T = np.linspace(100.0, 400.0, R)
    J = np.linspace(-3e11, 3e11, R)
    ctx = _batch(mm, sizes, seeds, T, J, demag)
    try:
        m0 = []
        for r, (nx, ny) in enumerate(sizes):
            m = W.m_perp(W.Grid(nx, ny, 1, *CELL), seed=200 + r, tilt=0.2)
            mm.mm_set_m(ctx, r, m)
            m0.append(m)
        n = 25
        mm.mm_step(ctx, n)
        terms = ("exchange", "anisotropy", "zeeman") + (("demag",) if demag else ())
        for r, (nx, ny) in enumerate(sizes):
            p = oracle_problem(W.Grid(nx, ny, 1, *CELL), MAT)
            o = Solver(p, m0[r], terms=terms, T=T[r], seed=int(seeds[r]), dt=1e-14,
                       torque=Torque(kind="stt", J=J[r], p=(0, 0, 1), P=0.5, Lambda=1.3))
            for _ in range(n):
                o.dm_step()
            err = np.abs(mm.mm_get_m(ctx, r, m0[r].shape) - o.m).max()
            assert err <= 1e-5, (r, sizes[r], err)
    finally:
        mm.mm_destroy(ctx)


# -- adaptive variant -------------------------------------------------------------
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_adaptive_dm_replay_matches_oracle(prec, ci):
    """The oracle's accepted adaptive steps replayed on the GPU (mm_step_dt):
    same trajectory within the bars."""
    mm = need_gpu()
    name, grid, mat, B = CASES[ci]
    m0 = W.random_m(grid, seed=80 + ci)
    o = _oracle(grid, mat, m0, B, dt=1e-14, rtol=1e-5)
    dts = [o.dm_adaptive_step() for _ in range(25)]
    ctx = make_ctx(mm, grid, mat, precision=prec, integrator="dma", demag=True, B=B, dt=1e-14, rtol=1e-5)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_step_dt(ctx, dts)
        err = np.abs(mm.mm_get_m(ctx, 0, m0.shape) - o.m).max()
        assert err <= (1e-11 if prec == 64 else 1e-5), err
    finally:
        mm.mm_destroy(ctx)


def test_adaptive_dm_controller_follows_oracle_fp64():
    """FP64: the device controller takes the oracle's accept/reject decisions
    and step sizes (a rejection included: the first step is oversized)."""
    mm = need_gpu()
    name, grid, mat, B = CASES[0]
    m0 = W.random_m(grid, seed=90)
    o = _oracle(grid, mat, m0, B, dt=2e-12, rtol=1e-5)
    for _ in range(20):
        o.dm_adaptive_step()
    assert o.rejected >= 1
    ctx = make_ctx(mm, grid, mat, precision=64, integrator="dma", demag=True, B=B, dt=2e-12, rtol=1e-5)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_step(ctx, 20)
        st = mm.mm_get_stats(ctx)
        assert st["accepted"] == 20 and st["rejected"] == o.rejected
        assert abs(st["t"] - o.t) < 1e-9 * o.t and abs(st["dt"] - o.dt) < 1e-9 * o.dt
        assert np.abs(mm.mm_get_m(ctx, 0, m0.shape) - o.m).max() <= 1e-11
    finally:
        mm.mm_destroy(ctx)


def test_adaptive_dm_run_lands_on_t_end():
    mm = need_gpu()
    name, grid, mat, B = CASES[2]
    ctx = make_ctx(mm, grid, mat, precision=32, integrator="dma", demag=True, B=B, dt=1e-13, rtol=1e-5)
    try:
        mm.mm_set_m(ctx, 0, W.random_m(grid, seed=91))
        mm.mm_run(ctx, 3.3e-12)
        t, _, _ = mm.mm_get_time(ctx)
        assert abs(t - 3.3e-12) < 1e-24
        with pytest.raises(mm.MMError):
            make_ctx(mm, grid, mat, precision=32, integrator="dma", demag=False, T=300.0)
    finally:
        mm.mm_destroy(ctx)
