"""GPU parity of replica batching (Methods, "Replica batching"): replicas of
uneven sizes, each with its own Philox key, temperature and spin-orbit
current, advanced by one persistent launch per Heun stage, against the FP64
oracle run replica by replica; the batched path against the single-instance
path; the launch-shape autotuner restores the state it perturbs.

Bar: max |m_gpu - m_oracle| <= 1e-5 (FP32) after the stated steps."""
import numpy as np
import pytest

import workloads as W
from gpu_util import need_gpu, oracle_problem

pytestmark = pytest.mark.gpu

MAT = W.Material(Ms=1.1e6, A=2e-11, alpha=0.01, Ku1=9e5, u=(0.0, 0.0, 1.0))
CELL = (2e-9, 2e-9, 1e-9)


def _batch(mm, sizes, seeds, T, J, demag=True, dt=1e-14):
    grids = [mm.make_grid(nx, ny, 1, *CELL) for nx, ny in sizes]
    M = mm.Material(MAT.Ms, MAT.A, MAT.alpha, MAT.Ku1, MAT.u, MAT.D)
    cfg = mm.make_config(precision=32, integrator=mm.MM_HEUN,
                         demag=mm.MM_DEMAG_EXACT if demag else mm.MM_DEMAG_OFF, dt=dt, T=0.0)
    ctx = mm.mm_create_batch(grids, M.s, cfg, seeds)
    ctx._mat = M
    mm.mm_set_temperature(ctx, T)
    mm.mm_set_torque(ctx, mm.make_torque(mm.MM_TORQUE_SOT, p=(0, 1, 0), theta_SH=0.1), J)
    return ctx


@pytest.mark.parametrize("shape", ["persistent", "stacked"])
@pytest.mark.parametrize("demag", [True, False])
def test_uneven_replicas_match_oracle(demag, shape):
    """Both launch shapes: the persistent per-stage kernel and the stacked
    per-size-class passes (sizes interleaved, so storage regroups them)."""
    mm = need_gpu()
    from oracle.llg import Solver, Torque
    sizes = [(32, 32), (48, 48), (17, 9), (64, 64), (32, 32), (96, 96), (24, 40)]
    R = len(sizes)
    seeds = np.arange(1, R + 1, dtype=np.uint64) * np.uint64(7919)
    T = np.linspace(100.0, 400.0, R)
    J = np.linspace(1e11, 3e11, R)
    ctx = _batch(mm, sizes, seeds, T, J, demag)
    if shape == "stacked":
        mm.mm_batch_set_shape(ctx, 0)
    try:
        m0 = []
        for r, (nx, ny) in enumerate(sizes):
            g = W.Grid(nx, ny, 1, *CELL)
            m = W.m_perp(g, seed=100 + r, tilt=0.2)
            mm.mm_set_m(ctx, r, m)
            m0.append(m)
        n = 25
        mm.mm_step(ctx, n)
        terms = ("exchange", "anisotropy", "zeeman") + (("demag",) if demag else ())
        for r, (nx, ny) in enumerate(sizes):
            g = W.Grid(nx, ny, 1, *CELL)
            p = oracle_problem(g, MAT)
            o = Solver(p, m0[r], terms=terms, T=T[r], seed=int(seeds[r]), dt=1e-14,
                       torque=Torque(kind="sot", J=J[r], p=(0, 1, 0), theta_SH=0.1))
            for _ in range(n):
                o.heun_step()
            err = np.abs(mm.mm_get_m(ctx, r, m0[r].shape) - o.m).max()
            assert err <= 1e-5, (r, sizes[r], err)
    finally:
        mm.mm_destroy(ctx)


@pytest.mark.parametrize("shape", ["persistent", "stacked"])
def test_batched_replica_equals_single_instance(shape):
    """The batched engine and the single-instance path agree replica by
    replica (the paper's R = 1 regression, generalised to every replica)."""
    mm = need_gpu()
    sizes = [(64, 64), (32, 32), (48, 48), (32, 32)]
    seeds = np.array([11, 22, 33, 44], dtype=np.uint64)
    T = np.array([300.0, 300.0, 150.0, 0.0])
    J = np.array([2e11, 1e11, 3e11, 2e11])
    ctx = _batch(mm, sizes, seeds, T, J)
    if shape == "stacked":
        mm.mm_batch_set_shape(ctx, 0)
    try:
        singles = []
        for r, (nx, ny) in enumerate(sizes):
            g = W.Grid(nx, ny, 1, *CELL)
            m = W.m_perp(g, seed=r, tilt=0.3)
            mm.mm_set_m(ctx, r, m)
            G = mm.make_grid(nx, ny, 1, *CELL)
            M = mm.Material(MAT.Ms, MAT.A, MAT.alpha, MAT.Ku1, MAT.u, MAT.D)
            cfg = mm.make_config(precision=32, integrator=mm.MM_HEUN, demag=mm.MM_DEMAG_EXACT, dt=1e-14, T=T[r])
            s = mm.mm_create_batch([G], M.s, cfg, seeds[r:r + 1])
            s._mat = M
            mm.mm_set_m(s, 0, m)
            mm.mm_set_torque(s, mm.make_torque(mm.MM_TORQUE_SOT, p=(0, 1, 0), theta_SH=0.1), J[r:r + 1])
            singles.append(s)
        mm.mm_step(ctx, 40)
        for r, s in enumerate(singles):
            mm.mm_step(s, 40)
            shp = (3, 1, sizes[r][1], sizes[r][0])
            assert np.abs(mm.mm_get_m(ctx, r, shp) - mm.mm_get_m(s, 0, shp)).max() < 2e-6
    finally:
        mm.mm_destroy(ctx)
        for s in singles:
            mm.mm_destroy(s)


def test_autotune_restores_state_and_is_cached(tmp_path):
    mm = need_gpu()
    sizes = [(32, 32), (64, 64), (48, 48), (32, 32)] * 3
    R = len(sizes)
    ctx = _batch(mm, sizes, None, np.full(R, 300.0), np.full(R, 2e11))
    try:
        for r, (nx, ny) in enumerate(sizes):
            mm.mm_set_m(ctx, r, W.m_perp(W.Grid(nx, ny, 1, *CELL), seed=r, tilt=0.2))
        mm.mm_step(ctx, 3)
        before = [mm.mm_get_m(ctx, r, (3, 1, ny, nx)) for r, (nx, ny) in enumerate(sizes)]
        t0 = mm.mm_get_time(ctx)
        cache = str(tmp_path / "tune.json")
        nt, blocks = mm.mm_batch_autotune(ctx, cache)
        assert (nt, blocks) == (0, 0) or (nt in (256, 512) and 1 <= blocks <= R)
        after = [mm.mm_get_m(ctx, r, (3, 1, ny, nx)) for r, (nx, ny) in enumerate(sizes)]
        assert all(np.array_equal(a, b) for a, b in zip(before, after))
        assert mm.mm_get_time(ctx) == t0
        assert mm.mm_batch_autotune(ctx, cache) == (nt, blocks)     # served from the cache
        mm.mm_step(ctx, 3)
    finally:
        mm.mm_destroy(ctx)


def test_batched_observables_per_replica():
    mm = need_gpu()
    from oracle.demag import demag_spectrum
    from oracle.observables import energy
    sizes = [(32, 24), (40, 40)]
    ctx = _batch(mm, sizes, None, np.zeros(2), np.zeros(2))
    try:
        for r, (nx, ny) in enumerate(sizes):
            g = W.Grid(nx, ny, 1, *CELL)
            m = W.random_m(g, seed=r)
            mm.mm_set_m(ctx, r, m)
            md = mm.mm_get_m(ctx, r, m.shape)
            p = oracle_problem(g, MAT)
            E = mm.mm_energy(ctx, r)
            ref = energy(md, p, demag_spectrum(p.shape, p.d), terms=("exchange", "anisotropy", "zeeman", "demag"))
            assert abs(E[5] - ref["total"]) <= 2e-6 * max(abs(v) for v in ref.values())
    finally:
        mm.mm_destroy(ctx)
