"""GPU parity of the batched trial engine (Results, "Replica batching"):
one-cell replicas (the macrospin ensemble, one thread per slot with the
moment in registers for blocks of steps), small films without demag (one
CTA per replica, state in shared memory), and retire/refill on one-cell and
8 x 8 film replicas (with and without demag), against the oracle's trials
run one by one.

Bars: per-replica max |m_gpu - m_oracle| <= 1e-5 (FP32).  Trial outcomes:
the step count and stop flag of every trial equal the oracle's, except
where the FP32 and FP64 trajectories straddle the threshold: there the
oracle's mean projection at the first of the two decision steps lies within
1e-4 of the threshold."""
import numpy as np
import pytest

import workloads as W
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

D1 = 4e-9


def _spec(grid, mat, terms, J, T, dt, thr, max_steps, tilt=0.05, seed=9):
    from oracle.fields import Problem
    from oracle.llg import Torque
    from oracle.trials import TrialSpec
    p = Problem.from_workload(grid, mat)
    m0 = np.zeros((3,) + p.shape)
    m0[0] = tilt
    m0[2] = -1.0
    m0 /= np.sqrt((m0 ** 2).sum(axis=0))
    tq = Torque(kind="stt", p=(0, 0, 1), P=0.6, Lambda=1.0)
    return TrialSpec(p=p, m_init=m0, J=np.asarray(J, float), T=np.asarray(T, float), terms=terms, torque=tq,
                     base_seed=seed, dt=dt, axis=(0, 0, -1), threshold=thr, max_steps=max_steps)


def _oracle_projections(spec, q, n):
    """mean(m . axis) after each of the first n steps of trial q."""
    from oracle.llg import dot
    from oracle.trials import _advance, _solver
    s = _solver(spec, q)
    a = np.asarray(spec.axis, float)
    a /= np.linalg.norm(a)
    out = []
    for _ in range(n):
        _advance(s, spec)
        out.append(float(dot(s.m, np.broadcast_to(a[:, None, None, None], s.m.shape))[s.p.present].mean()))
    return out


def _context(mm, spec, R, integrator, terms_mask, demag):
    g = spec.p.shape
    grid = mm.make_grid(g[2], g[1], 1, *spec.p.d)
    Ms = float(spec.p.Ms.flat[0])
    M = mm.Material(Ms, float(spec.p.A.flat[0]), float(spec.p.alpha.flat[0]), float(spec.p.Ku1.flat[0]),
                    tuple(spec.p.u[:, 0, 0, 0]), 0.0)
    cfg = mm.make_config(precision=32, integrator=integrator, demag=mm.MM_DEMAG_EXACT if demag else mm.MM_DEMAG_OFF,
                         dt=spec.dt, T=0.0, terms=terms_mask)
    ctx = mm.mm_create_batch([grid] * R, M.s, cfg, None)
    ctx._mat = M
    tq = spec.torque
    mm.mm_set_torque(ctx, mm.make_torque(mm.MM_TORQUE_STT, p=tq.p, P=tq.P, Lambda=tq.Lambda), np.zeros(R))
    return ctx


def _compare_outcomes(spec, steps, stopped):
    from oracle.trials import run_trial
    marginal = 0
    for q in range(len(spec.J)):
        n_o, stop_o, _ = run_trial(spec, q)
        if (steps[q], bool(stopped[q])) == (n_o, stop_o):
            continue
        k = min(steps[q], n_o)
        proj = _oracle_projections(spec, q, k)[k - 1]
        assert abs(proj - spec.threshold) < 1e-4, (q, steps[q], stopped[q], n_o, stop_o, proj)
        marginal += 1
    assert marginal <= 1


def _run_to_completion(mm, ctx, n, chunk=100, limit=100000):
    done = 0
    total = 0
    while done < n and total < limit:
        mm.mm_step(ctx, chunk)
        total += chunk
        steps, stopped, done = mm.mm_trials_result(ctx)
    assert done == n
    return steps, stopped


@pytest.mark.parametrize("integ", ["dm", "heun"])
def test_one_cell_replicas_match_oracle(integ):
    """64 macrospins (anisotropy, STT, thermal field), each with its own key,
    temperature and current, 300 steps in blocks inside one thread each."""
    mm = need_gpu()
    from oracle.fields import Problem
    from oracle.llg import Solver, Torque
    R, n, dt = 64, 300, 2e-13
    grid = W.Grid(1, 1, 1, D1, D1, D1)
    mat = W.Material(Ms=1e6, A=1e-11, alpha=0.05, Ku1=6e5, u=(0, 0, 1))
    seeds = (np.arange(R, dtype=np.uint64) + np.uint64(5)) * np.uint64(104729)
    T = np.linspace(0.0, 400.0, R)
    J = np.linspace(-2e12, 3e12, R)
    G = mm.make_grid(1, 1, 1, D1, D1, D1)
    M = mm.Material(mat.Ms, mat.A, mat.alpha, mat.Ku1, mat.u, 0.0)
    cfg = mm.make_config(precision=32, integrator=mm.MM_DM if integ == "dm" else mm.MM_HEUN,
                         demag=mm.MM_DEMAG_OFF, dt=dt, T=0.0, terms=4 | 8 | 32)
    ctx = mm.mm_create_batch([G] * R, M.s, cfg, seeds)
    ctx._mat = M
    try:
        mm.mm_set_temperature(ctx, T)
        mm.mm_set_torque(ctx, mm.make_torque(mm.MM_TORQUE_STT, p=(0, 0, 1), P=0.6, Lambda=1.2), J)
        rng = np.random.default_rng(1)
        m0 = []
        for r in range(R):
            v = rng.normal(size=3)
            v /= np.linalg.norm(v)
            m0.append(v.reshape(3, 1, 1, 1))
            mm.mm_set_m(ctx, r, m0[-1])
        mm.mm_step(ctx, n)
        t, _, steps = mm.mm_get_time(ctx)
        assert steps == n and abs(t - n * dt) < 1e-20
        p = Problem.from_workload(grid, mat)
        for r in range(R):
            o = Solver(p, m0[r], terms=("anisotropy", "zeeman"), T=T[r], seed=int(seeds[r]), dt=dt,
                       torque=Torque(kind="stt", J=J[r], p=(0, 0, 1), P=0.6, Lambda=1.2))
            for _ in range(n):
                if integ == "dm":
                    o.dm_step()
                else:
                    o.heun_step()
            err = np.abs(mm.mm_get_m(ctx, r, (3, 1, 1, 1)) - o.m).max()
            assert err <= 1e-5, (r, err)
    finally:
        mm.mm_destroy(ctx)


def test_retire_refill_macrospins_match_oracle():
    """24 trials over 8 one-cell slots: every trial's stop step equals the
    oracle's trial run alone."""
    mm = need_gpu()
    grid = W.Grid(1, 1, 1, D1, D1, D1)
    mat = W.Material(Ms=1e6, A=1e-11, alpha=0.05, Ku1=6e5, u=(0, 0, 1))
    n = 24
    spec = _spec(grid, mat, ("anisotropy", "zeeman"), np.linspace(2e11, 2.5e12, n), np.full(n, 300.0), 2e-13,
                 0.9, 600)
    ctx = _context(mm, spec, 8, mm.MM_DM, 4 | 8 | 32, False)
    try:
        mm.mm_trials_start(ctx, spec.J, spec.T, spec.m_init, axis=spec.axis, threshold=spec.threshold,
                           max_steps=spec.max_steps, base_seed=spec.base_seed, refill=True)
        steps, stopped = _run_to_completion(mm, ctx, n)
        assert stopped.any() and not stopped.all()
        _compare_outcomes(spec, steps, stopped)
    finally:
        mm.mm_destroy(ctx)


@pytest.mark.parametrize("shape", ["persistent", "stacked"])
def test_retire_refill_films_match_oracle(shape):
    """10 trials over 4 slots of 8 x 8 films with exchange, anisotropy,
    demag, STT and the thermal field, on both launch shapes: one persistent
    launch per stage with the stop test inside the corrector, or the
    per-class passes with idle slots skipped and a per-slot stop-test
    launch after the corrector."""
    mm = need_gpu()
    grid = W.Grid(8, 8, 1, D1, D1, D1)
    mat = W.Material(Ms=1e6, A=1.5e-11, alpha=0.05, Ku1=1.1e6, u=(0, 0, 1))
    n = 10
    spec = _spec(grid, mat, ("exchange", "anisotropy", "zeeman", "demag"), np.linspace(5e11, 6e12, n),
                 np.full(n, 300.0), 1e-13, 0.98, 300)
    ctx = _context(mm, spec, 4, mm.MM_DM, 1 | 4 | 8 | 16 | 32, True)
    try:
        if shape == "stacked":
            mm.mm_batch_set_shape(ctx, 0)
        mm.mm_trials_start(ctx, spec.J, spec.T, spec.m_init, axis=spec.axis, threshold=spec.threshold,
                           max_steps=spec.max_steps, base_seed=spec.base_seed, refill=True)
        steps, stopped = _run_to_completion(mm, ctx, n, chunk=50)
        assert stopped.any() and not stopped.all()
        _compare_outcomes(spec, steps, stopped)
    finally:
        mm.mm_destroy(ctx)


def test_without_refill_only_the_first_slots_run():
    mm = need_gpu()
    grid = W.Grid(1, 1, 1, D1, D1, D1)
    mat = W.Material(Ms=1e6, A=1e-11, alpha=0.05, Ku1=6e5, u=(0, 0, 1))
    n, R = 20, 8
    spec = _spec(grid, mat, ("anisotropy", "zeeman"), np.full(n, 3e12), np.full(n, 300.0), 2e-13, 0.9, 400)
    ctx = _context(mm, spec, R, mm.MM_DM, 4 | 8 | 32, False)
    try:
        mm.mm_trials_start(ctx, spec.J, spec.T, spec.m_init, axis=spec.axis, threshold=spec.threshold,
                           max_steps=spec.max_steps, base_seed=spec.base_seed, refill=False)
        mm.mm_step(ctx, 500)
        steps, stopped, done = mm.mm_trials_result(ctx)
        assert done == R
        assert (steps[:R] > 0).all() and (steps[R:] == -1).all()
        mm.mm_step(ctx, 10)           # idle slots stay idle
        assert mm.mm_trials_result(ctx)[2] == R
    finally:
        mm.mm_destroy(ctx)


def test_trial_api_errors():
    mm = need_gpu()
    G1 = mm.make_grid(1, 1, 1, D1, D1, D1)
    G2 = mm.make_grid(2, 2, 1, D1, D1, D1)
    M = mm.Material(1e6, 1e-11, 0.05, 6e5, (0, 0, 1), 0.0)
    cfg = mm.make_config(precision=32, integrator=mm.MM_DM, demag=mm.MM_DEMAG_OFF, dt=1e-13, terms=4 | 8 | 32)
    m0 = np.array([0.0, 0.0, 1.0]).reshape(3, 1, 1, 1)
    single = mm.mm_create(G1, M.s, cfg)
    mixed = mm.mm_create_batch([G1, G2], M.s, cfg, None)
    try:
        with pytest.raises(mm.MMError):
            mm.mm_trials_start(single, [1e11], [0.0], m0)
        with pytest.raises(mm.MMError):
            mm.mm_trials_start(mixed, [1e11], [0.0], m0)
    finally:
        mm.mm_destroy(single)
        mm.mm_destroy(mixed)
    with pytest.raises(mm.MMError):
        demag_cfg = mm.make_config(precision=32, integrator=mm.MM_DM, demag=mm.MM_DEMAG_EXACT, dt=1e-13)
        mm.mm_create_batch([G1, G1], M.s, demag_cfg, None)


@pytest.mark.parametrize("integ", ["dm", "heun"])
def test_small_films_without_demag_match_oracle(integ):
    """Films of at most 1024 cells without demag run one CTA per replica with
    the state in shared memory for blocks of steps: uneven sizes, interfacial
    and bulk DMI, anisotropy, Zeeman, STT and the thermal field."""
    mm = need_gpu()
    from oracle.llg import Solver, Torque
    sizes = [(8, 8), (16, 16), (32, 32), (17, 9), (5, 31), (1, 12)]
    R = len(sizes)
    cell = (2e-9, 2e-9, 1e-9)
    mat = W.Material(Ms=1.1e6, A=2e-11, alpha=0.05, Ku1=9e5, u=(0, 0, 1), D=1.5e-3, Db=-1e-3)
    M = mm.Material(mat.Ms, mat.A, mat.alpha, mat.Ku1, mat.u, mat.D, Db=mat.Db)
    cfg = mm.make_config(precision=32, integrator=mm.MM_DM if integ == "dm" else mm.MM_HEUN,
                         demag=mm.MM_DEMAG_OFF, dt=1e-14, terms=1 | 2 | 4 | 8 | 32)
    seeds = (np.arange(R, dtype=np.uint64) + np.uint64(3)) * np.uint64(7919)
    ctx = mm.mm_create_batch([mm.make_grid(nx, ny, 1, *cell) for nx, ny in sizes], M.s, cfg, seeds)
    ctx._mat = M
    T = np.linspace(50.0, 400.0, R)
    J = np.linspace(-2e11, 3e11, R)
    try:
        mm.mm_set_field(ctx, 0, (0.01, 0.0, 0.02))
        mm.mm_set_temperature(ctx, T)
        mm.mm_set_torque(ctx, mm.make_torque(mm.MM_TORQUE_STT, p=(0, 0.3, 1), P=0.5, Lambda=1.4), J)
        m0 = []
        for r, (nx, ny) in enumerate(sizes):
            m0.append(W.m_perp(W.Grid(nx, ny, 1, *cell), seed=300 + r, tilt=0.3))
            mm.mm_set_m(ctx, r, m0[-1])
        n = 40
        mm.mm_step(ctx, n)
        t, _, steps = mm.mm_get_time(ctx)
        assert steps == n
        for r, (nx, ny) in enumerate(sizes):
            from gpu_util import oracle_problem
            p = oracle_problem(W.Grid(nx, ny, 1, *cell), mat, (0.01, 0.0, 0.02))
            o = Solver(p, m0[r], terms=("exchange", "dmi", "anisotropy", "zeeman"), T=T[r], seed=int(seeds[r]),
                       dt=1e-14, torque=Torque(kind="stt", J=J[r], p=(0, 0.3, 1), P=0.5, Lambda=1.4))
            for _ in range(n):
                if integ == "dm":
                    o.dm_step()
                else:
                    o.heun_step()
            err = np.abs(mm.mm_get_m(ctx, r, m0[r].shape) - o.m).max()
            assert err <= 1e-5, (r, sizes[r], err)
    finally:
        mm.mm_destroy(ctx)


def test_retire_refill_small_films_without_demag():
    """Retire/refill in the shared-memory film kernel: 12 trials over 4 slots
    of 8 x 8 films with exchange, anisotropy, STT and 300 K."""
    mm = need_gpu()
    grid = W.Grid(8, 8, 1, D1, D1, D1)
    mat = W.Material(Ms=1e6, A=1.5e-11, alpha=0.05, Ku1=1.1e6, u=(0, 0, 1))
    n = 12
    spec = _spec(grid, mat, ("exchange", "anisotropy", "zeeman"), np.linspace(5e11, 8e12, n),
                 np.full(n, 300.0), 1e-13, 0.98, 300)
    ctx = _context(mm, spec, 4, mm.MM_DM, 1 | 4 | 8 | 32, False)
    try:
        mm.mm_trials_start(ctx, spec.J, spec.T, spec.m_init, axis=spec.axis, threshold=spec.threshold,
                           max_steps=spec.max_steps, base_seed=spec.base_seed, refill=True)
        steps, stopped = _run_to_completion(mm, ctx, n, chunk=50)
        assert stopped.any() and not stopped.all()
        _compare_outcomes(spec, steps, stopped)
    finally:
        mm.mm_destroy(ctx)
