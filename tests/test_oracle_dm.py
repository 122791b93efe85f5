"""Pins of the oracle's Depondt-Mertens rotation scheme (Methods,
"Integrators" and "Replica batching"): the rotation form of Eq. 1 against
the independently pinned slope, exactness for a constant rotation vector
(matrix exponential), second order against the closed-form damped
macrospin and the closed-form spin-orbit relaxation, |m| kept without
renormalisation, one thermal draw per step, and the Langevin equilibrium
<m_z> = L(xi) the paper validates its thermal field against (Results,
"Replica batching")."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import workloads as W
from oracle.constants import GAMMA0, HBAR, KB, MU0, QE
from oracle.fields import Problem
from oracle.llg import Solver, Torque, cross, dot
from oracle.philox import thermal_field


def _film(seed=1, shape=(12, 8, 2)):
    grid = W.Grid(*shape, 2e-9, 2e-9, 2e-9)
    mat = W.Material(Ms=6e5, A=1.3e-11, alpha=0.3, Ku1=3e5, u=(0, 0, 1), D=2e-3)
    p = Problem.from_workload(grid, mat, B_ext=(0.02, 0.0, 0.05))
    return grid, p, W.random_m(grid, seed=seed)


def _cell(alpha, Ms=8e5, B=(0.0, 0.0, 0.0), d=2e-9):
    grid = W.Grid(1, 1, 1, d, d, d)
    return Problem.from_workload(grid, W.Material(Ms=Ms, A=1e-11, alpha=alpha), B_ext=B)


def _m(v):
    v = np.asarray(v, dtype=np.float64)
    return (v / np.linalg.norm(v)).reshape(3, 1, 1, 1)


def _skew(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


TORQUES = [
    Torque(),
    Torque(kind="sot", J=3e11, p=(0.3, 1.0, 0.2), theta_SH=0.12, fl_ratio=0.4),
    Torque(kind="stt", J=-2e11, p=(0.0, 0.4, 1.0), P=0.5, Lambda=1.7, eps_prime=0.05),
    Torque(kind="zl", J=1e12, P=0.6, xi=0.07, direction=(1.0, 0.5, 0.0)),
]


@pytest.mark.parametrize("tq", TORQUES, ids=["none", "sot", "stt", "zl"])
def test_rotation_vector_reproduces_the_slope(tq):
    """Omega x m equals the LLG slope (field terms, demag and each spin
    torque), cell by cell."""
    grid, p, m = _film()
    s = Solver(p, m, torque=tq)
    k = s.slope(s.m)
    w = s.omega(s.m)
    assert np.abs(cross(w, s.m) - k).max() <= 1e-12 * np.abs(k).max()


def test_exact_for_a_constant_rotation_vector():
    """alpha = 0 in a uniform applied field: Omega = gamma0 mu0 H is
    constant, so every step is exact however large: the result equals
    expm(dt [Omega]x) applied to m, a rotation of 0.7 rad per step."""
    b = np.array([0.3, -0.5, 0.8])
    b = b / np.linalg.norm(b)
    H0 = 4e5
    p = _cell(0.0, B=tuple(MU0 * H0 * b))
    m0 = _m([1.0, 0.2, -0.1])
    w = GAMMA0 * MU0 * H0 * b
    dt = 0.7 / np.linalg.norm(w)
    s = Solver(p, m0, terms=("zeeman",))
    for _ in range(9):
        s.dm_step(dt)
    exp = expm(9 * dt * _skew(w)) @ m0[:, 0, 0, 0]
    assert np.abs(s.m[:, 0, 0, 0] - exp).max() < 1e-13


def test_field_like_torque_rotates_about_p_exactly():
    """alpha = 0, no field, a purely field-like torque (Slonczewski form with
    P = 0, so h_DL = 0, and eps' > 0): Omega = gamma0 mu0 h_FL p is constant
    and the steps are exact, p's component along m included."""
    Ms, tF, J, epsp = 1.1e6, 2e-9, 4e11, 0.3
    p = _cell(0.0, Ms=Ms)
    pol = np.array([0.2, 1.0, -0.4])
    tq = Torque(kind="stt", J=J, p=tuple(pol), P=0.0, Lambda=1.0, eps_prime=epsp, t_F=tF)
    pol = pol / np.linalg.norm(pol)
    w = GAMMA0 * MU0 * epsp * HBAR * J / (QE * MU0 * Ms * tF) * pol
    dt = 0.9 / np.linalg.norm(w)
    m0 = _m([1.0, -0.3, 0.5])
    s = Solver(p, m0, terms=(), torque=tq)
    for _ in range(6):
        s.dm_step(dt)
    exp = expm(6 * dt * _skew(w)) @ m0[:, 0, 0, 0]
    assert np.abs(s.m[:, 0, 0, 0] - exp).max() < 1e-13


def _dl_closed_form(t, theta0, rate):
    return 2 * math.atan(math.tan(theta0 / 2) * math.exp(-rate * t))


def test_damping_like_relaxation_second_order():
    """alpha = 0, no field, damping-like SOT only (fl_ratio = 0): the angle to
    p obeys d theta/dt = -gamma0 mu0 h_DL sin theta, so tan(theta/2) decays
    as exp(-gamma0 mu0 h_DL t) in a fixed plane; halving dt quarters the
    error."""
    Ms, tF, J, th = 1.1e6, 2e-9, 5e11, 0.2
    p = _cell(0.0, Ms=Ms)
    tq = Torque(kind="sot", J=J, p=(0, 0, 1), theta_SH=th, fl_ratio=0.0, t_F=tF)
    hDL = 0.5 * th * HBAR * J / (QE * MU0 * Ms * tF)
    rate = GAMMA0 * MU0 * hDL
    theta0 = 2.5
    m0 = _m([math.sin(theta0), 0.0, math.cos(theta0)])
    T = 3.0 / rate
    errs = []
    for n in (100, 200, 400):
        s = Solver(p, m0, terms=(), torque=tq)
        for _ in range(n):
            s.dm_step(T / n)
        th_t = _dl_closed_form(T, theta0, rate)
        exp = np.array([math.sin(th_t), 0.0, math.cos(th_t)])
        errs.append(np.abs(s.m[:, 0, 0, 0] - exp).max())
    rates = math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])
    assert all(1.8 < r < 2.3 for r in rates), (errs, rates)


def _damped_closed_form(t, alpha, H0, theta0, phi0):
    gp = GAMMA0 / (1 + alpha ** 2)
    th = 2 * math.atan(math.tan(theta0 / 2) * math.exp(-gp * alpha * MU0 * H0 * t))
    ph = phi0 + gp * MU0 * H0 * t
    return np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])


def test_damped_precession_second_order():
    alpha, H0 = 0.05, 5e5
    p = _cell(alpha, B=(0, 0, MU0 * H0))
    m0 = _m([math.sin(1.0) * math.cos(0.3), math.sin(1.0) * math.sin(0.3), math.cos(1.0)])
    T = 20e-12
    errs = []
    for n in (200, 400, 800):
        s = Solver(p, m0, terms=("zeeman",))
        for _ in range(n):
            s.dm_step(T / n)
        errs.append(np.abs(s.m[:, 0, 0, 0] - _damped_closed_form(T, alpha, H0, 1.0, 0.3)).max())
    rates = math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])
    assert all(1.8 < r < 2.3 for r in rates), (errs, rates)
    assert errs[-1] < 1e-4


def test_norm_kept_without_renormalising():
    """Every term, demag and an STT current, 60 steps: |m| = 1 to rounding,
    although no step rescales m.  The same steps taken by Heun without its
    final rescaling drift by orders of magnitude more."""
    grid, p, m = _film()
    tq = TORQUES[2]
    s = Solver(p, m, torque=tq)
    for _ in range(60):
        s.dm_step(2e-14)
    assert np.abs(np.sqrt(dot(s.m, s.m)) - 1).max() < 1e-14
    h = Solver(p, m, torque=tq)
    mm = h.m.copy()
    for _ in range(60):
        k1 = h.slope(mm)
        k2 = h.slope(mm + 2e-14 * k1)
        mm = mm + 1e-14 * (k1 + k2)
    assert np.abs(np.sqrt(dot(mm, mm)) - 1).max() > 1e3 * np.abs(np.sqrt(dot(s.m, s.m)) - 1).max()


def test_one_thermal_draw_acts_as_a_fixed_field_within_a_step():
    """T > 0: a step equals the T = 0 step in which the applied field is the
    step's thermal draw (the same field in the predictor and the corrector,
    Stratonovich), for the step counter the solver is at."""
    grid, p, m = _film(seed=3, shape=(6, 5, 1))
    T, dt, seed = 300.0, 1e-14, 11
    s = Solver(p, m, T=T, seed=seed)
    s.step = 7
    s.dm_step(dt)
    h = thermal_field(p, T, dt, seed, 7)
    q = Problem(**{**p.__dict__, "B_ext": p.B_ext + MU0 * h})
    ref = Solver(q, m)
    ref.dm_step(dt)
    assert np.abs(s.m - ref.m).max() < 1e-14
    # and a different step counter gives a different draw
    s2 = Solver(p, m, T=T, seed=seed)
    s2.step = 8
    s2.dm_step(dt)
    assert np.abs(s2.m - s.m).max() > 1e-6


def _langevin(x):
    return 1.0 / math.tanh(x) - 1.0 / x


def test_langevin_equilibrium():
    """Results, "Replica batching": an isotropic macrospin in a field at
    temperature T relaxes to <m_z> = L(xi), xi = mu0 Ms V H / (kB T).  4096
    independent cells (no exchange, no demag) with xi = 3, time average
    after equilibration: L(3) = 0.6716."""
    n = 64
    d = 2e-9
    Ms, alpha, Tk = 4e5, 0.5, 300.0
    V = d ** 3
    H = 3.0 * KB * Tk / (MU0 * Ms * V)
    grid = W.Grid(n, n, 1, d, d, d)
    p = Problem.from_workload(grid, W.Material(Ms=Ms, A=1e-11, alpha=alpha), B_ext=(0, 0, MU0 * H))
    m0 = np.zeros((3, 1, n, n))
    m0[2] = 1.0
    gp = GAMMA0 / (1 + alpha ** 2)
    t_relax = 1.0 / (alpha * gp * MU0 * H)       # damping time in the field
    dt = 0.02 * t_relax
    s = Solver(p, m0, terms=("zeeman",), T=Tk, seed=5)
    samples = []
    for k in range(1500):
        s.dm_step(dt)
        if k >= 300 and k % 10 == 0:
            samples.append(s.m[2].mean())
    mz = float(np.mean(samples))
    assert abs(mz - _langevin(3.0)) < 0.01, mz


# -- retire / refill ------------------------------------------------------------
from oracle.trials import TrialSpec, run_ensemble, run_trial  # noqa: E402


def _stt_spec(n_trials, max_steps=400, T=300.0, seed=9):
    """A perpendicular macrospin (m near -z, p = +z) driven by Slonczewski
    STT at a spread of currents around its instability threshold."""
    d = 4e-9
    grid = W.Grid(1, 1, 1, d, d, d)
    p = Problem.from_workload(grid, W.Material(Ms=1e6, A=1e-11, alpha=0.05, Ku1=6e5, u=(0, 0, 1)),
                              B_ext=(0.0, 0.0, 0.0))
    m0 = _m([0.05, 0.0, -1.0])
    J = np.linspace(2e11, 2.5e12, n_trials)
    Ts = np.full(n_trials, T)
    tq = Torque(kind="stt", p=(0, 0, 1), P=0.6, Lambda=1.0)
    return TrialSpec(p=p, m_init=m0, J=J, T=Ts, terms=("anisotropy",), torque=tq, base_seed=seed,
                     dt=2e-13, axis=(0, 0, -1), threshold=0.0, max_steps=max_steps)


def test_refill_keeps_every_trial_independent_of_its_slot():
    """Each trial's outcome equals the same trial run alone, whatever slot and
    start step the ensemble gave it; with refill no slot idles while trials
    wait, without refill only the first R trials run."""
    spec = _stt_spec(10, max_steps=1000)
    alone = {q: run_trial(spec, q)[:2] for q in range(10)}
    assert any(v[1] for v in alone.values()) and not all(v[1] for v in alone.values())
    res, starts, g = run_ensemble(spec, 10, R=3, refill=True)
    assert res == alone
    assert sorted(starts) == list(range(10))
    # no idle slot while trials wait: a slot's next trial starts right after
    # its previous one retired
    by_slot = {}
    for q, (r, s0) in starts.items():
        by_slot.setdefault(r, []).append((s0, q))
    for r, lst in by_slot.items():
        lst.sort()
        for (s0, q), (s1, _) in zip(lst, lst[1:]):
            assert s1 == s0 + res[q][0]
    res0, starts0, _ = run_ensemble(spec, 10, R=3, refill=False)
    assert sorted(res0) == [0, 1, 2] and all(res0[q] == alone[q] for q in range(3))


def test_switching_needs_current_at_zero_temperature():
    """T = 0: below the STT instability (J small) the trial never stops, far
    above it the trial switches; the stop step falls as J grows."""
    spec = _stt_spec(3, max_steps=4000, T=0.0)
    spec.J = np.array([1e11, 3.0e12, 5.0e12])
    out = [run_trial(spec, q)[:2] for q in range(3)]
    assert out[0] == (4000, False)
    assert out[1][1] and out[2][1] and out[2][0] < out[1][0]


# -- adaptive variant -------------------------------------------------------------
def test_adaptive_tracks_the_closed_form_and_its_tolerance():
    """Damped precession in a constant field: every accepted step's embedded
    error is below rtol, the trajectory error against the closed form falls
    with rtol, and the step grows where the motion is slow (the end of the
    relaxation) and shrinks after a rejection."""
    from oracle.llg import rotate  # noqa: F401  (the step rotates)
    alpha, H0 = 0.1, 5e5
    p = _cell(alpha, B=(0, 0, MU0 * H0))
    m0 = _m([math.sin(1.0) * math.cos(0.3), math.sin(1.0) * math.sin(0.3), math.cos(1.0)])
    T = 60e-12
    errs = []
    for rtol in (1e-3, 1e-4, 1e-5):
        s = Solver(p, m0, terms=("zeeman",), dt=1e-13, rtol=rtol, dt_max=1e-11)
        dts = []
        while s.t < T:
            dts.append(s.dm_adaptive_step())
        errs.append(np.abs(s.m[:, 0, 0, 0] - _damped_closed_form(s.t, alpha, H0, 1.0, 0.3)).max())
        assert s.accepted == len(dts)
    # the global error follows the tolerance: about rtol, a decade per decade
    for e, rtol in zip(errs, (1e-3, 1e-4, 1e-5)):
        assert e < 3 * rtol, errs
    assert all(5 < errs[i] / errs[i + 1] < 20 for i in range(2)), errs


def test_adaptive_rejects_an_oversized_step():
    """A first step far above what rtol allows is rejected and retried
    smaller; the accepted step then meets the tolerance."""
    grid, p, m = _film(seed=4)
    s = Solver(p, m, dt=5e-12, rtol=1e-5)
    dt = s.dm_adaptive_step()
    assert s.rejected >= 1 and dt < 5e-12
    s2 = Solver(p, m)
    w1 = s2.omega(s2.m)
    from oracle.llg import rotate
    ms = rotate(s2.m, w1, dt)
    w2 = s2.omega(ms)
    mn = rotate(s2.m, 0.5 * (w1 + w2), dt)
    assert np.abs(mn - s.m).max() < 1e-15
    assert np.sqrt(((mn - ms) ** 2).sum(axis=0)).max() <= 1e-5


def test_adaptive_refuses_finite_temperature():
    grid, p, m = _film()
    with pytest.raises(ValueError):
        Solver(p, m, T=300.0).dm_adaptive_step()


def test_trial_stop_step_is_the_switching_time_of_the_macrospin():
    """Deterministic trials (T = 0) of a perpendicular STT macrospin with
    p = -z, stopped at m_z <= 0: below the threshold current J_c0 a trial
    runs out its steps; above it the stop step is the first step past the
    time at which the polar angle, following its scalar equation (integrated
    by scipy), reaches pi/2."""
    from scipy.integrate import solve_ivp

    Ms, Ku, alpha, P, Lam, dz, dt = 1e6, 1e6, 0.02, 0.6, 2.0, 1e-9, 1e-13
    grid = W.Grid(1, 1, 1, 2e-9, 2e-9, dz)
    p = Problem.from_workload(grid, W.Material(Ms=Ms, A=1e-11, alpha=alpha, Ku1=Ku, u=(0, 0, 1)))
    HK, L2 = 2 * Ku / (MU0 * Ms), Lam ** 2
    Jc0 = alpha * HK * QE * MU0 * Ms * dz / (HBAR * P * L2 / 2)
    mult = np.array([0.5, 2.0, 3.0])
    th0 = 0.1
    m0 = np.array([math.sin(th0), 0.0, math.cos(th0)]).reshape(3, 1, 1, 1)
    spec = TrialSpec(p=p, m_init=m0, J=mult * Jc0, T=np.zeros(3), terms=("anisotropy",),
                     torque=Torque(kind="stt", p=(0, 0, -1), P=P, Lambda=Lam), dt=dt, axis=(0, 0, 1),
                     threshold=0.0, max_steps=8000, integrator="dm")
    gp = GAMMA0 / (1 + alpha ** 2)
    for q in range(3):
        n, stopped, m = run_trial(spec, q)
        if mult[q] < 1:
            assert not stopped and n == spec.max_steps and m[2, 0, 0, 0] > math.cos(th0)
            continue
        base = HBAR * mult[q] * Jc0 / (QE * MU0 * Ms * dz)

        def rhs(_, y, base=base):
            eps = P * L2 / ((L2 + 1) - (L2 - 1) * math.cos(y[0]))
            return [gp * MU0 * math.sin(y[0]) * (eps * base - alpha * HK * math.cos(y[0]))]

        def half(_, y):
            return y[0] - math.pi / 2
        half.terminal = True
        t_star = solve_ivp(rhs, (0, spec.max_steps * dt), [th0], rtol=1e-12, atol=1e-14,
                           events=half).t_events[0][0]
        assert stopped and m[2, 0, 0, 0] <= 0
        assert abs(n - t_star / dt) < 3
