"""Pins of the oracle's LLG right-hand side, spin torques and integrators:
the closed-form macrospin trajectory, convergence orders, the Dormand-Prince
order conditions, |m| = 1 and energy dissipation."""
import math
from fractions import Fraction as F

import numpy as np
import pytest

import workloads as W
from oracle.constants import GAMMA0, MU0
from oracle.fields import Problem
from oracle.llg import DP_A, DP_B4, DP_B5, DP_C, Solver, Torque, cross, dot, spin_torque, zhang_li_torque
from oracle.observables import energy


def test_dormand_prince_order_conditions():
    c, b, bh = DP_C, DP_B5, DP_B4
    for i in range(1, 7):
        assert sum(DP_A[i]) == c[i]
    assert DP_A[6] == b[:6]                       # first same as last
    assert sum(b) == 1 and sum(bh) == 1
    # 5th-order quadrature conditions of b, 4th of b_hat
    for q in range(1, 6):
        assert sum(bi * ci ** (q - 1) for bi, ci in zip(b, c)) == F(1, q)
    for q in range(1, 5):
        assert sum(bi * ci ** (q - 1) for bi, ci in zip(bh, c)) == F(1, q)
    A = [row + [F(0)] * (7 - len(row)) for row in DP_A]
    # sum_i b_i sum_j a_ij c_j = 1/6, sum_i b_i c_i sum_j a_ij c_j = 1/8
    Ac = [sum(A[i][j] * c[j] for j in range(7)) for i in range(7)]
    assert sum(b[i] * Ac[i] for i in range(7)) == F(1, 6)
    assert sum(b[i] * c[i] * Ac[i] for i in range(7)) == F(1, 8)
    Ac2 = [sum(A[i][j] * c[j] ** 2 for j in range(7)) for i in range(7)]
    assert sum(b[i] * Ac2[i] for i in range(7)) == F(1, 12)
    AAc = [sum(A[i][j] * Ac[j] for j in range(7)) for i in range(7)]
    assert sum(b[i] * AAc[i] for i in range(7)) == F(1, 24)
    # a 5th-order condition
    assert sum(b[i] * c[i] ** 2 * Ac[i] for i in range(7)) == F(1, 10)


def _macrospin(alpha=0.1, H0=8e5, theta0=1.0, phi0=0.3):
    # a cube cell: self-demag is parallel to m and exerts no torque
    grid = W.Grid(1, 1, 1, 2e-9, 2e-9, 2e-9)
    p = Problem.from_workload(grid, W.Material(Ms=8e5, A=1e-11, alpha=alpha), B_ext=(0, 0, MU0 * H0))
    m0 = np.array([math.sin(theta0) * math.cos(phi0), math.sin(theta0) * math.sin(phi0), math.cos(theta0)])
    return p, m0.reshape(3, 1, 1, 1)


def _closed_form(t, alpha, H0, theta0, phi0):
    gp = GAMMA0 / (1 + alpha ** 2)
    th = 2 * math.atan(math.tan(theta0 / 2) * math.exp(-gp * alpha * MU0 * H0 * t))
    ph = phi0 + gp * MU0 * H0 * t
    return np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])


def test_macrospin_dopri_matches_closed_form():
    alpha, H0 = 0.1, 8e5
    p, m0 = _macrospin(alpha, H0)
    s = Solver(p, m0, terms=("zeeman", "demag"), dt=1e-13, rtol=1e-9)
    while s.t < 50e-12:
        s.rk45_step()
    exp = _closed_form(s.t, alpha, H0, 1.0, 0.3)
    assert np.max(np.abs(s.m[:, 0, 0, 0] - exp)) < 1e-8


def test_heun_second_order_and_dopri_fifth_order():
    alpha, H0 = 0.05, 5e5
    p, m0 = _macrospin(alpha, H0)
    T = 20e-12
    errs_h, errs_d = [], []
    for n in (200, 400, 800):
        s = Solver(p, m0, terms=("zeeman",))
        for _ in range(n):
            s.heun_step(T / n)
        errs_h.append(np.abs(s.m[:, 0, 0, 0] - _closed_form(T, alpha, H0, 1.0, 0.3)).max())
    for n in (20, 40, 80):
        s = Solver(p, m0, terms=("zeeman",))
        for _ in range(n):
            s.rk45_step_fixed(T / n)
        errs_d.append(np.abs(s.m[:, 0, 0, 0] - _closed_form(T, alpha, H0, 1.0, 0.3)).max())
    rate_h = math.log2(errs_h[0] / errs_h[1]), math.log2(errs_h[1] / errs_h[2])
    rate_d = math.log2(errs_d[0] / errs_d[1]), math.log2(errs_d[1] / errs_d[2])
    assert all(1.8 < r < 2.3 for r in rate_h), rate_h
    assert all(4.6 < r < 6.5 for r in rate_d), rate_d


def test_dopri_error_estimate_is_the_fourth_order_local_error():
    """The embedded estimate |m5 - m4| that drives the step controller falls
    as h^5 over one step (the local error of the 4th-order solution), while
    the 5th-order solution's own local error against the closed form falls
    as h^6 and stays well below the estimate (Dormand & Prince 1980: the
    5th-order solution is propagated, the 4th-order one only measured).  A
    wrong 4th-order weight lowers the estimate's order; a wrong stage or
    5th-order weight lowers the local error's."""
    alpha, H0 = 0.05, 5e5
    p, m0 = _macrospin(alpha, H0)
    errs, locs = [], []
    for h in (2e-12, 1e-12, 5e-13):
        s = Solver(p, m0, terms=("zeeman",))
        m5, err, _ = s.dopri_attempt(h)
        errs.append(err)
        locs.append(np.abs(m5[:, 0, 0, 0] - _closed_form(h, alpha, H0, 1.0, 0.3)).max())
    r_err = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    r_loc = [math.log2(locs[i] / locs[i + 1]) for i in range(2)]
    assert all(4.8 < r < 5.2 for r in r_err), r_err
    assert all(5.7 < r < 6.4 for r in r_loc), r_loc
    assert all(loc < 0.1 * e for loc, e in zip(locs, errs)), (locs, errs)


def test_rk4_fourth_order_on_the_macrospin():
    """Classical RK4 against the closed-form damped precession: halving the
    step divides the error by ~16."""
    alpha, H0 = 0.05, 5e5
    p, m0 = _macrospin(alpha, H0)
    T = 20e-12
    errs = []
    for n in (40, 80, 160):
        s = Solver(p, m0, terms=("zeeman",))
        for _ in range(n):
            s.rk4_step(T / n)
        errs.append(np.abs(s.m[:, 0, 0, 0] - _closed_form(T, alpha, H0, 1.0, 0.3)).max())
    rates = math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])
    assert all(3.6 < r < 4.5 for r in rates), rates
    assert errs[-1] < 1e-7


def test_rk4_single_step_is_the_classical_tableau():
    """One RK4 step of dm/dt = f(m) written out by hand for a linear field-free
    precession about z (f is linear in m for a Zeeman-only macrospin without
    damping), compared with the solver's step before renormalisation."""
    p, m0 = _macrospin(alpha=0.0, H0=4e5)
    s = Solver(p, m0, terms=("zeeman",))
    dt = 3e-13
    m = s.m.copy()
    f = s.slope
    k1 = f(m); k2 = f(m + dt / 2 * k1); k3 = f(m + dt / 2 * k2); k4 = f(m + dt * k3)
    ref = m + dt * (k1 / 6 + k2 / 3 + k3 / 3 + k4 / 6)
    ref = ref / np.sqrt((ref ** 2).sum())
    s.rk4_step(dt)
    assert np.abs(s.m - ref).max() < 1e-15
    # rotation angle per step of the exact solution: RK4 keeps the phase to O(dt^5)
    w = GAMMA0 * MU0 * 4e5 * dt
    assert abs(math.atan2(s.m[1, 0, 0, 0], s.m[0, 0, 0, 0]) - math.atan2(m0[1, 0, 0, 0], m0[0, 0, 0, 0]) - w) < 1e-4 * w


def test_precession_sense_follows_eq1():
    # m = x, H = z: dm/dt = -gamma' mu0 m x H = +gamma' mu0 H y
    p, _ = _macrospin(alpha=0.0)
    s = Solver(p, np.array([1.0, 0, 0]).reshape(3, 1, 1, 1), terms=("zeeman",))
    k = s.slope(s.m)[:, 0, 0, 0]
    assert k[1] > 0 and abs(k[0]) < 1e-6 * k[1] and abs(k[2]) < 1e-6 * k[1]


def _film(seed=1, D=2e-3, Ku=3e5, shape=(12, 8, 2)):
    grid = W.Grid(*shape, 2e-9, 2e-9, 2e-9)
    mat = W.Material(Ms=6e5, A=1.3e-11, alpha=0.3, Ku1=Ku, u=(0, 0, 1), D=D)
    p = Problem.from_workload(grid, mat, B_ext=(0.02, 0.0, 0.05))
    return grid, p, W.random_m(grid, seed=seed)


def test_norm_preserved_and_energy_dissipated():
    """alpha > 0, T = 0, static field, no current: E never increases over
    accepted RK45 steps (free DMI edges included), |m| = 1 to rounding."""
    grid, p, m = _film()
    s = Solver(p, m, dt=1e-14, rtol=1e-7)
    E = [energy(s.m, p, s.K_hat)["total"]]
    for _ in range(60):
        s.rk45_step()
        n = np.sqrt(dot(s.m, s.m))
        assert np.abs(n - 1).max() < 1e-15 * 4
        E.append(energy(s.m, p, s.K_hat)["total"])
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-12 * np.abs(E[:-1])), np.diff(E).max()
    assert E[-1] < E[0]


def test_sot_special_cases():
    grid = W.Grid(1, 1, 1, 2e-9, 2e-9, 1e-9)
    p = Problem.from_workload(grid, W.Material(Ms=1.1e6, A=2e-11, alpha=0.0))
    tq = Torque(kind="sot", J=2e11, p=(0, 1, 0), theta_SH=0.1)
    m_par = np.array([0, 1.0, 0]).reshape(3, 1, 1, 1)
    assert np.abs(spin_torque(m_par, p, tq, 1)).max() == 0
    m = np.array([0.6, 0.0, 0.8]).reshape(3, 1, 1, 1)
    t = spin_torque(m, p, tq, 1)[:, 0, 0, 0]
    from oracle.constants import HBAR, QE
    hDL = 0.1 * HBAR * 2e11 / (2 * QE * MU0 * 1.1e6 * 1e-9)
    pv = np.array([0, 1.0, 0])
    mv = m[:, 0, 0, 0]
    # alpha = 0: pure rotation toward p, magnitude gamma0 mu0 h_DL |p - m(m.p)|
    assert np.allclose(t, GAMMA0 * MU0 * hDL * (pv - mv * np.dot(mv, pv)), rtol=1e-12)
    assert np.dot(t, pv) > 0


def test_stt_efficiency_limits_and_direction():
    grid = W.Grid(1, 1, 1, 2e-9, 2e-9, 1e-9)
    p = Problem.from_workload(grid, W.Material(Ms=1e6, A=2e-11, alpha=0.0))
    Lam, P = 2.0, 0.6
    tq = Torque(kind="stt", J=1e11, p=(0, 0, 1), P=P, Lambda=Lam)
    th = 0.4
    for mz_sign, eps in [(+1, P / 2), (-1, P * Lam ** 2 / 2)]:
        # near the limits m.p -> +-1 the torque magnitude / |p - m(m.p)| -> eps * base
        m = np.array([math.sin(1e-3), 0, mz_sign * math.cos(1e-3)]).reshape(3, 1, 1, 1)
        t = spin_torque(m, p, tq, 1)[:, 0, 0, 0]
        mv = m[:, 0, 0, 0]
        perp = np.array([0, 0, 1.0]) - mv * mv[2]
        from oracle.constants import HBAR, QE
        base = HBAR * 1e11 / (QE * MU0 * 1e6 * 1e-9)
        assert np.allclose(t, GAMMA0 * MU0 * eps * base * perp, rtol=1e-3)
    m = np.array([math.sin(th), 0, math.cos(th)]).reshape(3, 1, 1, 1)
    t = spin_torque(m, p, tq, 1)[:, 0, 0, 0]
    assert t[2] > 0      # J > 0 pulls m toward p


def test_zhang_li_uniform_is_zero_and_wall_translates():
    grid = W.Grid(8, 3, 1, 2e-9, 2e-9, 1e-9)
    p = Problem.from_workload(grid, W.Material(Ms=8e5, A=1.3e-11, alpha=0.02))
    tq = Torque(kind="zl", J=1e12, P=0.5, xi=0.02)
    m = np.zeros((3,) + p.shape)
    m[2] = 1.0
    assert np.abs(zhang_li_torque(m, p, tq)).max() == 0
    # xi = alpha: a Bloch wall in a chain translates rigidly, m(x,t) = m(x + u t, 0)
    n, dx = 200, 1e-9
    Ms, A, K = 8e5, 1.3e-11, 5e5
    grid = W.Grid(n, 1, 1, dx, dx, dx)
    p = Problem.from_workload(grid, W.Material(Ms=Ms, A=A, alpha=0.05, Ku1=K, u=(0, 0, 1)))
    delta = math.sqrt(A / K)
    x = (np.arange(n) - n / 2 + 0.5) * dx
    th = 2 * np.arctan(np.exp(x / delta))
    m = np.zeros((3,) + p.shape)
    m[1, 0, 0] = np.sin(th)
    m[2, 0, 0] = np.cos(th)
    s = Solver(p, m, terms=("exchange", "anisotropy"), dt=1e-14, rtol=1e-8)
    for _ in range(2000):          # relax the discrete wall first
        s.rk45_step()
        if s.t > 20e-12:
            break
    from oracle.constants import MU_B, QE
    J, P = 2e12, 0.5
    u = J * P * MU_B / (QE * Ms)
    s.torque = Torque(kind="zl", J=J, P=P, xi=0.05)
    mz0 = s.m[2].mean()
    t0 = s.t
    while s.t - t0 < 50e-12:
        s.rk45_step()
    shift = (s.m[2].mean() - mz0) * n * dx / 2      # <mz> = 2 x_centre / L for this wall
    assert abs(shift - (-u * (s.t - t0))) < 0.03 * u * (s.t - t0)


@pytest.mark.parametrize("J_over_Jc0,eps_prime", [(2.0, 0.0), (0.5, 0.0), (1.5, 0.3)])
def test_stt_macrospin_polar_angle_follows_its_scalar_equation(J_over_Jc0, eps_prime):
    """Perpendicular macrospin with p = -z: precession and the m x p terms
    only turn the azimuth, so the polar angle obeys the scalar equation
    dtheta/dt = gamma' mu0 sin(theta) [h_DL(theta) + alpha h_FL - alpha H_K cos(theta)]
    with h_DL = eps(m.p) hbar J / (e mu0 Ms t_F), m.p = -cos(theta); below
    the threshold J_c0 = alpha H_K e mu0 Ms t_F / (hbar eps(-1)) the state
    relaxes, above it the current reverses it.  The oracle's 3-D integration
    must follow that equation (integrated here by scipy)."""
    from scipy.integrate import solve_ivp

    from oracle.constants import HBAR, QE
    Ms, Ku, alpha, P, Lam, dz = 1e6, 1e6, 0.02, 0.6, 2.0, 1e-9
    grid = W.Grid(1, 1, 1, 2e-9, 2e-9, dz)
    p = Problem.from_workload(grid, W.Material(Ms=Ms, A=1e-11, alpha=alpha, Ku1=Ku, u=(0, 0, 1)))
    HK = 2 * Ku / (MU0 * Ms)
    L2 = Lam ** 2
    Jc0 = alpha * HK * QE * MU0 * Ms * dz / (HBAR * P * L2 / 2)
    J = J_over_Jc0 * Jc0
    base = HBAR * J / (QE * MU0 * Ms * dz)
    gp = GAMMA0 / (1 + alpha ** 2)

    def rhs(_, y):
        th = y[0]
        eps = P * L2 / ((L2 + 1) - (L2 - 1) * math.cos(th))
        return [gp * MU0 * math.sin(th) * (eps * base + alpha * eps_prime * base - alpha * HK * math.cos(th))]

    th0, t_end = 0.2, 150e-12
    ref = solve_ivp(rhs, (0, t_end), [th0], rtol=1e-12, atol=1e-14).y[0, -1]
    m0 = np.array([math.sin(th0), 0.0, math.cos(th0)]).reshape(3, 1, 1, 1)
    tq = Torque(kind="stt", J=J, p=(0, 0, -1), P=P, Lambda=Lam, eps_prime=eps_prime)
    s = Solver(p, m0, terms=("anisotropy",), torque=tq, dt=1e-14, rtol=1e-10)
    while s.t < t_end:
        s.dt = min(s.dt, t_end - s.t)
        s.rk45_step()
    th = math.acos(float(s.m[2, 0, 0, 0]))
    assert abs(th - ref) < 1e-7
    assert (th > th0) == (J_over_Jc0 > 1)


def test_zhang_li_wall_velocity_follows_the_one_dimensional_model():
    """A wall in a uniaxial chain (no transverse anisotropy, so no Walker
    limit) driven by the Zhang-Li torque moves steadily at
    v = u (1 + alpha xi) / (1 + alpha^2) while its plane precesses at
    |xi - alpha| u / (delta (1 + alpha^2)) (the rigid-profile solution of the
    collective-coordinate equations).  alpha = 0.5 makes the xi dependence
    large; the common lattice factor of the central difference
    (about -(dx/delta)^2/6) cancels in the ratios."""
    from oracle.constants import MU_B, QE
    n, dx = 200, 1e-9
    Ms, A, K, alpha = 8e5, 1.3e-11, 5e5, 0.5
    grid = W.Grid(n, 1, 1, dx, dx, dx)
    p = Problem.from_workload(grid, W.Material(Ms=Ms, A=A, alpha=alpha, Ku1=K, u=(0, 0, 1)))
    delta = math.sqrt(A / K)
    x = (np.arange(n) - n / 2 + 0.5) * dx
    th = 2 * np.arctan(np.exp(x / delta))
    m = np.zeros((3,) + p.shape)
    m[1, 0, 0] = np.sin(th)
    m[2, 0, 0] = np.cos(th)
    s = Solver(p, m, terms=("exchange", "anisotropy"), dt=1e-14, rtol=1e-8)
    while s.t < 20e-12:
        s.rk45_step()
    m_rel = s.m.copy()
    J, P = 2e12, 0.5
    u = J * P * MU_B / (QE * Ms)
    v = {}
    for xi in (0.0, 0.5, 1.0):
        s = Solver(p, m_rel, terms=("exchange", "anisotropy"), dt=1e-14, rtol=1e-8,
                   torque=Torque(kind="zl", J=J, P=P, xi=xi))
        mz0 = s.m[2].mean()
        phi0 = math.atan2(s.m[1].sum(), s.m[0].sum())            # azimuth of the wall's moment
        while s.t < 50e-12:
            s.rk45_step()
        v[xi] = -(s.m[2].mean() - mz0) * n * dx / 2 / s.t       # <mz> = 2 x_centre / L
        lattice = 1 - (dx / delta) ** 2 / 6
        assert abs(v[xi] / (u * lattice * (1 + alpha * xi) / (1 + alpha ** 2)) - 1) < 2e-3, (xi, v[xi])
        # the wall drifts along -x (as the rigid translation at xi = alpha
        # shows), so for this wall the plane turns at -(xi - alpha) u / (delta (1 + alpha^2))
        rate = (math.atan2(s.m[1].sum(), s.m[0].sum()) - phi0) / s.t
        want = -(xi - alpha) * u / (delta * (1 + alpha ** 2))
        assert abs(rate - want) < 2e-3 * u / delta, (xi, rate, want)
    assert abs(v[1.0] / v[0.0] - (1 + alpha)) < 1e-4
    assert abs(v[0.5] / v[0.0] - (1 + alpha * 0.5)) < 1e-4
