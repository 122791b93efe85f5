"""LLG right-hand side, spin torques and integrators of the oracle.

Methods, "Physics and discretization", Eq. 1:
    dm/dt = -gamma' mu0 (m x H) - gamma' alpha mu0 m x (m x H),
    gamma' = gamma0 / (1 + alpha^2),
with the spin torques entering every integrator stage (Slonczewski STT, spin-orbit
torque, Zhang-Li), and Methods, "Integrators": Heun (stochastic LLG,
Stratonovich: the same thermal field in predictor and corrector), RK45
Dormand-Prince (adaptive, first-same-as-last), classical RK4 and the
norm-exact Depondt-Mertens rotation scheme (Rodrigues update).

Spin-torque forms (the paper names the torques, not their formulas).  A
damping-like coefficient h_DL and a field-like coefficient h_FL (A/m) along
the polarisation p enter the Gilbert form as
    -gamma0 mu0 h_DL m x (m x p)  and  -gamma0 mu0 h_FL m x p;
converted to Eq. 1's Landau-Lifshitz form they read
    tau = -gamma' mu0 [ (h_DL + alpha h_FL) m x (m x p) + (h_FL - alpha h_DL) m x p ].
 * SOT (spin Hall):   h_DL = theta_SH hbar J / (2 e mu0 Ms t_F), h_FL = r_FL h_DL
 * Slonczewski STT:   h_DL = eps(m) hbar J/(e mu0 Ms t_F), h_FL = eps' hbar J/(e mu0 Ms t_F),
                      eps = P L^2 / ((L^2 + 1) + (L^2 - 1)(m.p))
 * Zhang-Li (Methods): u = J P mu_B / (e Ms) along the current direction,
                      without 1/(1+xi^2) unless the mumax3-matching option is set;
   tau = 1/(1+alpha^2) [ -(1 + alpha xi) m x (m x (u.grad)m) - (xi - alpha) m x (u.grad)m ],
   (u.grad)m by central differences with the absent neighbour taken as the
   cell itself.

Integrator readings (the paper names only an adaptive DOPRI5 with FSAL reuse):
stages are not renormalised; err = max over cells of |m5 - m4|_2; accept
when err <= rtol; dt_new = dt * clamp(0.9 (rtol/err)^(1/5), 0.2, 5), with
the factor capped at 1 on the step after a rejection; dt clamped to
[dt_min, dt_max] (below dt_min is an error); on accept m <- m5/|m5| and the
FSAL slope k7 = f(m5) is reused unchanged.  Heun: the predictor is not
renormalised; the corrector result is.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction as F

import numpy as np

from .constants import GAMMA0, HBAR, MU0, MU_B, QE
from .demag import demag_spectrum, h_demag
from .fields import Problem, _shift, h_local
from .philox import splitmix64, thermal_field

# Dormand & Prince (1980) RK5(4)7FSAL coefficients, as exact fractions.
DP_C = [F(0), F(1, 5), F(3, 10), F(4, 5), F(8, 9), F(1), F(1)]
DP_A = [
    [],
    [F(1, 5)],
    [F(3, 40), F(9, 40)],
    [F(44, 45), F(-56, 15), F(32, 9)],
    [F(19372, 6561), F(-25360, 2187), F(64448, 6561), F(-212, 729)],
    [F(9017, 3168), F(-355, 33), F(46732, 5247), F(49, 176), F(-5103, 18656)],
    [F(35, 384), F(0), F(500, 1113), F(125, 192), F(-2187, 6784), F(11, 84)],
]
DP_B5 = [F(35, 384), F(0), F(500, 1113), F(125, 192), F(-2187, 6784), F(11, 84), F(0)]
DP_B4 = [F(5179, 57600), F(0), F(7571, 16695), F(393, 640), F(-92097, 339200), F(187, 2100), F(1, 40)]


def cross(a, b):
    return np.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


def dot(a, b):
    return (a * b).sum(axis=0)


@dataclass
class Torque:
    """Spin-torque description.  kind in {"none", "sot", "stt", "zl"}."""
    kind: str = "none"
    J: float = 0.0                       # A/m^2
    p: tuple = (0.0, 1.0, 0.0)           # polarisation (SOT, STT)
    theta_SH: float = 0.0                # SOT spin Hall angle
    fl_ratio: float = 0.0                # SOT field-like / damping-like ratio
    P: float = 0.0                       # STT, ZL polarisation
    Lambda: float = 1.0                  # STT asymmetry
    eps_prime: float = 0.0               # STT secondary term
    t_F: float = 0.0                     # free-layer thickness (0 -> nz * dz)
    xi: float = 0.0                      # ZL non-adiabaticity
    direction: tuple = (1.0, 0.0, 0.0)   # ZL current direction
    match_mumax: bool = False            # ZL: divide u by (1 + xi^2)


def llg_rhs(m, H, p: Problem):
    """Eq. 1 (Landau-Lifshitz form)."""
    gp = GAMMA0 / (1.0 + p.alpha ** 2)
    mxH = cross(m, H)
    out = -gp * MU0 * (mxH + p.alpha * cross(m, mxH))
    return np.where(p.present, out, 0.0)


def _st_coefficients(m, p: Problem, tq: Torque, nz: int):
    """Damping-like and field-like coefficients h_DL, h_FL (A/m) and the unit
    polarisation p of the SOT / Slonczewski STT term, or None."""
    pol = np.asarray(tq.p, dtype=np.float64)
    pol = pol / np.linalg.norm(pol)
    pv = np.broadcast_to(pol[:, None, None, None], m.shape)
    t_F = tq.t_F if tq.t_F > 0 else nz * p.d[2]
    with np.errstate(divide="ignore", invalid="ignore"):
        base = np.where(p.present, HBAR * tq.J / (QE * MU0 * np.where(p.present, p.Ms, 1.0) * t_F), 0.0)
    if tq.kind == "sot":
        hDL = 0.5 * tq.theta_SH * base
        hFL = tq.fl_ratio * hDL
    elif tq.kind == "stt":
        L2 = tq.Lambda ** 2
        eps = tq.P * L2 / ((L2 + 1.0) + (L2 - 1.0) * dot(m, pv))
        hDL = eps * base
        hFL = tq.eps_prime * base
    else:
        return None
    return hDL, hFL, pv


def spin_torque(m, p: Problem, tq: Torque, nz: int):
    """SOT or Slonczewski STT term in Landau-Lifshitz form."""
    c = _st_coefficients(m, p, tq, nz)
    if c is None:
        return np.zeros_like(m)
    hDL, hFL, pv = c
    gp = GAMMA0 / (1.0 + p.alpha ** 2)
    mxp = cross(m, pv)
    out = -gp * MU0 * ((hDL + p.alpha * hFL) * cross(m, mxp) + (hFL - p.alpha * hDL) * mxp)
    return np.where(p.present, out, 0.0)


def _zl_drive(m, p: Problem, tq: Torque):
    """(u.grad) m of the Zhang-Li torque (A/m per m/s: the drift u times the
    central-difference gradient, the absent neighbour taken as the cell)."""
    d = np.asarray(tq.direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.where(p.present, tq.J * tq.P * MU_B / (QE * np.where(p.present, p.Ms, 1.0)), 0.0)
    if tq.match_mumax:
        u = u / (1.0 + tq.xi ** 2)
    grad = np.zeros_like(m)
    for direction in range(3):
        if d[direction] == 0.0:
            continue
        per = bool(p.pbc[direction])
        Ms_p = _shift(p.Ms, direction, +1, per)
        Ms_m = _shift(p.Ms, direction, -1, per)
        mp = np.where(Ms_p > 0, _shift(m, direction, +1, per), m)
        mm = np.where(Ms_m > 0, _shift(m, direction, -1, per), m)
        grad += d[direction] * (mp - mm) / (2.0 * p.d[direction])
    return u * grad


def zhang_li_torque(m, p: Problem, tq: Torque):
    ug = _zl_drive(m, p, tq)
    mxug = cross(m, ug)
    out = (-(1.0 + p.alpha * tq.xi) * cross(m, mxug) - (tq.xi - p.alpha) * mxug) / (1.0 + p.alpha ** 2)
    return np.where(p.present, out, 0.0)


def rotate(m, w, dt):
    """Rotation of every cell's m about its own axis w / |w| by the angle
    |w| dt (right-handed), Rodrigues' formula
        R m = m cos a + (n x m) sin a + n (n . m)(1 - cos a),  a = |w| dt,
    so that for constant w the result solves dm/dt = w x m exactly.  Cells
    with w = 0 are unchanged."""
    wn = np.sqrt(dot(w, w))
    a = wn * dt
    n = w / np.where(wn > 0, wn, 1.0)
    c, s = np.cos(a), np.sin(a)
    return m * c + cross(n, m) * s + n * (dot(n, m) * (1.0 - c))


def _unit(m, present):
    n = np.sqrt(dot(m, m))
    return np.where(present, m / np.where(n > 0, n, 1.0), 0.0)


@dataclass
class Solver:
    """One instance advanced by Heun or RK45 in FP64.

    ``terms`` selects the effective-field contributions; ``T`` > 0 adds the
    Philox thermal field (Heun and Depondt-Mertens only, as adaptive
    stepping with white noise is not defined).
    """
    p: Problem
    m: np.ndarray
    terms: tuple = ("exchange", "dmi", "anisotropy", "zeeman", "demag")
    torque: Torque = field(default_factory=Torque)
    T: float = 0.0
    seed: int = 0
    dt: float = 1e-14
    rtol: float = 1e-6
    dt_min: float = 1e-20
    dt_max: float = 1e-11
    t: float = 0.0
    step: int = 0
    K_hat: np.ndarray = None
    k1: np.ndarray = None
    last_rejected: bool = False
    accepted: int = 0
    rejected: int = 0

    def __post_init__(self):
        self.m = _unit(np.array(self.m, dtype=np.float64), self.p.present)
        if "demag" in self.terms and self.K_hat is None:
            self.K_hat = demag_spectrum(self.p.shape, self.p.d, images=tuple(int(v) for v in self.p.pbc))

    # -- field and slope ----------------------------------------------------
    def field(self, m, h_th=None):
        H = np.zeros_like(m)
        for v in h_local(m, self.p, self.terms).values():
            H += v
        if "demag" in self.terms:
            H += h_demag(m, self.p, self.K_hat)
        if h_th is not None:
            H += h_th
        return np.where(self.p.present, H, 0.0)

    def slope(self, m, h_th=None):
        k = llg_rhs(m, self.field(m, h_th), self.p)
        if self.torque.kind in ("sot", "stt"):
            k = k + spin_torque(m, self.p, self.torque, self.p.shape[0])
        elif self.torque.kind == "zl":
            k = k + zhang_li_torque(m, self.p, self.torque)
        return k

    # -- Heun ---------------------------------------------------------------
    def thermal(self, dt):
        if self.T <= 0:
            return None
        return thermal_field(self.p, self.T, dt, self.seed, self.step)

    def heun_step(self, dt=None):
        dt = self.dt if dt is None else dt
        h_th = self.thermal(dt)
        k1 = self.slope(self.m, h_th)
        m_star = self.m + dt * k1
        k2 = self.slope(m_star, h_th)
        self.m = _unit(self.m + 0.5 * dt * (k1 + k2), self.p.present)
        self.t += dt
        self.step += 1
        self.accepted += 1

    # -- classical Runge-Kutta (fixed step) -----------------------------------
    def rk4_step(self, dt=None):
        """Methods, "Integrators" (RK4, fixed step): four slopes, the weighted
        sum (k1 + 2 k2 + 2 k3 + k4) / 6, stages not renormalised, |m| = 1
        restored after the step."""
        dt = self.dt if dt is None else dt
        k1 = self.slope(self.m)
        k2 = self.slope(self.m + 0.5 * dt * k1)
        k3 = self.slope(self.m + 0.5 * dt * k2)
        k4 = self.slope(self.m + dt * k3)
        self.m = _unit(self.m + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4), self.p.present)
        self.t += dt
        self.step += 1
        self.accepted += 1

    # -- Depondt-Mertens rotation scheme ---------------------------------------
    def omega(self, m, h_th=None):
        """Methods, "Integrators" (norm-exact Depondt-Mertens scheme): Eq. 1
        written as a rotation, dm/dt = Omega x m.  Since -m x H = H x m and
        -m x (m x H) = (m x H) x m,
            Omega = gamma' mu0 (H + alpha m x H)
        and the spin torques above contribute, by the same two identities,
            gamma' mu0 [ (h_DL + alpha h_FL) m x p + (h_FL - alpha h_DL) p ]
            (1 + alpha xi) m x u' + (xi - alpha) u'   over (1 + alpha^2)
        (SOT/STT; Zhang-Li with u' = (u.grad) m).  Omega x m is the slope."""
        p = self.p
        H = self.field(m, h_th)
        gp = GAMMA0 / (1.0 + p.alpha ** 2)
        w = gp * MU0 * (H + p.alpha * cross(m, H))
        if self.torque.kind in ("sot", "stt"):
            hDL, hFL, pv = _st_coefficients(m, p, self.torque, p.shape[0])
            w = w + gp * MU0 * ((hDL + p.alpha * hFL) * cross(m, pv) + (hFL - p.alpha * hDL) * pv)
        elif self.torque.kind == "zl":
            tq = self.torque
            ug = _zl_drive(m, p, tq)
            w = w + ((1.0 + p.alpha * tq.xi) * cross(m, ug) + (tq.xi - p.alpha) * ug) / (1.0 + p.alpha ** 2)
        return np.where(p.present, w, 0.0)

    def dm_step(self, dt=None):
        """Methods, "Integrators" and "Replica batching" (Depondt and Mertens,
        2009): a predictor-corrector on rotations.  Omega_1 = Omega(m_n);
        the predictor m* rotates m_n about Omega_1 for dt; Omega_2 =
        Omega(m*); m_{n+1} rotates m_n about (Omega_1 + Omega_2) / 2 for dt.
        One thermal draw serves both Omega evaluations (Stratonovich).  A
        rotation keeps |m|, so nothing is renormalised."""
        dt = self.dt if dt is None else dt
        h_th = self.thermal(dt)
        w1 = self.omega(self.m, h_th)
        m_star = rotate(self.m, w1, dt)
        w2 = self.omega(m_star, h_th)
        self.m = np.where(self.p.present, rotate(self.m, 0.5 * (w1 + w2), dt), 0.0)
        self.t += dt
        self.step += 1
        self.accepted += 1

    def dm_adaptive_step(self):
        """Methods, "Integrators": the Depondt-Mertens scheme, which the paper
        allows to run adaptively.  Reading (it gives no controller): the predictor
        m* (a first-order rotation) and the corrector m_{n+1} (second order)
        form an embedded pair; err = max over cells |m_{n+1} - m*|; accept
        when err <= rtol; dt_new = dt * clamp(0.9 (rtol/err)^(1/2), 0.2, 5),
        capped at 1 right after a rejection; dt within [dt_min, dt_max].
        T must be 0.  Returns the accepted dt."""
        if self.T > 0:
            raise ValueError("adaptive stepping with white noise is not defined")
        while True:
            dt = self.dt
            w1 = self.omega(self.m)
            m_star = rotate(self.m, w1, dt)
            w2 = self.omega(m_star)
            m_new = np.where(self.p.present, rotate(self.m, 0.5 * (w1 + w2), dt), 0.0)
            d = m_new - np.where(self.p.present, m_star, 0.0)
            err = float(np.sqrt(dot(d, d)).max()) if d.size else 0.0
            fac = 0.9 * (self.rtol / err) ** 0.5 if err > 0 else 5.0
            fac = min(max(fac, 0.2), 5.0)
            if err <= self.rtol:
                if self.last_rejected:
                    fac = min(fac, 1.0)
                self.m = m_new
                self.t += dt
                self.step += 1
                self.accepted += 1
                self.last_rejected = False
                self.dt = min(dt * fac, self.dt_max)
                return dt
            self.rejected += 1
            self.last_rejected = True
            new_dt = dt * fac
            if new_dt < self.dt_min:
                raise FloatingPointError("Depondt-Mertens time step underflow")
            self.dt = new_dt

    # -- Dormand-Prince -----------------------------------------------------
    def dopri_attempt(self, dt):
        """Returns (m5, err, k7) for one attempted step from self.m."""
        if self.k1 is None:
            self.k1 = self.slope(self.m)
        k = [self.k1]
        for s in range(1, 7):
            ms = self.m.copy()
            for j, a in enumerate(DP_A[s]):
                if a != 0:
                    ms = ms + dt * float(a) * k[j]
            k.append(self.slope(ms))
        m5 = ms                              # row 7 of A equals the 5th-order weights
        delta = np.zeros_like(self.m)
        for j in range(7):
            e = DP_B5[j] - DP_B4[j]
            if e != 0:
                delta = delta + dt * float(e) * k[j]
        err = float(np.sqrt(dot(delta, delta)).max()) if delta.size else 0.0
        return m5, err, k[6]

    def rk45_step_fixed(self, dt):
        """Advance by exactly dt (replay of a known accepted step sequence)."""
        m5, err, k7 = self.dopri_attempt(dt)
        self.m = _unit(m5, self.p.present)
        self.k1 = k7
        self.t += dt
        self.step += 1
        self.accepted += 1
        return err

    def rk45_step(self):
        """Attempt steps until one is accepted; returns the accepted dt."""
        while True:
            dt = self.dt
            m5, err, k7 = self.dopri_attempt(dt)
            if err > 0:
                fac = 0.9 * (self.rtol / err) ** 0.2
            else:
                fac = 5.0
            fac = min(max(fac, 0.2), 5.0)
            if err <= self.rtol:
                if self.last_rejected:
                    fac = min(fac, 1.0)
                self.m = _unit(m5, self.p.present)
                self.k1 = k7
                self.t += dt
                self.step += 1
                self.accepted += 1
                self.last_rejected = False
                self.dt = min(dt * fac, self.dt_max)
                return dt
            self.rejected += 1
            self.last_rejected = True
            new_dt = dt * fac
            if new_dt < self.dt_min:
                raise FloatingPointError("RK45 time step underflow")
            self.dt = new_dt


def replica_seed(base_seed: int, r: int) -> int:
    return splitmix64((int(base_seed) + int(r)) & ((1 << 64) - 1))
