"""Pins of the oracle's counter-based thermal field: exactness of the
uniforms, the statistics of the normals, counter/key sensitivity, and the
macrospin Langevin equilibrium the paper validates sigma against
(<m_z> = L(3) = coth 3 - 1/3 = 0.672; the paper measures 0.675)."""
import math
import os

import numpy as np

import workloads as W
from oracle.constants import KB, MU0
from oracle.fields import Problem
from oracle.llg import Solver
from oracle.philox import normals, philox4x32_10, raw, splitmix64, uniforms


def test_uniforms_are_exact_multiples_in_unit_interval():
    x = np.array([0, 255, 256, 0xFFFFFFFF, 0x12345678], dtype=np.uint64)
    u = uniforms(x)
    assert u[0] == 2.0 ** -24 and u[1] == 2.0 ** -24 and u[2] == 2.0 ** -23
    assert u[3] == 1.0
    k = u * 2 ** 24
    assert np.all(k == np.round(k)) and np.all((u > 0) & (u <= 1))
    # float32 holds every value exactly
    assert np.all(u.astype(np.float32).astype(np.float64) == u)


def test_philox_outputs_are_uniform_and_decorrelated():
    x0, x1, x2, x3 = raw(seed=12345, step=7, ncell=1 << 16)
    bits = np.concatenate([x0, x1, x2, x3]).astype(np.uint64)
    # every bit position set about half of the time
    frac = np.array([((bits >> np.uint64(b)) & np.uint64(1)).mean() for b in range(32)])
    assert np.all(np.abs(frac - 0.5) < 0.01)
    # byte histogram is flat (chi-square, 255 dof)
    h = np.bincount((bits & np.uint64(0xFF)).astype(np.int64), minlength=256)
    e = len(bits) / 256
    chi2 = ((h - e) ** 2 / e).sum()
    assert chi2 < 350
    # adjacent counters / adjacent output words are uncorrelated
    u = uniforms(x0)
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.02
    assert abs(np.corrcoef(uniforms(x0), uniforms(x1))[0, 1]) < 0.02


def test_philox_avalanche_on_counter_and_key():
    base = philox4x32_10(np.arange(4096), 5, 0, 0, 0xDEADBEEF, 0x1234)
    flips = []
    for args in [(np.arange(4096) ^ 1, 5, 0, 0, 0xDEADBEEF, 0x1234),
                 (np.arange(4096), 4, 0, 0, 0xDEADBEEF, 0x1234),
                 (np.arange(4096), 5, 0, 0, 0xDEADBEEE, 0x1234),
                 (np.arange(4096), 5, 0, 1, 0xDEADBEEF, 0x1234)]:
        other = philox4x32_10(*args)
        diff = np.concatenate([(a ^ b) for a, b in zip(base, other)]).astype(np.uint64)
        ones = sum(((diff >> np.uint64(b)) & np.uint64(1)).sum() for b in range(32))
        flips.append(ones / (diff.size * 32))
    assert all(abs(f - 0.5) < 0.01 for f in flips), flips


def test_normals_statistics():
    g = normals(seed=99, step=3, ncell=200000).ravel()
    assert abs(g.mean()) < 0.01
    assert abs(g.var() - 1) < 0.01
    assert abs((g ** 4).mean() - 3) < 0.05          # Gaussian kurtosis
    g2 = normals(seed=99, step=4, ncell=200000).ravel()
    assert abs(np.corrcoef(g, g2)[0, 1]) < 0.01
    assert np.all(normals(seed=99, step=3, ncell=1000) == normals(seed=99, step=3, ncell=1000))


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_philox_known_answer_vectors():
    """The generator's published known-answer vectors (all-zero, all-ones and
    pi-digit counters and keys)."""
    rows = _rows("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for row in rows:
        c0, c1, c2, c3, k0, k1, *want = (int(v, 16) for v in row)
        got = philox4x32_10([c0], [c1], [c2], [c3], [k0], [k1])
        assert [int(x[0]) for x in got] == want


def test_splitmix64_known_answer_sequence():
    rows = _rows("splitmix64_kat.txt")
    assert rows[0][0] == "state"
    state = int(rows[0][1])
    for row in rows[1:]:
        assert splitmix64(state) == int(row[0])
        state = (state + 0x9E3779B97F4A7C15) % (1 << 64)


def test_splitmix64_is_a_bijective_mixer():
    outs = {splitmix64(i) for i in range(20000)}
    assert len(outs) == 20000
    assert splitmix64(0) != splitmix64(1) and splitmix64(0) < 2 ** 64


def test_langevin_equilibrium_of_macrospins():
    """Independent single-cell moments in a field at temperature T: the
    time/ensemble average of m.z approaches the Langevin function
    L(xi) = coth xi - 1/xi with xi = mu0 Ms V H / kB T, at the paper's
    xi = 3 (tests/golden/langevin_macrospin.txt)."""
    fx = {row[0]: float(row[2]) for row in _rows("langevin_macrospin.txt")}
    xi = fx["xi"]
    n = 2048
    T = 300.0
    cell = 2e-9
    V = cell ** 3
    Ms = 8e5
    H = xi * KB * T / (MU0 * Ms * V)
    grid = W.Grid(n, 1, 1, cell, cell, cell)
    # no exchange: every cell is an independent macrospin
    p = Problem.from_workload(grid, W.Material(Ms=Ms, A=0.0, alpha=1.0), B_ext=(0.0, 0.0, MU0 * H))
    m0 = np.zeros((3,) + p.shape)
    m0[2] = 1.0
    s = Solver(p, m0, terms=("zeeman",), T=T, seed=2024, dt=2e-14)
    acc = []
    for it in range(3000):
        s.heun_step()
        if it >= 1000 and it % 10 == 0:
            acc.append(s.m[2].mean())
    mz = float(np.mean(acc))
    L_xi = 1.0 / math.tanh(xi) - 1.0 / xi
    assert round(L_xi, 3) == fx["L_xi_printed"]
    assert abs(mz - L_xi) < 0.015, (mz, L_xi)
    # the paper's own measurement sits as far from L(3) as this sampling allows
    assert abs(fx["mz_measured_printed"] - L_xi) < 0.015
