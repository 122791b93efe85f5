"""Parity at the full sizes of the benchmark workloads.

* 128x32x1 thin film, FP64 RK45 (rtol 1e-6) for the whole 0.5 ns: the GPU
  replays the oracle's accepted step sequence; every cell compared.
* 256x256x16 DMI film: FP32 and FP64 replays of the oracle's first 20
  accepted RK45 steps from a random state; energy and topological charge of
  the final state against the oracle's compensated sums.
* 512x512x64 vortex (16.7 M cells, padded 1024x1024x128): its demag field
  against the oracle at every cell and at sampled cells by direct sums; too
  large for the oracle to step, so the FP32 run is held to the FP64 GPU run
  (itself held to the oracle at the smaller sizes) on the same steps, plus
  |m| = 1 and energy decay (alpha > 0, no applied field).
* 1024 uneven replicas: 200 Heun steps at 300 K with SOT, ten replicas
  covering every size class against the oracle.

Bars: FP64 max|dm| <= 1e-11, FP32 max|dm| <= 1e-5 (Methods, "Physics and
discretization": LLG of Eq. 1 integrated by the Dormand-Prince pair)."""
import functools

import numpy as np
import pytest

import workloads as W
from gpu_util import make_ctx, need_gpu, oracle_problem

pytestmark = pytest.mark.gpu


def _solver(w, m0, **kw):
    from oracle.demag import demag_spectrum
    from oracle.llg import Solver
    p = oracle_problem(w.grid, w.mat, w.B_ext)
    return Solver(p, m0, K_hat=demag_spectrum(p.shape, p.d), **kw), p


def test_thin_film_full_run_fp64():
    mm = need_gpu()
    w = W.film_128x32()
    m0 = W.m_uniform_perturbed(w.grid, seed=w.seed)
    o, p = _solver(w, m0, dt=1e-14, rtol=w.rtol)
    dts = []
    while o.t < w.t_end:
        dts.append(o.rk45_step())
    ctx = make_ctx(mm, w.grid, w.mat, precision=64, demag=True, B=w.B_ext, dt=1e-14, rtol=w.rtol)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_step_dt(ctx, dts)
        t, _, n = mm.mm_get_time(ctx)
        assert n == len(dts) and t >= w.t_end
        err = np.abs(mm.mm_get_m(ctx, 0, m0.shape) - o.m).max()
        assert err <= 1e-11, (len(dts), err)
    finally:
        mm.mm_destroy(ctx)


_DMI_REPLAY_STEPS = 20


@functools.lru_cache(maxsize=1)
def _dmi_oracle_run():
    """The oracle's first 20 accepted RK45 steps of the 256x256x16 DMI film
    from its seeded random state (about 10 s per step on one host core),
    shared by both precisions."""
    w = W.dmi_256x256x16()
    m0 = W.m_random_sphere(w.grid, seed=w.seed)
    o, p = _solver(w, m0, dt=1e-14, rtol=w.rtol)
    dts = [o.rk45_step() for _ in range(_DMI_REPLAY_STEPS)]
    return w, m0, dts, o.m.copy(), p, o.K_hat


@pytest.mark.parametrize("prec", [64, 32])
def test_dmi_film_256x256x16_replay(prec):
    mm = need_gpu()
    from oracle.observables import energy, topological_charge
    w, m0, dts, m_ref, p, K_hat = _dmi_oracle_run()
    ctx = make_ctx(mm, w.grid, w.mat, precision=prec, demag=True, B=w.B_ext, dt=1e-14, rtol=w.rtol)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_step_dt(ctx, dts)
        m = mm.mm_get_m(ctx, 0, m0.shape)
        err = np.abs(m - m_ref).max()
        assert err <= (1e-11 if prec == 64 else 1e-5), err
        if prec == 64:
            E = mm.mm_energy(ctx, 0)
            ref = energy(m, p, K_hat)
            assert abs(E[5] - ref["total"]) <= 1e-12 * max(abs(v) for v in ref.values())
            Q = mm.mm_topo_charge(ctx, 0)
            assert abs(Q - topological_charge(m, p)) <= 1e-9
    finally:
        mm.mm_destroy(ctx)


def test_vortex_512x512x64_fp32_against_fp64():
    mm = need_gpu()
    w = W.vortex_512x512x64()
    m0 = W.m_vortex(w.grid, seed=w.seed)
    c64 = make_ctx(mm, w.grid, w.mat, precision=64, demag=True, dt=1e-14, rtol=w.rtol)
    try:
        mm.mm_set_m(c64, 0, m0)
        E0 = mm.mm_energy(c64, 0)[5]
        ts = [0.0]
        for _ in range(3):
            mm.mm_step(c64, 1)
            ts.append(mm.mm_get_time(c64, 0)[0])
        dts = np.diff(ts)
        m64 = mm.mm_get_m(c64, 0, m0.shape)
        E1 = mm.mm_energy(c64, 0)[5]
    finally:
        mm.mm_destroy(c64)
    assert E1 <= E0
    assert np.abs(np.sqrt((m64 ** 2).sum(axis=0)) - 1.0).max() < 1e-12
    c32 = make_ctx(mm, w.grid, w.mat, precision=32, demag=True, dt=1e-14, rtol=w.rtol)
    try:
        mm.mm_set_m(c32, 0, m0)
        mm.mm_step_dt(c32, dts)
        m32 = mm.mm_get_m(c32, 0, m0.shape)
    finally:
        mm.mm_destroy(c32)
    assert np.abs(np.sqrt((m32 ** 2).sum(axis=0)) - 1.0).max() < 1e-6
    err = np.abs(m32 - m64).max()
    assert err <= 1e-5, err


def test_vortex_512x512x64_demag_field_sampled():
    """The 512x512x64 demag field (FP32, padded 1024x1024x128: the split-line
    z convolution) at sampled cells -- corners, edges, the vortex core and
    random cells -- against the oracle's direct sum over all 16.7 M source
    cells; tolerance 5e-6 of Ms, the FP32 demag bar of the small grids."""
    mm = need_gpu()
    from oracle.demag import h_demag_at
    from gpu_util import TERMS
    w = W.vortex_512x512x64()
    g = w.grid
    ctx = make_ctx(mm, g, w.mat, precision=32, demag=True)
    try:
        m = W.m_vortex(g, seed=w.seed)
        mm.mm_set_m(ctx, 0, m)
        m_dev = mm.mm_get_m(ctx, 0, m.shape)
        H = mm.mm_get_heff(ctx, 0, m.shape, TERMS["demag"])
    finally:
        mm.mm_destroy(ctx)
    rng = np.random.default_rng(55)
    targets = [(0, 0, 0), (63, 511, 511), (0, 511, 0), (63, 0, 511), (31, 255, 256), (32, 256, 255),
               (0, 300, 0), (63, 17, 400)]
    targets += [tuple(int(v) for v in rng.integers(0, (64, 512, 512))) for _ in range(6)]
    ref = h_demag_at(m_dev, oracle_problem(g, w.mat), targets)
    got = np.stack([H[:, k, j, i] for (k, j, i) in targets])
    err = np.abs(got - ref).max()
    assert err <= 5e-6 * w.mat.Ms, err


def test_vortex_512x512x64_demag_field_every_cell():
    """The same field at every one of the 16.7 M cells against the oracle's
    FFT route (full complex numpy FFTs of the 1024x1024x128 padded tensor and
    magnetisation; about 30 GB of host memory, a few minutes)."""
    mm = need_gpu()
    from oracle.demag import demag_spectrum, h_demag
    from gpu_util import TERMS
    w = W.vortex_512x512x64()
    g = w.grid
    ctx = make_ctx(mm, g, w.mat, precision=32, demag=True)
    try:
        m = W.m_vortex(g, seed=w.seed)
        mm.mm_set_m(ctx, 0, m)
        m_dev = mm.mm_get_m(ctx, 0, m.shape)
        H = mm.mm_get_heff(ctx, 0, m.shape, TERMS["demag"])
    finally:
        mm.mm_destroy(ctx)
    p = oracle_problem(g, w.mat)
    ref = h_demag(m_dev, p, demag_spectrum(p.shape, p.d))
    err = np.abs(H - ref).max()
    assert err <= 5e-6 * np.abs(ref).max(), err


def test_newell_entries_at_the_largest_displacements():
    """FP64 Newell entries of the 512x512x64 grid of 3 nm cubes at the far
    corners of the padded tensor, against the oracle's evaluation."""
    mm = need_gpu()
    from oracle.demag import newell_at
    ijk = np.array([[511, 511, 63], [511, 0, 0], [0, 511, 0], [0, 0, 63], [300, 200, 40], [1, 511, 63],
                    [2, 0, 0], [3, 2, 1]], dtype=np.int32)
    d = (3e-9, 3e-9, 3e-9)
    g = mm.mm_newell(ijk, d)
    o = newell_at(ijk, d)
    scale = np.abs(o).max(axis=1, keepdims=True)
    assert np.all(np.abs(g - o) <= 1e-11 * scale + 1e-18)


def _far_field_second_order(ijk, h):
    """-(V/4 pi) [d_a d_b 1/R + sum_d h_d^2/12 d_d^2 d_a d_b 1/R]: the cell
    average of the point-dipole kernel to second order (the moments of the
    difference of two uniform points per axis), from the closed forms of the
    second and fourth derivatives of 1/R; relative error O((h/R)^4)."""
    x = np.asarray(ijk, float) * np.asarray(h, float)
    R2 = float(x @ x)
    R = np.sqrt(R2)
    V = h[0] * h[1] * h[2]
    dlt = np.eye(3)

    def t2(i, j):
        return 3 * x[i] * x[j] / R ** 5 - dlt[i, j] / R ** 3

    def t4(i, j, k, l):
        xs = x
        return (105 * xs[i] * xs[j] * xs[k] * xs[l] / R ** 9
                - 15 * (dlt[i, j] * xs[k] * xs[l] + dlt[i, k] * xs[j] * xs[l] + dlt[i, l] * xs[j] * xs[k]
                        + dlt[j, k] * xs[i] * xs[l] + dlt[j, l] * xs[i] * xs[k] + dlt[k, l] * xs[i] * xs[j]) / R ** 7
                + 3 * (dlt[i, j] * dlt[k, l] + dlt[i, k] * dlt[j, l] + dlt[i, l] * dlt[j, k]) / R ** 5)

    out = []
    for a, b in [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]:
        s = t2(a, b) + sum(h[d] ** 2 / 12.0 * t4(a, b, d, d) for d in range(3))
        out.append(-V / (4 * np.pi) * s)
    return np.array(out)


def test_newell_far_band_against_the_far_field_expansion():
    """The GPU's FP64 Newell entries beyond 128 cells (its 3-point quadrature
    band) against the second-order far-field expansion of the cell-averaged
    dipole kernel -- a check that does not go through the oracle: the
    difference must stay within (h/R)^4 (the expansion's own truncation)."""
    mm = need_gpu()
    for h in [(3e-9, 3e-9, 3e-9), (2e-9, 2e-9, 1e-9), (3.90625e-9, 3.90625e-9, 3e-9)]:
        ijk = np.array([[511, 511, 63], [511, 0, 0], [0, 511, 0], [300, 200, 40], [140, 0, 0], [0, 135, 20],
                        [-200, 150, -10], [130, 60, 63]], dtype=np.int32)
        g = mm.mm_newell(ijk, h)
        for q in range(ijk.shape[0]):
            A = _far_field_second_order(ijk[q], h)
            dist = np.linalg.norm(ijk[q] * np.asarray(h)) / max(h)
            rel = np.abs(g[q] - A).max() / np.abs(A).max()
            assert rel <= 2.0 / dist ** 4, (h, tuple(ijk[q]), rel)


def test_skyrmion_film_512x512_replay_fp32():
    """The 512x512x1 DMI film (the surrogate workload's exact path: one-row-per-
    warp X passes with the stage combine fused in, the fused inverse-X +
    field kernel) against the oracle after 10 of the oracle's accepted RK45
    steps, replayed."""
    mm = need_gpu()
    w = W.skyrmion_512()
    m0 = W.m_skyrmion_lattice(w.grid, seed=w.seed, spacing=40e-9, radius=8e-9)
    o, p = _solver(w, m0, dt=1e-14, rtol=w.rtol)
    dts = [o.rk45_step() for _ in range(10)]
    ctx = make_ctx(mm, w.grid, w.mat, precision=32, demag=True, B=w.B_ext, dt=1e-14, rtol=w.rtol)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_step_dt(ctx, dts)
        err = np.abs(mm.mm_get_m(ctx, 0, m0.shape) - o.m).max()
        assert err <= 1e-5, err
    finally:
        mm.mm_destroy(ctx)


def test_replicas_1024_sampled_against_oracle():
    """All 1024 perpendicular free layers of uneven sizes in one batch
    (T = 300 K, per-replica Philox keys splitmix64(3 + r), SOT current per
    replica), 200 Heun steps; ten replicas -- the first of every size class,
    the smallest, the largest, the first and the last -- against the oracle
    run replica by replica (same thermal words, same current)."""
    mm = need_gpu()
    from oracle.llg import Solver, Torque, replica_seed
    R = 1024
    sizes = W.replica_sizes(R, seed=3)
    J = W.replica_currents(R)
    mat = W.Material(Ms=1.1e6, A=2e-11, alpha=0.01, Ku1=9e5, u=(0.0, 0.0, 1.0))
    M = mm.Material(mat.Ms, mat.A, mat.alpha, mat.Ku1, mat.u, mat.D)
    grids = [mm.make_grid(n, n, 1, 2e-9, 2e-9, 1e-9) for n in sizes]
    cfg = mm.make_config(precision=32, integrator=mm.MM_HEUN, demag=mm.MM_DEMAG_EXACT, dt=1e-14, T=300.0, seed=3)
    ctx = mm.mm_create_batch(grids, M.s, cfg, None)
    ctx._mat = M
    try:
        mm.mm_set_torque(ctx, mm.make_torque(mm.MM_TORQUE_SOT, p=(0, 1, 0), theta_SH=0.1), J)
        m0 = []
        for r, n in enumerate(sizes):
            m = W.m_perp(W.Grid(n, n, 1, 2e-9, 2e-9, 1e-9), seed=1000 + r, tilt=0.05)
            mm.mm_set_m(ctx, r, m)
            m0.append(m)
        n_steps = 200
        mm.mm_step(ctx, n_steps)
        picks = {0, R - 1, int(np.argmin(sizes)), int(np.argmax(sizes))}
        picks |= {sizes.index(n) for n in sorted(set(sizes))}
        picks |= {int(v) for v in np.random.default_rng(8).integers(0, R, 10 - len(picks))}
        assert len(picks) >= 8 and len({sizes[r] for r in picks}) == 5
        for r in sorted(picks):
            g = W.Grid(sizes[r], sizes[r], 1, 2e-9, 2e-9, 1e-9)
            p = oracle_problem(g, mat)
            o = Solver(p, m0[r], terms=("exchange", "anisotropy", "zeeman", "demag"), T=300.0,
                       seed=replica_seed(3, r), dt=1e-14,
                       torque=Torque(kind="sot", J=J[r], p=(0, 1, 0), theta_SH=0.1))
            for _ in range(n_steps):
                o.heun_step()
            err = np.abs(mm.mm_get_m(ctx, r, m0[r].shape) - o.m).max()
            assert err <= 1e-5, (r, sizes[r], err)
    finally:
        mm.mm_destroy(ctx)


def test_mumag_sp4_field_a():
    """muMAG standard problem 4, field A (Results, "Validation against the
    muMAG standard problems"): the s-state (uniform [1,1,1] relaxed 5 ns with
    alpha = 1 in zero field), then 1 ns at alpha = 0.02 in (-24.6, 4.3, 0) mT.
    <m_x>(1 ns) lies within the spread of the solvers the paper compares
    (-0.969 ... -0.984 against the reference -0.986): within 0.02 of the
    reference; FP32 and FP64 trajectories agree to 1e-4."""
    mm = need_gpu()
    g = W.film_128x32().grid
    out = {}
    for prec in (64, 32):
        relax = make_ctx(mm, g, W.Material(Ms=8e5, A=1.3e-11, alpha=1.0), precision=prec, demag=True, dt=1e-13)
        try:
            m0 = np.full((3,) + g.shape, 1 / np.sqrt(3.0))
            mm.mm_set_m(relax, 0, m0)
            mm.mm_run(relax, 5e-9)
            ms = mm.mm_get_m(relax, 0, m0.shape)
        finally:
            mm.mm_destroy(relax)
        dyn = make_ctx(mm, g, W.Material(Ms=8e5, A=1.3e-11, alpha=0.02), precision=prec, demag=True, dt=1e-13,
                       B=(-24.6e-3, 4.3e-3, 0.0))
        try:
            mm.mm_set_m(dyn, 0, ms)
            mx = []
            for k in range(1, 21):
                mm.mm_run(dyn, k * 50e-12)
                mx.append(float(mm.mm_get_m(dyn, 0, m0.shape)[0].mean()))
            out[prec] = (float(ms[0].mean()), np.array(mx))
        finally:
            mm.mm_destroy(dyn)
    s_mx, traj = out[64]
    assert 0.95 < s_mx < 0.99                      # an s-state, not saturation
    assert traj[0] > 0 > traj[-1]                  # switched
    assert abs(traj[-1] - (-0.986)) < 0.02, traj[-1]
    assert np.abs(out[32][1] - traj).max() < 1e-4
