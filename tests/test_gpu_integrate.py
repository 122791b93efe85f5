"""GPU parity of whole steps: RK45 replayed on the oracle's accepted step
sequence (so accept/reject decisions cannot diverge), Heun with the Philox
thermal field and spin torques, and the device-side step controller.

Bar: max over cells of |m_gpu - m_oracle| after the stated number of steps
<= 1e-11 in FP64 and <= 1e-5 in FP32."""
import numpy as np
import pytest

import workloads as W
from gpu_util import make_ctx, need_gpu, oracle_problem

pytestmark = pytest.mark.gpu


def _oracle_solver(grid, mat, m, B=(0, 0, 0), **kw):
    from oracle.llg import Solver
    p = oracle_problem(grid, mat, B)
    return Solver(p, m, **kw)


CASES = [
    ("film3d", W.Grid(12, 8, 3, 2e-9, 2e-9, 2e-9),
     W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.1, Ku1=8e5, u=(0, 0, 1), D=3e-3), (0.0, 0.0, 0.0)),
    ("film2d", W.Grid(32, 8, 1, 3.90625e-9, 3.90625e-9, 3e-9),
     W.Material(Ms=8e5, A=1.3e-11, alpha=0.02), (-24.6e-3, 4.3e-3, 0.0)),
    ("odd", W.Grid(17, 5, 2, 2e-9, 3e-9, 1e-9),
     W.Material(Ms=7e5, A=1.1e-11, alpha=0.3, Ku1=2e5, u=(0.6, 0, 0.8), D=1.5e-3), (0.0, 0.02, 0.01)),
    # half length 64 on a small grid: the stage combine runs in the CTA-wide X
    # pass (the one-row-per-warp kernel of this length forms no stage)
    ("rows64", W.Grid(64, 12, 2, 2e-9, 2e-9, 2e-9),
     W.Material(Ms=6e5, A=1.3e-11, alpha=0.2, Ku1=3e5, u=(0, 0, 1), D=2e-3), (0.0, 0.01, 0.03)),
    # half length 192: the FP32 stage combine runs inside the X pass; granular
    # regions with holes exercise the per-cell Ms there
    ("fused", W.Grid(170, 12, 2, 2e-9, 2e-9, 2e-9),
     W.with_cells(W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.1, Ku1=8e5, u=(0, 0, 1), D=3e-3),
                  W.random_material_cells(W.Grid(170, 12, 2, 2e-9, 2e-9, 2e-9), 9)), (0.0, 0.0, 0.05)),
    # one material, nx = 128 (half length 128): in FP32 the inverse X pass
    # runs inside the field kernel (H_demag stays in shared memory)
    ("c2r_field", W.Grid(128, 6, 2, 2e-9, 2e-9, 2e-9),
     W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.1, Ku1=8e5, u=(0, 0, 1), D=3e-3), (0.01, 0.0, 0.02)),
    # the same kernel with a ragged last CTA: 7 rows, CTAs of 4 rows
    ("c2r_field_ragged", W.Grid(128, 7, 1, 2e-9, 2e-9, 2e-9),
     W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.1, Ku1=8e5, u=(0, 0, 1), D=3e-3), (0.0, 0.01, 0.02)),
]


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_rk45_replay_matches_oracle(prec, ci):
    mm = need_gpu()
    name, grid, mat, B = CASES[ci]
    m0 = W.random_m(grid, seed=20 + ci)
    o = _oracle_solver(grid, mat, m0, B, dt=1e-14, rtol=1e-6)
    nsteps = 40
    dts = [o.rk45_step() for _ in range(nsteps)]
    ctx = make_ctx(mm, grid, mat, precision=prec, demag=True, B=B, dt=1e-14, rtol=1e-6)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_step_dt(ctx, dts)
        m = mm.mm_get_m(ctx, 0, m0.shape)
        t, _, n = mm.mm_get_time(ctx)
        assert n == nsteps and abs(t - sum(dts)) < 1e-24
        err = np.abs(m - o.m).max()
        assert err <= (1e-11 if prec == 64 else 1e-5), err
    finally:
        mm.mm_destroy(ctx)


def test_rk45_controller_follows_oracle_fp64():
    """Free adaptive run: the device controller takes the same accepted
    step sizes as the oracle's (FP64, same tableau and controller)."""
    mm = need_gpu()
    name, grid, mat, B = CASES[0]
    m0 = W.random_m(grid, seed=5)
    o = _oracle_solver(grid, mat, m0, B, dt=1e-14, rtol=1e-6)
    ctx = make_ctx(mm, grid, mat, precision=64, demag=True, B=B, dt=1e-14, rtol=1e-6)
    try:
        mm.mm_set_m(ctx, 0, m0)
        for _ in range(30):
            o.rk45_step()
        mm.mm_step(ctx, 30)
        t, dt, n = mm.mm_get_time(ctx)
        assert n == 30
        assert abs(t - o.t) <= 1e-9 * o.t
        assert abs(dt - o.dt) <= 1e-8 * o.dt
        assert np.abs(mm.mm_get_m(ctx, 0, m0.shape) - o.m).max() < 1e-9
    finally:
        mm.mm_destroy(ctx)


def test_run_lands_on_t_end():
    mm = need_gpu()
    name, grid, mat, B = CASES[1]
    ctx = make_ctx(mm, grid, mat, precision=32, demag=True, B=B, dt=1e-14, rtol=1e-6)
    try:
        mm.mm_set_m(ctx, 0, W.m_uniform_perturbed(grid, seed=1))
        mm.mm_run(ctx, 7.3e-12)
        t, _, n = mm.mm_get_time(ctx)
        assert abs(t - 7.3e-12) < 1e-24 and n > 0
        m = mm.mm_get_m(ctx, 0, (3, grid.nz, grid.ny, grid.nx))
        assert np.abs(np.sqrt((m * m).sum(0)) - 1).max() < 1e-6
    finally:
        mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("torque", ["sot", "stt", "zl"])
def test_heun_thermal_with_torque_matches_oracle(prec, torque):
    mm = need_gpu()
    from oracle.llg import Torque, replica_seed
    grid = W.Grid(20, 12, 1, 2e-9, 2e-9, 1e-9)
    mat = W.Material(Ms=1.1e6, A=2e-11, alpha=0.01, Ku1=9e5, u=(0, 0, 1))
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
    o = _oracle_solver(grid, mat, m0, terms=("exchange", "anisotropy", "demag"), torque=tq_o, T=300.0,
                       seed=replica_seed(seed, 0), dt=1e-14)
    ctx = make_ctx(mm, grid, mat, precision=prec, integrator="heun", demag=True, dt=1e-14, T=300.0, seed=seed)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_set_torque(ctx, tq_g, [J])
        n = 60
        for _ in range(n):
            o.heun_step()
        mm.mm_step(ctx, n)
        err = np.abs(mm.mm_get_m(ctx, 0, m0.shape) - o.m).max()
        assert err <= (1e-11 if prec == 64 else 1e-5), err
    finally:
        mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("integ", ["heun", "dm"])
def test_fused_inverse_x_field_heun_and_dm(prec, integ):
    """Heun and Depondt-Mertens steps at 300 K with spin-orbit torque on a
    one-material 256 x 4 film: in FP32 both the predictor and the corrector
    take the demag field from the fused inverse-X + field kernel."""
    mm = need_gpu()
    from oracle.llg import Torque, replica_seed
    grid = W.Grid(256, 4, 1, 2e-9, 2e-9, 1e-9)
    mat = W.Material(Ms=1.1e6, A=2e-11, alpha=0.02, Ku1=9e5, u=(0, 0, 1), D=1e-3)
    J = 2.0e11
    tq_o = Torque(kind="sot", J=J, p=(0, 1, 0), theta_SH=0.1, fl_ratio=0.2)
    tq_g = mm.make_torque(mm.MM_TORQUE_SOT, p=(0, 1, 0), theta_SH=0.1, fl_ratio=0.2)
    m0 = W.m_perp(grid, seed=5, tilt=0.3)
    seed = 13
    o = _oracle_solver(grid, mat, m0, terms=("exchange", "dmi", "anisotropy", "demag"), torque=tq_o, T=300.0,
                       seed=replica_seed(seed, 0), dt=1e-14)
    ctx = make_ctx(mm, grid, mat, precision=prec, integrator=integ, demag=True, dt=1e-14, T=300.0, seed=seed)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_set_torque(ctx, tq_g, [J])
        n = 40
        for _ in range(n):
            if integ == "heun":
                o.heun_step()
            else:
                o.dm_step()
        mm.mm_step(ctx, n)
        err = np.abs(mm.mm_get_m(ctx, 0, m0.shape) - o.m).max()
        assert err <= (1e-11 if prec == 64 else 1e-5), err
    finally:
        mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", [64, 32])
def test_zhang_li_with_rk45_replay(prec):
    mm = need_gpu()
    from oracle.llg import Torque
    grid = W.Grid(24, 6, 2, 2e-9, 2e-9, 2e-9)
    mat = W.Material(Ms=8e5, A=1.3e-11, alpha=0.05, Ku1=5e5, u=(0, 0, 1), D=1e-3)
    m0 = W.random_m(grid, seed=9)
    tq_o = Torque(kind="zl", J=3e12, P=0.6, xi=0.1, direction=(1, 0, 0), match_mumax=True)
    o = _oracle_solver(grid, mat, m0, torque=tq_o, dt=1e-14, rtol=1e-6)
    dts = [o.rk45_step() for _ in range(25)]
    ctx = make_ctx(mm, grid, mat, precision=prec, demag=True, dt=1e-14)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_set_torque(ctx, mm.make_torque(mm.MM_TORQUE_ZL, P=0.6, xi=0.1, direction=(1, 0, 0), match_mumax=1),
                         [3e12])
        mm.mm_step_dt(ctx, dts)
        err = np.abs(mm.mm_get_m(ctx, 0, m0.shape) - o.m).max()
        assert err <= (1e-11 if prec == 64 else 1e-5), err
    finally:
        mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_rk4_matches_oracle(prec, ci):
    """Classical RK4 (fixed step) against the oracle's RK4, same steps."""
    mm = need_gpu()
    name, grid, mat, B = CASES[ci]
    m0 = W.random_m(grid, seed=40 + ci)
    dt, nsteps = 5e-15, 30
    o = _oracle_solver(grid, mat, m0, B, dt=dt)
    for _ in range(nsteps):
        o.rk4_step(dt)
    ctx = make_ctx(mm, grid, mat, precision=prec, integrator="rk4", demag=True, B=B, dt=dt)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_step(ctx, nsteps)
        t, _, n = mm.mm_get_time(ctx)
        assert n == nsteps and abs(t - nsteps * dt) < 1e-25
        err = np.abs(mm.mm_get_m(ctx, 0, m0.shape) - o.m).max()
        assert err <= (1e-11 if prec == 64 else 1e-5), err
    finally:
        mm.mm_destroy(ctx)


def test_rk4_rejects_finite_temperature():
    mm = need_gpu()
    name, grid, mat, B = CASES[0]
    with pytest.raises(mm.MMError):
        make_ctx(mm, grid, mat, precision=32, integrator="rk4", demag=False, T=300.0)


@pytest.mark.parametrize("prec", [32, 64])
def test_state_written_back_unchanged_keeps_the_fsal_slope(prec):
    """mm_set_m with the state mm_get_m just returned leaves the state bit for
    bit as it was, so the next RK45 step keeps its first-same-as-last slope:
    it launches fewer kernels than the same step after a real change (one
    cell turned), and the trajectory equals one that never left the device."""
    mm = need_gpu()
    grid = W.Grid(32, 16, 4, 3e-9, 3e-9, 3e-9)
    mat = W.Material(Ms=8e5, A=1.3e-11, alpha=0.02)
    m0 = W.m_random_sphere(grid, seed=12)
    dts = np.full(1, 2e-14)
    ctx = make_ctx(mm, grid, mat, precision=prec, dt=2e-14)
    try:
        mm.mm_set_m(ctx, 0, m0)
        mm.mm_step_dt(ctx, np.full(4, 2e-14))
        m = mm.mm_get_m(ctx, 0, m0.shape)
        s0 = mm.mm_get_stats(ctx)
        mm.mm_set_m(ctx, 0, m)
        mm.mm_step_dt(ctx, dts)
        s1 = mm.mm_get_stats(ctx)
        m2 = mm.mm_get_m(ctx, 0, m0.shape)
        m2[:, 0, 0, 0] = [0.0, 0.0, 1.0]
        mm.mm_set_m(ctx, 0, m2)
        mm.mm_step_dt(ctx, dts)
        s2 = mm.mm_get_stats(ctx)
        same = s1["kernel_launches"] - s0["kernel_launches"]
        changed = s2["kernel_launches"] - s1["kernel_launches"]
        assert changed > same, (same, changed)
    finally:
        mm.mm_destroy(ctx)
    res = []
    for roundtrip in (False, True):
        ctx = make_ctx(mm, grid, mat, precision=prec, dt=2e-14)
        try:
            mm.mm_set_m(ctx, 0, m0)
            mm.mm_step_dt(ctx, np.full(4, 2e-14))
            if roundtrip:
                mm.mm_set_m(ctx, 0, mm.mm_get_m(ctx, 0, m0.shape))
            mm.mm_step_dt(ctx, np.full(3, 2e-14))
            res.append(mm.mm_get_m(ctx, 0, m0.shape))
        finally:
            mm.mm_destroy(ctx)
    assert np.array_equal(res[0], res[1])
