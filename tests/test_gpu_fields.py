"""GPU parity of the effective field: every term of libmm's fused field
kernel, the FP64 Newell tensor and the pruned FFT demag path against the
FP64 oracle, on odd and ragged grids, with holes and several materials.

Tolerances (max over cells, relative to the largest |H|): FP64 1e-11,
FP32 2e-6 for the local terms (float rounding of m_j - m_i under the
1/dx^2 exchange factor) and 5e-6 for demag (FP32 FFT round-off over
log2(P) passes)."""
import numpy as np
import pytest

import workloads as W
from gpu_util import TERMS, make_ctx, need_gpu, oracle_problem, rel_err

pytestmark = pytest.mark.gpu

GRIDS = [
    W.Grid(17, 9, 2, 2e-9, 3e-9, 1.5e-9),
    W.Grid(8, 8, 1, 2e-9, 2e-9, 1e-9),
    W.Grid(33, 5, 1, 3.90625e-9, 3.90625e-9, 3e-9),
    W.Grid(16, 12, 3, 2e-9, 2e-9, 2e-9),
    W.Grid(1, 1, 1, 2e-9, 2e-9, 2e-9),
    W.Grid(40, 1, 1, 1e-9, 1e-9, 1e-9),
]


def _mat(grid, seed, cells):
    mat = W.Material(Ms=6e5, A=1.3e-11, alpha=0.1, Ku1=4e5, u=(0.3, 0.2, 0.9), D=2.5e-3)
    if cells:
        mat = W.with_cells(mat, W.random_material_cells(grid, seed))
    return mat


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("gi", range(len(GRIDS)))
@pytest.mark.parametrize("cells", [False, True])
def test_local_terms_match_oracle(prec, gi, cells):
    mm = need_gpu()
    from oracle.fields import h_anisotropy, h_dmi, h_exchange, h_zeeman
    grid = GRIDS[gi]
    mat = _mat(grid, gi, cells)
    B = (0.01, -0.02, 0.05)
    ctx = make_ctx(mm, grid, mat, precision=prec, demag=False, B=B)
    try:
        m = W.random_m(grid, seed=gi + 1)
        mm.mm_set_m(ctx, 0, m)
        m_dev = mm.mm_get_m(ctx, 0, m.shape)
        p = oracle_problem(grid, mat, B)
        # compare against the oracle on the state the GPU actually holds
        tol = 1e-11 if prec == 64 else 2e-6
        from oracle.constants import MU0
        # natural scale of each term: its coefficient times |m| = 1 (a single
        # cell's ghost terms cancel to rounding, so |ref| alone can be 0)
        hmin = min(grid.dx, grid.dy, grid.dz)
        coef = {"exchange": 2 * mat.A / (MU0 * mat.Ms * hmin ** 2), "dmi": 2 * mat.D / (MU0 * mat.Ms * hmin),
                "anisotropy": 2 * mat.Ku1 / (MU0 * mat.Ms), "zeeman": np.abs(B).max() / MU0}
        for name, fn in (("exchange", lambda: h_exchange(m_dev, p)), ("dmi", lambda: h_dmi(m_dev, p)),
                         ("anisotropy", lambda: h_anisotropy(m_dev, p)), ("zeeman", lambda: h_zeeman(p))):
            H = mm.mm_get_heff(ctx, 0, m.shape, TERMS[name])
            ref = np.where(p.present, fn(), 0.0)
            scale = max(np.abs(ref).max(), coef[name])
            assert np.abs(H - ref).max() <= tol * scale, (name, np.abs(H - ref).max() / scale)
    finally:
        mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", [64, 32])
def test_periodic_exchange_and_dmi(prec):
    mm = need_gpu()
    from oracle.fields import h_dmi, h_exchange
    grid = W.Grid(12, 7, 3, 2e-9, 2e-9, 2e-9, (1, 1, 1))
    mat = _mat(grid, 0, False)
    ctx = make_ctx(mm, grid, mat, precision=prec, demag=False)
    try:
        m = W.random_m(grid, seed=3)
        mm.mm_set_m(ctx, 0, m)
        m_dev = mm.mm_get_m(ctx, 0, m.shape)
        p = oracle_problem(grid, mat)
        tol = 1e-11 if prec == 64 else 2e-6
        assert rel_err(mm.mm_get_heff(ctx, 0, m.shape, TERMS["exchange"]), h_exchange(m_dev, p)) < tol
        assert rel_err(mm.mm_get_heff(ctx, 0, m.shape, TERMS["dmi"]), h_dmi(m_dev, p)) < tol
    finally:
        mm.mm_destroy(ctx)


def test_newell_tensor_matches_oracle():
    mm = need_gpu()
    from oracle.demag import newell_at
    rng = np.random.default_rng(0)
    ijk = np.concatenate([
        np.array([(i, j, k) for i in range(-3, 4) for j in range(-3, 4) for k in range(-2, 3)]),
        rng.integers(-300, 301, size=(300, 3)) * np.array([1, 1, 0]),
        rng.integers(-40, 41, size=(300, 3)),
    ])
    for cell in [(2e-9, 2e-9, 2e-9), (2e-9, 2e-9, 1e-9), (3.90625e-9, 3.90625e-9, 3e-9), (3e-9, 2e-9, 2.5e-9)]:
        g = mm.mm_newell(ijk, cell)
        o = newell_at(ijk, cell)
        scale = np.abs(o).max(axis=1, keepdims=True)
        assert np.all(np.abs(g - o) <= 1e-11 * scale + 1e-18), np.max(np.abs(g - o) / scale)


DEMAG_GRIDS = [
    W.Grid(8, 8, 1, 2e-9, 2e-9, 1e-9),
    W.Grid(17, 9, 2, 2e-9, 3e-9, 1.5e-9),
    W.Grid(16, 12, 3, 2e-9, 2e-9, 2e-9),
    W.Grid(24, 20, 1, 3.90625e-9, 3.90625e-9, 3e-9),
    W.Grid(10, 1, 4, 2e-9, 2e-9, 2e-9),
    W.Grid(1, 1, 1, 2e-9, 2e-9, 2e-9),
    W.Grid(48, 48, 1, 2e-9, 2e-9, 1e-9),
    W.Grid(32, 16, 8, 3e-9, 3e-9, 3e-9),
    # FP32 3-D fast paths: padded y lengths 48 / 128 / 32 (direct column
    # passes, ragged final CTA), padded z lengths 32 / 16 / 8 (z line in
    # registers, ragged final column block)
    W.Grid(40, 24, 16, 2e-9, 2e-9, 2e-9),
    W.Grid(24, 64, 8, 2e-9, 2e-9, 1e-9),
    W.Grid(13, 16, 4, 3e-9, 2e-9, 2e-9),
    # one-row-per-warp X passes: half lengths 192 (odd nx: scalar loads) and 512
    W.Grid(171, 10, 1, 2e-9, 2e-9, 1e-9),
    W.Grid(500, 4, 2, 2e-9, 2e-9, 2e-9),
    # 3-smooth compile-time lengths: half lengths 108 / 81 / 216 / 162 / 324,
    # column lengths 108 / 81 (odd) / 48 / 324
    W.Grid(100, 50, 1, 2.5e-9, 2.5e-9, 3e-9),
    W.Grid(75, 41, 3, 2e-9, 2e-9, 2e-9),
    W.Grid(200, 20, 2, 2e-9, 2e-9, 2e-9),
    W.Grid(150, 24, 24, 3e-9, 3e-9, 3e-9),
    W.Grid(300, 150, 1, 2e-9, 2e-9, 1e-9),
    # middle pass split over several threads per line (four-step): padded z
    # lengths 64 / 81 (n_in at its maximum 41) / 96 / 128 / 81 (ragged n_in),
    # padded y lengths (2-D) 32 / 64 / 128 / 192 / 256 / 512
    W.Grid(12, 10, 32, 2e-9, 2e-9, 2e-9),
    W.Grid(9, 6, 41, 3e-9, 3e-9, 3e-9),
    W.Grid(10, 8, 48, 2e-9, 2e-9, 1e-9),
    W.Grid(6, 5, 64, 3e-9, 3e-9, 3e-9),
    W.Grid(7, 4, 37, 2e-9, 3e-9, 2e-9),
    W.Grid(16, 16, 1, 2e-9, 2e-9, 1e-9),
    W.Grid(20, 32, 1, 2e-9, 2e-9, 1e-9),
    W.Grid(30, 64, 1, 2e-9, 2e-9, 1e-9),
    W.Grid(12, 96, 1, 2e-9, 2e-9, 1e-9),
    W.Grid(9, 128, 1, 2e-9, 2e-9, 1e-9),
    W.Grid(6, 256, 1, 2e-9, 2e-9, 1e-9),
    # Y passes split over several threads per column: padded y lengths 512
    # and 1024 with ragged n_in (250 and 500 rows)
    W.Grid(6, 250, 3, 2e-9, 2e-9, 2e-9),
    W.Grid(4, 500, 2, 3e-9, 2e-9, 2e-9),
]


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("gi", range(len(DEMAG_GRIDS)))
def test_demag_field_matches_oracle(prec, gi):
    mm = need_gpu()
    from oracle.demag import demag_spectrum, h_demag
    grid = DEMAG_GRIDS[gi]
    mat = _mat(grid, gi, cells=(gi % 2 == 1))
    ctx = make_ctx(mm, grid, mat, precision=prec, demag=True)
    try:
        m = W.random_m(grid, seed=10 + gi)
        mm.mm_set_m(ctx, 0, m)
        m_dev = mm.mm_get_m(ctx, 0, m.shape)
        p = oracle_problem(grid, mat)
        ref = np.where(p.present, h_demag(m_dev, p, demag_spectrum(p.shape, p.d)), 0.0)
        H = mm.mm_get_heff(ctx, 0, m.shape, TERMS["demag"])
        tol = 1e-11 if prec == 64 else 5e-6
        assert rel_err(H, ref) < tol, rel_err(H, ref)
    finally:
        mm.mm_destroy(ctx)


def test_demag_field_full_size_256x256x16():
    """The benchmark's grid (256x256x16 cells of 2 nm, padded 512x512x32) in
    FP32 against the FP64 oracle, every cell compared."""
    mm = need_gpu()
    from oracle.demag import demag_spectrum, h_demag
    w = W.dmi_256x256x16()
    grid = w.grid
    ctx = make_ctx(mm, grid, w.mat, precision=32, demag=True)
    try:
        m = W.m_random_sphere(grid, seed=2)
        mm.mm_set_m(ctx, 0, m)
        m_dev = mm.mm_get_m(ctx, 0, m.shape)
        p = oracle_problem(grid, w.mat)
        ref = h_demag(m_dev, p, demag_spectrum(p.shape, p.d))
        H = mm.mm_get_heff(ctx, 0, m.shape, TERMS["demag"])
        assert rel_err(H, ref) < 5e-6, rel_err(H, ref)
    finally:
        mm.mm_destroy(ctx)


def test_demag_tensor_spectrum_matches_oracle_fft():
    """For power-of-two grids both sides pad to exactly 2n: the stored real
    spectrum equals -Re(FFT(N))/(Px Py Pz) of the oracle's padded tensor."""
    mm = need_gpu()
    from oracle.demag import demag_spectrum
    for grid in (W.Grid(16, 8, 4, 2e-9, 2e-9, 1e-9), W.Grid(32, 16, 1, 2e-9, 2e-9, 1e-9)):
        ctx = make_ctx(mm, grid, W.Material(Ms=8e5, A=1.3e-11, alpha=0.02), precision=64, demag=True)
        try:
            K, (Px, Py, Pz) = mm.mm_get_demag_kernel(ctx)
            assert (Px, Py, Pz) == (2 * grid.nx, 2 * grid.ny if grid.ny > 1 else 1, 2 * grid.nz if grid.nz > 1 else 1)
            S = demag_spectrum((grid.nz, grid.ny, grid.nx), (grid.dx, grid.dy, grid.dz))
            # the oracle pads a singleton axis to 2 (one nonzero entry): its k = 0
            # plane is the unpadded transform the GPU stores
            Sz = S[:, : Pz // 2 + 1] if grid.nz > 1 else S[:, :1]
            ref = -Sz[:, :, : Py // 2 + 1, : Px // 2 + 1].real / (Px * Py * Pz)
            ncomp = K.shape[0]
            err = np.abs(K - ref[:ncomp]).max() / np.abs(ref).max()
            assert err < 1e-12, err
        finally:
            mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", [64, 32])
def test_thermal_stream_is_bit_exact(prec):
    mm = need_gpu()
    from oracle.philox import raw, thermal_field
    from oracle.llg import replica_seed
    grid = W.Grid(13, 7, 2, 2e-9, 2e-9, 1e-9)
    mat = W.with_cells(W.Material(Ms=1.1e6, A=2e-11, alpha=0.01), W.random_material_cells(grid, 4))
    ctx = make_ctx(mm, grid, mat, precision=prec, integrator="heun", demag=False, dt=1e-14, T=300.0, seed=77)
    try:
        seed_r = replica_seed(77, 0)
        for step in (0, 1, 123456789012):
            r, h = mm.mm_get_thermal(ctx, 0, step, grid.n)
            o = np.stack(raw(seed_r, step, grid.n), axis=1).ravel()
            assert np.array_equal(r, o)
            p = oracle_problem(grid, mat)
            ref = thermal_field(p, 300.0, 1e-14, seed_r, step).reshape(-1)
            tol = 1e-12 if prec == 64 else 2e-6
            assert np.max(np.abs(h - ref)) <= tol * np.abs(ref).max()
    finally:
        mm.mm_destroy(ctx)
