"""Pins of the oracle's demagnetising field: FFT convolution against the
brute-force double sum, exact symmetry results for uniformly magnetised
cubes, the thin-film limit, periodic images, and Kittel precession of a
single cell."""
import numpy as np
import pytest

import workloads as W
from oracle.demag import demag_spectrum, h_demag, h_demag_at, h_demag_direct, newell_octant
from oracle.fields import Problem


def _problem(grid, seed=0, holes=True):
    mat = W.Material(Ms=8e5, A=1.3e-11, alpha=0.02)
    if holes:
        mat = W.with_cells(mat, W.random_material_cells(grid, seed))
    return Problem.from_workload(grid, mat)


@pytest.mark.parametrize("shape,cell", [((4, 4, 1), (2e-9, 2e-9, 1e-9)),
                                        ((6, 5, 3), (3e-9, 2e-9, 2.5e-9)),
                                        ((7, 3, 2), (1e-9, 1e-9, 1e-9)),
                                        ((1, 1, 1), (2e-9, 2e-9, 2e-9)),
                                        ((5, 1, 1), (2e-9, 1e-9, 1e-9))])
def test_fft_convolution_equals_direct_sum(shape, cell):
    nx, ny, nz = shape
    grid = W.Grid(nx, ny, nz, *cell)
    p = _problem(grid, seed=nx * 31 + ny)
    m = W.random_m(grid, seed=7)
    H_fft = h_demag(m, p, demag_spectrum(p.shape, p.d))
    H_dir = h_demag_direct(m, p)
    scale = np.abs(H_dir).max()
    assert np.max(np.abs(H_fft - H_dir)) <= 1e-12 * scale


@pytest.mark.parametrize("shape,cell", [((5, 4, 3), (3e-9, 2e-9, 2.5e-9)), ((6, 1, 1), (2e-9, 1e-9, 1e-9))])
def test_sampled_direct_sum_equals_brute_force(shape, cell):
    """The per-target sum with the parity-extended octant is the brute-force
    double sum (which evaluates the tensor at every signed displacement) at
    every cell, holes and several materials included."""
    nx, ny, nz = shape
    grid = W.Grid(nx, ny, nz, *cell)
    p = _problem(grid, seed=nx + 7 * ny)
    m = W.random_m(grid, seed=11)
    H_dir = h_demag_direct(m, p)
    targets = [(k, j, i) for k in range(nz) for j in range(ny) for i in range(nx)]
    H_at = h_demag_at(m, p, targets)
    ref = np.stack([H_dir[:, k, j, i] for (k, j, i) in targets])
    assert np.max(np.abs(H_at - ref)) <= 1e-12 * np.abs(ref).max()


def test_sampled_direct_sum_uniform_cube_centre():
    """Independently of the brute-force route: the centre of a uniformly
    magnetised 5x5x5 cube of cubic cells sees -Ms m / 3 (cubic symmetry and
    the trace identity), for m along each axis and along a diagonal."""
    grid = W.Grid(5, 5, 5, 2e-9, 2e-9, 2e-9)
    p = _problem(grid, holes=False)
    for u in ((1.0, 0, 0), (0, 1.0, 0), (0, 0, 1.0), (0.6, 0.0, 0.8)):
        m = np.broadcast_to(np.array(u)[:, None, None, None], (3, 5, 5, 5)).copy()
        H = h_demag_at(m, p, [(2, 2, 2)])[0]
        assert np.allclose(H, -8e5 * np.array(u) / 3.0, rtol=0, atol=1e-9 * 8e5)


@pytest.mark.parametrize("n", [3, 5, 7])
def test_uniform_cube_centre_is_minus_third(n):
    """Cubic symmetry + trace identity: the centre cell of a uniformly
    magnetised cube made of n^3 cubic cells has H = -Ms m / 3 exactly."""
    grid = W.Grid(n, n, n, 2e-9, 2e-9, 2e-9)
    p = _problem(grid, holes=False)
    for mdir in [(1, 0, 0), (0, 0, 1), (1, 1, 1)]:
        v = np.asarray(mdir, float) / np.linalg.norm(mdir)
        m = np.broadcast_to(v[:, None, None, None], (3, n, n, n)).copy()
        H = h_demag(m, p, demag_spectrum(p.shape, p.d))
        c = n // 2
        assert np.allclose(H[:, c, c, c], -p.Ms[0, 0, 0] * v / 3.0, rtol=0, atol=1e-10 * p.Ms[0, 0, 0])
        # body-averaged factor of a cube is 1/3 along every axis
        avg = H.reshape(3, -1).mean(axis=1)
        assert np.allclose(avg, -p.Ms[0, 0, 0] * v / 3.0, rtol=0, atol=1e-10 * p.Ms[0, 0, 0])


def test_interior_trace_identity():
    """Sum over sources of tr N = 1 for every target: a uniformly magnetised
    body has div H = 0 inside, so sum_a H_a(m = e_a) = -Ms."""
    grid = W.Grid(6, 4, 3, 2e-9, 3e-9, 1e-9)
    p = _problem(grid, holes=False)
    Kh = demag_spectrum(p.shape, p.d)
    tot = np.zeros(p.shape)
    for a in range(3):
        m = np.zeros((3,) + p.shape)
        m[a] = 1.0
        tot += h_demag(m, p, Kh)[a]
    assert np.allclose(tot, -p.Ms, rtol=0, atol=1e-10 * p.Ms.max())


def test_thin_film_limit():
    """A laterally large film magnetised along z approaches H_z = -Ms at its
    centre, N_xx = N_yy -> 0, with a deficit shrinking ~ thickness/size."""
    deficits = []
    for L in (16, 32, 64):
        grid = W.Grid(L, L, 1, 2e-9, 2e-9, 1e-9)
        p = _problem(grid, holes=False)
        Kh = demag_spectrum(p.shape, p.d)
        m = np.zeros((3,) + p.shape)
        m[2] = 1.0
        Hz = h_demag(m, p, Kh)[2, 0, L // 2, L // 2] / p.Ms[0, 0, 0]
        deficits.append(1.0 + Hz)
        m = np.zeros((3,) + p.shape)
        m[0] = 1.0
        Hx = h_demag(m, p, Kh)[0, 0, L // 2, L // 2] / p.Ms[0, 0, 0]
        assert -0.2 < Hx < 0
    assert all(0 < d < 0.2 for d in deficits)
    assert deficits[1] < 0.6 * deficits[0] and deficits[2] < 0.6 * deficits[1]


def test_octant_symmetric_extension_matches_direct_evaluation():
    """The padded kernel built from the octant by parity equals the tensor
    evaluated directly at negative displacements (checked via a direct sum)."""
    grid = W.Grid(5, 4, 2, 2e-9, 2e-9, 1e-9)
    p = _problem(grid, seed=3)
    m = W.random_m(grid, seed=3)
    oct_ = newell_octant(p.shape, p.d)
    H = h_demag(m, p, demag_spectrum(p.shape, p.d, oct_))
    assert np.allclose(H, h_demag_direct(m, p), rtol=0, atol=1e-12 * np.abs(H).max())


# -- periodic boundaries (image sums) -------------------------------------------
@pytest.mark.parametrize("images", [(2, 1, 0), (0, 0, 1), (1, 2, 1)])
def test_periodic_field_is_the_replicated_sample(images):
    """With R images per periodic axis the field equals the open-boundary
    field of the sample repeated 2R + 1 times along that axis, in the central
    copy (computed independently through the pinned open-boundary path)."""
    nx, ny, nz = 5, 4, 2
    grid = W.Grid(nx, ny, nz, 2e-9, 3e-9, 1.5e-9, images)
    p = _problem(grid, seed=3)
    m = W.random_m(grid, seed=8)
    H = h_demag(m, p, demag_spectrum(p.shape, p.d, images=images))
    Rx, Ry, Rz = images
    big = W.Grid(nx * (2 * Rx + 1), ny * (2 * Ry + 1), nz * (2 * Rz + 1), 2e-9, 3e-9, 1.5e-9)
    reps = (1, 2 * Rz + 1, 2 * Ry + 1, 2 * Rx + 1)
    pb = Problem.from_workload(big, W.with_cells(W.Material(Ms=8e5, A=1.3e-11, alpha=0.02),
                                                 {"Ms": np.tile(p.Ms, reps[1:])}))
    Hb = h_demag(np.tile(m, reps), pb, demag_spectrum(pb.shape, pb.d))
    c = Hb[:, Rz * nz:(Rz + 1) * nz, Ry * ny:(Ry + 1) * ny, Rx * nx:(Rx + 1) * nx]
    assert np.abs(H - c).max() < 1e-10 * np.abs(c).max()


def test_periodic_film_limit():
    """A film periodic in x and y approaches the infinite slab as the images
    grow: H = -Ms m_z z for uniform m, and no in-plane field."""
    n = 8
    errs_z, errs_x = [], []
    for R in (2, 8, 32):
        grid = W.Grid(n, n, 1, 4e-9, 4e-9, 1e-9, (R, R, 0))
        p = Problem.from_workload(grid, W.Material(Ms=8e5, A=1.3e-11, alpha=0.02))
        K = demag_spectrum(p.shape, p.d, images=(R, R, 0))
        mz = np.zeros((3,) + p.shape); mz[2] = 1
        mx = np.zeros((3,) + p.shape); mx[0] = 1
        errs_z.append(np.abs(h_demag(mz, p, K)[2] / 8e5 + 1).max())
        errs_x.append(np.abs(h_demag(mx, p, K)[0] / 8e5).max())
    assert errs_z[0] > errs_z[1] > errs_z[2] and errs_z[2] < 2e-3, errs_z
    assert errs_x[0] > errs_x[1] > errs_x[2] and errs_x[2] < 2e-3, errs_x


def test_periodic_rod_limit():
    """A square rod periodic along x: magnetised along the rod there is no
    field; across it the field tends to -Ms/2 (N_yy = N_zz = 1/2)."""
    grid = W.Grid(6, 1, 1, 2e-9, 2e-9, 2e-9, (200, 0, 0))
    p = Problem.from_workload(grid, W.Material(Ms=8e5, A=1.3e-11, alpha=0.02))
    K = demag_spectrum(p.shape, p.d, images=(200, 0, 0))
    mx = np.zeros((3,) + p.shape); mx[0] = 1
    my = np.zeros((3,) + p.shape); my[1] = 1
    assert np.abs(h_demag(mx, p, K)[0] / 8e5).max() < 2e-3
    assert np.abs(h_demag(my, p, K)[1] / 8e5 + 0.5).max() < 2e-3


def test_single_cell_precesses_at_the_kittel_frequency():
    """A single cell is magnetised uniformly, so its demagnetising field is
    -Ms (Nx mx, Ny my, Nz mz) with the prism factors of the cell.  Small-angle
    precession about an applied field along x then follows Kittel's formula
    w = gamma0 sqrt((B + mu0 Ms (Ny - Nx)) (B + mu0 Ms (Nz - Nx))), with the
    factors taken from Aharoni's closed form (independent of the oracle)."""
    import math

    from oracle.constants import GAMMA0, MU0
    from oracle.llg import Solver
    from prism import prism_factor

    d, Ms, B = (4e-9, 2e-9, 1e-9), 8e5, 0.05
    grid = W.Grid(1, 1, 1, *d)
    p = Problem.from_workload(grid, W.Material(Ms=Ms, A=1.3e-11, alpha=0.0), B_ext=(B, 0.0, 0.0))
    a, b, c = (v / 2 for v in d)
    Nx, Ny, Nz = prism_factor(b, c, a), prism_factor(c, a, b), prism_factor(a, b, c)
    w_kittel = GAMMA0 * math.sqrt((B + MU0 * Ms * (Ny - Nx)) * (B + MU0 * Ms * (Nz - Nx)))
    eps = 1e-4
    m0 = np.array([math.sqrt(1 - eps * eps), eps, 0.0]).reshape(3, 1, 1, 1)
    s = Solver(p, m0, terms=("zeeman", "demag"))
    period = 2 * math.pi / w_kittel
    dt = period / 400
    ts, ys = [0.0], [float(s.m[1, 0, 0, 0])]
    for _ in range(1400):
        s.rk45_step_fixed(dt)
        ts.append(s.t)
        ys.append(float(s.m[1, 0, 0, 0]))
    # downward zero crossings of m_y (it starts at its maximum)
    cross = [ts[i] + (ts[i + 1] - ts[i]) * ys[i] / (ys[i] - ys[i + 1])
             for i in range(len(ys) - 1) if ys[i] > 0 >= ys[i + 1]]
    assert len(cross) >= 3
    measured = (cross[-1] - cross[0]) / (len(cross) - 1)
    assert abs(measured / period - 1) < 1e-6
    # the field alone (no shape anisotropy) would give gamma0 B: far off
    assert abs(2 * math.pi / (GAMMA0 * B) / measured - 1) > 0.5
