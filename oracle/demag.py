"""Open-boundary demagnetising field of the oracle.

Methods, "Physics and discretization": open-boundary demagnetisation by FFT
convolution with the Newell tensor, zero-padded to 2N.  The oracle follows
the definition directly:

    H_a(r) = - sum_{r'} sum_b N_ab(r - r') Ms(r') m_b(r')

evaluated (i) as a brute-force O(N^2) double sum (``h_demag_direct``) and
(ii) as a circular convolution on the grid zero-padded to 2n per axis with
full complex numpy FFTs (``h_demag``) -- no pruning, no symmetry
compression.  The tensor itself comes from ``newell.c`` (closed form near,
tent quadrature far).

Readings: the source-cell Ms multiplies m (per-cell Ms); the padded length
is 2n on every axis (2 on a singleton axis, where only the zero
displacement exists).

Periodic boundaries (Methods: "periodic-boundary demagnetization by an
image-sum kernel"; the number of images is not printed).  With R_x images
on a periodic x axis (likewise y, z) the field is that of the sample and
its 2R_x + 1 copies shifted by multiples of the box length, evaluated in
the central copy:

    H_a(r) = - sum_{|p| <= R} sum_{r'} sum_b N_ab(r - r' - p L) Ms m_b(r'),

so the tensor becomes the image sum  sum_p N(d - p L)  over displacements
|d| < n, and the same zero-padded convolution applies unchanged.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_library(force: bool = False) -> str:
    """Compile newell.c into oracle/liboracle.so with gcc (-O2, OpenMP)."""
    src = os.path.join(_HERE, "newell.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _get_lib():
    global _lib
    with _lock:
        if _lib is None:
            build_library()
            lib = ctypes.CDLL(_LIB_PATH)
            d = ctypes.c_double
            P = ctypes.POINTER(ctypes.c_double)
            lib.oracle_newell_f.restype = d
            lib.oracle_newell_f.argtypes = [d, d, d]
            lib.oracle_newell_g.restype = d
            lib.oracle_newell_g.argtypes = [d, d, d]
            for fn in (lib.oracle_newell_analytic, lib.oracle_newell_at):
                fn.restype = None
                fn.argtypes = [d, d, d, d, d, d, P]
            lib.oracle_newell_quadrature.restype = None
            lib.oracle_newell_quadrature.argtypes = [d, d, d, d, d, d, ctypes.c_int, P]
            lib.oracle_newell_octant.restype = None
            lib.oracle_newell_octant.argtypes = [ctypes.c_int] * 3 + [d, d, d, P]
            lib.oracle_newell_list.restype = None
            lib.oracle_newell_list.argtypes = [ctypes.c_long, ctypes.POINTER(ctypes.c_int), d, d, d, P]
            _lib = lib
    return _lib


def newell_f(x, y, z):
    return _get_lib().oracle_newell_f(x, y, z)


def newell_g(x, y, z):
    return _get_lib().oracle_newell_g(x, y, z)


def _six(fn, *args):
    out = (ctypes.c_double * 6)()
    fn(*args, out)
    return np.array(out[:])


def newell_analytic(X, Y, Z, d):
    """Closed form (xx, yy, zz, xy, xz, yz) at displacement (X,Y,Z) metres."""
    return _six(_get_lib().oracle_newell_analytic, X, Y, Z, *d)


def newell_quadrature(X, Y, Z, d, nq):
    return _six(_get_lib().oracle_newell_quadrature, X, Y, Z, d[0], d[1], d[2], nq)


def newell_at(ijk, d) -> np.ndarray:
    """Tensor at integer displacements ijk (count, 3) -> (count, 6)."""
    ijk = np.ascontiguousarray(np.asarray(ijk, dtype=np.int32).reshape(-1, 3))
    out = np.zeros((ijk.shape[0], 6))
    _get_lib().oracle_newell_list(ijk.shape[0], ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  d[0], d[1], d[2], out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def newell_octant(shape, d) -> np.ndarray:
    """Tensor on displacements 0 <= i<nx, 0<=j<ny, 0<=k<nz -> (6, nz, ny, nx)."""
    nz, ny, nx = shape
    out = np.zeros((6, nz, ny, nx))
    _get_lib().oracle_newell_octant(nx, ny, nz, d[0], d[1], d[2],
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def newell_octant_images(shape, d, images) -> np.ndarray:
    """Image-summed tensor on the octant displacements: sum over
    a in [-R_x, R_x], b in [-R_y, R_y], c in [-R_z, R_z] of
    N(i + a nx, j + b ny, k + c nz) -> (6, nz, ny, nx)."""
    nz, ny, nx = shape
    Rx, Ry, Rz = (int(v) for v in images)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    out = np.zeros((nz * ny * nx, 6))
    for a in range(-Rx, Rx + 1):
        for b in range(-Ry, Ry + 1):
            for c in range(-Rz, Rz + 1):
                out += newell_at(base + np.array([a * nx, b * ny, c * nz]), d)
    return out.T.reshape(6, nz, ny, nx)


# parity of each component under (x -> -x, y -> -y, z -> -z)
_PARITY = {0: (1, 1, 1), 1: (1, 1, 1), 2: (1, 1, 1),
           3: (-1, -1, 1), 4: (-1, 1, -1), 5: (1, -1, -1)}
# component index of the (a, b) tensor element
COMP = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}


def padded_kernel(shape, d, octant=None) -> np.ndarray:
    """Tensor placed on the zero-padded (2nz, 2ny, 2nx) grid at wrap-around
    positions (displacement i at index i mod 2nx); the index n (no
    displacement) stays zero.  Other octants by parity of each component."""
    nz, ny, nx = shape
    if octant is None:
        octant = newell_octant(shape, d)
    P = (2 * nz, 2 * ny, 2 * nx)
    K = np.zeros((6,) + P)
    for c in range(6):
        px, py, pz = _PARITY[c]
        for sz in (1, -1):
            for sy in (1, -1):
                for sx in (1, -1):
                    sign = (px if sx < 0 else 1) * (py if sy < 0 else 1) * (pz if sz < 0 else 1)
                    # a mirrored octant excludes its zero plane (owned by the + side)
                    k0, j0, i0 = (0 if sz > 0 else 1), (0 if sy > 0 else 1), (0 if sx > 0 else 1)
                    kk = (sz * np.arange(k0, nz)) % P[0]
                    jj = (sy * np.arange(j0, ny)) % P[1]
                    ii = (sx * np.arange(i0, nx)) % P[2]
                    K[c][np.ix_(kk, jj, ii)] = sign * octant[c][k0:, j0:, i0:]
    return K


def demag_spectrum(shape, d, octant=None, images=(0, 0, 0)) -> np.ndarray:
    """Full complex FFT of each padded tensor component -> (6, 2nz, 2ny, 2nx);
    images: periodic image counts per axis (x, y, z), 0 = open."""
    if octant is None and any(images):
        octant = newell_octant_images(shape, d, images)
    K = padded_kernel(shape, d, octant)
    return np.fft.fftn(K, axes=(1, 2, 3))


def h_demag(m: np.ndarray, p, K_hat: np.ndarray) -> np.ndarray:
    """H_a = -IFFT( sum_b K_hat_ab * FFT(Ms m_b) ), cropped to the grid."""
    nz, ny, nx = p.shape
    P = K_hat.shape[1:]
    M_hat = []
    for b in range(3):
        M = np.zeros(P)
        M[:nz, :ny, :nx] = p.Ms * m[b]
        M_hat.append(np.fft.fftn(M))
    H = np.zeros_like(m)
    for a in range(3):
        acc = np.zeros(P, dtype=complex)
        for b in range(3):
            acc += K_hat[COMP[(a, b)]] * M_hat[b]
        H[a] = -np.fft.ifftn(acc).real[:nz, :ny, :nx]
    return H


def h_demag_at(m: np.ndarray, p, targets, octant=None) -> np.ndarray:
    """H at the listed target cells, rows (k, j, i), by the double sum of the
    definition over every source cell: -sum_{r'} sum_b N_ab(r - r') Ms m_b(r').
    The tensor at a displacement with negative components is the octant
    entry at its absolute value times each component's parity, which is
    what lets large grids be sampled (one octant, then one O(N) sum per
    target).  Returns (len(targets), 3)."""
    nz, ny, nx = p.shape
    if octant is None:
        octant = newell_octant(p.shape, p.d)
    M = p.Ms[None] * m
    out = np.zeros((len(targets), 3))
    for n, (kt, jt, it) in enumerate(targets):
        dk, dj, di = kt - np.arange(nz), jt - np.arange(ny), it - np.arange(nx)   # target - source
        N = []
        for c in range(6):
            px, py, pz = _PARITY[c]
            sx = np.where(di < 0, px, 1.0)
            sy = np.where(dj < 0, py, 1.0)
            sz = np.where(dk < 0, pz, 1.0)
            N.append(octant[c][np.ix_(np.abs(dk), np.abs(dj), np.abs(di))]
                     * sz[:, None, None] * sy[None, :, None] * sx[None, None, :])
        for a in range(3):
            out[n, a] = -sum(float(np.vdot(N[COMP[(a, b)]], M[b])) for b in range(3))
    return out


def h_demag_direct(m: np.ndarray, p) -> np.ndarray:
    """Brute-force double sum over all target/source pairs (tiny grids only)."""
    nz, ny, nx = p.shape
    H = np.zeros_like(m)
    idx = np.array([(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)])
    for t in range(len(idx)):
        disp = idx[t][None, :] - idx                 # target - source
        N = newell_at(disp, p.d)                     # (nsrc, 6)
        src = idx
        M = p.Ms[src[:, 2], src[:, 1], src[:, 0]][None, :] * m[:, src[:, 2], src[:, 1], src[:, 0]]
        it, jt, kt = idx[t]
        for a in range(3):
            s = 0.0
            for b in range(3):
                s += np.dot(N[:, COMP[(a, b)]], M[b])
            H[a, kt, jt, it] = -s
    return H
