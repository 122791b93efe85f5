"""ctypes binding of libmm (include/mm.h): the same function names as the C
ABI, argument marshalling only.  Every step of the hot path runs in the
library's CUDA kernels.

Host arrays are float64 numpy arrays in the ABI layout (component-major,
x fastest: shape (3, nz, ny, nx)).  Device arrays may be torch tensors (their
data_ptr is passed) in the context's precision.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_HERE, "libmm.so")
_lib = None
_lock = threading.Lock()

MM_OK, MM_ERR_ARG, MM_ERR_DEVICE, MM_ERR_OOM, MM_ERR_CUDA = 0, 1, 2, 3, 4
MM_ERR_NONFINITE, MM_ERR_DT_UNDERFLOW, MM_ERR_TIMEOUT, MM_ERR_STATE = 5, 6, 7, 8
MM_HEUN, MM_RK45, MM_RK4, MM_DM, MM_DM_ADAPTIVE = 0, 1, 2, 3, 4
MM_DEMAG_OFF, MM_DEMAG_EXACT, MM_DEMAG_SURROGATE = 0, 1, 2
MM_TERM_EXCHANGE, MM_TERM_DMI, MM_TERM_ANISOTROPY = 1, 2, 4
MM_TERM_ZEEMAN, MM_TERM_DEMAG, MM_TERM_THERMAL = 8, 16, 32
MM_TERM_CUBIC, MM_TERM_SURFACE, MM_TERM_RKKY, MM_TERM_MEL, MM_TERM_ALL = 64, 128, 256, 512, 1023
MM_E_EXCHANGE, MM_E_DMI, MM_E_ANISOTROPY, MM_E_ZEEMAN, MM_E_DEMAG, MM_E_TOTAL = range(6)
MM_E_CUBIC, MM_E_SURFACE, MM_E_RKKY, MM_E_MEL, MM_NENERGY = 6, 7, 8, 9, 10
MM_TORQUE_NONE, MM_TORQUE_SOT, MM_TORQUE_STT, MM_TORQUE_ZL = 0, 1, 2, 3

_D = C.POINTER(C.c_double)


class mm_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("pbc", C.c_int * 3)]


class mm_material(C.Structure):
    _fields_ = [("Ms", C.c_double), ("A", C.c_double), ("alpha", C.c_double), ("Ku1", C.c_double),
                ("u", C.c_double * 3), ("D", C.c_double),
                ("Ms_cell", _D), ("A_cell", _D), ("alpha_cell", _D), ("Ku1_cell", _D),
                ("u_cell", _D), ("D_cell", _D), ("D_bulk", C.c_double), ("D_bulk_cell", _D),
                ("Kc1", C.c_double), ("Kc2", C.c_double), ("c1", C.c_double * 3), ("c2", C.c_double * 3),
                ("Ks", C.c_double), ("B1", C.c_double), ("B2", C.c_double)]


class mm_config(C.Structure):
    _fields_ = [("precision", C.c_int), ("integrator", C.c_int), ("demag", C.c_int), ("terms", C.c_uint),
                ("dt", C.c_double), ("rtol", C.c_double), ("dt_min", C.c_double), ("dt_max", C.c_double),
                ("T", C.c_double), ("seed", C.c_uint64)]


class mm_torque(C.Structure):
    _fields_ = [("kind", C.c_int), ("p", C.c_double * 3), ("theta_SH", C.c_double), ("fl_ratio", C.c_double),
                ("P", C.c_double), ("Lambda", C.c_double), ("eps_prime", C.c_double), ("t_F", C.c_double),
                ("xi", C.c_double), ("dir", C.c_double * 3), ("match_mumax", C.c_int)]


class mm_stats(C.Structure):
    _fields_ = [("accepted", C.c_longlong), ("rejected", C.c_longlong), ("attempts", C.c_longlong),
                ("kernel_launches", C.c_longlong), ("t", C.c_double), ("dt", C.c_double)]


class mm_profile_entry(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_longlong), ("total_ms", C.c_double),
                ("bytes_per_launch", C.c_double)]


class mm_train_cfg(C.Structure):
    _fields_ = [("n_snapshots", C.c_int), ("snap_every", C.c_int), ("max_gap", C.c_int), ("crop", C.c_int),
                ("batch", C.c_int), ("steps", C.c_int), ("lr", C.c_double), ("seed", C.c_uint64)]


class mm_surrogate_stats(C.Structure):
    _fields_ = [("exact_evals", C.c_longlong), ("surrogate_evals", C.c_longlong), ("refreshes", C.c_longlong),
                ("fallback", C.c_int), ("last_error", C.c_double), ("max_error", C.c_double),
                ("train_loss", C.c_double), ("c_in", C.c_double), ("c_out", C.c_double)]


class mm_trials(C.Structure):
    _fields_ = [("n_trials", C.c_longlong), ("J", _D), ("T", _D), ("m_init", _D), ("axis", C.c_double * 3),
                ("threshold", C.c_double), ("max_steps", C.c_longlong), ("base_seed", C.c_uint64),
                ("refill", C.c_int)]


class MMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libmm status {status}: {msg}")
        self.status = status


_SIGS = {
    "mm_create": [C.POINTER(mm_grid), C.POINTER(mm_material), C.POINTER(mm_config), C.POINTER(C.c_void_p)],
    "mm_create_batch": [C.c_int, C.POINTER(mm_grid), C.POINTER(mm_material), C.POINTER(mm_config),
                        C.POINTER(C.c_uint64), C.POINTER(C.c_void_p)],
    "mm_destroy": [C.c_void_p],
    "mm_set_stream": [C.c_void_p, C.c_void_p],
    "mm_set_m": [C.c_void_p, C.c_int, _D],
    "mm_get_m": [C.c_void_p, C.c_int, _D],
    "mm_set_m_device": [C.c_void_p, C.c_void_p],
    "mm_get_m_device": [C.c_void_p, C.c_void_p],
    "mm_set_field": [C.c_void_p, C.c_int, _D, _D],
    "mm_set_temperature": [C.c_void_p, _D],
    "mm_set_strain": [C.c_void_p, _D, _D],
    "mm_set_rkky": [C.c_void_p, C.c_int, C.c_int, C.c_double],
    "mm_set_torque": [C.c_void_p, C.POINTER(mm_torque), _D],
    "mm_step": [C.c_void_p, C.c_long],
    "mm_step_dt": [C.c_void_p, _D, C.c_long],
    "mm_run": [C.c_void_p, C.c_double],
    "mm_get_heff": [C.c_void_p, C.c_int, _D, C.c_uint],
    "mm_energy": [C.c_void_p, C.c_int, _D],
    "mm_topo_charge": [C.c_void_p, C.c_int, C.c_int, _D],
    "mm_mean_m": [C.c_void_p, C.c_int, C.c_int, _D],
    "mm_get_time": [C.c_void_p, C.c_int, _D, _D, C.POINTER(C.c_longlong)],
    "mm_get_stats": [C.c_void_p, C.POINTER(mm_stats)],
    "mm_get_state": [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)],
    "mm_set_state": [C.c_void_p, C.c_void_p, C.c_size_t],
    "mm_get_thermal": [C.c_void_p, C.c_int, C.c_longlong, C.POINTER(C.c_uint32), _D],
    "mm_get_demag_kernel": [C.c_void_p, _D, C.c_size_t, C.POINTER(C.c_int)],
    "mm_newell": [C.c_long, C.POINTER(C.c_int), C.c_double, C.c_double, C.c_double, _D],
    "mm_topo_charge_noalloc": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                               C.c_void_p, C.c_void_p],
    "mm_batch_autotune": [C.c_void_p, C.c_char_p, C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "mm_batch_set_shape": [C.c_void_p, C.c_int, C.c_int],
    "mm_trials_start": [C.c_void_p, C.POINTER(mm_trials)],
    "mm_trials_result": [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.POINTER(C.c_longlong)],
    "mm_surrogate_train": [C.c_void_p, C.POINTER(mm_train_cfg), _D],
    "mm_surrogate_set": [C.c_void_p, C.c_int, C.c_double],
    "mm_surrogate_get_stats": [C.c_void_p, C.POINTER(mm_surrogate_stats)],
    "mm_surrogate_weights": [C.c_void_p, _D, _D, C.c_size_t, _D],
    "mm_surrogate_forward": [C.c_void_p, C.c_int, C.c_int, C.c_int, _D, _D, C.c_int],
    "mm_surrogate_grad": [C.c_void_p, C.c_int, C.c_int, C.c_int, _D, _D, _D, _D, C.c_int],
    "mm_set_profiling": [C.c_void_p, C.c_int],
    "mm_get_profile": [C.c_void_p, C.POINTER(mm_profile_entry), C.POINTER(C.c_int)],
    "mm_debug_inject": [C.c_void_p, C.c_int],
    "mm_last_error": [C.c_void_p],
    "mm_status_string": [C.c_int],
    "mm_measure_peak": [C.c_int, _D],
}


def load(path: str | None = None):
    """Load libmm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or lib_path
            if not os.path.exists(p):
                raise MMError(-1, f"{p} is missing: build it with paper_2608_15253_gb300/build.py "
                                  "(there is no CPU fallback)")
            lib = C.CDLL(p)
            for name, args in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = C.c_char_p if name in ("mm_last_error", "mm_status_string") else C.c_int
            _lib = lib
    return _lib


def _check(status, ctx=None):
    if status != MM_OK:
        lib = load()
        msg = lib.mm_last_error(ctx).decode() if lib.mm_last_error(ctx) else ""
        raise MMError(status, msg)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


# ---------------------------------------------------------------------------
# C functions under their C names (argument marshalling only)
# ---------------------------------------------------------------------------

def mm_create(grid: mm_grid, mat: mm_material, cfg: mm_config):
    ctx = C.c_void_p()
    _check(load().mm_create(C.byref(grid), C.byref(mat), C.byref(cfg), C.byref(ctx)))
    return ctx


def mm_create_batch(grids, mat: mm_material, cfg: mm_config, seeds=None):
    arr = (mm_grid * len(grids))(*grids)
    sp = None
    if seeds is not None:
        s = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
        sp = s.ctypes.data_as(C.POINTER(C.c_uint64))
    ctx = C.c_void_p()
    _check(load().mm_create_batch(len(grids), arr, C.byref(mat), C.byref(cfg), sp, C.byref(ctx)))
    return ctx


def mm_destroy(ctx):
    _check(load().mm_destroy(ctx))


def mm_set_stream(ctx, stream_ptr: int | None):
    _check(load().mm_set_stream(ctx, C.c_void_p(stream_ptr) if stream_ptr else None), ctx)


def mm_set_m(ctx, replica: int, m):
    a = _f64(m)
    _check(load().mm_set_m(ctx, replica, _dptr(a)), ctx)


def mm_get_m(ctx, replica: int, shape, out=None):
    """out: optional C-contiguous float64 array of `shape` to fill (e.g. a
    view of page-locked memory)."""
    if out is None:
        out = np.zeros(shape, dtype=np.float64)
    elif out.dtype != np.float64 or not out.flags.c_contiguous or out.shape != tuple(shape):
        raise ValueError("out must be a C-contiguous float64 array of the given shape")
    _check(load().mm_get_m(ctx, replica, _dptr(out)), ctx)
    return out


def mm_set_m_device(ctx, dev_ptr: int):
    _check(load().mm_set_m_device(ctx, C.c_void_p(dev_ptr)), ctx)


def mm_get_m_device(ctx, dev_ptr: int):
    _check(load().mm_get_m_device(ctx, C.c_void_p(dev_ptr)), ctx)


def mm_set_field(ctx, replica: int, B, B_cell=None):
    b = _f64(B, 3)
    bc = _f64(B_cell) if B_cell is not None else None
    _check(load().mm_set_field(ctx, replica, _dptr(b), _dptr(bc) if bc is not None else None), ctx)


def mm_set_temperature(ctx, T):
    t = _f64(np.atleast_1d(T))
    _check(load().mm_set_temperature(ctx, _dptr(t)), ctx)


def mm_set_torque(ctx, tq: mm_torque, J):
    j = _f64(np.atleast_1d(J))
    _check(load().mm_set_torque(ctx, C.byref(tq), _dptr(j)), ctx)


def mm_step(ctx, n: int):
    _check(load().mm_step(ctx, int(n)), ctx)


def mm_step_dt(ctx, dts):
    d = _f64(dts)
    _check(load().mm_step_dt(ctx, _dptr(d), d.size), ctx)


def mm_run(ctx, t_end: float):
    _check(load().mm_run(ctx, float(t_end)), ctx)


def mm_get_heff(ctx, replica: int, shape, term_mask: int = MM_TERM_ALL):
    out = np.zeros(shape, dtype=np.float64)
    _check(load().mm_get_heff(ctx, replica, _dptr(out), term_mask), ctx)
    return out


def mm_set_strain(ctx, eps=None, eps_cell=None):
    """Uniform strain eps[6] (xx, yy, zz, xy, xz, yz) or per cell (6, nz, ny, nx)."""
    e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
    ec = None if eps_cell is None else _f64(eps_cell)
    _check(load().mm_set_strain(ctx, _dptr(e) if e is not None else None, _dptr(ec) if ec is not None else None),
           ctx)


def mm_set_rkky(ctx, k1: int, k2: int, J: float):
    _check(load().mm_set_rkky(ctx, int(k1), int(k2), float(J)), ctx)


def mm_energy(ctx, replica: int = 0):
    out = np.zeros(MM_NENERGY, dtype=np.float64)
    _check(load().mm_energy(ctx, replica, _dptr(out)), ctx)
    return out


def mm_topo_charge(ctx, replica: int = 0, layer: int = -1):
    q = C.c_double()
    _check(load().mm_topo_charge(ctx, replica, layer, C.byref(q)), ctx)
    return q.value


def mm_mean_m(ctx, replica: int = 0, layer: int = -1):
    out = np.zeros(3, dtype=np.float64)
    _check(load().mm_mean_m(ctx, replica, layer, _dptr(out)), ctx)
    return out


def mm_get_time(ctx, replica: int = 0):
    t, dt, n = C.c_double(), C.c_double(), C.c_longlong()
    _check(load().mm_get_time(ctx, replica, C.byref(t), C.byref(dt), C.byref(n)), ctx)
    return t.value, dt.value, n.value


def mm_get_stats(ctx):
    s = mm_stats()
    _check(load().mm_get_stats(ctx, C.byref(s)), ctx)
    return {k: getattr(s, k) for k, _ in mm_stats._fields_}


def mm_get_state(ctx) -> bytes:
    n = C.c_size_t(0)
    _check(load().mm_get_state(ctx, None, C.byref(n)), ctx)
    buf = C.create_string_buffer(n.value)
    _check(load().mm_get_state(ctx, buf, C.byref(n)), ctx)
    return buf.raw


def mm_set_state(ctx, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _check(load().mm_set_state(ctx, buf, len(blob)), ctx)


def mm_get_thermal(ctx, replica: int, step: int, ncell: int, raw=True, field=True):
    r = np.zeros(4 * ncell, dtype=np.uint32) if raw else None
    h = np.zeros(3 * ncell, dtype=np.float64) if field else None
    _check(load().mm_get_thermal(ctx, replica, step,
                                 r.ctypes.data_as(C.POINTER(C.c_uint32)) if raw else None,
                                 _dptr(h) if field else None), ctx)
    return r, h


def mm_get_demag_kernel(ctx):
    dims = (C.c_int * 4)()
    _check(load().mm_get_demag_kernel(ctx, None, 0, dims), ctx)
    ncomp, Px, Py, Pz = dims[:]
    shape = (ncomp, Pz // 2 + 1, Py // 2 + 1, Px // 2 + 1)
    out = np.zeros(shape, dtype=np.float64)
    _check(load().mm_get_demag_kernel(ctx, _dptr(out), out.size, dims), ctx)
    return out, (Px, Py, Pz)


def mm_newell(ijk, d):
    a = np.ascontiguousarray(np.asarray(ijk, dtype=np.int32).reshape(-1, 3))
    out = np.zeros((a.shape[0], 6), dtype=np.float64)
    _check(load().mm_newell(a.shape[0], a.ctypes.data_as(C.POINTER(C.c_int)), d[0], d[1], d[2], _dptr(out)))
    return out


def mm_topo_charge_noalloc(m_dev: int, precision: int, nx: int, ny: int, nz: int, dx: float, dy: float,
                           layer: int, q_dev: int, stream: int | None = None):
    """Device pointers in and out (ints, e.g. torch data_ptr()); allocates nothing."""
    _check(load().mm_topo_charge_noalloc(C.c_void_p(m_dev), precision, nx, ny, nz, dx, dy, layer, C.c_void_p(q_dev),
                                         C.c_void_p(stream) if stream else None))


def mm_batch_autotune(ctx, cache_path: str | None = None):
    nt, blocks = C.c_int(0), C.c_int(0)
    _check(load().mm_batch_autotune(ctx, cache_path.encode() if cache_path else None, C.byref(nt), C.byref(blocks)),
           ctx)
    return nt.value, blocks.value


def mm_batch_set_shape(ctx, nt: int, blocks: int = 0):
    """nt = 0: stacked shape; 256 or 512 threads with `blocks` persistent CTAs."""
    _check(load().mm_batch_set_shape(ctx, int(nt), int(blocks)), ctx)


def mm_trials_start(ctx, J, T, m_init, axis=(0.0, 0.0, 1.0), threshold=0.0, max_steps=1000, base_seed=0,
                    refill=True):
    """Retire/refill over len(J) trials; J, T per trial, m_init (3, 1, ny, nx)."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    m0 = np.ascontiguousarray(m_init, dtype=np.float64)
    if J.shape != T.shape:
        raise ValueError("J and T need one entry per trial")
    sp = mm_trials(J.size, _dptr(J), _dptr(T), _dptr(m0), (C.c_double * 3)(*axis), threshold, max_steps,
                   int(base_seed), 1 if refill else 0)
    _check(load().mm_trials_start(ctx, C.byref(sp)), ctx)
    ctx._trials_n = J.size


def mm_trials_result(ctx):
    """(steps[n], stopped[n], done): steps -1 while a trial is unfinished."""
    n = ctx._trials_n
    steps = np.zeros(n, dtype=np.int64)
    stopped = np.zeros(n, dtype=np.int32)
    done = C.c_longlong(0)
    _check(load().mm_trials_result(ctx, steps.ctypes.data_as(C.POINTER(C.c_longlong)),
                                   stopped.ctypes.data_as(C.POINTER(C.c_int)), C.byref(done)), ctx)
    return steps, stopped.astype(bool), done.value


SURROGATE_NPARAMS = 56099


def mm_surrogate_train(ctx, cfg: mm_train_cfg) -> float:
    loss = C.c_double(0.0)
    _check(load().mm_surrogate_train(ctx, C.byref(cfg), C.byref(loss)), ctx)
    return loss.value


def mm_surrogate_set(ctx, k: int, tol: float = 1e-3):
    _check(load().mm_surrogate_set(ctx, int(k), float(tol)), ctx)


def mm_surrogate_get_stats(ctx):
    s = mm_surrogate_stats()
    _check(load().mm_surrogate_get_stats(ctx, C.byref(s)), ctx)
    return {k: getattr(s, k) for k, _ in mm_surrogate_stats._fields_}


def mm_surrogate_weights(ctx, set_params=None, c_in=None):
    """Returns (params, c_in); set_params (56099 values) replaces them first."""
    get = np.zeros(SURROGATE_NPARAMS)
    st = _f64(set_params, SURROGATE_NPARAMS) if set_params is not None else None
    ci = C.c_double(c_in if c_in is not None else 1.0)
    _check(load().mm_surrogate_weights(ctx, _dptr(get), _dptr(st) if st is not None else None, SURROGATE_NPARAMS,
                                       C.byref(ci) if (c_in is not None or st is None) else None), ctx)
    return get, ci.value


def mm_surrogate_forward(ctx, x, path: int = 0):
    x = _f64(x)
    B, _, H, W = x.shape
    y = np.zeros((B, 3, H, W))
    _check(load().mm_surrogate_forward(ctx, B, H, W, _dptr(x), _dptr(y), path), ctx)
    return y


def mm_surrogate_grad(ctx, x, t, path: int = 0):
    x = _f64(x)
    t = _f64(t)
    B, _, H, W = x.shape
    loss = C.c_double(0.0)
    g = np.zeros(SURROGATE_NPARAMS)
    _check(load().mm_surrogate_grad(ctx, B, H, W, _dptr(x), _dptr(t), C.byref(loss), _dptr(g), path), ctx)
    return loss.value, g


def make_train_cfg(n_snapshots=24, snap_every=4, max_gap=6, crop=128, batch=16, steps=1000, lr=1e-3, seed=4):
    return mm_train_cfg(n_snapshots, snap_every, max_gap, crop, batch, steps, lr, seed)


def mm_set_profiling(ctx, on: bool):
    _check(load().mm_set_profiling(ctx, 1 if on else 0), ctx)


def mm_get_profile(ctx):
    n = C.c_int(0)
    _check(load().mm_get_profile(ctx, None, C.byref(n)), ctx)
    arr = (mm_profile_entry * max(1, n.value))()
    _check(load().mm_get_profile(ctx, arr, C.byref(n)), ctx)
    return [{"name": arr[q].name.decode(), "launches": arr[q].launches, "total_ms": arr[q].total_ms,
             "bytes_per_launch": arr[q].bytes_per_launch} for q in range(n.value)]


def mm_measure_peak(precision: int) -> float:
    """Measured FP32 (32) or FP64 (64) fused multiply-add throughput, flop/s."""
    v = C.c_double()
    _check(load().mm_measure_peak(precision, C.byref(v)))
    return v.value


def mm_debug_inject(ctx, fault: int):
    _check(load().mm_debug_inject(ctx, fault), ctx)


def mm_last_error(ctx=None) -> str:
    v = load().mm_last_error(ctx)
    return v.decode() if v else ""


def mm_status_string(s: int) -> str:
    return load().mm_status_string(s).decode()


# ---------------------------------------------------------------------------
# struct builders (marshalling helpers)
# ---------------------------------------------------------------------------

def make_grid(nx, ny, nz, dx, dy, dz, pbc=(0, 0, 0)) -> mm_grid:
    g = mm_grid(nx, ny, nz, dx, dy, dz)
    g.pbc[:] = list(pbc)
    return g


class Material:
    """mm_material plus ownership of its per-cell arrays (kept alive here)."""

    def __init__(self, Ms, A, alpha, Ku1=0.0, u=(0.0, 0.0, 1.0), D=0.0, cells=None, Db=0.0, Kc1=0.0, Kc2=0.0,
                 c1=(1.0, 0.0, 0.0), c2=(0.0, 1.0, 0.0), Ks=0.0, B1=0.0, B2=0.0):
        self.s = mm_material(Ms, A, alpha, Ku1)
        self.s.u[:] = list(u)
        self.s.D = D
        self.s.D_bulk = Db
        self.s.Kc1, self.s.Kc2, self.s.Ks, self.s.B1, self.s.B2 = Kc1, Kc2, Ks, B1, B2
        self.s.c1[:] = list(c1)
        self.s.c2[:] = list(c2)
        self._keep = []
        for name, arr in (cells or {}).items():
            a = _f64(arr)
            self._keep.append(a)
            setattr(self.s, f"{'D_bulk' if name == 'Db' else name}_cell", _dptr(a))


def make_config(precision=32, integrator=MM_RK45, demag=MM_DEMAG_EXACT, terms=0, dt=1e-14, rtol=1e-6,
                dt_min=0.0, dt_max=0.0, T=0.0, seed=0) -> mm_config:
    return mm_config(precision, integrator, demag, terms, dt, rtol, dt_min, dt_max, T, seed)


def make_torque(kind=MM_TORQUE_NONE, p=(0.0, 1.0, 0.0), theta_SH=0.0, fl_ratio=0.0, P=0.0, Lambda=1.0,
                eps_prime=0.0, t_F=0.0, xi=0.0, direction=(1.0, 0.0, 0.0), match_mumax=0) -> mm_torque:
    t = mm_torque()
    t.kind = kind
    t.p[:] = list(p)
    t.theta_SH, t.fl_ratio, t.P, t.Lambda, t.eps_prime, t.t_F, t.xi = theta_SH, fl_ratio, P, Lambda, eps_prime, t_F, xi
    t.dir[:] = list(direction)
    t.match_mumax = match_mumax
    return t
