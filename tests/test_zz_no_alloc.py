"""The allocation-free topological charge (for callers that may not allocate
device memory, e.g. inside a CUDA graph capture or a framework-owned memory
pool) must agree with the allocating entry point mm_topo_charge.  Collected
last so that a run stopping at the first failure has run everything else."""
import numpy as np
import pytest

import workloads as W
from gpu_util import make_ctx, need_gpu

pytestmark = pytest.mark.gpu


def _skyrmion(grid, R, w):
    x = (np.arange(grid.nx) - grid.nx / 2 + 0.5) * grid.dx
    y = (np.arange(grid.ny) - grid.ny / 2 + 0.5) * grid.dy
    X, Y = np.meshgrid(x, y)
    r = np.hypot(X, Y)
    th = 2 * np.arctan(np.exp(-(r - R) / w))
    ph = np.arctan2(Y, X)
    m = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    return np.broadcast_to(m[:, None], (3, grid.nz, grid.ny, grid.nx)).copy()


@pytest.mark.parametrize("prec", [32, 64])
def test_noalloc_charge_matches_allocating_entry_point(prec):
    mm = need_gpu()
    import torch
    grid = W.Grid(96, 80, 3, 1e-9, 1e-9, 1e-9)
    ctx = make_ctx(mm, grid, W.Material(Ms=5.8e5, A=1.5e-11, alpha=0.1), precision=prec, demag=False)
    try:
        m = _skyrmion(grid, 12e-9, 3e-9)
        m[:, 1] = W.random_m(W.Grid(96, 80, 1, 1e-9, 1e-9, 1e-9), seed=4)[:, 0]   # a layer with another charge
        mm.mm_set_m(ctx, 0, m)
        dtype = torch.float32 if prec == 32 else torch.float64
        m_dev = torch.empty(3 * grid.n, dtype=dtype, device="cuda")
        mm.mm_get_m_device(ctx, m_dev.data_ptr())
        q_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        torch.cuda.synchronize()
        for layer in (-1, 1):           # two calls in a row share the scratch array
            mm.mm_topo_charge_noalloc(m_dev.data_ptr(), prec, grid.nx, grid.ny, grid.nz, grid.dx, grid.dy, layer,
                                      q_dev.data_ptr(), stream)
            torch.cuda.synchronize()
            q_new = float(q_dev.item())
            q_ref = mm.mm_topo_charge(ctx, 0, layer)
            assert abs(q_new - q_ref) <= 1e-12 * max(1.0, abs(q_ref)), (layer, q_new, q_ref)
    finally:
        mm.mm_destroy(ctx)


def test_noalloc_charge_rejects_oversized_input():
    mm = need_gpu()
    import torch
    q_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    m_dev = torch.zeros(3, dtype=torch.float32, device="cuda")
    with pytest.raises(mm.MMError) as e:
        # 4097 x 4096 cells exceed the fixed partial-sum array; rejected before any launch
        mm.mm_topo_charge_noalloc(m_dev.data_ptr(), 32, 4097, 4096, 1, 1e-9, 1e-9, -1, q_dev.data_ptr())
    assert e.value.status == mm.MM_ERR_ARG
