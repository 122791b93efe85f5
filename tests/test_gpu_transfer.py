"""Host transfers through the C ABI from page-locked and pageable host
buffers give the same state (renormalised per cell, absent cells zero), in
FP32 and FP64."""
import numpy as np
import pytest

import workloads as W
from gpu_util import make_ctx, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [32, 64])
def test_pinned_and_pageable_transfers_agree(prec):
    mm = need_gpu()
    import torch
    grid = W.Grid(24, 10, 3, 2e-9, 2e-9, 2e-9)
    mat = W.with_cells(W.Material(Ms=6e5, A=1.3e-11, alpha=0.1), W.random_material_cells(grid, 2))
    ctx = make_ctx(mm, grid, mat, precision=prec, demag=False)
    try:
        rng = np.random.default_rng(3)
        m = rng.normal(size=(3,) + grid.shape) * 2.0          # not unit length
        pinned = torch.empty(m.size, dtype=torch.float64, pin_memory=True)
        mp = pinned.numpy().reshape(m.shape)
        mp[...] = m
        mm.mm_set_m(ctx, 0, mp)                               # page-locked source
        a = mm.mm_get_m(ctx, 0, m.shape)                      # pageable read-back
        mm.mm_set_m(ctx, 0, m)                                # pageable source
        out = torch.empty(m.size, dtype=torch.float64, pin_memory=True)
        b = out.numpy().reshape(m.shape)
        mm.mm_get_m(ctx, 0, m.shape, out=b)                   # page-locked read-back
        assert np.array_equal(a, b)
        present = mat.cell["Ms"] > 0
        n = np.sqrt((m ** 2).sum(axis=0))
        ref = np.where(present, m / n, 0.0)
        assert np.abs(a - ref).max() < (1e-15 if prec == 64 else 1e-7)
    finally:
        mm.mm_destroy(ctx)
