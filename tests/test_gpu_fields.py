"""Field transfers through the C ABI: pinned host buffers (read and written by the packing
kernels directly) give the same values as pageable ones (staged through device memory)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_pinned_and_pageable_transfers_agree(gpu, precision):
    import torch
    C = gpu
    N = 20
    grid = C.icon_grid_build(2, 2, N)
    st = C.icon_state_init_ex(grid, 3, C.ICON_CASE_JET, noise_K=0.1, precision=precision)
    try:
        C.icon_dycore_step(st, 300.0, 5)
        for f in ("vn", "w", "rho", "theta_v", "exner", "mflx", "wflx"):
            page = C.icon_state_copy_field(st, grid, N, f)
            pinned = torch.empty(page.shape, dtype=torch.float64, pin_memory=True).numpy()
            C.icon_state_copy_field(st, grid, N, f, pinned)
            assert np.array_equal(page, pinned), f
        # write through pinned memory, read back through pageable memory
        for f in ("vn", "w", "rho", "theta_v", "exner"):
            x = C.icon_state_copy_field(st, grid, N, f)
            y = x * (1.0 + 1e-3) if f != "w" else x
            if f == "w":
                y = x.copy()
                y[:, 1:-1] += 1e-4
            src = torch.empty(y.shape, dtype=torch.float64, pin_memory=True).numpy()
            src[...] = y
            C.icon_state_set_field(st, grid, N, f, src)
            back = C.icon_state_copy_field(st, grid, N, f)
            expect = y.astype(np.float32).astype(np.float64) if (precision == 1 and f == "vn") else y
            assert np.array_equal(back, expect), f
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)
