"""GPU grid builder vs the oracle: integer tables bit-exact, FP64 geometry to 1e-14."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

INT = ["c2v", "c2e", "e2c", "e2v", "v2e", "v2c", "vdeg", "e2vt", "e2q"]
GEOM = ["x_c", "x_e", "x_v", "n_e", "t_e", "l_e", "d_e", "A_c", "A_v", "f_e", "vt_w", "kin_w", "lsq_w",
        "L34", "s_ce", "s_ve"]


@pytest.mark.parametrize("bis", [0, 1, 2, 3, 5])
def test_tables_match_oracle(gpu, bis):
    C = gpu
    grid = C.icon_grid_build(2, bis, 4)
    try:
        g = O.build_grid(2, bis)
        assert C.icon_grid_counts(grid) == (g.nc, g.ne, g.nv)
        for name in INT:
            got = C.icon_grid_copy_table(grid, name)
            want = getattr(g, name)
            assert np.array_equal(got, want.reshape(got.shape)), name
        for name in GEOM:
            got = C.icon_grid_copy_table(grid, name)
            want = getattr(g, name).reshape(got.shape)
            scale = np.max(np.abs(want))
            err = np.max(np.abs(got - want)) / scale
            assert err <= 1e-14, (name, err)
    finally:
        C.icon_grid_free(grid)


def test_large_grid_invariants(gpu):
    """R2B8 (the paper's 10 km grid): counts, Euler, 12 pentagons, areas tile the sphere."""
    C = gpu
    grid = C.icon_grid_build(2, 8, 2)
    try:
        nc, ne, nv = C.icon_grid_counts(grid)
        assert (nc, ne, nv) == (5242880, 7864320, 2621442)
        assert nv - ne + nc == 2
        deg = C.icon_grid_copy_table(grid, "vdeg")
        assert np.sum(deg == 5) == 12 and np.sum(deg == 6) == nv - 12
        R = O.R_EARTH
        for name in ("A_c", "A_v"):
            a = C.icon_grid_copy_table(grid, name)
            assert abs(a.sum() / (4 * np.pi * R * R) - 1) < 1e-12
        e2c = C.icon_grid_copy_table(grid, "e2c")
        assert np.all(e2c[:, 0] < e2c[:, 1]) and e2c.min() >= 0
        # every cell appears exactly three times as an edge neighbour
        assert np.all(np.bincount(e2c.ravel(), minlength=nc) == 3)
    finally:
        C.icon_grid_free(grid)
