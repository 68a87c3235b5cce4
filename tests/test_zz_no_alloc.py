"""The allocation-free mass entry point against the ordinary one.

icon_global_mass_noalloc serves callers that cannot allocate device memory when
they need the integral (a component whose device memory belongs to a host model's
pool allocator, or a loop that forbids allocations after start-up). It reduces a
caller-owned density array with partial sums kept in one fixed array inside the
library. Here it must agree with icon_global_mass on the same density, on two
calls in a row, for a second density after a step (nothing stale is carried
over), for a padded row layout, on terrain-following levels when given the
columns' own layer thicknesses (and with the oracle's mass there), and refuse
what it cannot hold or read.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-14          # relative; the mass comparisons of the parity tests use the same bound


def _rel(a, b):
    return abs(a - b) / abs(b)


def test_noalloc_mass_matches_ordinary_mass(gpu):
    import torch
    C = gpu
    N = 30
    grid = C.icon_grid_build(2, 4, N)
    st = C.icon_state_init_ex(grid, 3, C.ICON_CASE_JET, noise_K=0.1)
    try:
        m_ref = C.icon_global_mass(st)
        rho = torch.from_numpy(C.icon_state_copy_field(st, grid, N, "rho")).cuda()
        torch.cuda.synchronize()
        m1 = C.icon_global_mass_noalloc(grid, rho.data_ptr(), N)
        m2 = C.icon_global_mass_noalloc(grid, rho.data_ptr(), N)
        assert _rel(m1, m_ref) <= TOL and _rel(m2, m_ref) <= TOL
        assert m1 == m2                                   # deterministic

        # a different density after one step: the shared scratch keeps nothing that matters
        C.icon_dycore_step(st, 360.0, 5)
        m_ref2 = C.icon_global_mass(st)
        rho2 = torch.from_numpy(C.icon_state_copy_field(st, grid, N, "rho")).cuda()
        torch.cuda.synchronize()
        assert _rel(C.icon_global_mass_noalloc(grid, rho2.data_ptr(), N), m_ref2) <= TOL

        # padded rows: only levels 0..N-1 of each row of stride ld are read
        ld = N + 6
        padded = torch.full((rho2.shape[0], ld), 1e30, dtype=torch.float64, device="cuda")
        padded[:, :N] = rho2
        torch.cuda.synchronize()
        assert _rel(C.icon_global_mass_noalloc(grid, padded.data_ptr(), ld), m_ref2) <= TOL

        # refusals: stride below the level count, NULL density
        with pytest.raises(C.IconError) as ei:
            C.icon_global_mass_noalloc(grid, rho2.data_ptr(), N - 1)
        assert ei.value.status == C.ICON_EINVAL
        with pytest.raises(C.IconError):
            C.icon_global_mass_noalloc(grid, 0, N)
        # host memory is not device memory of the current device: refused before any launch
        host = np.ones((rho2.shape[0], N))
        with pytest.raises(C.IconError) as ei:
            C.icon_global_mass_noalloc(grid, host.ctypes.data, N)
        assert ei.value.status == C.ICON_EINVAL and "not device memory" in str(ei.value)
        with pytest.raises(C.IconError) as ei:
            C.icon_global_mass_noalloc(grid, rho2.data_ptr(), N, dev_dz_ptr=host.ctypes.data)
        assert ei.value.status == C.ICON_EINVAL and "dev_dz" in str(ei.value)
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)


def test_noalloc_mass_refuses_grids_beyond_its_scratch(gpu):
    import torch
    C = gpu
    grid = C.icon_grid_build(2, 9, 2)          # R2B9: 20,971,520 cells > 16,777,216
    try:
        dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
        with pytest.raises(C.IconError) as ei:
            C.icon_global_mass_noalloc(grid, dummy.data_ptr(), 2)
        assert ei.value.status == C.ICON_EINVAL and "exceed the maximum" in str(ei.value)
    finally:
        C.icon_grid_free(grid)


def test_noalloc_mass_on_terrain_following_levels(gpu):
    """With the columns' own layer thicknesses the allocation-free integral is the terrain
    state's mass (icon_global_mass and the oracle's); with the flat thicknesses it is not."""
    import torch
    import oracle as O
    import oracle.terrain as OT
    C = gpu
    N, bis, h0, a = 20, 3, 1500.0, 1.5e6
    grid = C.icon_grid_build(2, bis, N)
    st = C.icon_state_init_ex(grid, 5, C.ICON_CASE_JET, noise_K=0.1, topo_height_m=h0, topo_radius_m=a)
    try:
        g = O.build_grid(2, bis)
        v = O.vertical_grid(N)
        t = OT.terrain_geometry(g, v, OT.mountain(g.x_c, h0, a))
        m_oracle = OT.terrain_mass(g, t, O.init_state(g, v, 5, O.CASE_JET, noise_K=0.1, terrain=t))
        m_ref = C.icon_global_mass(st)
        ld = N + 4
        rho = torch.zeros((g.nc, ld), dtype=torch.float64, device="cuda")
        rho[:, :N] = torch.from_numpy(C.icon_state_copy_field(st, grid, N, "rho"))
        dz = torch.zeros((g.nc, ld), dtype=torch.float64, device="cuda")
        dz[:, :N] = torch.from_numpy(t.dz_c)
        torch.cuda.synchronize()
        m1 = C.icon_global_mass_noalloc(grid, rho.data_ptr(), ld, dev_dz_ptr=dz.data_ptr())
        m2 = C.icon_global_mass_noalloc(grid, rho.data_ptr(), ld, dev_dz_ptr=dz.data_ptr())
        assert m1 == m2
        assert _rel(m1, m_ref) <= TOL and _rel(m1, m_oracle) <= 1e-13
        m_flat = C.icon_global_mass_noalloc(grid, rho.data_ptr(), ld)
        assert _rel(m_flat, m_ref) > 1e-6               # the flat thicknesses give another integral
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)
