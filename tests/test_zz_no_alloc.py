"""The allocation-free mass entry point against the ordinary one.

icon_global_mass_noalloc serves callers that cannot allocate device memory when
they need the integral (a component whose device memory belongs to a host model's
pool allocator, or a loop that forbids allocations after start-up). It reduces a
caller-owned density array with partial sums kept in one fixed array inside the
library. Here it must agree with icon_global_mass on the same density, on two
calls in a row, for a second density after a step (nothing stale is carried
over), for a padded row layout, and refuse what it cannot hold.
"""
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
