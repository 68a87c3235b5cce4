"""The recorded mixed step's second graph branch (each stage's edge diagnostics and cell
kinetic energy beside the previous stage's column, recorded on flat levels of grids of
327,680 cells and more) changes no result: steps from the graph with the branch, from the
graph without it (ICON_STEP_OVERLAP=0 when the graph is recorded) and eagerly with one
stream (the profiled step) agree bit for bit on R2B6, with and without divergence damping and
with a ragged level count; over terrain and on coarser grids no branch is recorded."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

PROG = ("vn", "w", "rho", "theta_v", "exner", "mflx", "wflx")


def run(C, grid, nlev, mode, damp, topo=0.0, dt=300.0):
    st = C.icon_state_init_ex(grid, 5, C.ICON_CASE_JET, noise_K=0.1, precision=C.ICON_MIXED,
                              topo_height_m=topo, topo_radius_m=1.5e6 if topo > 0 else 0.0)
    try:
        if not damp:
            C.icon_state_set_option(st, C.ICON_OPT_DIVDAMP4, 0.0)
        kernels = C.icon_state_step_kernels(st, dt, 5)
        for _ in range(2):
            if mode == "eager":
                C.icon_dycore_step_profile(st, dt, 5)
            else:
                C.icon_dycore_step(st, dt, 5)
        return {f: C.icon_state_copy_field(st, grid, nlev, f) for f in PROG}, kernels
    finally:
        C.icon_state_free(st)


@pytest.mark.parametrize("nlev,damp", [(30, True), (47, True), (30, False)])
def test_branch_changes_no_result(gpu, monkeypatch, nlev, damp):
    C = gpu
    grid = C.icon_grid_build(2, 6, nlev)            # R2B6: 327,680 cells
    try:
        monkeypatch.delenv("ICON_STEP_OVERLAP", raising=False)
        a, ka = run(C, grid, nlev, "graph", damp, dt=90.0)
        monkeypatch.setenv("ICON_STEP_OVERLAP", "0")
        b, kb = run(C, grid, nlev, "graph", damp, dt=90.0)
        monkeypatch.delenv("ICON_STEP_OVERLAP")
        c, _ = run(C, grid, nlev, "eager", damp, dt=90.0)
    finally:
        C.icon_grid_free(grid)
    assert ka == kb
    for f in PROG:
        assert np.array_equal(a[f], b[f]), f
        assert np.array_equal(a[f], c[f]), f


def test_terrain_records_one_branch(gpu, monkeypatch):
    C = gpu
    grid = C.icon_grid_build(2, 2, 30)
    try:
        monkeypatch.delenv("ICON_STEP_OVERLAP", raising=False)
        a, _ = run(C, grid, 30, "graph", True, topo=1500.0)
        c, _ = run(C, grid, 30, "eager", True, topo=1500.0)
    finally:
        C.icon_grid_free(grid)
    for f in PROG:
        assert np.array_equal(a[f], c[f]), f
