"""Long runs on the GPU: the benchmark's jet state stays finite, bounded and mass-conserving
over many simulated hours, in both precisions, on flat and on terrain-following levels.

R2B4/90 at dt 360 s has the horizontal sound Courant number of the R2B6/90 benchmark at dt 90 s
(the grid spacing halves with each bisection); 200 steps are 20 simulated hours. The R2B6/90
run covers one simulated day of the benchmark configuration itself, which is what a figure
in simulated days per day rests on.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(C, bis, nlev, dt, nsteps, precision, check_every, topo_m=0.0):
    grid = C.icon_grid_build(2, bis, nlev)
    st = C.icon_state_init_ex(grid, 2, C.ICON_CASE_JET, noise_K=0.1, precision=precision, topo_height_m=topo_m,
                              topo_radius_m=800e3 if topo_m > 0 else 0.0)
    try:
        m0 = C.icon_global_mass(st)
        w_max = vn_max = 0.0
        for n in range(1, nsteps + 1):
            C.icon_dycore_step_async(st, dt, 5)
            if n % check_every == 0 or n == nsteps:
                C.icon_state_status(st)                    # raises ICON_ENONFINITE
                w = C.icon_state_copy_field(st, grid, nlev, "w")
                vn = C.icon_state_copy_field(st, grid, nlev, "vn")
                w_max = max(w_max, float(np.abs(w).max()))
                vn_max = max(vn_max, float(np.abs(vn).max()))
        m1 = C.icon_global_mass(st)
        return abs(m1 - m0) / m0, w_max, vn_max
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)


@pytest.mark.parametrize("precision", [0, 1])
def test_twenty_hours_at_the_benchmark_courant_number(gpu, precision):
    drift, w_max, vn_max = _run(gpu, 4, 90, 360.0, 200, precision, 25)
    assert drift <= 200 * 1e-13, drift
    assert w_max < 1.0 and vn_max < 60.0, (w_max, vn_max)


@pytest.mark.parametrize("precision", [0, 1])
def test_one_simulated_day_of_the_benchmark_configuration(gpu, precision):
    drift, w_max, vn_max = _run(gpu, 6, 90, 90.0, 960, precision, 120)
    assert drift <= 960 * 1e-13, drift
    assert w_max < 1.0 and vn_max < 60.0, (w_max, vn_max)


@pytest.mark.parametrize("precision", [0, 1])
def test_twenty_hours_over_the_mountain(gpu, precision):
    """The same twenty hours on terrain-following levels over the benchmark's 1500 m mountain
    (radius 800 km): both precisions, the mixed one with the lean column on these levels."""
    drift, w_max, vn_max = _run(gpu, 4, 90, 360.0, 200, precision, 25, topo_m=1500.0)
    assert drift <= 200 * 1e-13, drift
    assert w_max < 1.0 and vn_max < 60.0, (w_max, vn_max)
