"""Ragged and maximum level counts: one step of the FP64 form and of every mixed column form
against the oracle, element by element, at level counts that end a few levels past a window,
lane-group or transpose-chunk boundary of the kernels (33 = 32 + 1, 47 = 31 + 16) and at the
largest count the library takes (256 levels, on the coarsest grid)."""
import numpy as np
import pytest

from tests.test_gpu_mixed import TOL_WIND, d_min, gpu_run, oracle_run
from tests.test_gpu_step import check_step
from tests.tolerances import thermo_bound_mixed, w_bound_mixed
from tests.conftest import rel_l2

pytestmark = pytest.mark.gpu

# (bisections, levels, case, dt): dt keeps N dtau below the explicit buoyancy limit at 256 levels
CASES = [(1, 33, 2, 300.0), (1, 47, 1, 300.0), (0, 256, 2, 300.0)]
IDS = ["R2B1-33", "R2B1-47", "R2B0-256"]


@pytest.mark.parametrize("bis,nlev,case,dt", CASES, ids=IDS)
def test_fp64_ragged_and_maximum_levels(gpu, bis, nlev, case, dt):
    out, m0, m1 = gpu_run(gpu, bis, nlev, 8, case, dt, 5, 1, gpu.ICON_FP64, 0.05)
    ref = oracle_run(bis, nlev, 8, case, dt, 5, 1, 0.05)
    check_step(out, ref, dt, 5, 1)
    assert abs(m1 - m0) / m0 <= 1e-13


@pytest.mark.parametrize("form", ["lean", "stored", "recompute"])
@pytest.mark.parametrize("bis,nlev,case,dt", CASES, ids=IDS)
def test_mixed_ragged_and_maximum_levels(gpu, monkeypatch, form, bis, nlev, case, dt):
    monkeypatch.setenv("ICON_MIXED_COLUMN", form)
    out, m0, m1 = gpu_run(gpu, bis, nlev, 8, case, dt, 5, 1, gpu.ICON_MIXED, 0.05)
    ref = oracle_run(bis, nlev, 8, case, dt, 5, 1, 0.05)
    assert rel_l2(out["vn"], ref["vn"]) <= TOL_WIND
    assert rel_l2(out["mflx"], ref["mflx"]) <= TOL_WIND
    for f in ("rho", "theta_v", "exner"):
        assert rel_l2(out[f], ref[f]) <= thermo_bound_mixed(dt, 5, 1, d_min(bis)), f
    assert np.sqrt(np.mean((out["w"] - ref["w"]) ** 2)) <= w_bound_mixed(dt, 5, 1)
    assert abs(m1 - m0) / m0 <= 1e-13
