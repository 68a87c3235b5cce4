"""Mixed-precision step (FP32 stencils, FP64 column solve and prognostic updates)
against the FP64 oracle and against the FP64 GPU step."""
import numpy as np
import pytest

import oracle as O
from tests.conftest import rel_l2
from tests.tolerances import thermo_bound_mixed, w_bound_mixed

pytestmark = pytest.mark.gpu

PROG = ("vn", "w", "rho", "theta_v", "exner")
TOL_WIND = 1e-5          # rel L2 of the horizontal wind after one step (FP32 stencils)


def d_min(bis):
    """Shortest dual edge of the grid (m), from the oracle's grid builder."""
    return float(O.build_grid(2, bis).d_e.min())


def gpu_run(C, bis, nlev, seed, case, dt, nsub, nsteps, precision, noise=-1.0):
    grid = C.icon_grid_build(2, bis, nlev)
    st = C.icon_state_init_ex(grid, seed, case, noise_K=noise, precision=precision)
    try:
        assert C.icon_state_precision(st) == precision
        m0 = C.icon_global_mass(st)
        for _ in range(nsteps):
            C.icon_dycore_step(st, dt, nsub)
        out = {f: C.icon_state_copy_field(st, grid, nlev, f) for f in PROG + ("mflx", "wflx")}
        m1 = C.icon_global_mass(st)
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)
    return out, m0, m1


def oracle_run(bis, nlev, seed, case, dt, nsub, nsteps, noise=None):
    g = O.build_grid(2, bis)
    v = O.vertical_grid(nlev)
    s = O.init_state(g, v, seed, case, noise_K=noise)
    for _ in range(nsteps):
        s, acc = O.dycore_step(g, v, s, dt, nsub)
        s = dict(s, **acc)
    return s


def test_mixed_initial_state(gpu):
    C = gpu
    grid = C.icon_grid_build(2, 2, 20)
    a = C.icon_state_init_ex(grid, 4, C.ICON_CASE_JET, noise_K=0.1, precision=C.ICON_FP64)
    b = C.icon_state_init_ex(grid, 4, C.ICON_CASE_JET, noise_K=0.1, precision=C.ICON_MIXED)
    try:
        for f in PROG:
            x = C.icon_state_copy_field(a, grid, 20, f)
            y = C.icon_state_copy_field(b, grid, 20, f)
            if f == "vn":
                assert np.array_equal(y, x.astype(np.float32).astype(np.float64))
            else:
                assert np.array_equal(x, y), f
        assert C.icon_global_mass(a) == C.icon_global_mass(b) or \
            abs(C.icon_global_mass(a) / C.icon_global_mass(b) - 1) < 1e-15
    finally:
        C.icon_state_free(a)
        C.icon_state_free(b)
        C.icon_grid_free(grid)


FORMS = ["lean", "stored", "recompute"]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("bis,nlev,case,dt,noise", [(2, 20, 1, 300.0, 0.01), (3, 30, 2, 150.0, 0.1),
                                                    (1, 60, 3, 400.0, 0.0)])
def test_mixed_one_step_vs_oracle(gpu, monkeypatch, bis, nlev, case, dt, noise, form):
    """Every form of the mixed column (lean: FP32 rows and factors with an FP64 base and FP64
    substitution, the default; stored: the frozen FP64 parts kept by the predictor for the
    corrector; recompute: both stages compute them) against the FP64 oracle."""
    monkeypatch.setenv("ICON_MIXED_COLUMN", form)
    out, m0, m1 = gpu_run(gpu, bis, nlev, 6, case, dt, 5, 1, gpu.ICON_MIXED, noise)
    ref = oracle_run(bis, nlev, 6, case, dt, 5, 1, noise)
    assert rel_l2(out["vn"], ref["vn"]) <= TOL_WIND
    assert rel_l2(out["mflx"], ref["mflx"]) <= TOL_WIND
    for f in ("rho", "theta_v", "exner"):
        assert rel_l2(out[f], ref[f]) <= thermo_bound_mixed(dt, 5, 1, d_min(bis)), f
    rms = np.sqrt(np.mean((out["w"] - ref["w"]) ** 2))
    assert rms <= w_bound_mixed(dt, 5, 1), rms
    assert abs(m1 - m0) / m0 <= 1e-13                          # FP64 flux sums conserve mass


@pytest.mark.parametrize("form", FORMS)
def test_mixed_rest_stays_at_rest(gpu, monkeypatch, form):
    monkeypatch.setenv("ICON_MIXED_COLUMN", form)
    out, m0, m1 = gpu_run(gpu, 2, 20, 0, 0, 300.0, 5, 2, gpu.ICON_MIXED)
    assert np.all(out["vn"] == 0.0)
    assert np.abs(out["w"]).max() <= 1e-6
    assert abs(m1 - m0) / m0 <= 1e-14


def test_mixed_vs_fp64_gpu_larger(gpu):
    """R2B5 with 60 levels, jet with noise, 2 steps: mixed against the FP64 GPU step."""
    a, am0, am1 = gpu_run(gpu, 5, 60, 2, 2, 180.0, 5, 2, gpu.ICON_FP64, 0.1)
    b, bm0, bm1 = gpu_run(gpu, 5, 60, 2, 2, 180.0, 5, 2, gpu.ICON_MIXED, 0.1)
    assert rel_l2(b["vn"], a["vn"]) <= 2 * TOL_WIND
    for f in ("rho", "theta_v", "exner"):
        assert rel_l2(b[f], a[f]) <= thermo_bound_mixed(180.0, 5, 2, d_min(5)), f
    assert abs(bm1 - bm0) / bm0 <= 2e-13
    assert am0 == bm0 or abs(am0 / bm0 - 1) < 1e-15


def test_integer_pipe_conversions_match_hardware(gpu):
    """The FP32<->FP64 conversions built from the IEEE-754 encodings agree bit for bit
    with the hardware conversions on 2^22 random finite inputs and halfway cases."""
    assert gpu.icon_selftest(1 << 22) == 0


@pytest.mark.parametrize("form", ["lean", "recompute"])
def test_mixed_column_forms_agree(gpu, monkeypatch, form):
    """R2B4 / 60 levels, 2 steps: the lean and the recomputing column against the
    stored-factor one (different operation order and precision of the coefficients)."""
    monkeypatch.setenv("ICON_MIXED_COLUMN", "stored")
    a, am0, am1 = gpu_run(gpu, 4, 60, 3, 2, 240.0, 5, 2, gpu.ICON_MIXED, 0.1)
    monkeypatch.setenv("ICON_MIXED_COLUMN", form)
    b, bm0, bm1 = gpu_run(gpu, 4, 60, 3, 2, 240.0, 5, 2, gpu.ICON_MIXED, 0.1)
    assert rel_l2(b["vn"], a["vn"]) <= TOL_WIND
    for f in ("rho", "theta_v", "exner"):
        assert rel_l2(b[f], a[f]) <= thermo_bound_mixed(240.0, 5, 2, d_min(4)), f
    assert np.sqrt(np.mean((b["w"] - a["w"]) ** 2)) <= w_bound_mixed(240.0, 5, 2)
    assert abs(am1 / am0 - 1) <= 1e-13 and abs(bm1 / bm0 - 1) <= 1e-13
