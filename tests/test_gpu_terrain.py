"""The step on terrain-following levels over a Gaussian mountain against the oracle's
(oracle.terrain), through the C ABI: initial state, one and two steps, with and without
the step options, mass, tracers, the mixed-precision form, and the argument checks of
the topography."""
import numpy as np
import pytest

import oracle as O
import oracle.terrain as T
from tests.conftest import rel_l2
from tests.tolerances import w_bound, thermo_bound_mixed, w_bound_mixed
from tests.test_gpu_mixed import d_min, TOL_WIND

pytestmark = pytest.mark.gpu

PROG = ("vn", "w", "rho", "theta_v", "exner")
H0, RADIUS = 1500.0, 800e3


def run_gpu(C, bis, nlev, seed, case, dt, nsub, nsteps, c4=0.0, d4=0.0, ut=False, h0=H0, radius=RADIUS,
            precision=0):
    grid = C.icon_grid_build(2, bis, nlev)
    st = C.icon_state_init_ex(grid, seed, case, noise_K=0.1, topo_height_m=h0, topo_radius_m=radius,
                              precision=precision)
    try:
        init = {f: C.icon_state_copy_field(st, grid, nlev, f) for f in PROG}
        C.icon_state_set_option(st, C.ICON_OPT_DIVDAMP4, c4)
        C.icon_state_set_option(st, C.ICON_OPT_DIFF4, d4)
        C.icon_state_set_option(st, C.ICON_OPT_UPWIND_THETA, 1.0 if ut else 0.0)
        m0 = C.icon_global_mass(st)
        for _ in range(nsteps):
            C.icon_dycore_step(st, dt, nsub)
        out = {f: C.icon_state_copy_field(st, grid, nlev, f) for f in PROG + ("mflx", "wflx")}
        m1 = C.icon_global_mass(st)
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)
    return init, out, m0, m1


def run_oracle(bis, nlev, seed, case, dt, nsub, nsteps, c4=0.0, d4=0.0, ut=False):
    g = O.build_grid(2, bis)
    v = O.vertical_grid(nlev)
    t = T.terrain_geometry(g, v, T.mountain(g.x_c, H0, RADIUS))
    s0 = O.init_state(g, v, seed, case, noise_K=0.1, terrain=t)
    s = s0
    for _ in range(nsteps):
        s, acc = T.terrain_step(g, v, t, s, dt, nsub, divdamp4=c4, diff4=d4, upwind_theta=ut)
    return s0, dict(s, **acc), T.terrain_mass(g, t, s0), T.terrain_mass(g, t, s)


CASES = [(2, 20, 2, 300.0, 1), (3, 30, 3, 200.0, 2), (1, 2, 2, 300.0, 1), (1, 3, 3, 300.0, 1)]


@pytest.mark.parametrize("bis,nlev,case,dt,nsteps", CASES)
def test_terrain_step_vs_oracle(gpu, bis, nlev, case, dt, nsteps):
    gi, go, m0, m1 = run_gpu(gpu, bis, nlev, 8, case, dt, 5, nsteps)
    oi, oo, om0, om1 = run_oracle(bis, nlev, 8, case, dt, 5, nsteps)
    for f in ("vn", "rho", "theta_v", "exner"):
        assert rel_l2(gi[f], oi[f]) <= 1e-14, f                     # heights, hydrostatic integration
    assert np.all(gi["w"] == 0.0)
    for f in ("vn", "rho", "theta_v", "exner", "mflx"):
        assert rel_l2(go[f], oo[f]) <= 1e-12 * nsteps, f
    assert np.sqrt(np.mean((go["w"] - oo["w"]) ** 2)) <= w_bound(dt, 5, nsteps)
    assert np.sqrt(np.mean((go["wflx"] - oo["wflx"]) ** 2)) <= 1.5 * w_bound(dt, 5, nsteps)
    # the ground w is the terrain-following one, nonzero over the mountain
    assert np.max(np.abs(go["w"][:, -1])) > 1e-4
    assert abs(m0 / om0 - 1.0) <= 1e-14
    assert abs(m1 / m0 - 1.0) <= 1e-13 and abs(om1 / om0 - 1.0) <= 1e-13


def test_terrain_with_options_vs_oracle(gpu):
    c4, d4 = 0.004, 0.005
    _, go, m0, m1 = run_gpu(gpu, 2, 20, 8, 2, 300.0, 5, 1, c4=c4, d4=d4, ut=True)
    _, oo, _, _ = run_oracle(2, 20, 8, 2, 300.0, 5, 1, c4=c4, d4=d4, ut=True)
    for f in ("vn", "rho", "theta_v", "exner", "mflx"):
        assert rel_l2(go[f], oo[f]) <= 1e-12, f
    assert np.sqrt(np.mean((go["w"] - oo["w"]) ** 2)) <= w_bound(300.0, 5, 1)
    assert abs(m1 / m0 - 1.0) <= 1e-13


def test_mountain_changes_the_flow(gpu):
    """The same jet over flat ground and over the mountain differ after one step, most
    near the mountain (90E 30N)."""
    _, go, _, _ = run_gpu(gpu, 3, 20, 8, 2, 300.0, 5, 1)
    _, gf, _, _ = run_gpu(gpu, 3, 20, 8, 2, 300.0, 5, 1, h0=0.0, radius=0.0)
    d = np.max(np.abs(go["vn"] - gf["vn"]), axis=1)
    g = O.build_grid(2, 3)
    hs_e = T.mountain(g.x_e, H0, RADIUS)
    assert d.max() > 1e-2
    assert d[hs_e > 0.5 * H0].mean() > 20.0 * d[hs_e < 1e-3 * H0].mean()


def test_topography_arguments(gpu):
    C = gpu
    grid = C.icon_grid_build(2, 1, 10)
    try:
        for h0, a, prec in [(-100.0, RADIUS, 0), (3000.0, RADIUS, 0), (1000.0, 10.0, 0), (1000.0, 10.0, 1)]:
            with pytest.raises(C.IconError) as ei:
                C.icon_state_init_ex(grid, 1, 2, topo_height_m=h0, topo_radius_m=a, precision=prec)
            assert ei.value.status == C.ICON_EINVAL
        # the persistent ensemble runs on flat levels only
        m = C.icon_state_init_ex(grid, 1, 3, precision=1, topo_height_m=1000.0, topo_radius_m=RADIUS)
        try:
            with pytest.raises(C.IconError) as ei:
                C.icon_ensemble_create([m])
            assert ei.value.status == C.ICON_EINVAL
        finally:
            C.icon_state_free(m)
    finally:
        C.icon_grid_free(grid)


def test_tracer_over_terrain_vs_oracle(gpu):
    """Two tracers (uniform and a smooth field) on the terrain-following levels through
    two steps: the uniform one stays uniform, the other matches the oracle's transport
    with the oracle's terrain fluxes, and tracer mass is conserved."""
    C = gpu
    bis, nlev, dt = 2, 20, 300.0
    g = O.build_grid(2, bis)
    v = O.vertical_grid(nlev)
    t = T.terrain_geometry(g, v, T.mountain(g.x_c, H0, RADIUS))
    q0 = 1.0 + 0.5 * g.x_c[:, 2:3] + 0.01 * np.arange(nlev)[None, :]
    grid = C.icon_grid_build(2, bis, nlev)
    st = C.icon_state_init_ex(grid, 8, 2, noise_K=0.1, topo_height_m=H0, topo_radius_m=RADIUS)
    try:
        C.icon_state_add_tracers(st, 2)
        C.icon_state_set_tracer(st, grid, nlev, 0, np.full((g.nc, nlev), 3.7))
        C.icon_state_set_tracer(st, grid, nlev, 1, q0)
        for _ in range(2):
            C.icon_dycore_step(st, dt, 5)
        gq = [C.icon_state_copy_tracer(st, grid, nlev, i) for i in range(2)]
        grho = C.icon_state_copy_field(st, grid, nlev, "rho")
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)
    s = O.init_state(g, v, 8, 2, noise_K=0.1, terrain=t)
    m0 = O.tracer_mass(g, v, s["rho"], q0, terrain=t)
    q = q0
    for _ in range(2):
        s1, acc = T.terrain_step(g, v, t, s, dt, 5)
        q = O.tracer_step(g, v, q, s["rho"], s1["rho"], acc["mflx"], acc["wflx"], dt, terrain=t)
        s = s1
    assert np.max(np.abs(gq[0] / 3.7 - 1.0)) < 1e-13
    assert np.max(np.abs(gq[1] - q)) < 1e-12
    assert np.max(np.abs(gq[1] - q0)) > 1e-5                         # it moved (7e-5)
    assert abs(O.tracer_mass(g, v, grho, gq[1], terrain=t) / m0 - 1.0) < 1e-13


# ------------------------------------------------------------------ mixed precision
@pytest.mark.parametrize("form", ["lean", "recompute"])
@pytest.mark.parametrize("bis,nlev,case,dt", [(2, 20, 2, 300.0), (3, 30, 3, 200.0)])
def test_mixed_terrain_one_step_vs_oracle(gpu, monkeypatch, bis, nlev, case, dt, form):
    """The mixed form on terrain-following levels (FP32 stencils and metric terms; the lean
    column with each cell's spacings and the contravariant vertical velocity, the default,
    or the recomputing FP64 column) against the FP64 oracle, with the mixed form's
    tolerances."""
    monkeypatch.setenv("ICON_MIXED_COLUMN", form)
    gi, go, m0, m1 = run_gpu(gpu, bis, nlev, 8, case, dt, 5, 1, precision=1)
    oi, oo, _, _ = run_oracle(bis, nlev, 8, case, dt, 5, 1)
    for f in ("rho", "theta_v", "exner"):
        assert np.array_equal(gi[f], oi[f]) or rel_l2(gi[f], oi[f]) <= 1e-14, f
    assert rel_l2(go["vn"], oo["vn"]) <= TOL_WIND
    assert rel_l2(go["mflx"], oo["mflx"]) <= TOL_WIND
    for f in ("rho", "theta_v", "exner"):
        assert rel_l2(go[f], oo[f]) <= thermo_bound_mixed(dt, 5, 1, d_min(bis)), f
    assert np.sqrt(np.mean((go["w"] - oo["w"]) ** 2)) <= w_bound_mixed(dt, 5, 1)
    assert abs(m1 - m0) / m0 <= 1e-13


def test_mixed_terrain_vs_fp64_gpu_larger(gpu):
    """R2B4 with 60 levels over the mountain, 2 steps: mixed against the FP64 GPU step."""
    _, a, am0, _ = run_gpu(gpu, 4, 60, 2, 2, 240.0, 5, 2)
    _, b, bm0, bm1 = run_gpu(gpu, 4, 60, 2, 2, 240.0, 5, 2, precision=1)
    assert rel_l2(b["vn"], a["vn"]) <= 2 * TOL_WIND
    for f in ("rho", "theta_v", "exner"):
        assert rel_l2(b[f], a[f]) <= thermo_bound_mixed(240.0, 5, 2, d_min(4)), f
    assert abs(bm1 - bm0) / bm0 <= 2e-13
    assert abs(am0 / bm0 - 1) < 1e-15


def test_mixed_terrain_tracer_stays_uniform(gpu):
    C = gpu
    grid = C.icon_grid_build(2, 2, 20)
    st = C.icon_state_init_ex(grid, 8, 2, noise_K=0.1, precision=1, topo_height_m=H0, topo_radius_m=RADIUS)
    try:
        C.icon_state_add_tracers(st, 1)
        C.icon_state_set_tracer(st, grid, 20, 0, np.full((1280, 20), 3.7))
        for _ in range(2):
            C.icon_dycore_step(st, 300.0, 5)
        q = C.icon_state_copy_tracer(st, grid, 20, 0)
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)
    assert np.max(np.abs(q / 3.7 - 1.0)) < 1e-13
