"""Tracer transport on the GPU against the oracle's (T1-T5), and its consistency and
conservation in both precisions."""
import numpy as np
import pytest

import oracle as O
import oracle.tracer as T
from tests.conftest import rel_l2
from tests.tolerances import thermo_bound_mixed

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-12


def q_init(g, v):
    """A smooth tracer: varies with position on the sphere and with height."""
    zf = np.asarray(v.z_f)[None, :]
    return 1.0 + 0.5 * g.x_c[:, 2:3] + 0.3 * g.x_c[:, 0:1] * g.x_c[:, 1:2] + 2e-5 * zf


def test_tables_match_oracle(gpu):
    C = gpu
    g = O.build_grid(2, 3)
    grid = C.icon_grid_build(2, 3, 10)
    try:
        assert np.array_equal(C.icon_grid_copy_table(grid, "c2c"), T.cell_neighbours(g))
        G = C.icon_grid_copy_table(grid, "lsq_c").reshape(g.nc, 3, 3)
        Go = T.cell_lsq_weights(g)
        assert np.max(np.abs(G - Go)) / np.max(np.abs(Go)) < 1e-13
        roff = C.icon_grid_copy_table(grid, "roff").reshape(g.ne, 2, 3)
        ro = (g.x_e[:, None, :] - g.x_c[g.e2c]) * O.R_EARTH
        assert np.max(np.abs(roff - ro)) / np.max(np.abs(ro)) < 1e-14
    finally:
        C.icon_grid_free(grid)


def run_gpu(C, bis, nlev, seed, case, dt, nsub, nsteps, q0s, precision=0, noise=0.1):
    grid = C.icon_grid_build(2, bis, nlev)
    st = C.icon_state_init_ex(grid, seed, case, noise_K=noise, precision=precision)
    try:
        C.icon_state_add_tracers(st, len(q0s))
        assert C.icon_state_tracers(st) == len(q0s)
        for t, q0 in enumerate(q0s):
            C.icon_state_set_tracer(st, grid, nlev, t, q0)
        rho0 = C.icon_state_copy_field(st, grid, nlev, "rho")
        for _ in range(nsteps):
            C.icon_dycore_step(st, dt, nsub)
        qs = [C.icon_state_copy_tracer(st, grid, nlev, t) for t in range(len(q0s))]
        rho1 = C.icon_state_copy_field(st, grid, nlev, "rho")
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)
    return qs, rho0, rho1


@pytest.mark.parametrize("bis,nlev,case,dt,nsteps", [(2, 20, 2, 300.0, 1), (3, 30, 1, 200.0, 2), (1, 12, 3, 400.0, 1)])
def test_transport_vs_oracle(gpu, bis, nlev, case, dt, nsteps):
    g = O.build_grid(2, bis)
    v = O.vertical_grid(nlev)
    q0 = q_init(g, v)
    (qg,), _, _ = run_gpu(gpu, bis, nlev, 4, case, dt, 5, nsteps, [q0])
    s = O.init_state(g, v, 4, case, noise_K=0.1)
    q = q0
    for _ in range(nsteps):
        s1, acc = O.dycore_step(g, v, s, dt, 5)
        q = O.tracer_step(g, v, q, s["rho"], s1["rho"], acc["mflx"], acc["wflx"], dt)
        s = s1
    assert rel_l2(qg, q) <= TOL_STEP * nsteps
    # the change itself is linear in the step-mean fluxes: the horizontal ones agree to
    # 1e-12, the vertical one inherits w's absolute rounding (tolerances.w_bound), which is
    # ~1e-10 relative to its small size (measured: 2e-12 on the change)
    assert rel_l2(qg - q0, q - q0) <= 1e-10


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_uniform_tracer_and_tracer_mass(gpu, precision):
    """Uniform stays uniform (the step-mean fluxes are the ones that moved rho) and the
    tracer mass sum A dz rho q is conserved, in both precisions."""
    C = gpu
    bis, nlev, dt = 3, 30, 200.0
    g = O.build_grid(2, bis)
    v = O.vertical_grid(nlev)
    q0 = q_init(g, v)
    (qu, qs), rho0, rho1 = run_gpu(C, bis, nlev, 2, 2, dt, 5, 2, [np.full((g.nc, nlev), 2.5), q0], precision)
    assert np.max(np.abs(qu / 2.5 - 1.0)) < 1e-12
    m0 = O.tracer_mass(g, v, rho0, q0)
    m1 = O.tracer_mass(g, v, rho1, qs)
    assert abs(m1 / m0 - 1.0) < 1e-13
    assert np.max(np.abs(qs - q0)) > 1e-6


def test_mixed_tracer_vs_fp64(gpu):
    C = gpu
    bis, nlev, dt = 4, 40, 240.0
    g = O.build_grid(2, bis)
    v = O.vertical_grid(nlev)
    q0 = q_init(g, v)
    (qa,), _, _ = run_gpu(C, bis, nlev, 3, 2, dt, 5, 2, [q0], 0)
    (qb,), _, _ = run_gpu(C, bis, nlev, 3, 2, dt, 5, 2, [q0], 1)
    assert rel_l2(qb, qa) <= thermo_bound_mixed(dt, 5, 2, float(g.d_e.min()))


def test_tracer_api_errors(gpu):
    C = gpu
    grid = C.icon_grid_build(2, 1, 10)
    st = C.icon_state_init(grid, 1, 1)
    try:
        with pytest.raises(C.IconError):
            C.icon_state_add_tracers(st, 0)
        with pytest.raises(C.IconError):
            C.icon_state_add_tracers(st, 9)
        C.icon_state_add_tracers(st, 2)
        with pytest.raises(C.IconError):
            C.icon_state_add_tracers(st, 1)
        with pytest.raises(C.IconError):
            C.icon_state_copy_tracer(st, grid, 10, 2)
        assert np.all(C.icon_state_copy_tracer(st, grid, 10, 1) == 0.0)
        m = C.icon_state_init_ex(grid, 1, 1, precision=1)
        try:
            C.icon_state_add_tracers(m, 1)
            with pytest.raises(C.IconError):
                C.icon_ensemble_create([m])
        finally:
            C.icon_state_free(m)
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)
