"""The step options on the GPU against the oracle's: fourth-order divergence damping
(DD), fourth-order background diffusion (BD) and upwind theta_v in the heat fluxes
(UT), both precisions."""
import numpy as np
import pytest

import oracle as O
from tests.conftest import rel_l2
from tests.test_gpu_mixed import d_min
from tests.tolerances import thermo_bound_mixed, w_bound, w_bound_mixed

pytestmark = pytest.mark.gpu

PROG = ("vn", "w", "rho", "theta_v", "exner")
C4 = 0.004           # divergence damping coefficient
D4 = 0.005           # background diffusion coefficient


def run_gpu(C, bis, nlev, seed, case, dt, nsub, nsteps, precision, c4=C4, d4=0.0, ut=False):
    grid = C.icon_grid_build(2, bis, nlev)
    st = C.icon_state_init_ex(grid, seed, case, noise_K=0.1, precision=precision)
    try:
        C.icon_state_set_option(st, C.ICON_OPT_DIVDAMP4, c4)
        C.icon_state_set_option(st, C.ICON_OPT_DIFF4, d4)
        C.icon_state_set_option(st, C.ICON_OPT_UPWIND_THETA, 1.0 if ut else 0.0)
        m0 = C.icon_global_mass(st)
        for _ in range(nsteps):
            C.icon_dycore_step(st, dt, nsub)
        out = {f: C.icon_state_copy_field(st, grid, nlev, f) for f in PROG + ("mflx",)}
        m1 = C.icon_global_mass(st)
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)
    return out, m0, m1


def run_oracle(bis, nlev, seed, case, dt, nsub, nsteps, c4=C4, d4=0.0, ut=False):
    g = O.build_grid(2, bis)
    v = O.vertical_grid(nlev)
    s = O.init_state(g, v, seed, case, noise_K=0.1)
    for _ in range(nsteps):
        s, acc = O.dycore_step(g, v, s, dt, nsub, divdamp4=c4, diff4=d4, upwind_theta=ut)
    return dict(s, **acc)


OPTS = [(C4, 0.0, False), (0.0, D4, False), (0.0, 0.0, True), (C4, D4, True)]
IDS = ["dd", "bd", "ut", "dd+bd+ut"]


@pytest.mark.parametrize("c4,d4,ut", OPTS, ids=IDS)
@pytest.mark.parametrize("bis,nlev,case,dt,nsteps", [(2, 20, 2, 300.0, 1), (3, 30, 3, 200.0, 2)])
def test_fp64_vs_oracle(gpu, bis, nlev, case, dt, nsteps, c4, d4, ut):
    go, m0, m1 = run_gpu(gpu, bis, nlev, 8, case, dt, 5, nsteps, 0, c4, d4, ut)
    oo = run_oracle(bis, nlev, 8, case, dt, 5, nsteps, c4, d4, ut)
    for f in ("vn", "rho", "theta_v", "exner", "mflx"):
        assert rel_l2(go[f], oo[f]) <= 1e-12 * nsteps, f
    assert np.sqrt(np.mean((go["w"] - oo["w"]) ** 2)) <= w_bound(dt, 5, nsteps)
    assert abs(m1 / m0 - 1.0) <= 1e-13
    # it acts: the oracle without the options differs
    ou = run_oracle(bis, nlev, 8, case, dt, 5, nsteps, c4=0.0, d4=0.0)
    assert rel_l2(ou["vn"], oo["vn"]) > 1e-9 or rel_l2(ou["theta_v"], oo["theta_v"]) > 1e-9


@pytest.mark.parametrize("c4,d4,ut", OPTS, ids=IDS)
def test_mixed_vs_oracle(gpu, c4, d4, ut):
    bis, nlev, case, dt = 3, 30, 2, 150.0
    go, m0, m1 = run_gpu(gpu, bis, nlev, 8, case, dt, 5, 1, 1, c4, d4, ut)
    oo = run_oracle(bis, nlev, 8, case, dt, 5, 1, c4, d4, ut)
    assert rel_l2(go["vn"], oo["vn"]) <= 1e-5
    for f in ("rho", "theta_v", "exner"):
        assert rel_l2(go[f], oo[f]) <= thermo_bound_mixed(dt, 5, 1, d_min(bis)), f
    assert np.sqrt(np.mean((go["w"] - oo["w"]) ** 2)) <= w_bound_mixed(dt, 5, 1)
    assert abs(m1 / m0 - 1.0) <= 1e-13


def test_option_errors_and_ensemble(gpu):
    C = gpu
    grid = C.icon_grid_build(2, 1, 10)
    st = C.icon_state_init_ex(grid, 1, 1, precision=1)
    try:
        with pytest.raises(C.IconError):
            C.icon_state_set_option(st, 99, 0.0)
        with pytest.raises(C.IconError):
            C.icon_state_set_option(st, C.ICON_OPT_DIVDAMP4, -0.1)
        with pytest.raises(C.IconError):
            C.icon_state_set_option(st, C.ICON_OPT_DIVDAMP4, 1.0)
        C.icon_state_set_option(st, C.ICON_OPT_DIVDAMP4, 0.004)
        ens = C.icon_ensemble_create([st])             # the ensemble runs the damping
        C.icon_ensemble_free(ens)
        C.icon_state_set_option(st, C.ICON_OPT_DIVDAMP4, 0.0)
        with pytest.raises(C.IconError):
            C.icon_state_set_option(st, C.ICON_OPT_DIFF4, 0.02)
        C.icon_state_set_option(st, C.ICON_OPT_DIFF4, 0.005)
        with pytest.raises(C.IconError):
            C.icon_ensemble_create([st])
        C.icon_state_set_option(st, C.ICON_OPT_DIFF4, 0.0)
        with pytest.raises(C.IconError):
            C.icon_state_set_option(st, C.ICON_OPT_UPWIND_THETA, 0.5)
        C.icon_state_set_option(st, C.ICON_OPT_UPWIND_THETA, 1.0)
        with pytest.raises(C.IconError):
            C.icon_ensemble_create([st])
        C.icon_state_set_option(st, C.ICON_OPT_UPWIND_THETA, 0.0)
        ens = C.icon_ensemble_create([st])
        C.icon_ensemble_free(ens)
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)
