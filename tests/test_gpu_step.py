"""FP64 dycore step on the GPU vs the FP64 oracle, element by element."""
import numpy as np
import pytest

import oracle as O
from tests.conftest import rel_l2
from tests.tolerances import w_bound

pytestmark = pytest.mark.gpu

PROG = ("vn", "w", "rho", "theta_v", "exner")
TOL_STEP = 1e-12          # rel L2 per field after one FP64 step
TOL_INIT = 1e-14
def check_step(go, oo, dt, nsub, nsteps):
    for f in PROG + ("mflx", "wflx"):
        if f in ("w", "wflx"):
            scale = 1.0 if f == "w" else float(np.max(np.abs(oo["rho"])))
            rms = np.sqrt(np.mean((go[f] - oo[f]) ** 2))
            assert rms <= w_bound(dt, nsub, nsteps) * scale, (f, rms)
        else:
            err = rel_l2(go[f], oo[f])
            assert err <= TOL_STEP * max(nsteps, 1), (f, err)


def run_gpu(C, bis, nlev, seed, case, dt, nsub, nsteps, noise=-1.0):
    grid = C.icon_grid_build(2, bis, nlev)
    st = C.icon_state_init_ex(grid, seed, case, noise_K=noise)
    try:
        init = {f: C.icon_state_copy_field(st, grid, nlev, f) for f in PROG}
        m0 = C.icon_global_mass(st)
        for _ in range(nsteps):
            C.icon_dycore_step(st, dt, nsub)
        out = {f: C.icon_state_copy_field(st, grid, nlev, f) for f in PROG + ("mflx", "wflx")}
        m1 = C.icon_global_mass(st)
        m1b = C.icon_global_mass(st)
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)
    return init, out, (m0, m1, m1b)


def run_oracle(bis, nlev, seed, case, dt, nsub, nsteps, noise=None):
    g = O.build_grid(2, bis)
    v = O.vertical_grid(nlev)
    s = O.init_state(g, v, seed, case, noise_K=noise)
    init = dict(s)
    m0 = O.global_mass(g, v, s)
    acc = None
    for _ in range(nsteps):
        s, acc = O.dycore_step(g, v, s, dt, nsub)
    return init, dict(s, **(acc or {})), (m0, O.global_mass(g, v, s))


@pytest.mark.parametrize("case", [0, 1, 2, 3])
def test_initial_state_parity(gpu, case):
    ginit, _, _ = run_gpu(gpu, 2, 20, 11, case, 300.0, 5, 0)
    oinit, _, _ = run_oracle(2, 20, 11, case, 300.0, 5, 0)
    for f in PROG:
        if f in ("vn", "w") and not np.any(oinit[f]):
            assert np.all(ginit[f] == 0.0)
            continue
        assert rel_l2(ginit[f], oinit[f]) <= TOL_INIT, f


def test_one_step_r2b2_sbr(gpu):
    """The R2B2/20-level solid-body-rotation case: one step of 5 substeps, dt = 300 s."""
    _, go, gm = run_gpu(gpu, 2, 20, 1, O.CASE_SBR, 300.0, 5, 1, noise=0.01)
    _, oo, om = run_oracle(2, 20, 1, O.CASE_SBR, 300.0, 5, 1, noise=0.01)
    check_step(go, oo, 300.0, 5, 1)
    assert abs(gm[0] - om[0]) / om[0] < 1e-14 and abs(gm[1] - om[1]) / om[1] < 1e-14
    assert gm[1] == gm[2]                                  # deterministic mass sum
    assert abs(gm[1] - gm[0]) / gm[0] < 1e-13              # mass conserved


@pytest.mark.parametrize("bis,nlev,case,dt,nsteps", [(1, 30, 2, 400.0, 3), (3, 20, 3, 150.0, 1), (0, 2, 1, 600.0, 2)])
def test_steps_various(gpu, bis, nlev, case, dt, nsteps):
    _, go, _ = run_gpu(gpu, bis, nlev, 5, case, dt, 5, nsteps, noise=0.1)
    _, oo, _ = run_oracle(bis, nlev, 5, case, dt, 5, nsteps, noise=0.1)
    check_step(go, oo, dt, 5, nsteps)


def test_rest_stays_at_rest(gpu):
    _, go, gm = run_gpu(gpu, 2, 20, 0, O.CASE_REST, 300.0, 5, 2)
    assert np.all(go["vn"] == 0.0)
    assert np.abs(go["w"]).max() <= 1e-12
    assert gm[0] == gm[1] or abs(gm[1] - gm[0]) / gm[0] < 1e-15


def test_bad_arguments(gpu):
    C = gpu
    grid = C.icon_grid_build(2, 0, 10)
    st = C.icon_state_init(grid, 1, 1)
    try:
        with pytest.raises(C.IconError):
            C.icon_dycore_step(st, -1.0, 5)
        with pytest.raises(C.IconError):
            C.icon_dycore_step(st, 10.0, 0)
        with pytest.raises(C.IconError):
            C.icon_state_init(grid, 1, 9)
        with pytest.raises(C.IconError):
            C._check(C._lib.icon_grid_copy_table(grid, 0, None, 4))       # NULL destination
        with pytest.raises(C.IconError):
            C._check(C._lib.icon_grid_copy_table(grid, 0, C.np.zeros(4).ctypes.data, 4))   # wrong size
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)
