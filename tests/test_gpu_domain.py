"""The decomposed FP64 step (parts with halo exchanges) against the single-domain step and
the oracle: owned rows bit-identical to the single-domain step for 2 and 4 parts, the mass
of the parts' sums equal to the single-domain mass, and one step within the FP64 parity
bounds of the oracle."""
import numpy as np
import pytest

import oracle as O
from tests.conftest import rel_l2
from tests.tolerances import w_bound

pytestmark = pytest.mark.gpu

FIELDS = ("vn", "w", "rho", "theta_v", "exner", "mflx", "wflx")


@pytest.mark.parametrize("nparts,rings", [(2, 3), (4, 3), (3, 4)])
def test_decomposed_step_is_bit_identical(gpu, nparts, rings):
    C = gpu
    N, dt = 30, 240.0
    grid = C.icon_grid_build(2, 3, N)
    ref = C.icon_state_init_ex(grid, 5, C.ICON_CASE_JET, noise_K=0.1)
    src = C.icon_state_init_ex(grid, 5, C.ICON_CASE_JET, noise_K=0.1)
    dom = None
    try:
        dom = C.icon_domain_create(src, nparts, rings)
        m0 = C.icon_global_mass(ref)
        assert abs(C.icon_domain_global_mass(dom) / m0 - 1.0) <= 1e-14
        for _ in range(2):
            C.icon_dycore_step(ref, dt, 5)
            C.icon_domain_step(dom, dt, 5)
        for f in FIELDS:
            a = C.icon_state_copy_field(ref, grid, N, f)
            b = C.icon_domain_copy_field(dom, grid, N, f)
            assert np.array_equal(a, b), (f, np.abs(a - b).max())
        assert abs(C.icon_domain_global_mass(dom) / C.icon_global_mass(ref) - 1.0) <= 1e-14
        own = sum(int(C.icon_domain_part_counts(dom, p)[0]) for p in range(nparts))
        assert own == 20 * 4 ** 4
    finally:
        if dom is not None:
            C.icon_domain_free(dom)
        C.icon_state_free(ref)
        C.icon_state_free(src)
        C.icon_grid_free(grid)


def test_decomposed_step_vs_oracle(gpu):
    C = gpu
    N, dt, bis = 20, 300.0, 2
    grid = C.icon_grid_build(2, bis, N)
    st = C.icon_state_init_ex(grid, 7, C.ICON_CASE_SBR, noise_K=0.01)
    dom = None
    try:
        dom = C.icon_domain_create(st, 2, 3)
        C.icon_domain_step(dom, dt, 5)
        g = O.build_grid(2, bis)
        v = O.vertical_grid(N)
        s, acc = O.dycore_step(g, v, O.init_state(g, v, 7, O.CASE_SBR, noise_K=0.01), dt, 5)
        s = dict(s, **acc)
        for f in FIELDS:
            got = C.icon_domain_copy_field(dom, grid, N, f)
            if f in ("w", "wflx"):
                scale = 1.0 if f == "w" else float(np.abs(s["rho"]).max())
                assert np.sqrt(np.mean((got - s[f]) ** 2)) <= w_bound(dt, 5, 1) * scale, f
            else:
                assert rel_l2(got, s[f]) <= 1e-12, f
    finally:
        if dom is not None:
            C.icon_domain_free(dom)
        C.icon_state_free(st)
        C.icon_grid_free(grid)


def test_domain_rejects_what_it_does_not_decompose(gpu):
    C = gpu
    grid = C.icon_grid_build(2, 1, 10)
    mx = C.icon_state_init_ex(grid, 1, C.ICON_CASE_SBR, precision=C.ICON_MIXED)
    fp = C.icon_state_init_ex(grid, 1, C.ICON_CASE_SBR)
    try:
        with pytest.raises(C.IconError) as ei:
            C.icon_domain_create(mx, 2, 3)
        assert ei.value.status == C.ICON_EINVAL
        with pytest.raises(C.IconError) as ei:
            C.icon_domain_create(fp, 2, 2)                       # halo too shallow for a stage
        assert ei.value.status == C.ICON_EINVAL
        C.icon_state_set_option(fp, C.ICON_OPT_DIFF4, 0.005)          # background diffusion: not decomposed
        with pytest.raises(C.IconError) as ei:
            C.icon_domain_create(fp, 2, 3)
        assert ei.value.status == C.ICON_EINVAL
    finally:
        C.icon_state_free(mx)
        C.icon_state_free(fp)
        C.icon_grid_free(grid)
