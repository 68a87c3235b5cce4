"""Batched ensemble (one persistent cooperative launch per step for all members),
autotuned tiles, and the fault paths (barrier timeout, non-finite state, failing
allocator) -- none of which faults, traps or hangs the GPU."""
import ctypes

import numpy as np
import pytest

from tests.conftest import rel_l2
from tests.tolerances import w_bound_mixed

pytestmark = pytest.mark.gpu

# A member advanced inside the persistent ensemble kernel runs the same per-item device
# code as a solo step, but the FP32 stencils are inlined into a different kernel and the
# compiler may fuse a different set of FP32 multiply-adds: the two agree to FP32 rounding.
TOL_MEMBER = 1e-6

PROG = ("vn", "w", "rho", "theta_v", "exner")


def _fields(C, st, grid, N):
    return {f: C.icon_state_copy_field(st, grid, N, f) for f in PROG + ("mflx", "wflx")}


@pytest.mark.parametrize("form", ["lean", "stored"])
def test_ensemble_members_equal_solo_runs(gpu, monkeypatch, form):
    """Members of one persistent launch against the same states stepped alone, for the lean
    column (the default) and the stored-factor column."""
    monkeypatch.setenv("ICON_MIXED_COLUMN", form)
    C = gpu
    N = 60
    grids = [C.icon_grid_build(2, 2, N), C.icon_grid_build(2, 3, N)]
    spec = [(0, 0, 300.0), (0, 1, 300.0), (1, 2, 150.0), (1, 3, 150.0)]     # (grid, member, dt)
    ens_states = [C.icon_state_init_ex(grids[g], 3, C.ICON_CASE_MEMBER, precision=C.ICON_MIXED, member=m)
                  for g, m, _ in spec]
    solo_states = [C.icon_state_init_ex(grids[g], 3, C.ICON_CASE_MEMBER, precision=C.ICON_MIXED, member=m)
                   for g, m, _ in spec]
    ens = C.icon_ensemble_create(ens_states)
    try:
        C.icon_ensemble_step(ens, [dt for _, _, dt in spec], 5, 2)
        for (g, _, dt), so in zip(spec, solo_states):
            C.icon_dycore_step(so, dt, 5)
            C.icon_dycore_step(so, dt, 5)
        for (g, _, dt), a, b in zip(spec, ens_states, solo_states):
            fa, fb = _fields(C, a, grids[g], N), _fields(C, b, grids[g], N)
            for f in fa:
                if f in ("w", "wflx"):
                    rms = np.sqrt(np.mean((fa[f] - fb[f]) ** 2))
                    assert rms <= w_bound_mixed(dt, 5, 2) * (1.0 if f == "w" else 2.0), f
                else:
                    assert rel_l2(fa[f], fb[f]) <= TOL_MEMBER, f
        # members really differ from each other (independent perturbations)
        v0 = C.icon_state_copy_field(ens_states[0], grids[0], N, "vn")
        v1 = C.icon_state_copy_field(ens_states[1], grids[0], N, "vn")
        assert not np.array_equal(v0, v1)
    finally:
        C.icon_ensemble_free(ens)
        for s in ens_states + solo_states:
            C.icon_state_free(s)
        for g in grids:
            C.icon_grid_free(g)


def test_results_do_not_depend_on_tiles(gpu):
    """Every stencil tile (8, 16 or 32 lanes per entity, 64 to 512 threads per block) and
    every launch shape of the lean column (registers held for 6 to 12 blocks per SM) gives
    bit-identical results; the autotuner's choices lie in the candidate sets."""
    C = gpu
    N = 40
    grid = C.icon_grid_build(2, 3, N)
    kinds = [C.KIND_MX_VERTEX, C.KIND_MX_EDGE, C.KIND_MX_CELL_KE, C.KIND_MX_EDGE_TEND, C.KIND_MX_COLUMN_PREP,
             C.KIND_MX_DIFF_VERTEX]
    out = []
    try:
        for (lanes, block), shape in (((32, 128), (2, 10)), ((16, 512), (2, 12)), ((8, 64), (2, 6)),
                                      ((16, 256), (2, 8)), ((8, 128), (2, 9)), ((0, 0), (0, 0))):
            st = C.icon_state_init_ex(grid, 9, C.ICON_CASE_JET, noise_K=0.1, precision=C.ICON_MIXED)
            for k in kinds:
                C.icon_state_set_tiling(st, k, lanes, block)
            C.icon_state_set_tiling(st, C.KIND_MX_LEAN, *shape)
            C.icon_dycore_step(st, 150.0, 5)
            tiles = [C.icon_state_tiling(st, k) for k in kinds]
            if lanes:
                assert all(t == (lanes, block) for t in tiles)
                assert C.icon_state_tiling(st, C.KIND_MX_LEAN) == shape
            else:        # chosen by the autotuner
                assert all(t[0] in (8, 16, 32) and t[1] in (64, 128, 256, 512) for t in tiles), tiles
                assert C.icon_state_tiling(st, C.KIND_MX_LEAN) in C.LEAN_SHAPES
            out.append(_fields(C, st, grid, N))
            C.icon_state_free(st)
        for o in out[1:]:
            for f in out[0]:
                assert np.array_equal(out[0][f], o[f]), f
        st = C.icon_state_init_ex(grid, 9, C.ICON_CASE_JET, precision=C.ICON_MIXED)
        try:
            for kind, lanes, block in ((C.KIND_MX_VERTEX, 4, 128), (C.KIND_MX_VERTEX, 16, 96),
                                       (C.KIND_MX_LEAN, 1, 10), (C.KIND_MX_LEAN, 2, 7)):
                with pytest.raises(C.IconError) as ei:
                    C.icon_state_set_tiling(st, kind, lanes, block)
                assert ei.value.status == C.ICON_EINVAL
        finally:
            C.icon_state_free(st)
    finally:
        C.icon_grid_free(grid)


def test_barrier_timeout_is_reported_not_hung(gpu):
    """Block 0 skips its first barrier arrival: the other blocks' bounded waits run out,
    the kernel returns, the step reports ICON_ETIMEOUT and the context stays usable."""
    C = gpu
    grid = C.icon_grid_build(2, 1, 20)
    sts = [C.icon_state_init_ex(grid, 3, C.ICON_CASE_MEMBER, precision=C.ICON_MIXED, member=m) for m in range(2)]
    ens = C.icon_ensemble_create(sts)
    try:
        C.icon_ensemble_set_option(ens, C.ICON_ENS_SPIN_LIMIT, 1 << 16)
        C.icon_ensemble_set_option(ens, C.ICON_ENS_TEST_SKIP_BARRIER, 1)
        with pytest.raises(C.IconError) as ei:
            C.icon_ensemble_step(ens, [300.0, 300.0], 5, 1)
        assert ei.value.status == C.ICON_ETIMEOUT
        # the GPU context is still healthy: a fresh state steps normally
        st = C.icon_state_init_ex(grid, 1, C.ICON_CASE_SBR, precision=C.ICON_MIXED)
        C.icon_dycore_step(st, 300.0, 5)
        C.icon_state_free(st)
        # and the ensemble itself recovers once the hook is off
        C.icon_ensemble_set_option(ens, C.ICON_ENS_TEST_SKIP_BARRIER, 0)
        C.icon_ensemble_set_option(ens, C.ICON_ENS_SPIN_LIMIT, 1 << 24)
        fresh = [C.icon_state_init_ex(grid, 3, C.ICON_CASE_MEMBER, precision=C.ICON_MIXED, member=m) for m in range(2)]
        for f in PROG:
            for a, b in zip(sts, fresh):
                C.icon_state_set_field(a, grid, 20, f, C.icon_state_copy_field(b, grid, 20, f))
        C.icon_ensemble_step(ens, [300.0, 300.0], 5, 1)
        for s in fresh:
            C.icon_state_free(s)
    finally:
        C.icon_ensemble_free(ens)
        for s in sts:
            C.icon_state_free(s)
        C.icon_grid_free(grid)


@pytest.mark.parametrize("precision", [0, 1])
def test_nonfinite_state_is_reported(gpu, precision):
    C = gpu
    N = 20
    grid = C.icon_grid_build(2, 1, N)
    st = C.icon_state_init_ex(grid, 1, C.ICON_CASE_SBR, precision=precision)
    try:
        th = C.icon_state_copy_field(st, grid, N, "theta_v")
        th[17, 5] = np.nan
        C.icon_state_set_field(st, grid, N, "theta_v", th)
        with pytest.raises(C.IconError) as ei:
            C.icon_dycore_step(st, 300.0, 5)
        assert ei.value.status == C.ICON_ENONFINITE
    finally:
        C.icon_state_free(st)
        C.icon_grid_free(grid)


def test_failing_allocator_gives_enomem_without_leaks(gpu):
    import torch
    import paper_2511_02021_gb300 as P
    C = gpu
    live = {}
    budget = [25]

    def alloc(n):
        if budget[0] <= 0:
            return 0
        budget[0] -= 1
        p = torch.cuda.caching_allocator_alloc(n, 0, torch.cuda.current_stream())
        live[p] = n
        return p

    def dealloc(p):
        live.pop(p)
        torch.cuda.caching_allocator_delete(p)

    C.icon_set_allocator(alloc, dealloc)
    try:
        h = ctypes.c_void_p()
        rc = C._lib.icon_grid_build(2, 2, 20, ctypes.byref(h))
        assert rc == C.ICON_ENOMEM and h.value is None
        assert live == {}                                  # every block handed out was returned
    finally:
        P.use_torch_allocator(0)


def test_ensemble_phase_profile(gpu):
    """The phase-timed step advances the members exactly as a plain ensemble step (same
    kernel, same work lists), reports every phase the step runs with one barrier per
    phase and substep stage, and its phase times add up to the launch."""
    C = gpu
    N, nsub = 30, 5
    grids = [C.icon_grid_build(2, 2, N), C.icon_grid_build(2, 3, N)]
    spec = [(0, 0, 300.0), (1, 1, 150.0)]
    dts = [dt for _, _, dt in spec]
    a = [C.icon_state_init_ex(grids[g], 4, C.ICON_CASE_MEMBER, precision=C.ICON_MIXED, member=m) for g, m, _ in spec]
    b = [C.icon_state_init_ex(grids[g], 4, C.ICON_CASE_MEMBER, precision=C.ICON_MIXED, member=m) for g, m, _ in spec]
    ea, eb = C.icon_ensemble_create(a), C.icon_ensemble_create(b)
    try:
        C.icon_ensemble_step(ea, dts, nsub, 1)
        ms, cnt = C.icon_ensemble_step_profile(eb, dts, nsub)
        for (g, _, _), sa, sb in zip(spec, a, b):
            for f in PROG:
                assert np.array_equal(C.icon_state_copy_field(sa, grids[g], N, f),
                                      C.icon_state_copy_field(sb, grids[g], N, f)), f
        names = [C.icon_ensemble_phase_name(k) for k in range(C.ICON_ENS_PHASE_COUNT)]
        got = {names[k]: int(cnt[k]) for k in range(C.ICON_ENS_PHASE_COUNT) if cnt[k]}
        # lean column with damping (the defaults): the damping's edge update is in the gather
        per_stage = {"vertex": 2, "edge_diag": 2, "cell_ke": 2, "edge_tend": 2, "gather": 2, "column": 2}
        want = {k: v * nsub for k, v in per_stage.items()}
        want.update(zero=1, dd_div=nsub, dd_lap=nsub, diff_vertex=1, diff_edge=1, diff_theta=1)
        assert got == want
        assert np.all(ms >= 0.0) and ms.sum() > 0.0
        assert C.icon_ensemble_phase_name(C.ICON_ENS_PHASE_COUNT) is None
        # a second profiled step accumulates
        ms2, cnt2 = C.icon_ensemble_step_profile(eb, dts, nsub, ms.copy(), cnt.copy())
        assert np.array_equal(cnt2, 2 * cnt) and ms2.sum() > ms.sum()
    finally:
        C.icon_ensemble_free(ea)
        C.icon_ensemble_free(eb)
        for s in a + b:
            C.icon_state_free(s)
        for g in grids:
            C.icon_grid_free(g)
