"""Pins of the oracle's initial states and whole dycore step (no GPU)."""
import copy

import numpy as np
import pytest

import oracle as O
from oracle import dycore as D
from oracle import state as S
from tests.conftest import golden_path
from tests.tolerances import EPS, w_bound


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_splitmix64_published_outputs():
    for line in open(golden_path("splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, idx, out = line.split()
        assert int(O.splitmix64(int(seed), int(idx))) == int(out, 16)
    u = O.uniform01(5, np.arange(100000, dtype=np.uint64))
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def test_member_parameters_ranges():
    for m in range(64):
        ms, amp, lon, lat = O.member_params(3, m)
        assert 0.5 <= amp < 2.0 and 0.0 <= lon < 2 * np.pi and -np.pi / 2 <= lat <= np.pi / 2
    assert len({O.member_params(3, m)[0] for m in range(64)}) == 64


@pytest.mark.parametrize("which", ["sbr", "jet"])
def test_analytic_states_are_balanced(which):
    """Hydrostatic and gradient-wind balance of the analytic states, by finite differences."""
    phi = np.deg2rad(np.linspace(-80, 80, 33))
    x = np.stack([np.cos(phi), np.zeros_like(phi), np.sin(phi)], axis=1)
    z = np.linspace(500.0, 30000.0, 25)
    fn = S.sbr_state if which == "sbr" else S.jet_state
    lnp, T, u = fn(x, z)
    hz = 1.0
    lnp_zp, _, _ = fn(x, z + hz)
    lnp_zm, _, _ = fn(x, z - hz)
    dlnp_dz = (lnp_zp - lnp_zm) / (2 * hz)
    assert np.allclose(dlnp_dz, -S.GRAV / (S.RD * T), rtol=1e-6, atol=0)
    hp = 1e-5
    def at(ph):
        xx = np.stack([np.cos(ph), np.zeros_like(ph), np.sin(ph)], axis=1)
        return fn(xx, z)[0]
    dlnp_dphi = (at(phi + hp) - at(phi - hp)) / (2 * hp)
    R = O.R_EARTH
    res = (u * u * np.tan(phi)[:, None] / R + 2 * O.OMEGA * np.sin(phi)[:, None] * u
           + S.RD * T / R * dlnp_dphi)
    assert np.abs(res).max() < 1e-7 * np.abs(2 * O.OMEGA * u).max()
    if which == "jet":
        x45 = np.array([[np.sqrt(0.5), 0.0, np.sqrt(0.5)]])
        assert fn(x45, np.array([S.JET_ZJ]))[2][0, 0] == pytest.approx(35.0, rel=1e-13)
        assert T.min() > 150.0 and T.max() < 400.0
        assert np.all(u >= 0.0)


def test_jet_state_is_statically_stable():
    """The jet stand-in has a positive buoyancy frequency squared everywhere (a statically
    unstable initial state overturns within hours, which no time step survives)."""
    lat = np.deg2rad(np.linspace(-89.0, 89.0, 179))
    x = np.stack([np.cos(lat), np.zeros_like(lat), np.sin(lat)], axis=1)
    z = np.linspace(0.0, 40000.0, 801)
    lnp, T, u = S.jet_state(x, z)
    theta = T * np.exp(-(S.RD / S.CPD) * (lnp - np.log(S.P0)))
    N2 = S.GRAV * np.diff(np.log(theta), axis=1) / np.diff(z)[None, :]
    assert N2.min() > 1.2e-4, N2.min()
    # the shift of Phi leaves the wind untouched where T = T_j (z = z_j): u(45 deg) = 35 m/s
    x45 = np.array([[np.sqrt(0.5), 0.0, np.sqrt(0.5)]])
    assert S.jet_state(x45, np.array([S.JET_ZJ]))[2][0, 0] == pytest.approx(35.0, rel=1e-13)


def test_initial_state_structure():
    g = O.build_grid(2, 1)
    v = O.vertical_grid(20)
    s = O.init_state(g, v, 1, O.CASE_REST)
    # rest: horizontally uniform, discrete hydrostatic balance, state equation
    for f in ("rho", "theta_v", "exner"):
        assert np.all(s[f] == s[f][0:1])
    assert np.all(s["vn"] == 0.0) and np.all(s["w"] == 0.0)
    T = s["theta_v"] * s["exner"]
    assert np.allclose(T, 250.0, rtol=2e-3)
    p = S.P0 * s["exner"] ** (S.CPD / S.RD)
    assert np.allclose(p, s["rho"] * S.RD * T, rtol=1e-13)
    # noise: bounded by the amplitude, seeded, reproducible
    s1 = O.init_state(g, v, 1, O.CASE_SBR)
    s1b = O.init_state(g, v, 1, O.CASE_SBR, noise_K=0.0)
    d = s1["theta_v"] - s1b["theta_v"]
    assert np.abs(d).max() <= 0.01 and np.abs(d).max() > 0.009
    assert np.array_equal(s1["theta_v"], O.init_state(g, v, 1, O.CASE_SBR)["theta_v"])
    assert not np.array_equal(s1["theta_v"], O.init_state(g, v, 2, O.CASE_SBR)["theta_v"])


def test_rest_state_stays_at_rest():
    g = O.build_grid(2, 1)
    v = O.vertical_grid(20)
    s = O.init_state(g, v, 0, O.CASE_REST)
    s1, acc = O.dycore_step(g, v, s, 300.0, 5)
    assert np.all(s1["vn"] == 0.0)
    assert np.abs(s1["w"]).max() <= 1e-12
    for f in ("rho", "theta_v", "exner"):
        assert rel(s1[f], s[f]) < 1e-14
    assert np.all(acc["mflx"] == 0.0)


def _sbr_drift(g, nlev=20, dt=300.0, nsteps=1):
    v = O.vertical_grid(nlev)
    s0 = O.init_state(g, v, 1, O.CASE_SBR, noise_K=0.0)
    s = s0
    for _ in range(nsteps):
        s, _ = O.dycore_step(g, v, s, dt, 5)
    return rel(s["vn"], s0["vn"])


def test_sbr_drift_bounded_and_shrinking():
    d = [_sbr_drift(O.build_grid(2, b)) for b in (0, 1, 2)]
    assert d[-1] < 2e-4
    assert d[0] > d[1] > d[2]


def test_planted_sign_errors_break_balance():
    """A wrong vorticity or Coriolis sign in the oracle fails the balance pin by orders of magnitude."""
    g = O.build_grid(2, 1)
    good = _sbr_drift(g)
    bad_f = copy.copy(g)
    bad_f.f_e = -g.f_e
    bad_z = copy.copy(g)
    bad_z.s_ve = -g.s_ve
    assert _sbr_drift(bad_f) > 30 * good
    assert _sbr_drift(bad_z) > 3 * good


def test_mass_conserved_and_fluxes_consistent():
    g = O.build_grid(2, 1)
    v = O.vertical_grid(20)
    s = O.init_state(g, v, 2, O.CASE_JET, noise_K=0.1)
    m0 = O.global_mass(g, v, s)
    s1, acc = O.dycore_step(g, v, s, 300.0, 5)
    m1 = O.global_mass(g, v, s1)
    assert abs(m1 - m0) / m0 < 1e-13
    # the step-mean mass fluxes reproduce the density change of each column
    div = D.divergence(g, acc["mflx"])
    vert = (acc["wflx"][:, :-1] - acc["wflx"][:, 1:]) / v.dz[None, :]
    drho = -300.0 * (div + vert)
    assert rel(s["rho"] + drho, s1["rho"]) < 1e-13
    assert np.abs(acc["wflx"][:, 0]).max() == 0.0 and np.abs(acc["wflx"][:, -1]).max() == 0.0


def test_diffusion_properties():
    g = O.build_grid(2, 1)
    v = O.vertical_grid(20)
    s = O.init_state(g, v, 0, O.CASE_REST)
    s1, Kh = D.diffusion(g, v, s, 300.0)
    assert np.all(s1["theta_v"] == s["theta_v"]) and np.all(Kh == 0.0)
    s = O.init_state(g, v, 2, O.CASE_JET, noise_K=0.5)
    s1, Kh = D.diffusion(g, v, s, 300.0)
    assert np.all(Kh >= 0.0)
    assert np.all(s1["rho"] == s["rho"])
    # flux form: the area-weighted theta_v sum is unchanged
    tot0 = np.sum(g.A_c[:, None] * s["theta_v"], axis=0)
    tot1 = np.sum(g.A_c[:, None] * s1["theta_v"], axis=0)
    assert np.all(np.abs(tot1 - tot0) < 1e-13 * tot0)
    # diffusion reduces the theta_v variance on every level
    var0 = np.var(s["theta_v"], axis=0)
    var1 = np.var(s1["theta_v"], axis=0)
    assert np.all(var1 <= var0)


def test_w_conditioning():
    """The oracle's own w moves by far more than eps under one-ulp input perturbations,
    while the other fields move by O(eps): the premise of w_bound."""
    g = O.build_grid(2, 2)
    v = O.vertical_grid(20)
    s = O.init_state(g, v, 1, O.CASE_SBR, noise_K=0.01)
    a, _ = O.dycore_step(g, v, s, 300.0, 5)
    sp = dict(s)
    sp["exner"] = s["exner"] * (1 + EPS * np.random.default_rng(0).choice([-1, 1], size=s["exner"].shape))
    b, _ = O.dycore_step(g, v, sp, 300.0, 5)
    assert rel(b["w"], a["w"]) > 1e-12
    assert np.sqrt(np.mean((b["w"] - a["w"]) ** 2)) < w_bound(300.0, 5, 1)
    for f in ("vn", "rho", "theta_v", "exner"):
        assert rel(b[f], a[f]) < 1e-14


# ------------------------------------------------------------------ vertical advection and the linearised
# state equation, pinned against the mathematics (a mistake planted in the oracle fails these)
import inspect


def _planted(module, func, old, new, count=1):
    """A copy of module.func with the source text `old` replaced by `new` (a planted mistake)."""
    src = inspect.getsource(getattr(module, func))
    assert src.count(old) == count, (func, old)
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), "<planted %s>" % func, "exec"), ns)
    return ns[func]


def _linear_column_state(g, v, b_vn, c_w, d_w):
    """Horizontally uniform column state: vn = 3 + b_vn z at every edge (full levels), w = c_w + d_w z
    at every cell (half levels); the scalars are irrelevant to the tendencies."""
    vn = np.repeat((3.0 + b_vn * v.z_f)[None, :], g.ne, axis=0)
    w = np.repeat((c_w + d_w * v.z_h)[None, :], g.nc, axis=0)
    return {"vn": vn, "w": w}


def _vertical_advection_errors(tend, g, v, flat_terrain=None):
    """Max deviation of the vertical advection terms of `tend` from -w dvn/dz and -w dw/dz
    (momentum equation in advective form, z upward) for linear profiles, where the centred
    differences and the linear interpolation to half levels are exact. The vn term is the
    difference of A_vn with and without w (the horizontal terms do not depend on w). The
    terrain-following form advects with the contravariant velocity, which is 0 at the lid and
    the ground by definition (R-Z4); the layers next to them then see half their w."""
    N = v.N
    b, c, d = 2.0e-3, 0.3, -1.5e-5              # dvn/dz (1/s), w = c + d z
    s = _linear_column_state(g, v, b, c, d)
    s0 = dict(s, w=np.zeros_like(s["w"]))
    call = (lambda st: tend(g, v, st)) if flat_terrain is None else (lambda st: tend(g, v, flat_terrain, st))
    A_vn, A_w = call(s)[:2]
    A_vn0 = call(s0)[0]
    wh = c + d * v.z_h
    if flat_terrain is not None:
        wh[0] = wh[N] = 0.0
    wbar = 0.5 * (wh[:-1] + wh[1:])              # mean of the two half-level w of a layer
    exp_vn = -wbar * b
    # top and bottom full levels: the half level outside takes the adjacent full value (R-B1),
    # so the one-layer difference sees half the gradient there
    exp_vn_edge = -wbar * b / 2.0
    dvn = A_vn - A_vn0
    err_vn = max(np.abs(dvn[:, 1:N - 1] - exp_vn[None, 1:N - 1]).max(),
                 np.abs(dvn[:, [0, N - 1]] - exp_vn_edge[None, [0, N - 1]]).max())
    exp_w = -(c + d * v.z_h[1:N]) * d             # -w dw/dz at the interior half levels
    err_w = np.abs(A_w[:, 1:N] - exp_w[None, :]).max()
    scale_vn = np.abs(exp_vn).max()
    scale_w = np.abs(exp_w).max()
    return err_vn / scale_vn, err_w / scale_w


def test_vertical_advection_matches_the_advective_form():
    g = O.build_grid(2, 0)
    v = O.vertical_grid(20)
    e_vn, e_w = _vertical_advection_errors(D.tendencies, g, v)
    assert e_vn < 1e-10 and e_w < 1e-12, (e_vn, e_w)


def test_vertical_advection_of_the_terrain_oracle_over_flat_ground():
    from oracle import terrain as T
    g = O.build_grid(2, 0)
    v = O.vertical_grid(20)
    t = T.terrain_geometry(g, v, np.zeros(g.nc))
    e_vn, e_w = _vertical_advection_errors(T.tendencies, g, v, flat_terrain=t)
    assert e_vn < 1e-10 and e_w < 1e-12, (e_vn, e_w)


@pytest.mark.parametrize("old,new,which", [
    ("- wbar * (vn_ie[:, :N] - vn_ie[:, 1:])", "+ wbar * (vn_ie[:, :N] - vn_ie[:, 1:])", 0),
    ("- w[:, 1:N] * (w[:, 0:N - 1]", "+ w[:, 1:N] * (w[:, 0:N - 1]", 1),
    # a denominator over one level interval while the centred difference of w spans two
    ("(v.z_h[0:N - 1] - v.z_h[2:N + 1])", "(v.z_f[0:N - 1] - v.z_f[1:N])", 1),
])
def test_planted_vertical_advection_mistakes_fail(old, new, which):
    g = O.build_grid(2, 0)
    v = O.vertical_grid(20)
    bad = _planted(D, "tendencies", old, new)
    errs = _vertical_advection_errors(bad, g, v)
    assert errs[which] > 0.3, errs


def _state_equation_residual(substep, g, v, s, dtau, terrain=None):
    """max |pi - (Rd rho theta_v / p0)^(Rd/cvd)| / pi after one predictor-corrector substep."""
    acc = {"mflx": np.zeros((g.ne, v.N)), "wflx": np.zeros((g.nc, v.N + 1))}
    if terrain is None:
        s1 = substep(g, v, s, dtau, 1, acc)
    else:
        s1 = substep(g, v, terrain, s, dtau, 1, acc)
    eos = (S.RD * s1["rho"] * s1["theta_v"] / S.P0) ** (S.RD / S.CVD)
    return np.abs(s1["exner"] / eos - 1.0).max()


def _moving_state(g, v, terrain=None):
    """Solid-body rotation with theta_v noise and a smooth vertical velocity, so that both the
    explicit and the implicit vertical fluxes change Theta at first order in dtau."""
    s = O.init_state(g, v, 3, O.CASE_SBR, noise_K=0.05, terrain=terrain)
    zz = v.z_h / v.z_top
    w = 0.4 * np.sin(np.pi * zz)[None, :] * (1.0 + 0.5 * g.x_c[:, 0:1])
    return dict(s, w=w)


def _orders(substep, g, v, s, terrain=None, dtaus=(20.0, 10.0, 5.0)):
    r = [_state_equation_residual(substep, g, v, s, dt, terrain) for dt in dtaus]
    return [r[i] / r[i + 1] for i in range(len(r) - 1)], r


def test_linearised_state_equation_is_second_order():
    """The column updates Exner by the state equation linearised about S^n,
    pi^{n+1} - pi^n = (Rd/cvd)(pi/Theta)(Theta^{n+1} - Theta^n); the state equation itself,
    pi = (Rd rho theta_v/p0)^(Rd/cvd), then holds up to a residual quadratic in the increment:
    halving dtau divides it by about 4."""
    g = O.build_grid(2, 0)
    v = O.vertical_grid(20)
    s = _moving_state(g, v)
    eos0 = (S.RD * s["rho"] * s["theta_v"] / S.P0) ** (S.RD / S.CVD)
    assert np.abs(s["exner"] / eos0 - 1.0).max() < 1e-14
    ratios, r = _orders(D.substep, g, v, s)
    assert all(3.5 < q < 4.5 for q in ratios), (ratios, r)


def test_linearised_state_equation_is_second_order_over_terrain():
    from oracle import terrain as T
    g = O.build_grid(2, 0)
    v = O.vertical_grid(20)
    t = T.terrain_geometry(g, v, T.mountain(g.x_c, 1500.0, 1.5e6))
    s = _moving_state(g, v, terrain=t)
    ratios, r = _orders(T.substep, g, v, s, terrain=t)
    assert all(3.5 < q < 4.5 for q in ratios), (ratios, r)


@pytest.mark.parametrize("old,new", [
    ("ex_x = ex + (RD / CVD)", "ex_x = ex + (RD / CPD)"),
    ("gam = (RD / CVD)", "gam = (RD / CPD)"),
])
def test_planted_state_equation_mistakes_fail(old, new, monkeypatch):
    """With Rd/cpd in place of Rd/cvd in either place the residual is first order in dtau."""
    g = O.build_grid(2, 0)
    v = O.vertical_grid(20)
    s = _moving_state(g, v)
    monkeypatch.setattr(D, "column", _planted(D, "column", old, new))
    ratios, r = _orders(D.substep, g, v, s)
    assert all(q < 2.6 for q in ratios), (ratios, r)


def test_long_run_stays_bounded():
    """120 steps (10 simulated hours) of the jet on R2B2/20 at the parity configuration's time
    step: finite, w and vn bounded, mass conserved (a statically unstable initial state or an
    unstable scheme grows w geometrically within a few dozen steps)."""
    g = O.build_grid(2, 1)
    v = O.vertical_grid(20)
    s = O.init_state(g, v, 2, O.CASE_JET, noise_K=0.1)
    m0 = O.global_mass(g, v, s)
    for _ in range(120):
        s, _ = O.dycore_step(g, v, s, 300.0, 5)
    assert np.all(np.isfinite(s["w"])) and np.abs(s["w"]).max() < 0.05
    assert np.abs(s["vn"]).max() < 40.0
    assert abs(O.global_mass(g, v, s) / m0 - 1.0) < 1e-12
