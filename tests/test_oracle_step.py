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
