"""Pins of the upwind-theta option (UT): the donor selection restated as a loop, the
monotonicity of the upwind flux-form transport of theta_v, and the step's invariants."""
import numpy as np

import oracle as O
from oracle.dycore import divergence, edge_mean, edge_upwind


def test_donor_selection_matches_a_loop():
    g = O.build_grid(2, 0)
    rng = np.random.default_rng(2)
    f = rng.standard_normal((g.nc, 3))
    vn = rng.standard_normal((g.ne, 3))
    got = edge_upwind(g, f, vn)
    for e in range(g.ne):
        for k in range(3):
            donor = g.e2c[e, 0] if vn[e, k] >= 0.0 else g.e2c[e, 1]
            assert got[e, k] == f[donor, k]


def test_upwind_flux_form_is_monotone():
    """Horizontal flux-form update of Theta = rho theta with rho updated by the same mass
    fluxes: with upwind theta every new theta lies within the range of the cell and its
    neighbours (Courant number below 1); with the centred theta it does not."""
    g = O.build_grid(2, 3)
    rng = np.random.default_rng(5)
    nb = np.stack([np.where(g.e2c[g.c2e[:, s], 0] == np.arange(g.nc), g.e2c[g.c2e[:, s], 1],
                            g.e2c[g.c2e[:, s], 0]) for s in range(3)], 1)
    rho = 1.0 + 0.1 * rng.random((g.nc, 1))
    theta = 280.0 + 40.0 * rng.random((g.nc, 1))
    vn = rng.standard_normal((g.ne, 1)) * 10.0
    dt = 0.3 * g.d_e.min() / (np.abs(vn).max() * 1.2)
    F = edge_mean(g, rho) * vn
    rho1 = rho - dt * divergence(g, F)
    lo = np.minimum(theta[:, 0], theta[nb, 0].min(axis=1))
    hi = np.maximum(theta[:, 0], theta[nb, 0].max(axis=1))

    def step(theta_e):
        return ((rho * theta - dt * divergence(g, F * theta_e)) / rho1)[:, 0]

    tu = step(edge_upwind(g, theta, vn))
    assert np.all(tu >= lo - 1e-9) and np.all(tu <= hi + 1e-9)
    tc = step(edge_mean(g, theta))
    assert np.any(tc < lo - 1e-6) or np.any(tc > hi + 1e-6)


def test_step_invariants():
    g = O.build_grid(2, 1)
    v = O.vertical_grid(10)
    s = O.init_state(g, v, 1, O.CASE_JET, noise_K=0.1)
    m0 = O.global_mass(g, v, s)
    s1, _ = O.dycore_step(g, v, s, 300.0, 5, upwind_theta=True)
    s2, _ = O.dycore_step(g, v, s, 300.0, 5)
    assert abs(O.global_mass(g, v, s1) / m0 - 1.0) < 1e-13
    assert np.max(np.abs(s1["theta_v"] - s2["theta_v"])) > 0.0
    # a uniform theta_v makes the option a no-op
    u = O.init_state(g, v, 1, O.CASE_REST)
    u1, _ = O.dycore_step(g, v, u, 300.0, 5, upwind_theta=True)
    u2, _ = O.dycore_step(g, v, u, 300.0, 5)
    for f in ("vn", "w", "rho", "theta_v", "exner"):
        assert np.array_equal(u1[f], u2[f]), f
