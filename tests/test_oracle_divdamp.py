"""Pins of the oracle's fourth-order divergence damping (DD, an option of the step)
against structure the operator must have: it leaves discretely non-divergent fields
alone, it is self-adjoint and non-positive in the edge inner product sum l_e d_e u v
(div and grad are adjoint), and in a step it keeps mass and the resting state."""
import numpy as np

import oracle as O
from oracle.dycore import divergence, divergence_damping, gradient

R = O.R_EARTH


def ip(g, u, v):
    return float(np.sum((g.l_e * g.d_e)[:, None] * u * v))


def test_rotational_field_is_untouched():
    g = O.build_grid(2, 3)
    psi = (g.x_v[:, 0] * g.x_v[:, 1] + g.x_v[:, 2])[:, None] * R
    vr = (psi[g.e2v[:, 1]] - psi[g.e2v[:, 0]]) / g.l_e[:, None]      # discrete rot psi: div == 0
    assert np.max(np.abs(divergence(g, vr))) * R / np.max(np.abs(vr)) < 1e-10
    out = divergence_damping(g, vr, 0.1)
    assert np.max(np.abs(out - vr)) / np.max(np.abs(vr)) < 1e-12


def test_self_adjoint_and_dissipative():
    g = O.build_grid(2, 3)
    rng = np.random.default_rng(7)
    u = rng.standard_normal((g.ne, 2))
    v = rng.standard_normal((g.ne, 2))
    c4 = 0.004
    Tu = divergence_damping(g, u, c4) - u
    Tv = divergence_damping(g, v, c4) - v
    assert abs(ip(g, u, Tv) - ip(g, Tu, v)) <= 1e-12 * abs(ip(g, u, Tv))
    assert ip(g, u, Tu) < 0.0 and ip(g, v, Tv) < 0.0
    # a damped random field has less divergence and no more energy
    ud = u + Tu
    assert np.linalg.norm(divergence(g, ud)) < np.linalg.norm(divergence(g, u))
    assert ip(g, ud, ud) < ip(g, u, u)


def test_gradient_field_is_damped_by_the_biharmonic():
    """For vn = grad(phi) the increment is T vn = -c4 Abar^2 grad(div grad (Lc phi)) with
    Lc = div grad. Using <grad a, u> = -sum_c A_c a_c (div u)_c twice (div and grad
    adjoint), <vn, T vn> = -c4 Abar^2 <grad Lc phi, grad Lc phi>: a transposed operand or a
    wrong sign anywhere breaks the identity."""
    g = O.build_grid(2, 2)
    rng = np.random.default_rng(3)
    phi = rng.standard_normal((g.nc, 1))
    vn = gradient(g, phi)
    c4 = 0.01
    T = divergence_damping(g, vn, c4) - vn
    abar = 4.0 * np.pi * R * R / g.nc
    Lphi = divergence(g, vn)
    # <grad phi, grad(div grad div grad phi)> = -<div grad phi, div grad(Lphi)>_A = ... = |grad Lphi|^2
    gl = gradient(g, Lphi)
    expect = -c4 * abar * abar * ip(g, gl, gl)
    assert abs(ip(g, vn, T) / expect - 1.0) < 1e-10


def test_step_with_damping_conserves_mass_and_rest():
    g = O.build_grid(2, 1)
    v = O.vertical_grid(10)
    s = O.init_state(g, v, 1, O.CASE_JET, noise_K=0.1)
    m0 = O.global_mass(g, v, s)
    s1, _ = O.dycore_step(g, v, s, 300.0, 5, divdamp4=0.004)
    assert abs(O.global_mass(g, v, s1) / m0 - 1.0) < 1e-13
    s2, _ = O.dycore_step(g, v, s, 300.0, 5)
    assert np.max(np.abs(s1["vn"] - s2["vn"])) > 0.0          # it acts
    r = O.init_state(g, v, 1, O.CASE_REST)
    r1, _ = O.dycore_step(g, v, r, 300.0, 5, divdamp4=0.004)
    assert np.all(r1["vn"] == 0.0)
