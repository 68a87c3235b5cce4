"""Pins of the oracle's fourth-order background diffusion option (BD): the O6 vector
Laplacian it squares is self-adjoint and non-positive in the l_e d_e inner product
(grad/div and rot/curl are adjoint pairs), so -c Abar^2 L(L(vn)) is self-adjoint and
non-positive; in a step it conserves mass, keeps rest at rest and damps the state."""
import numpy as np

import oracle as O
from oracle.dycore import vector_laplacian

R = O.R_EARTH


def ip(g, u, v):
    return float(np.sum((g.l_e * g.d_e)[:, None] * u * v))


def test_vector_laplacian_is_self_adjoint_and_non_positive():
    g = O.build_grid(2, 3)
    rng = np.random.default_rng(1)
    u = rng.standard_normal((g.ne, 2))
    v = rng.standard_normal((g.ne, 2))
    Lu, Lv = vector_laplacian(g, u), vector_laplacian(g, v)
    assert abs(ip(g, u, Lv) - ip(g, Lu, v)) <= 1e-12 * abs(ip(g, u, Lv))
    assert ip(g, u, Lu) < 0.0 and ip(g, v, Lv) < 0.0
    # the squared operator: <u, L L u> = <L u, L u> >= 0 (so -c L L dissipates)
    assert abs(ip(g, u, vector_laplacian(g, Lu)) / ip(g, Lu, Lu) - 1.0) < 1e-10


def test_solid_body_rotation_rotational_part():
    """Rigid rotation: L(u) = -2 u / R^2 on the sphere; the C grid's divergence part adds
    its known grid-scale error (about 5 %, not falling with refinement)."""
    for bis in (2, 3):
        g = O.build_grid(2, bis)
        un = np.sum(np.stack([-g.x_e[:, 1], g.x_e[:, 0], 0.0 * g.x_e[:, 0]], 1) * g.n_e, 1)[:, None] * 20.0
        L1 = vector_laplacian(g, un)
        assert np.linalg.norm(L1 + 2.0 / R ** 2 * un) / np.linalg.norm(2.0 / R ** 2 * un) < 0.06


def test_step_with_background_diffusion():
    g = O.build_grid(2, 1)
    v = O.vertical_grid(10)
    s = O.init_state(g, v, 1, O.CASE_JET, noise_K=0.1)
    m0 = O.global_mass(g, v, s)
    s1, _ = O.dycore_step(g, v, s, 300.0, 5, diff4=0.01)
    s2, _ = O.dycore_step(g, v, s, 300.0, 5)
    assert abs(O.global_mass(g, v, s1) / m0 - 1.0) < 1e-13
    ip0 = lambda x: float(np.sum((g.l_e * g.d_e)[:, None] * x * x))
    assert ip0(s1["vn"]) < ip0(s2["vn"])                     # it removes energy
    r = O.init_state(g, v, 1, O.CASE_REST)
    r1, _ = O.dycore_step(g, v, r, 300.0, 5, diff4=0.01)
    assert np.all(r1["vn"] == 0.0)
