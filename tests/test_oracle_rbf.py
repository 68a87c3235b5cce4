"""The RBF tangential reconstruction (ICON's vt on the same stencil) against the Perot
weights the step uses, for solid-body rotation on R2B1..R2B4: the evidence for keeping Perot
(no GPU)."""
import numpy as np
import pytest

import oracle as O
from oracle.rbf import rbf_tangential_weights, solid_body_vt_error


@pytest.fixture(scope="module")
def errors():
    out = {"perot": [], "stationary": [], "fixed": []}
    for bis in (1, 2, 3, 4):
        g = O.build_grid(2, bis)
        out["perot"].append(solid_body_vt_error(g, g.e2vt, g.vt_w))
        out["stationary"].append(solid_body_vt_error(g, *rbf_tangential_weights(g, 1.0 * g.l_e)))
        out["fixed"].append(solid_body_vt_error(g, *rbf_tangential_weights(g, np.full(g.ne, 1.0e6))))
    return {k: np.array(v) for k, v in out.items()}


def test_rbf_exact_for_its_own_interpolant():
    """Pin of the RBF weights themselves: a field that is one of the interpolant's basis
    functions, u(x) = phi(|x - x_j|) n_j, is reproduced exactly."""
    g = O.build_grid(2, 2)
    eps = np.full(g.ne, 8.0e5)
    st, w = rbf_tangential_weights(g, eps)
    e = 100
    j = st[e, 2]
    def u_at(x):
        r2 = np.sum((x - g.x_e[j]) ** 2, axis=-1) * O.R_EARTH ** 2
        return np.exp(-r2 / 8.0e5 ** 2)[..., None] * g.n_e[j]
    vn = np.sum(u_at(g.x_e[st[e]]) * g.n_e[st[e]], axis=1)
    vt = float(np.sum(w[e] * vn))
    assert vt == pytest.approx(float(np.dot(u_at(g.x_e[e]), g.t_e[e])), rel=1e-10, abs=1e-12)


def test_perot_converges_and_stationary_rbf_does_not(errors):
    p, s = errors["perot"], errors["stationary"]
    assert np.all(np.log2(p[:-1] / p[1:]) > 1.5)            # second order (measured 1.7, 1.6, 1.6)
    assert np.all(s > 0.1) and s[-1] > 0.9 * s[0]            # saturates near 17 %
    assert np.all(s > 10 * p) and s[-1] > 100 * p[-1]


def test_fixed_scale_rbf_converges_but_stays_behind_perot(errors):
    f, p = errors["fixed"], errors["perot"]
    assert f[-1] < 0.5 * f[-2]                               # converges once eps spans a few edges
    assert np.all(f > 5 * p)                                 # yet 5-40x less accurate than Perot
