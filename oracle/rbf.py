"""Radial-basis-function tangential velocity on the C grid: the study behind leaving the
RBF option out (FP64, plain numpy).

TEST INFRASTRUCTURE ONLY; the product library never imports this module.

ICON reconstructs the tangential velocity at an edge with vector RBF interpolation over
the four other edges of its two cells (the stencil of O4 without the edge itself). Reading
R-RBF of that reconstruction: the interpolant u(x) = sum_j c_j phi(|x - x_j|) n_j with the
Gaussian phi(r) = exp(-(r/eps)^2), fitted to the normal components, u(x_i).n_i = vn_i for
the four stencil edges i (a 4x4 system per edge), and evaluated as vt_e = u(x_e).t_e. So
vt_e = sum_i w_i vn_i with w = A^{-T} b, A_ij = phi(r_ij) n_i.n_j, b_j = phi(r_ej) n_j.t_e.
The shape parameter eps is either stationary (a multiple of the edge length) or fixed in
metres across resolutions.
"""
import numpy as np

from .grid import R_EARTH


def rbf_tangential_weights(g, eps):
    """R-RBF weights (Ne, 4) on the stencil g.e2vt[:, 1:5] for the shape parameter eps
    (metres, one value per edge); returns (stencil, weights)."""
    st = g.e2vt[:, 1:5]
    X = g.x_e[st] * R_EARTH
    Nn = g.n_e[st]
    d = X[:, :, None, :] - X[:, None, :, :]
    phi = np.exp(-np.sum(d * d, axis=3) / (eps[:, None, None] ** 2))
    A = phi * np.einsum("eik,ejk->eij", Nn, Nn)
    de = g.x_e[:, None, :] * R_EARTH - X
    b = np.exp(-np.sum(de * de, axis=2) / eps[:, None] ** 2) * np.einsum("ejk,ek->ej", Nn, g.t_e)
    w = np.linalg.solve(np.transpose(A, (0, 2, 1)), b[:, :, None])[:, :, 0]
    return st, w


def solid_body_vt_error(g, stencil, weights, u0=20.0):
    """Relative L2 error of a tangential reconstruction (weights on the stencil) for zonal
    solid-body rotation u = u0 cos(phi) against the exact u.t_e."""
    x = g.x_e
    cphi = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2)
    el = np.stack([-x[:, 1] / cphi, x[:, 0] / cphi, np.zeros_like(cphi)], axis=1)
    u = (u0 * cphi)[:, None] * el
    vn = np.sum(u * g.n_e, axis=1)
    exact = np.sum(u * g.t_e, axis=1)
    vt = np.sum(weights * vn[stencil], axis=1)
    return float(np.linalg.norm(vt - exact) / np.linalg.norm(exact))
