"""Tracer transport with the dycore's step-mean mass fluxes: the oracle (FP64, plain numpy).

TEST INFRASTRUCTURE ONLY; the product library never imports this module.

The paper's atmosphere carries water, CO2 and ozone tracers (Sec. "Overview of the
Problem") and prints no transport scheme. This is the builder's reading of a
flux-form, second-order, mass-consistent transport step that consumes the FP64
substep-averaged fluxes of one dycore step (M = mflx at edge-levels, positive from
c1 to c2; W = wflx at half levels, positive upward), one function per definition:

T1  cell neighbours: c2c[c, s] is the other cell of edge c2e[c, s].
T2  least-squares cell gradient: g_c = sum_s G_cs (q_c2c[c,s] - q_c), G_cs the
    3-vector weights (in the tangent plane at x_c) of argmin_g sum_s
    (q_s - q_c - g . d_cs)^2, d_cs = R (x_s - x_c) projected on that plane.
T3  edge value, upwind with a half-step back-trajectory (a Miura-type scheme):
    donor cd = c1 if M >= 0 else c2; rho_e = (rho_c1 + rho_c2) / 2 of the step's
    initial density; v_n = M / rho_e and v_t = M_t / rho_e with M_t the tangential
    mass flux from the dycore's tangential reconstruction (O4 weights applied to M);
    q_e = q_cd + g_cd . (R (x_e - x_cd) - dt/2 (v_n n_e + v_t t_e)).
T4  vertical half-level value at interior half levels: donor full level kd = h if
    W >= 0 (the level below) else h - 1; centred slope
    s_k = (q_{k-1} - q_{k+1}) / (z_{k-1} - z_{k+1}) (0 at the top and bottom level);
    w_h = W / rho_ic (rho_ic of the initial density, interpolated as in the dycore);
    q_h = q_kd + s_kd (z_h - z_kd - dt/2 w_h). No flux through the lid and the ground.
T5  update: (rho q)^{n+1} = rho^n q^n - dt [ (1/A_c) sum_s s_ce l_e M_e q_e
    + (W_k q_k - W_{k+1} q_{k+1}) / dz_k ],  q^{n+1} = (rho q)^{n+1} / rho^{n+1}.
With the dycore's own fluxes, rho^{n+1} = rho^n - dt div(M, W) up to rounding, so a
uniform tracer stays uniform and the tracer mass sum_c A_c sum_k dz_k rho q is
conserved (flux form). The scheme has no limiter.
T6  on terrain-following levels (oracle.terrain; M then carries the layer thickness,
    M = rho_e vn dz_e, and W is contravariant): v_n = M / (rho_e dz_e) and
    v_t = M_t / (rho_e dz_e) in T3; each cell's own full and half heights, spacings and
    interpolation weights in T4; in T5 the horizontal and vertical flux divergences
    together are divided by the cell's dz_k: (rho q)^{n+1} = rho^n q^n - dt [(1/A_c)
    sum_s s_ce l_e M_e q_e + W_k q_k - W_{k+1} q_{k+1}] / dz_ck.
"""
import numpy as np

from .grid import R_EARTH
from .state import to_half, to_half_w


def cell_neighbours(g):
    """T1: (Nc, 3) neighbour across each cell edge slot."""
    e = g.c2e
    c1, c2 = g.e2c[e, 0], g.e2c[e, 1]
    me = np.arange(g.nc)[:, None]
    return np.where(c1 == me, c2, c1)


def cell_lsq_weights(g):
    """T2: (Nc, 3, 3) weights G_cs as 3-vectors in the tangent plane at x_c."""
    nb = cell_neighbours(g)
    xc = g.x_c
    d = (g.x_c[nb] - xc[:, None, :]) * R_EARTH                 # (Nc, 3, 3)
    d = d - np.sum(d * xc[:, None, :], axis=2)[:, :, None] * xc[:, None, :]
    # orthonormal tangent basis at x_c
    ref = np.where(np.abs(xc[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    e1 = np.cross(ref, xc)
    e1 /= np.linalg.norm(e1, axis=1)[:, None]
    e2 = np.cross(xc, e1)
    p1 = np.sum(d * e1[:, None, :], axis=2)                    # (Nc, 3)
    p2 = np.sum(d * e2[:, None, :], axis=2)
    m11, m12, m22 = np.sum(p1 * p1, 1), np.sum(p1 * p2, 1), np.sum(p2 * p2, 1)
    det = m11 * m22 - m12 * m12
    i11, i12, i22 = m22 / det, -m12 / det, m11 / det
    q1 = i11[:, None] * p1 + i12[:, None] * p2
    q2 = i12[:, None] * p1 + i22[:, None] * p2
    return q1[:, :, None] * e1[:, None, :] + q2[:, :, None] * e2[:, None, :]


def cell_gradient(g, q, G=None):
    """T2: (Nc, 3, n) least-squares gradient 3-vectors of a cell field (Nc, n)."""
    if G is None:
        G = cell_lsq_weights(g)
    nb = cell_neighbours(g)
    out = np.zeros((g.nc, 3, q.shape[1]))
    for s in range(3):
        dq = q[nb[:, s]] - q
        out += G[:, s, :, None] * dq[:, None, :]
    return out


def edge_values(g, q, grad, M, rho, dt, terrain=None):
    """T3: (Ne, N) upwind edge values with the half-step back-trajectory."""
    c1, c2 = g.e2c[:, 0], g.e2c[:, 1]
    cd = np.where(M >= 0.0, c1[:, None], c2[:, None])          # (Ne, N) donor cells
    rho_e = 0.5 * (rho[c1] + rho[c2])
    if terrain is not None:
        rho_e = rho_e * terrain.dz_e                           # T6: M carries dz_e
    vn = M / rho_e
    Mt = np.zeros_like(M)
    for j in range(5):
        Mt += g.vt_w[:, j:j + 1] * M[g.e2vt[:, j]]
    vt = Mt / rho_e
    k = np.arange(M.shape[1])[None, :]
    off = ((g.x_e[:, None, :] - g.x_c[cd]) * R_EARTH
           - 0.5 * dt * (vn[:, :, None] * g.n_e[:, None, :] + vt[:, :, None] * g.t_e[:, None, :]))
    gd = np.moveaxis(grad, 1, 2)[cd, k]                        # (Ne, N, 3)
    return q[cd, k] + np.sum(gd * off, axis=2)


def half_values(v, q, W, rho, dt, terrain=None):
    """T4: (Nc, N+1) half-level values; 0 at the lid and the ground (no flux there)."""
    N = v.N
    nc = q.shape[0]
    if terrain is None:
        zf = np.broadcast_to(v.z_f[None, :], q.shape)
        zh = np.broadcast_to(v.z_h[None, :], (nc, N + 1))
        rho_ic = to_half(v, rho)
    else:                                                      # T6: each cell's own levels
        zf, zh = terrain.zf_c, terrain.zh_c
        rho_ic = to_half_w(terrain.wu_c, rho)
    s = np.zeros_like(q)
    if N >= 3:
        s[:, 1:N - 1] = (q[:, :N - 2] - q[:, 2:]) / (zf[:, :N - 2] - zf[:, 2:])
    rows = np.arange(nc)
    out = np.zeros((nc, N + 1))
    for h in range(1, N):
        up = W[:, h] >= 0.0
        kd = np.where(up, h, h - 1)
        qd = q[rows, kd]
        sd = s[rows, kd]
        wh = W[:, h] / rho_ic[:, h]
        out[:, h] = qd + sd * (zh[:, h] - zf[rows, kd] - 0.5 * dt * wh)
    return out


def tracer_step(g, v, q, rho_old, rho_new, mflx, wflx, dt, terrain=None):
    """T5: one transport step of the tracer q (Nc, N) with the step-mean fluxes (T6 on
    terrain-following levels)."""
    grad = cell_gradient(g, q)
    qe = edge_values(g, q, grad, mflx, rho_old, dt, terrain)
    F = mflx * qe
    div = np.zeros_like(q)
    for s in range(3):
        div += (g.s_ce[:, s] * g.l_e[g.c2e[:, s]])[:, None] * F[g.c2e[:, s]]
    div /= g.A_c[:, None]
    V = wflx * half_values(v, q, wflx, rho_old, dt, terrain)
    if terrain is not None:
        return (rho_old * q - dt * (div + (V[:, :v.N] - V[:, 1:])) / terrain.dz_c) / rho_new
    vert = (V[:, :v.N] - V[:, 1:]) / v.dz[None, :]
    return (rho_old * q - dt * (div + vert)) / rho_new


def tracer_mass(g, v, rho, q, terrain=None):
    """sum_c A_c sum_k dz_k rho q (kg of tracer per kg-of-air unit); each cell's own dz
    on terrain-following levels."""
    dz = v.dz[None, :] if terrain is None else terrain.dz_c
    return float(np.sum(g.A_c * np.sum(rho * q * dz, axis=1)))
