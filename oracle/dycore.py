"""Nonhydrostatic dynamical-core step on the triangular C-grid: the oracle (FP64, plain numpy).

TEST INFRASTRUCTURE ONLY; the product library never imports this module.

The paper names the method (a nonhydrostatic dynamical core on an
icosahedral-triangular C grid, Sec. "Current State of the Art"), its dominant
cost (memory-bound stencils with index lookups on triangles, hexagons and 12
pentagons, Sec. "Separation of Concerns") and nothing of its discretisation. The
operators and the step below are the builder's readings, one function per
definition, in the order the step applies them. Fields are (entity, level)
arrays; full level k = 0..N-1 runs top to bottom, half level h = 0..N with w = 0
at h = 0 (lid) and h = N (ground).

O1 gradient      (d psi/dn)_e = (psi_c2 - psi_c1) / d_e
O2 divergence    delta_c = (1/A_c) sum_e s_ce l_e u_e
O3 curl          zeta_v = (1/A_v) sum_e s_ve d_e vn_e
O4 tangential    vt_e = sum_j W_ej vn_j (Perot, 5 edges)
O5 cell KE       K_c = sum_e kappa_ce K_e,  K_e = (vn^2 + vt^2)/2
O6 vector Lapl.  L_e = (delta_c2 - delta_c1)/d_e - (zeta_v2 - zeta_v1)/l_e
O7 w advection   w_v = mean of w over the cells of v; at edges
                 a_e = vn_ie (w_c2 - w_c1)/d_e + vt_ie (w_v2 - w_v1)/l_e;
                 (v.grad w)_c = sum_e kappa_ce a_e; vertical part centred,
                 -w_h (w_{h-1} - w_{h+1}) / (z_{h-1} - z_{h+1}).
Step (dt, nsub substeps of dtau = dt/nsub, off-centring beta = 0.65):
  predictor  T0 = tend(S^n); vn* = vn^n + dtau (A_vn0 - cpd thv_e dpi/dn);
             column(S^n, vn*, A_w0) -> w*, rho*, thv*, pi*
  corrector  T* = tend(S*); vn^{n+1} = vn^n + dtau ((A_vn0 + A_vn*)/2 - cpd thv_e* dpi*/dn),
             divergence-damped with c4 = DIVDAMP4 (DD);
             column(S^n, vn^{n+1}, (A_w0 + A_w*)/2) with fluxes from rho_e*, thv_e*;
             mass-flux accumulators += rho_e* vn^{n+1} / nsub and
             rho_ic (beta w^{n+1} + (1-beta) w^n) / nsub.
  after the substeps: Smagorinsky diffusion with dt.
"""
import numpy as np

from .grid import R_EARTH
from .state import GRAV, RD, CPD, CVD, to_half

BETA = 0.65             # vertical off-centring (implicit weight)
CS_SMAG = 0.15          # Smagorinsky constant
# DD-base: fourth-order divergence damping of the corrector's vn in every substep with ICON's
# default coefficient; without it the C grid's grid-scale divergence noise grows at the
# pentagons under the jet and the R2B6/90 jet state goes non-finite after about 23 hours
DIVDAMP4 = 0.0025


# ------------------------------------------------------------------ operators
def gradient(g, psi):
    """O1: edge-normal gradient of a cell field (Nc, n) -> (Ne, n)."""
    return (psi[g.e2c[:, 1]] - psi[g.e2c[:, 0]]) / g.d_e[:, None]


def divergence(g, u):
    """O2: cell divergence of an edge-normal field (Ne, n) -> (Nc, n)."""
    acc = np.zeros((g.nc, u.shape[1]))
    for s in range(3):
        acc += (g.s_ce[:, s] * g.l_e[g.c2e[:, s]])[:, None] * u[g.c2e[:, s]]
    return acc / g.A_c[:, None]


def curl(g, vn):
    """O3: vertex relative vorticity (Nv, n), circulation counter-clockwise about v."""
    acc = np.zeros((g.nv, vn.shape[1]))
    for j in range(6):
        acc += (g.s_ve[:, j] * g.d_e[g.v2e[:, j]])[:, None] * vn[g.v2e[:, j]]
    return acc / g.A_v[:, None]


def tangential(g, vn):
    """O4: tangential velocity at edges from the 5-edge Perot stencil."""
    acc = np.zeros_like(vn)
    for j in range(5):
        acc += g.vt_w[:, j:j + 1] * vn[g.e2vt[:, j]]
    return acc


def cell_kinetic(g, Ke):
    """O5: cell kinetic energy from edge kinetic energies."""
    acc = np.zeros((g.nc, Ke.shape[1]))
    for s in range(3):
        acc += g.kin_w[:, s:s + 1] * Ke[g.c2e[:, s]]
    return acc


def vector_laplacian(g, vn):
    """O6: grad(div) - rot(curl), normal component at edges."""
    dl = divergence(g, vn)
    ze = curl(g, vn)
    return ((dl[g.e2c[:, 1]] - dl[g.e2c[:, 0]]) / g.d_e[:, None]
            - (ze[g.e2v[:, 1]] - ze[g.e2v[:, 0]]) / g.l_e[:, None])


def vertex_mean(g, f):
    """Mean of a cell field over the cells around each vertex (padding excluded)."""
    acc = np.zeros((g.nv, f.shape[1]))
    for j in range(5):
        acc += f[g.v2c[:, j]]
    acc += np.where(g.vdeg[:, None] == 6, f[g.v2c[:, 5]], 0.0)
    return acc / g.vdeg[:, None]


def edge_mean(g, f):
    """(f_c1 + f_c2) / 2 at edges."""
    return 0.5 * (f[g.e2c[:, 0]] + f[g.e2c[:, 1]])


def edge_upwind(g, f, vn):
    """UT (an option): the value of the cell the edge-normal flow comes from, f_c1 where
    vn >= 0 (flow from c1 to c2) else f_c2; used for theta_v in the heat flux."""
    return np.where(vn >= 0.0, f[g.e2c[:, 0]], f[g.e2c[:, 1]])


# ------------------------------------------------------------------ tendencies
def tendencies(g, v, s):
    """Explicit tendencies at state s: A_vn (Ne, N) at full levels and A_w (Nc, N+1),
    nonzero at interior half levels only."""
    N = v.N
    vn, w = s["vn"], s["w"]
    c1, c2 = g.e2c[:, 0], g.e2c[:, 1]
    v1, v2 = g.e2v[:, 0], g.e2v[:, 1]
    zeta = curl(g, vn)
    vt = tangential(g, vn)
    Ke = 0.5 * (vn * vn + vt * vt)
    Kc = cell_kinetic(g, Ke)
    vn_ie = to_half(v, vn)
    w_e = 0.5 * (w[c1] + w[c2])
    wbar = 0.5 * (w_e[:, :N] + w_e[:, 1:])
    zeta_e = 0.5 * (zeta[v1] + zeta[v2])
    A_vn = (-(Kc[c2] - Kc[c1]) / g.d_e[:, None]
            + (zeta_e + g.f_e[:, None]) * vt
            - wbar * (vn_ie[:, :N] - vn_ie[:, 1:]) / v.dz[None, :])

    w_v = vertex_mean(g, w)
    vt_ie = to_half(v, vt)
    a_e = (vn_ie * (w[c2] - w[c1]) / g.d_e[:, None]
           + vt_ie * (w_v[v2] - w_v[v1]) / g.l_e[:, None])
    hadv = cell_kinetic(g, a_e)                # same kappa weights as O5
    A_w = np.zeros((g.nc, N + 1))
    A_w[:, 1:N] = (-hadv[:, 1:N]
                   - w[:, 1:N] * (w[:, 0:N - 1] - w[:, 2:N + 1]) / (v.z_h[0:N - 1] - v.z_h[2:N + 1]))
    return A_vn, A_w


# ------------------------------------------------------------------ column solver
def thomas(lower, diag, upper, rhs):
    """Tridiagonal solve without pivoting, rows vectorised over columns.
    lower[:, 0] and upper[:, -1] are ignored."""
    n = diag.shape[1]
    cp = np.empty_like(diag)
    dp = np.empty_like(diag)
    cp[:, 0] = upper[:, 0] / diag[:, 0]
    dp[:, 0] = rhs[:, 0] / diag[:, 0]
    for i in range(1, n):
        m = diag[:, i] - lower[:, i] * cp[:, i - 1]
        cp[:, i] = upper[:, i] / m
        dp[:, i] = (rhs[:, i] - lower[:, i] * dp[:, i - 1]) / m
    x = np.empty_like(diag)
    x[:, n - 1] = dp[:, n - 1]
    for i in range(n - 2, -1, -1):
        x[:, i] = dp[:, i] - cp[:, i] * x[:, i + 1]
    return x


def column(g, v, s0, vn_new, A_w, rho_e, thv_e, dtau):
    """Vertically implicit update of (w, rho, theta_v, exner) for every cell, with
    coefficients frozen at s0 and horizontal mass/heat fluxes rho_e vn_new and
    rho_e thv_e vn_new. Returns the new fields and rho_ic of s0."""
    N = v.N
    rho, thv, ex, w = s0["rho"], s0["theta_v"], s0["exner"], s0["w"]
    F = rho_e * vn_new
    G = F * thv_e
    D_rho = divergence(g, F)
    D_th = divergence(g, G)
    Th = rho * thv
    rho_ic = to_half(v, rho)
    th_ic = to_half(v, thv)
    M = rho_ic * th_ic
    dz = v.dz[None, :]
    rho_x = rho - dtau * D_rho - dtau * (1.0 - BETA) * (rho_ic[:, :N] * w[:, :N] - rho_ic[:, 1:] * w[:, 1:]) / dz
    Th_x = Th - dtau * D_th - dtau * (1.0 - BETA) * (M[:, :N] * w[:, :N] - M[:, 1:] * w[:, 1:]) / dz
    ex_x = ex + (RD / CVD) * (ex / Th) * (Th_x - Th)
    dzh = v.dzh[None, 1:N]
    w_x = w[:, 1:N] + dtau * (A_w[:, 1:N]
                              - (1.0 - BETA) * CPD * th_ic[:, 1:N] * (ex[:, :N - 1] - ex[:, 1:N]) / dzh
                              - GRAV)
    a = dtau * BETA * CPD * th_ic[:, 1:N] / dzh
    gam = (RD / CVD) * (ex / Th) * dtau * BETA / dz
    lower = -a * gam[:, :N - 1] * M[:, :N - 1]
    diag = 1.0 + a * (gam[:, :N - 1] + gam[:, 1:N]) * M[:, 1:N]
    upper = -a * gam[:, 1:N] * M[:, 2:N + 1]
    rhs = w_x - a * (ex_x[:, :N - 1] - ex_x[:, 1:N])
    w_new = np.zeros((g.nc, N + 1))
    if N > 1:
        w_new[:, 1:N] = thomas(lower, diag, upper, rhs)
    w_new = w_new / (1.0 + dtau * v.rayleigh[None, :])
    q = M * w_new
    r = rho_ic * w_new
    Th_new = Th_x - dtau * BETA * (q[:, :N] - q[:, 1:]) / dz
    ex_new = ex_x - gam * (q[:, :N] - q[:, 1:])
    rho_new = rho_x - dtau * BETA * (r[:, :N] - r[:, 1:]) / dz
    return {"w": w_new, "rho": rho_new, "theta_v": Th_new / rho_new, "exner": ex_new}, rho_ic


def pressure_gradient(g, s):
    """cpd thv_e dpi/dn at edges."""
    return CPD * edge_mean(g, s["theta_v"]) * gradient(g, s["exner"])


# ------------------------------------------------------------------ diffusion
def vertex_vectors(g, vn):
    """Least-squares velocity 3-vectors at vertices (Nv, n, 3)."""
    u = np.zeros((g.nv, vn.shape[1], 3))
    for j in range(6):
        u += g.lsq_w[:, j, None, :] * vn[g.v2e[:, j]][:, :, None]
    return u


def smagorinsky_coefficient(g, vn):
    """K_h = cs^2 l_e d_e sqrt(D_T^2 + D_S^2) from quad-vertex velocities."""
    u = vertex_vectors(g, vn)
    u1, u2, u3, u4 = (u[g.e2q[:, j]] for j in range(4))
    n = g.n_e[:, None, :]
    t = g.t_e[:, None, :]
    d34 = u4 - u3
    d12 = u2 - u1
    DT = np.sum(d34 * n, axis=2) / g.L34[:, None] - np.sum(d12 * t, axis=2) / g.l_e[:, None]
    DS = np.sum(d34 * t, axis=2) / g.L34[:, None] + np.sum(d12 * n, axis=2) / g.l_e[:, None]
    return (CS_SMAG * CS_SMAG) * (g.l_e * g.d_e)[:, None] * np.sqrt(DT * DT + DS * DS)


def diffusion(g, v, s, dt, diff4=0.0):
    """Smagorinsky diffusion of vn and flux-form diffusion of theta_v (rho untouched,
    Exner adjusted at constant density). With diff4 > 0, fourth-order background
    diffusion of vn as well (BD, an option; ICON's background diffusion of order 4, the
    paper prints none): - diff4 Abar^2 L(L(vn)) with the O6 vector Laplacian L and the
    mean cell area Abar, applied once per step."""
    vn = s["vn"]
    Kh = smagorinsky_coefficient(g, vn)
    L1 = vector_laplacian(g, vn)
    vn_new = vn + dt * Kh * L1
    if diff4 > 0.0:
        abar = 4.0 * np.pi * R_EARTH * R_EARTH / g.nc
        vn_new = vn_new - (diff4 * abar * abar) * vector_laplacian(g, L1)
    thv = s["theta_v"]
    flux = (g.l_e[:, None] * Kh) * (thv[g.e2c[:, 1]] - thv[g.e2c[:, 0]]) / g.d_e[:, None]
    acc = np.zeros_like(thv)
    for sl in range(3):
        acc += g.s_ce[:, sl:sl + 1] * flux[g.c2e[:, sl]]
    dth = dt * acc / g.A_c[:, None]
    ex_new = s["exner"] * (1.0 + (RD / CVD) * dth / thv)
    out = dict(s)
    out.update(vn=vn_new, theta_v=thv + dth, exner=ex_new)
    return out, Kh


# ------------------------------------------------------------------ divergence damping (option)
def divergence_damping(g, vn, c4):
    """DD (fourth-order divergence damping, an option; ICON applies one in its corrector,
    the paper prints none): vn - c4 Abar^2 grad(div(grad(div vn))), Abar = 4 pi R^2 / Nc
    the mean cell area, with the O1/O2 operators. Rotational fields (div = 0) pass
    unchanged; a divergent mode of wavenumber k is scaled by about 1 - c4 Abar^2 k^4."""
    abar = 4.0 * np.pi * R_EARTH * R_EARTH / g.nc
    D = divergence(g, vn)
    L = divergence(g, gradient(g, D))
    return vn - (c4 * abar * abar) * gradient(g, L)


# ------------------------------------------------------------------ step and mass
def substep(g, v, s, dtau, nsub, acc, divdamp4=DIVDAMP4, upwind_theta=False):
    """One predictor-corrector substep; updates the accumulators in `acc`. With
    divdamp4 > 0 the corrector's vn^{n+1} is divergence-damped (DD) before its mass and
    heat fluxes are formed; with upwind_theta the heat fluxes carry the upwind theta_v (UT)
    instead of the centred one (the pressure gradient keeps the centred value)."""
    theta_e = (lambda st, vn: edge_upwind(g, st["theta_v"], vn)) if upwind_theta else \
        (lambda st, vn: edge_mean(g, st["theta_v"]))
    A_vn0, A_w0 = tendencies(g, v, s)
    vn_star = s["vn"] + dtau * (A_vn0 - pressure_gradient(g, s))
    cs, _ = column(g, v, s, vn_star, A_w0, edge_mean(g, s["rho"]), theta_e(s, vn_star), dtau)
    s_star = dict(cs, vn=vn_star)
    A_vn1, A_w1 = tendencies(g, v, s_star)
    vn_new = s["vn"] + dtau * (0.5 * (A_vn0 + A_vn1) - pressure_gradient(g, s_star))
    if divdamp4 > 0.0:
        vn_new = divergence_damping(g, vn_new, divdamp4)
    rho_e1 = edge_mean(g, s_star["rho"])
    cn, rho_ic0 = column(g, v, s, vn_new, 0.5 * (A_w0 + A_w1), rho_e1, theta_e(s_star, vn_new), dtau)
    acc["mflx"] += rho_e1 * vn_new / nsub
    acc["wflx"] += rho_ic0 * (BETA * cn["w"] + (1.0 - BETA) * s["w"]) / nsub
    return dict(cn, vn=vn_new)


def dycore_step(g, v, s, dt, nsub, divdamp4=DIVDAMP4, diff4=0.0, upwind_theta=False):
    """One step: nsub substeps of dt/nsub, then diffusion with dt. Returns
    (new state, accumulators {mflx (Ne,N), wflx (Nc,N+1)})."""
    dtau = dt / nsub
    acc = {"mflx": np.zeros((g.ne, v.N)), "wflx": np.zeros((g.nc, v.N + 1))}
    for _ in range(nsub):
        s = substep(g, v, s, dtau, nsub, acc, divdamp4, upwind_theta)
    s, _ = diffusion(g, v, s, dt, diff4)
    return s, acc


def global_mass(g, v, s):
    """Total air mass (kg): sum_c A_c sum_k dz_k rho_ck, pairwise summation."""
    col = np.sum(s["rho"] * v.dz[None, :], axis=1)
    return float(np.sum(g.A_c * col))
