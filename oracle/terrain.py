"""Terrain-following height coordinate over topography for the oracle (FP64, plain numpy).

TEST INFRASTRUCTURE ONLY; the product library never imports this module.

The paper's atmosphere uses a terrain-following hybrid height coordinate (Sec.
"Current State of the Art") and prints none of its formulas. The readings below
follow the published structure of ICON's coordinate and metric terms, written
out so that they can be checked by eye:

R-Z1 Levels (SLEVE type, one decay scale s_d = 4000 m): half level h of cell c at
     z_ch = zeta_h + hs_c b_h, b_h = sinh((z_top - zeta_h)/s_d) / sinh(z_top/s_d),
     zeta_h the flat levels of R-V1. b = 1 at the ground (levels follow the
     surface) and 0 at the lid (flat top). Full levels lie midway: zf = zeta_f +
     hs bf with bf_k = (b_k + b_{k+1})/2; layer thickness dz_ck = (zeta_k -
     zeta_{k+1}) + hs_c (b_k - b_{k+1}); centre spacing dzh_ch = zf_{c,h-1} -
     zf_{c,h}. An edge is a column at hs_e = (hs_c1 + hs_c2)/2 and a vertex one at
     the mean of its cells' hs, so every spacing follows the same formula.
R-Z2 Topography: hs = h0 exp(-(r/a)^2), r the great-circle distance to 90E 30N.
R-Z3 Horizontal derivatives run along the coordinate surfaces; only the pressure
     gradient carries the metric correction:
       (d pi/dn)_z = (pi'_c2 - pi'_c1)/d_e - sn_e,k (d pi'/dz)_e,k,
     pi' = pi - pi_ref(zf), pi_ref(z) = exp(-g z / (cpd 250 K)) (isothermal rest
     state, analytic), sn_e,k = (zf_c2,k - zf_c1,k)/d_e the slope of the full
     level, (d pi'/dz)_e the mean of the two cells' vertical derivatives
     (pi'_ic,k - pi'_ic,k+1)/dz_ck with pi'_ic the half-level interpolant, and
     (pi'_0 - pi'_1)/dzh_1, (pi'_{N-2} - pi'_{N-1})/dzh_{N-1} at the top and
     bottom full levels. Kinetic-energy gradient, vorticity and the horizontal
     advection of w take none (as ICON does).
R-Z4 Contravariant vertical velocity w_con = w - wcc, with the correction formed
     in ICON's order: at edges and full levels X_e,k = vn sn_e,k + vt st_e,k
     (full-level slopes: sn from the two cells, st = (zf_v2,k - zf_v1,k)/l_e from
     the two vertices), at cells X_c = sum_e kappa_ce X_e (the O5 weights), then
     interpolated to the interior half levels with the cell's own weights; at the
     ground wcc = sum_e kappa_ce (vn sn + vt st) with the lowest full level's wind
     and the surface slopes. w_con replaces w in the vertical advection of vn and
     w and in the vertical mass and heat fluxes; w_con = 0 at the lid and at the
     ground (free slip: the w a column leaves at the ground is its stage's wcc).
R-Z5 Flux form with layer thickness: the horizontal mass and heat fluxes carry
     dz_e (rho_e vn dz_e), each cell's budget is divided by its dz_c, and the
     vertical implicit solve is R-S's with each cell's own spacings. The
     step-mean fluxes are rho_e vn dz_e and rho_ic (beta w^{n+1} + (1 - beta)
     w^n - wcc).
R-Z6 A stage's wcc is that of the state its tendencies are taken at (S^n in the
     predictor, S* in the corrector). Rayleigh damping keeps the flat heights
     zeta_h. Diffusion and divergence damping act along coordinate surfaces.
With hs = 0 every formula reduces to the flat step of oracle.dycore.
"""
import numpy as np

from .grid import R_EARTH
from .state import GRAV, RD, CPD, CVD, to_half_w
from .dycore import (BETA, DIVDAMP4, curl, tangential, cell_kinetic, vertex_mean, edge_mean, edge_upwind,
                     divergence, thomas, diffusion, divergence_damping)

DECAY_M = 4000.0                    # SLEVE decay scale
T_REF = 250.0                       # temperature of the reference Exner profile
MOUNTAIN_LON, MOUNTAIN_LAT = np.deg2rad(90.0), np.deg2rad(30.0)


class Terrain:
    pass


def mountain(x, h0, radius_m):
    """R-Z2: Gaussian mountain h0 exp(-(r/a)^2) at unit positions x (n, 3)."""
    xc = np.array([np.cos(MOUNTAIN_LAT) * np.cos(MOUNTAIN_LON),
                   np.cos(MOUNTAIN_LAT) * np.sin(MOUNTAIN_LON), np.sin(MOUNTAIN_LAT)])
    cr = np.cross(x, xc[None, :])
    r = R_EARTH * np.arctan2(np.sqrt(np.sum(cr * cr, axis=1)), x @ xc)
    return h0 * np.exp(-(r / radius_m) ** 2)


def decay(v, decay_m=DECAY_M):
    """R-Z1: b at the half levels of the flat grid v."""
    return np.sinh((v.z_top - v.z_h) / decay_m) / np.sinh(v.z_top / decay_m)


def _column(v, b, hs):
    """Heights and spacings of columns standing on hs (n,): half and full heights,
    layer thickness, centre spacing and the upper weight of the half-level interpolant."""
    N = v.N
    bf = 0.5 * (b[:-1] + b[1:])
    zh = v.z_h[None, :] + hs[:, None] * b[None, :]
    zf = v.z_f[None, :] + hs[:, None] * bf[None, :]
    dz = v.dz[None, :] + hs[:, None] * (b[:-1] - b[1:])[None, :]
    dzh = np.zeros((len(hs), N + 1))
    dzh[:, 1:N] = (v.z_f[:-1] - v.z_f[1:])[None, :] + hs[:, None] * (bf[:-1] - bf[1:])[None, :]
    wu = np.zeros((len(hs), N + 1))
    wu[:, 1:N] = dz[:, 1:] / (dz[:, :-1] + dz[:, 1:])
    return zh, zf, dz, dzh, wu


def terrain_geometry(g, v, hs, decay_m=DECAY_M):
    """Metric fields of the terrain-following grid over cell topography hs (Nc,)."""
    t = Terrain()
    N = v.N
    t.hs = np.asarray(hs, dtype=np.float64)
    t.b = decay(v, decay_m)
    t.bf = 0.5 * (t.b[:-1] + t.b[1:])
    t.zh_c, t.zf_c, t.dz_c, t.dzh_c, t.wu_c = _column(v, t.b, t.hs)
    c1, c2 = g.e2c[:, 0], g.e2c[:, 1]
    t.hs_e = 0.5 * (t.hs[c1] + t.hs[c2])
    _, t.zf_e, t.dz_e, _, t.wu_e = _column(v, t.b, t.hs_e)
    t.hs_v = vertex_mean(g, t.hs[:, None])[:, 0]
    # slopes of the coordinate surfaces at edges: the zeta_h of the two columns cancel
    dn = (t.hs[c2] - t.hs[c1]) / g.d_e
    dt = (t.hs_v[g.e2v[:, 1]] - t.hs_v[g.e2v[:, 0]]) / g.l_e
    t.sn_s, t.st_s = dn, dt                            # at the ground (b = 1)
    t.sn_f = dn[:, None] * t.bf[None, :]               # full levels
    t.st_f = dt[:, None] * t.bf[None, :]
    t.ex_ref = np.exp(-GRAV * t.zf_c / (CPD * T_REF))
    t.N = N
    return t


# ------------------------------------------------------------------ metric terms
def vertical_derivative(t, f):
    """R-Z3: d f/dz at full levels of every cell, from the half-level interpolant;
    one-sided at the top and bottom full levels."""
    N = t.N
    d = np.zeros_like(f)
    if N < 2:
        return d
    fi = to_half_w(t.wu_c, f)
    d[:, 1:N - 1] = (fi[:, 1:N - 1] - fi[:, 2:N]) / t.dz_c[:, 1:N - 1]
    d[:, 0] = (f[:, 0] - f[:, 1]) / t.dzh_c[:, 1]
    d[:, N - 1] = (f[:, N - 2] - f[:, N - 1]) / t.dzh_c[:, N - 1]
    return d


def exner_gradient(g, t, ex):
    """R-Z3: horizontal gradient of Exner at constant height, normal to each edge."""
    c1, c2 = g.e2c[:, 0], g.e2c[:, 1]
    ep = ex - t.ex_ref
    dpz = vertical_derivative(t, ep)
    return (ep[c2] - ep[c1]) / g.d_e[:, None] - t.sn_f * (0.5 * (dpz[c1] + dpz[c2]))


def pressure_gradient(g, t, s):
    """cpd thv_e (d pi/dn)_z at edges."""
    return CPD * edge_mean(g, s["theta_v"]) * exner_gradient(g, t, s["exner"])


def contravariant_correction(g, t, vn, vt):
    """R-Z4: wcc at cells and half levels (Nc, N+1) for the edge velocities vn, vt."""
    N = t.N
    X = cell_kinetic(g, vn * t.sn_f + vt * t.st_f)
    wcc = to_half_w(t.wu_c, X)
    wcc[:, 0] = 0.0
    ground = vn[:, N - 1:N] * t.sn_s[:, None] + vt[:, N - 1:N] * t.st_s[:, None]
    wcc[:, N] = cell_kinetic(g, ground)[:, 0]
    return wcc


def tendencies(g, v, t, s):
    """A_vn (Ne, N), A_w (Nc, N+1) and wcc (Nc, N+1) at state s (R-Z3, R-Z4)."""
    N = v.N
    vn, w = s["vn"], s["w"]
    c1, c2 = g.e2c[:, 0], g.e2c[:, 1]
    v1, v2 = g.e2v[:, 0], g.e2v[:, 1]
    zeta = curl(g, vn)
    vt = tangential(g, vn)
    Kc = cell_kinetic(g, 0.5 * (vn * vn + vt * vt))
    vn_ie = to_half_w(t.wu_e, vn)
    vt_ie = to_half_w(t.wu_e, vt)
    wcc = contravariant_correction(g, t, vn, vt)
    wcon = w - wcc
    wcon[:, 0] = 0.0
    wcon[:, N] = 0.0
    wcon_e = 0.5 * (wcon[c1] + wcon[c2])
    wbar = 0.5 * (wcon_e[:, :N] + wcon_e[:, 1:])
    zeta_e = 0.5 * (zeta[v1] + zeta[v2])
    A_vn = (-(Kc[c2] - Kc[c1]) / g.d_e[:, None]
            + (zeta_e + g.f_e[:, None]) * vt
            - wbar * (vn_ie[:, :N] - vn_ie[:, 1:]) / t.dz_e)

    w_v = vertex_mean(g, w)
    a_e = (vn_ie * (w[c2] - w[c1]) / g.d_e[:, None]
           + vt_ie * (w_v[v2] - w_v[v1]) / g.l_e[:, None])
    hadv = cell_kinetic(g, a_e)
    A_w = np.zeros((g.nc, N + 1))
    A_w[:, 1:N] = (-hadv[:, 1:N]
                   - wcon[:, 1:N] * (w[:, 0:N - 1] - w[:, 2:N + 1]) / (t.zh_c[:, 0:N - 1] - t.zh_c[:, 2:N + 1]))
    return A_vn, A_w, wcc


# ------------------------------------------------------------------ column solver
def column(g, v, t, s0, vn_new, A_w, rho_e, thv_e, wcc, dtau):
    """R-Z5: the vertically implicit update of oracle.dycore.column on the terrain-following
    grid, with thickness-weighted horizontal fluxes and the contravariant explicit flux.
    Returns the new fields (w at the ground = wcc there) and rho_ic of s0."""
    N = v.N
    rho, thv, ex, w = s0["rho"], s0["theta_v"], s0["exner"], s0["w"]
    F = rho_e * vn_new * t.dz_e
    G = F * thv_e
    D_rho = divergence(g, F)
    D_th = divergence(g, G)
    Th = rho * thv
    rho_ic = to_half_w(t.wu_c, rho)
    th_ic = to_half_w(t.wu_c, thv)
    M = rho_ic * th_ic
    ve = (1.0 - BETA) * w - wcc                        # explicit part of the contravariant velocity
    ve[:, 0] = 0.0
    ve[:, N] = 0.0
    fr = rho_ic * ve
    ft = M * ve
    dz = t.dz_c
    rho_x = rho - dtau * (D_rho + fr[:, :N] - fr[:, 1:]) / dz
    Th_x = Th - dtau * (D_th + ft[:, :N] - ft[:, 1:]) / dz
    ex_x = ex + (RD / CVD) * (ex / Th) * (Th_x - Th)
    dzh = t.dzh_c[:, 1:N]
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
    w_out = w_new.copy()
    w_out[:, N] = wcc[:, N]
    return {"w": w_out, "rho": rho_new, "theta_v": Th_new / rho_new, "exner": ex_new}, rho_ic, w_new


# ------------------------------------------------------------------ step and mass
def substep(g, v, t, s, dtau, nsub, acc, divdamp4=DIVDAMP4, upwind_theta=False):
    """One predictor-corrector substep on the terrain-following grid (R-Z6)."""
    theta_e = (lambda st, vn: edge_upwind(g, st["theta_v"], vn)) if upwind_theta else \
        (lambda st, vn: edge_mean(g, st["theta_v"]))
    A_vn0, A_w0, wcc0 = tendencies(g, v, t, s)
    vn_star = s["vn"] + dtau * (A_vn0 - pressure_gradient(g, t, s))
    cs, _, _ = column(g, v, t, s, vn_star, A_w0, edge_mean(g, s["rho"]), theta_e(s, vn_star), wcc0, dtau)
    s_star = dict(cs, vn=vn_star)
    A_vn1, A_w1, wcc1 = tendencies(g, v, t, s_star)
    vn_new = s["vn"] + dtau * (0.5 * (A_vn0 + A_vn1) - pressure_gradient(g, t, s_star))
    if divdamp4 > 0.0:
        vn_new = divergence_damping(g, vn_new, divdamp4)
    rho_e1 = edge_mean(g, s_star["rho"])
    cn, rho_ic0, w_flux = column(g, v, t, s, vn_new, 0.5 * (A_w0 + A_w1), rho_e1, theta_e(s_star, vn_new),
                                 wcc1, dtau)
    N = v.N
    wc = BETA * w_flux + (1.0 - BETA) * s["w"] - wcc1
    wc[:, 0] = 0.0
    wc[:, N] = 0.0
    acc["mflx"] += rho_e1 * vn_new * t.dz_e / nsub
    acc["wflx"] += rho_ic0 * wc / nsub
    return dict(cn, vn=vn_new)


def terrain_step(g, v, t, s, dt, nsub, divdamp4=DIVDAMP4, diff4=0.0, upwind_theta=False):
    """One step on the terrain-following grid: nsub substeps of dt/nsub, then diffusion
    with dt. Returns (new state, accumulators {mflx (Ne,N), wflx (Nc,N+1)})."""
    dtau = dt / nsub
    acc = {"mflx": np.zeros((g.ne, v.N)), "wflx": np.zeros((g.nc, v.N + 1))}
    for _ in range(nsub):
        s = substep(g, v, t, s, dtau, nsub, acc, divdamp4, upwind_theta)
    s, _ = diffusion(g, v, s, dt, diff4)
    return s, acc


def terrain_mass(g, t, s):
    """Total air mass (kg): sum_c A_c sum_k dz_ck rho_ck."""
    return float(np.sum(g.A_c * np.sum(s["rho"] * t.dz_c, axis=1)))
