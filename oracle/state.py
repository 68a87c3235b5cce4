"""Vertical grid, constants and initial states for the oracle (test infrastructure, FP64).

TEST INFRASTRUCTURE ONLY; the product library never imports this module.

The paper fixes only that the atmosphere uses a nonhydrostatic formulation with a
terrain-following hybrid height coordinate, 90 levels at 10 km and 1.25 km
(Sec. "Current State of the Art"; Table 2). The definitions below are the
builder's readings:

R-C   Constants: g = 9.80665, Rd = 287.04, cpd = 1004.64, cvd = cpd - Rd, p0 = 1e5 Pa.
R-V1  Flat bottom, rigid lid z_top; half level i = 0..N (top to bottom) at
      z_top (exp(s (N-i)/N) - 1) / (exp(s) - 1). Defaults: N >= 60 -> z_top 75 km,
      s 5.5, damping base 45 km; otherwise z_top 30 km, s 2, damping base 20 km.
      Full level k (0-based) lies between half levels k and k+1.
R-V2  Rayleigh damping of w above z_d: w <- w / (1 + dtau r(z)),
      r = 0.05 sin^2(pi/2 (z - z_d)/(z_top - z_d)) 1/s.
R-I1  theta_v is taken from the analytic state; Exner at the lowest full level
      from the analytic pressure, then integrated upward in discrete hydrostatic
      balance  pi_{k-1} = pi_k - g dzh_k / (cpd theta_ic,k); rho from the state
      equation rho = p0 pi^(cvd/Rd) / (Rd theta_v).
R-I2  Noise: theta_v += a (2U - 1), U the draw number (cell * N + k) of the
      SplitMix64 stream of the seed, pi held fixed, rho recomputed.
Cases: 0 rest (isothermal 250 K); 1 solid-body rotation u = u0 cos(phi) in
      gradient balance, ln p = ln p0 - g z/(Rd T0) - (R Omega u0 + u0^2/2) sin^2(phi)/(Rd T0);
      2 balanced midlatitude jet (self-derived, see `jet_state`) plus a Gaussian
      zonal-wind bump of 1 m/s centred at 20E 40N with radius R/10;
      3 case 2 with the bump's amplitude in U(0.5, 2) m/s and its centre uniform
      on the sphere, drawn from a per-member seed.
"""
import numpy as np

from .grid import R_EARTH, OMEGA

GRAV = 9.80665
RD = 287.04
CPD = 1004.64
CVD = CPD - RD
P0 = 1.0e5

CASE_REST, CASE_SBR, CASE_JET, CASE_MEMBER = 0, 1, 2, 3

GOLDEN = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


# ------------------------------------------------------------------ SplitMix64
def splitmix64(seed, index):
    """Output number `index` (0-based) of the SplitMix64 generator (Steele, Lea, Flood 2014)
    started at `seed`: the state advances by the golden-ratio constant, then is mixed.
    `index` may be a numpy integer array; returns uint64."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (idx + np.uint64(1)) * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed, index):
    """53-bit uniform in [0, 1) from SplitMix64 output `index`."""
    return (splitmix64(seed, index) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def member_params(seed, member):
    """Case 3: (member seed, bump amplitude m/s, centre lon, centre lat) of one member."""
    ms = int(splitmix64(seed, member))
    amp = 0.5 + 1.5 * float(uniform01(ms, 0))
    lon = 2.0 * np.pi * float(uniform01(ms, 1))
    lat = float(np.arcsin(2.0 * float(uniform01(ms, 2)) - 1.0))
    return ms, amp, lon, lat


# ------------------------------------------------------------------ vertical grid
class Vertical:
    pass


def vertical_grid(nlev, top_m=None, stretch_s=None, damp_m=None):
    """R-V1 stretched height coordinate with the derived spacings and interpolation weights."""
    N = nlev
    if top_m is None:
        top_m = 75000.0 if N >= 60 else 30000.0
    if stretch_s is None:
        stretch_s = 5.5 if N >= 60 else 2.0
    if damp_m is None:
        damp_m = 45000.0 if N >= 60 else 20000.0
    v = Vertical()
    v.N, v.z_top, v.s, v.z_d = N, top_m, stretch_s, damp_m
    i = np.arange(N + 1, dtype=np.float64)
    v.z_h = top_m * (np.exp(stretch_s * (N - i) / N) - 1.0) / (np.exp(stretch_s) - 1.0)
    v.z_h[N] = 0.0
    v.z_h[0] = top_m
    v.dz = v.z_h[:-1] - v.z_h[1:]                      # layer thickness, full level k
    v.z_f = 0.5 * (v.z_h[:-1] + v.z_h[1:])
    v.dzh = np.zeros(N + 1)                            # full-level centre spacing at half level
    v.dzh[1:N] = v.z_f[:-1] - v.z_f[1:]
    v.wu = np.zeros(N + 1)                             # weight of the upper full level at half level
    v.wu[1:N] = v.dz[1:] / (v.dz[:-1] + v.dz[1:])
    # Rayleigh coefficient at half levels (0 at and below z_d)
    zz = v.z_h
    r = np.where(zz > damp_m, 0.05 * np.sin(0.5 * np.pi * (zz - damp_m) / (top_m - damp_m)) ** 2, 0.0)
    v.rayleigh = r
    return v


def to_half(v, f):
    """Linear-in-z interpolation of a full-level field (n, N) to half levels (n, N+1);
    the top and bottom half levels take the adjacent full value."""
    return to_half_w(v.wu, f)


def to_half_w(wu, f):
    """to_half with the weights of the upper full level given per half level (N+1,)
    or per point and half level (n, N+1) (a terrain-following grid)."""
    N = f.shape[1]
    out = np.empty((f.shape[0], N + 1))
    out[:, 0] = f[:, 0]
    out[:, N] = f[:, N - 1]
    out[:, 1:N] = wu[..., 1:N] * f[:, :N - 1] + (1.0 - wu[..., 1:N]) * f[:, 1:N]
    return out


# ------------------------------------------------------------------ analytic states
def _latlon_basis(x):
    """cos(phi), sin(phi), zonal and meridional unit vectors at unit positions x (n, 3)."""
    cphi = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2)
    sphi = x[:, 2]
    safe = np.where(cphi > 0.0, cphi, 1.0)
    e_lam = np.stack([-x[:, 1] / safe, x[:, 0] / safe, np.zeros(len(x))], axis=1)
    e_phi = np.stack([-sphi * x[:, 0] / safe, -sphi * x[:, 1] / safe, cphi], axis=1)
    return cphi, sphi, e_lam, e_phi


def heights(z):
    """Heights as a (1, m) row shared by every point, or the (n, m) heights of each point
    (a terrain-following grid)."""
    z = np.asarray(z, dtype=np.float64)
    return z if z.ndim == 2 else z[None, :]


def sbr_state(x, z, u0=20.0, T0=250.0):
    """Solid-body rotation: (ln p, T, u_lambda) at unit positions x (n,3), heights z (m,)
    or (n, m)."""
    cphi, sphi, _, _ = _latlon_basis(x)
    Z = heights(z)
    lnp = (np.log(P0) - GRAV * Z / (RD * T0)
           - ((R_EARTH * OMEGA * u0 + 0.5 * u0 * u0) * sphi[:, None] ** 2) / (RD * T0))
    T = np.full(lnp.shape, T0)
    u = (u0 * cphi)[:, None] + np.zeros(lnp.shape)
    return lnp, T, u


JET_ZJ = 10000.0        # jet level, m
JET_HJ = 10000.0        # vertical half-width of the jet, m
JET_PHI0 = 4.0 / 15.0   # shift of Phi: -Phi(equator) = Phi(pole) = 4/15
JET_T = 288.0           # temperature of the background and of the jet level, K
JET_U = 35.0            # jet speed at 45 deg latitude at the jet level, m/s


def jet_B():
    """Amplitude B such that u = 35 m/s at 45 deg latitude at the jet level.

    At z_j, S = 1 and S' = 0 so T = JET_T; the gradient-wind relation divided by
    sin(phi) reads u^2 / (R cos phi) + 2 Omega u = (Rd T / R) B S 4 cos^2 sin^2,
    and 4 cos^2 sin^2 = 1 at 45 degrees."""
    c45 = np.sqrt(0.5)
    return (JET_U * JET_U / (R_EARTH * c45) + 2.0 * OMEGA * JET_U) * R_EARTH / (RD * JET_T)


def jet_state(x, z):
    """Balanced midlatitude jet (self-derived stand-in for the baroclinic-wave state):

    ln p = ln p0 - z/H0 - B S(z) Phi(phi), H0 = Rd T_j / g,
    S(z) = exp(-((z - z_j)/h_j)^2), Phi = 4/15 - 4 (cos^3/3 - cos^5/5),
    T from hydrostatic balance: T = g / (Rd (1/H0 + B S'(z) Phi)),
    u from gradient-wind balance  u^2 tan(phi)/R + 2 Omega sin(phi) u = -(Rd T/R) d(ln p)/dphi,
    taking the root continuous with geostrophy (u = 0 at equator and poles).

    The constant 4/15 centres Phi (-4/15 at the equator, +4/15 at the poles): it adds a
    function of height alone to ln p, which leaves the wind's forcing dPhi/dphi unchanged
    and halves the largest temperature perturbation. With it and h_j = 10 km the state is
    statically stable everywhere (N^2 >= 1.4e-4 1/s^2); without it, or with h_j = 8 km,
    the lapse rate below the jet core exceeds the dry adiabatic one between about 20 and
    45 degrees latitude (N^2 < 0 near 9 km) and the state overturns within hours."""
    cphi, sphi, _, _ = _latlon_basis(x)
    B = jet_B()
    H0 = RD * JET_T / GRAV
    Z = heights(z)
    S = np.exp(-((Z - JET_ZJ) / JET_HJ) ** 2)
    dS = -2.0 * (Z - JET_ZJ) / (JET_HJ * JET_HJ) * S
    Phi = -4.0 * (cphi ** 3 / 3.0 - cphi ** 5 / 5.0) + JET_PHI0
    lnp = np.log(P0) - Z / H0 - B * S * Phi[:, None]
    T = GRAV / (RD * (1.0 / H0 + B * dS * Phi[:, None]))
    # divided by sin(phi): a u^2 + b u = c with a = 1/(R cos), b = 2 Omega,
    # c = (Rd T / R) B S * 4 cos^2 sin^2 (= -(Rd T/R) dlnp/dphi / sin)
    c = (RD * T / R_EARTH) * B * S * (4.0 * cphi ** 2 * sphi ** 2)[:, None]
    a = np.where(cphi > 1e-12, 1.0 / (R_EARTH * np.where(cphi > 1e-12, cphi, 1.0)), 0.0)[:, None]
    b = 2.0 * OMEGA
    u = 2.0 * c / (b + np.sqrt(b * b + 4.0 * a * c))
    return lnp, T, u


def _bump(x, amp, lon_c, lat_c):
    """amp * exp(-(r / (R/10))^2), r the great-circle distance to (lon_c, lat_c)."""
    xc = np.array([np.cos(lat_c) * np.cos(lon_c), np.cos(lat_c) * np.sin(lon_c), np.sin(lat_c)])
    cr = np.cross(x, xc[None, :])
    r = R_EARTH * np.arctan2(np.sqrt(np.sum(cr * cr, axis=1)), x @ xc)
    return amp * np.exp(-(r / (R_EARTH / 10.0)) ** 2)


def case_defaults(case):
    """Default theta_v noise amplitude (K) per case."""
    return {CASE_REST: 0.0, CASE_SBR: 0.01, CASE_JET: 0.0, CASE_MEMBER: 0.0}[case]


def init_state(g, v, seed, case, noise_K=None, member=0, terrain=None):
    """Initial prognostic state {vn (Ne,N), w (Nc,N+1), rho, theta_v, exner (Nc,N)}.
    With a terrain-following grid (`terrain`, from oracle.terrain.terrain_geometry) the
    analytic state is taken at each cell's and edge's own full-level heights and the
    hydrostatic integration runs with each cell's own spacings."""
    N = v.N
    if noise_K is None:
        noise_K = case_defaults(case)
    seed_used = seed
    bump = None
    if case == CASE_JET:
        bump = (1.0, np.deg2rad(20.0), np.deg2rad(40.0))
    elif case == CASE_MEMBER:
        ms, amp, lon, lat = member_params(seed, member)
        seed_used = ms
        bump = (amp, lon, lat)

    def analytic(x, z):
        if case == CASE_REST:
            lnp = np.log(P0) - GRAV * heights(z) / (RD * 250.0) + 0.0 * x[:, :1]
            return lnp, np.full(lnp.shape, 250.0), np.zeros(lnp.shape)
        if case == CASE_SBR:
            return sbr_state(x, z)
        if case in (CASE_JET, CASE_MEMBER):
            return jet_state(x, z)
        raise ValueError("unknown case")

    kappa = RD / CPD
    # scalars at cell centres, full levels
    zc = v.z_f if terrain is None else terrain.zf_c
    ze = v.z_f if terrain is None else terrain.zf_e
    lnp, T, _ = analytic(g.x_c, zc)
    ex_an = np.exp(kappa * (lnp - np.log(P0)))
    thv = T / ex_an
    ex = np.empty_like(thv)
    ex[:, N - 1] = ex_an[:, N - 1]
    th_ic = to_half(v, thv) if terrain is None else to_half_w(terrain.wu_c, thv)
    dzh = v.dzh[None, :] if terrain is None else terrain.dzh_c
    for k in range(N - 1, 0, -1):
        ex[:, k - 1] = ex[:, k] - GRAV * dzh[:, k] / (CPD * th_ic[:, k])
    if noise_K > 0.0:
        idx = np.arange(g.nc, dtype=np.uint64)[:, None] * np.uint64(N) + np.arange(N, dtype=np.uint64)[None, :]
        thv = thv + noise_K * (2.0 * uniform01(seed_used, idx) - 1.0)
    rho = P0 * ex ** (CVD / RD) / (RD * thv)

    # wind at edge midpoints
    _, _, u = analytic(g.x_e, ze)
    if bump is not None:
        u = u + _bump(g.x_e, *bump)[:, None]
    _, _, e_lam, _ = _latlon_basis(g.x_e)
    vn = u * np.sum(e_lam * g.n_e, axis=1)[:, None]
    w = np.zeros((g.nc, N + 1))
    return {"vn": vn, "w": w, "rho": rho, "theta_v": thv, "exner": ex}


def exner_ref(v):
    """Reference Exner of an isothermal 250 K rest column, same discrete integration."""
    lnp = np.log(P0) - GRAV * v.z_f / (RD * 250.0)
    ex_an = np.exp((RD / CPD) * (lnp - np.log(P0)))
    thv = 250.0 / ex_an
    N = v.N
    ex = np.empty(N)
    ex[N - 1] = ex_an[N - 1]
    th_ic = to_half(v, thv[None, :])[0]
    for k in range(N - 1, 0, -1):
        ex[k - 1] = ex[k] - GRAV * v.dzh[k] / (CPD * th_ic[k])
    return ex
