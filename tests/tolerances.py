"""Tolerances derived from the arithmetic, shared by the parity tests."""
EPS = 2.0 ** -52
GRAV = 9.80665


def w_bound(dt, nsub, nsteps):
    """Absolute RMS bound (m/s) on the GPU-oracle difference of w after nsteps steps.

    w is the residual of a balance between the vertical pressure-gradient force and
    gravity, each of size g * dtau per substep, so rounding differences of order
    eps * g * dtau per substep are not reduced by the (small) size of w itself: a
    one-ulp perturbation of the oracle's own input moves its w by ~1e-10 relative
    while every other field moves by O(eps) (test_w_conditioning). Bound:
    10 eps g dtau per substep, summed over the substeps."""
    return 10.0 * EPS * GRAV * (dt / nsub) * nsub * nsteps


EPS32 = 2.0 ** -23
U_MAX = 35.0            # largest wind speed of the analytic states, m/s


def thermo_bound_mixed(dt, nsub, nsteps, d_min):
    """Relative L2 bound for rho, theta_v and Exner of the mixed step against FP64.

    The horizontal mass and heat fluxes are FP32 (l_e rho_e vn): each flux carries a
    relative rounding of eps32, and the divergence of a nearly non-divergent flow does
    not cancel it, so each stage changes rho and Theta by up to eps32 times the
    advective Courant number dtau U / d. Bound: 10 times that per stage, summed over the
    2 stages of every substep."""
    return 10.0 * EPS32 * (dt / nsub) * U_MAX / d_min * 2 * nsub * nsteps


def w_bound_mixed(dt, nsub, nsteps):
    """Absolute RMS bound (m/s) for w of the mixed step: the FP32 advective tendency and
    the FP32 shadows of the provisional state perturb the FP64 w solve by about eps32
    times the size of the terms it balances (g * dtau per substep)."""
    return 10.0 * EPS32 * GRAV * (dt / nsub) * nsub * nsteps
