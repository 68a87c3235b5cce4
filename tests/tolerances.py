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
