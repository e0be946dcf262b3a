"""ES kernel and wall images (test infrastructure only).

phi(t; alpha, beta) = E(t)/Z with E(t) = exp(beta*(sqrt(1-(t/alpha)^2) - 1)) for |t| <= alpha
and 0 otherwise, Z = integral of E over [-alpha, alpha] (Eq. 54, Sec. III.E).  The 3D envelope
is the tensor product of phi in x, y and z (Eq. 53).  Near a no-slip wall the envelope is
replaced by itself minus its mirror image (Eq. 9), with the negative sign for both the monopole
and the dipole envelope (Sec. II).
"""

import numpy as np

from .params import BOTTOM_WALL, SLIT


def es_normalization(alpha, beta, n_gauss=128):
    """Z = int_{-alpha}^{alpha} E(t) dt (Eq. 54), by Gauss-Legendre quadrature after the
    substitution t = alpha*sin(theta), which gives the smooth integrand
    alpha * exp(beta*(cos(theta)-1)) * cos(theta) on [-pi/2, pi/2]."""
    x, w = np.polynomial.legendre.leggauss(n_gauss)
    theta = 0.5 * np.pi * x
    f = np.exp(beta * (np.cos(theta) - 1.0)) * np.cos(theta)
    return alpha * 0.5 * np.pi * np.dot(w, f)


def es(t, alpha, beta, Z=None):
    """phi(t; alpha, beta) of Eq. 54, vectorised over t; zero outside |t| <= alpha."""
    if Z is None:
        Z = es_normalization(alpha, beta)
    t = np.asarray(t, dtype=float)
    r = t / alpha
    inside = np.abs(r) <= 1.0
    arg = np.where(inside, 1.0 - r * r, 0.0)
    return np.where(inside, np.exp(beta * (np.sqrt(arg) - 1.0)), 0.0) / Z


def periodic_offset(xg, xp, L):
    """Minimum-image offset xg - xp in a periodic direction of period L."""
    d = np.asarray(xg) - xp
    return d - L * np.floor(d / L + 0.5)


def z_envelope(zc, zp, alpha, beta, mode, zmin, zmax, Z=None):
    """z factor of the wall envelope Delta^W (Eq. 9) at the nodes zc for a particle at zp.

    phi(zc - zp) - s_b*phi(zc - (2 zmin - zp)) - s_t*phi(zc - (2 zmax - zp)) with s_b = 1 for
    the bottom-wall and slit geometries, s_t = 1 for the slit (images in both walls,
    Appendix A), 0 otherwise.  An image term vanishes on [zmin, zmax] unless the particle is
    within alpha of that wall, so adding it always is the same as adding it below a threshold
    height z_im = alpha.
    """
    if Z is None:
        Z = es_normalization(alpha, beta)
    v = es(zc - zp, alpha, beta, Z)
    if mode in (BOTTOM_WALL, SLIT):
        v = v - es(zc - (2.0 * zmin - zp), alpha, beta, Z)
    if mode == SLIT:
        v = v - es(zc - (2.0 * zmax - zp), alpha, beta, Z)
    return v


# ---------------------------------------------------------------------------------------------
# Derivative kernels for the second torque route of Sec. III.D (spread the half-curl of the
# dipole envelope and interpolate the angular velocity with envelope derivatives, so that no extra
# transforms are needed).
# ---------------------------------------------------------------------------------------------

def es_derivative_cutoff(alpha, beta, iters=200):
    """|t| beyond which the derivative kernel is set to zero (footnote on the derivative route,
    Sec. III.D: truncate at the point where |phi'| is smallest before it blows up at the edge).

    With u = t/alpha and s = sqrt(1 - u^2), |phi'(t)| = beta |u| exp(beta (s - 1)) / (alpha s Z).
    Its logarithmic derivative in u vanishes where beta u^2 s = 1, i.e. beta v sqrt(1 - v) = 1
    with v = u^2.  v sqrt(1 - v) rises from 0 to 2/(3 sqrt 3) at v = 2/3 and falls back to 0 at
    v = 1, so for beta > 3 sqrt(3)/2 there are two roots: the smaller one is the maximum of |phi'|,
    the larger one (in (2/3, 1)) the minimum before the blow-up.  Returns alpha sqrt(v) for that
    larger root, found by bisection."""
    if not beta * (2.0 / 3.0) * np.sqrt(1.0 / 3.0) > 1.0:
        raise ValueError("beta too small: |phi'| has no interior minimum")
    lo, hi = 2.0 / 3.0, 1.0  # beta v sqrt(1-v) - 1 is > 0 at lo and < 0 at hi
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if beta * mid * np.sqrt(1.0 - mid) - 1.0 > 0.0:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-17:
            break
    return alpha * np.sqrt(0.5 * (lo + hi))


def es_derivative(t, alpha, beta, Z=None, cutoff=None):
    """phi'(t) = -beta t / (alpha^2 sqrt(1 - (t/alpha)^2)) phi(t) for |t| <= cutoff, zero beyond
    (the derivative of Eq. 54 with the truncation of es_derivative_cutoff)."""
    if Z is None:
        Z = es_normalization(alpha, beta)
    if cutoff is None:
        cutoff = es_derivative_cutoff(alpha, beta)
    t = np.asarray(t, dtype=float)
    inside = np.abs(t) <= cutoff
    r = np.where(inside, t / alpha, 0.0)
    s = np.sqrt(1.0 - r * r)
    return np.where(inside, -beta * r / (alpha * s) * np.exp(beta * (s - 1.0)) / Z, 0.0)


def z_envelope_derivative(zc, zp, alpha, beta, mode, zmin, zmax, Z=None, cutoff=None):
    """Derivative with respect to the node height zc of the z factor of Delta^W (Eq. 9):
    phi'(zc - zp) - s_b phi'(zc - (2 zmin - zp)) - s_t phi'(zc - (2 zmax - zp)).

    This is the exact derivative of the negatively imaged envelope.  Written as a fold-back of the
    part below the wall (the particle's own derivative kernel evaluated at the mirrored node
    2 zmin - zc), the folded term enters with a positive sign, since phi' is odd:
    -phi'(zc - (2 zmin - zp)) = +phi'((2 zmin - zc) - zp).  That is the sign the paper prescribes
    for the z derivative (footnote on the derivative route, Sec. III.D); it makes the whole
    gradient vanish for a particle on the wall."""
    if Z is None:
        Z = es_normalization(alpha, beta)
    if cutoff is None:
        cutoff = es_derivative_cutoff(alpha, beta)
    v = es_derivative(zc - zp, alpha, beta, Z, cutoff)
    if mode in (BOTTOM_WALL, SLIT):
        v = v - es_derivative(zc - (2.0 * zmin - zp), alpha, beta, Z, cutoff)
    if mode == SLIT:
        v = v - es_derivative(zc - (2.0 * zmax - zp), alpha, beta, Z, cutoff)
    return v
