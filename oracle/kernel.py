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
