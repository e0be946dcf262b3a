"""Particle <-> grid transfer with the ES envelope (test infrastructure only).

Spreading is step 1 of the algorithm in Sec. III.D: the force density of Eq. 7 sampled at the
grid nodes, f_i(x_g) = sum_j F_{j,i} Delta^W_M(x_g - r_j), and the torque field
t_i(x_g) = sum_j tau_{j,i} Delta^W_D(x_g - r_j) whose half-curl is added in Fourier-Chebyshev
space (the first of the two torque routes described after the algorithm in Sec. III.D).
Interpolation is step 8: the envelope integrals of Eqs. 10-11 evaluated with the trapezoid rule
in x, y (weight h^2) and Clenshaw-Curtis weights in z.

The second torque route of Sec. III.D (spread_curl, interpolate_curl) puts the half-curl of the
dipole envelope on the grid directly, (1/2) curl(tau Delta^W_D) = (1/2) grad Delta^W_D x tau, and
returns Omega_j = (1/2) h^2 sum_g w_c u(x_g) x grad Delta^W_D(x_g - r_j), which is Eq. 11 after
moving the curl onto the envelope by parts (no boundary term: u vanishes on a no-slip wall and
envelopes never reach an open boundary).  The gradient uses the truncated kernel derivative of
kernel.es_derivative in the differentiated direction and phi in the other two.

Grids are arrays of shape (3, nz, ny, nx): field, Chebyshev node (c = 0 at the top), y, x.
"""

import numpy as np

from . import cheb
from .kernel import (es, es_derivative, es_derivative_cutoff, es_normalization, periodic_offset, z_envelope,
                     z_envelope_derivative)
from .params import BOTTOM_WALL, FREE, SLIT


def kernel_params(p, which):
    """(alpha, beta) of the monopole ('M') or dipole ('D') envelope; alpha = m h / 2 (Sec. III.E)."""
    if which == "M":
        return p.alpha_M, p.beta_M
    if which == "D":
        return p.alpha_D, p.beta_D
    raise ValueError(which)


def check_positions(p, pos, which):
    """Reject heights outside [zmin, zmax] and envelopes crossing an open boundary
    (footnote to step 1 of Sec. III.D: kernels never extend through an open boundary)."""
    alpha, _ = kernel_params(p, which)
    z = pos[:, 2]
    if np.any(z < p.zmin) or np.any(z > p.zmax):
        raise ValueError("particle height outside [zmin, zmax]")
    if p.mode == FREE and np.any(z - alpha < p.zmin):
        raise ValueError("envelope crosses the open bottom boundary")
    if p.mode in (FREE, BOTTOM_WALL) and np.any(z + alpha > p.zmax):
        raise ValueError("envelope crosses the open top boundary")


def _particle_factors(p, xj, yj, zj, alpha, beta, Z, zn):
    xs = np.arange(p.nx) * p.h
    ys = np.arange(p.ny) * p.h
    fx = es(periodic_offset(xs, xj, p.Lx), alpha, beta, Z)
    fy = es(periodic_offset(ys, yj, p.Ly), alpha, beta, Z)
    fz = z_envelope(zn, zj, alpha, beta, p.mode, p.zmin, p.zmax, Z)
    ix = np.nonzero(fx)[0]
    iy = np.nonzero(fy)[0]
    iz = np.nonzero(fz)[0]
    return ix, iy, iz, fx[ix], fy[iy], fz[iz]


def _particle_gradient_factors(p, xj, yj, zj, zn):
    """Dipole-envelope factors and their derivatives on the particle's support: the index sets,
    phi in x, y and the imaged z factor, then phi' in x, y and d/dz of the imaged z factor."""
    alpha, beta = kernel_params(p, "D")
    Z = es_normalization(alpha, beta)
    cut = es_derivative_cutoff(alpha, beta)
    xs = np.arange(p.nx) * p.h
    ys = np.arange(p.ny) * p.h
    tx = periodic_offset(xs, xj, p.Lx)
    ty = periodic_offset(ys, yj, p.Ly)
    fx, fy = es(tx, alpha, beta, Z), es(ty, alpha, beta, Z)
    dx, dy = es_derivative(tx, alpha, beta, Z, cut), es_derivative(ty, alpha, beta, Z, cut)
    fz = z_envelope(zn, zj, alpha, beta, p.mode, p.zmin, p.zmax, Z)
    dz = z_envelope_derivative(zn, zj, alpha, beta, p.mode, p.zmin, p.zmax, Z, cut)
    ix = np.nonzero((fx != 0) | (dx != 0))[0]
    iy = np.nonzero((fy != 0) | (dy != 0))[0]
    iz = np.nonzero((fz != 0) | (dz != 0))[0]
    return ix, iy, iz, (fx[ix], fy[iy], fz[iz]), (dx[ix], dy[iy], dz[iz])


def _gradient_block(f, d):
    """The three components of grad Delta^W on the support block (z, y, x)."""
    (fx, fy, fz), (dx, dy, dz) = f, d
    gx = fz[:, None, None] * fy[None, :, None] * dx[None, None, :]
    gy = fz[:, None, None] * dy[None, :, None] * fx[None, None, :]
    gz = dz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    return gx, gy, gz


def spread(p, pos, vec, which="M"):
    """Grid values sum_j vec_j Delta^W(x_g - r_j) of Eq. 7 (step 1, Sec. III.D), one particle at
    a time.  pos, vec: (N, 3).  Returns (3, nz, ny, nx) float64."""
    pos = np.asarray(pos, dtype=float)
    vec = np.asarray(vec, dtype=float)
    check_positions(p, pos, which)
    alpha, beta = kernel_params(p, which)
    Z = es_normalization(alpha, beta)
    zn = cheb.nodes_z(p.nz, p.zmin, p.zmax)
    grid = np.zeros((3, p.nz, p.ny, p.nx))
    for j in range(pos.shape[0]):
        ix, iy, iz, fx, fy, fz = _particle_factors(p, pos[j, 0], pos[j, 1], pos[j, 2], alpha, beta, Z, zn)
        block = fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
        sel = np.ix_(iz, iy, ix)
        for i in range(3):
            grid[i][sel] += vec[j, i] * block
    return grid


def interpolate(p, pos, grid, which="M"):
    """Particle averages h^2 sum_g u_i(x_g) Delta^W(x_g - r_j) w_c of Eqs. 10-11 (step 8,
    Sec. III.D).  grid: (3, nz, ny, nx).  Returns (N, 3) float64."""
    pos = np.asarray(pos, dtype=float)
    check_positions(p, pos, which)
    alpha, beta = kernel_params(p, which)
    Z = es_normalization(alpha, beta)
    zn = cheb.nodes_z(p.nz, p.zmin, p.zmax)
    wz = cheb.clenshaw_curtis_weights(p.nz, p.H)
    out = np.zeros((pos.shape[0], 3))
    for j in range(pos.shape[0]):
        ix, iy, iz, fx, fy, fz = _particle_factors(p, pos[j, 0], pos[j, 1], pos[j, 2], alpha, beta, Z, zn)
        block = (fz * wz[iz])[:, None, None] * fy[None, :, None] * fx[None, None, :]
        sel = np.ix_(iz, iy, ix)
        for i in range(3):
            out[j, i] = p.h * p.h * np.sum(grid[i][sel] * block)
    return out


def spread_curl(p, pos, torque):
    """Grid values of the torque term of Eq. 7 by the derivative route: (1/2) grad Delta^W_D x tau_j
    summed over particles.  pos, torque: (N, 3).  Returns (3, nz, ny, nx) float64."""
    pos = np.asarray(pos, dtype=float)
    torque = np.asarray(torque, dtype=float)
    check_positions(p, pos, "D")
    zn = cheb.nodes_z(p.nz, p.zmin, p.zmax)
    grid = np.zeros((3, p.nz, p.ny, p.nx))
    for j in range(pos.shape[0]):
        ix, iy, iz, f, d = _particle_gradient_factors(p, pos[j, 0], pos[j, 1], pos[j, 2], zn)
        gx, gy, gz = _gradient_block(f, d)
        tx, ty, tz = torque[j]
        sel = np.ix_(iz, iy, ix)
        grid[0][sel] += 0.5 * (gy * tz - gz * ty)
        grid[1][sel] += 0.5 * (gz * tx - gx * tz)
        grid[2][sel] += 0.5 * (gx * ty - gy * tx)
    return grid


def interpolate_curl(p, pos, grid):
    """Angular velocities by the derivative route: Omega_j = (1/2) h^2 sum_g w_c u(x_g) x
    grad Delta^W_D(x_g - r_j).  grid: the velocity (3, nz, ny, nx).  Returns (N, 3) float64."""
    pos = np.asarray(pos, dtype=float)
    check_positions(p, pos, "D")
    zn = cheb.nodes_z(p.nz, p.zmin, p.zmax)
    wz = cheb.clenshaw_curtis_weights(p.nz, p.H)
    out = np.zeros((pos.shape[0], 3))
    for j in range(pos.shape[0]):
        ix, iy, iz, f, d = _particle_gradient_factors(p, pos[j, 0], pos[j, 1], pos[j, 2], zn)
        gx, gy, gz = _gradient_block(f, d)
        sel = np.ix_(iz, iy, ix)
        w = p.h * p.h * wz[iz][:, None, None]
        u, v, ww = grid[0][sel] * w, grid[1][sel] * w, grid[2][sel] * w
        out[j, 0] = 0.5 * np.sum(v * gz - ww * gy)
        out[j, 1] = 0.5 * np.sum(ww * gx - u * gz)
        out[j, 2] = 0.5 * np.sum(u * gy - v * gx)
    return out


def occupied_planes(p, pos, which_list=("M",)):
    """Sorted indices of the Chebyshev planes touched by at least one particle envelope
    (including images).  All other planes are exactly zero after spreading and are never read
    by interpolation."""
    zn = cheb.nodes_z(p.nz, p.zmin, p.zmax)
    occ = np.zeros(p.nz, dtype=bool)
    for which in which_list:
        alpha, beta = kernel_params(p, which)
        Z = es_normalization(alpha, beta)
        for zj in np.asarray(pos, dtype=float)[:, 2]:
            occ |= z_envelope(zn, zj, alpha, beta, p.mode, p.zmin, p.zmax, Z) != 0.0
    return np.nonzero(occ)[0]


__all__ = ["spread", "interpolate", "spread_curl", "interpolate_curl", "check_positions", "occupied_planes", "kernel_params", "SLIT"]
