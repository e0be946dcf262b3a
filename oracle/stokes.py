"""Spectral Stokes solve and the full mobility product (test infrastructure only).

Follows the eight steps of Sec. III.D in order, one wavenumber block at a time:
  1. spread forces (and torques) on the grid (transfer.spread);
  2. xy FFT of every Chebyshev plane, DCT-I in z to Chebyshev coefficients; the half-curl of the
     torque field is added in Fourier-Chebyshev space;
  3. per k != 0, the DP pressure BVP (Eqs. 15, 17), then the velocity BVPs (Eqs. 18, 22, 24);
  4. the wall correction: BW closed form (Eqs. 41-44), slit 8x8 system (Eqs. A4-A10, zero slip);
  5. the k = 0 mode (Sec. III.C; Appendix A.2);
  6. correction node values -> Chebyshev coefficients (DCT-I), added to the DP coefficients;
  7. curl in Fourier-Chebyshev space, inverse DCT-I and inverse xy FFT;
  8. interpolation (transfer.interpolate).
With torque_route='kernel_derivative' (the second torque route of Sec. III.D) step 1 adds the
half-curl of the dipole envelope to the force density instead of spreading a torque field, step 7
transforms the velocity only, and step 8 returns Omega with the envelope gradient
(transfer.spread_curl, transfer.interpolate_curl).

Readings where the paper is silent or ambiguous (each one is shared with the GPU path by
construction of its own code, never by shared code):
* Nyquist modes (n_x = -Nx/2 or n_y = -Ny/2 for even sizes) get a zero solution.
* In the open (free) geometry the k = 0 velocity is set to zero: the paper defers the
  backflow treatment (Sec. III), and zeroing matches the triply-periodic convention it cites.
* The slit correction is solved in the rescaled basis e^{-k(zmax - z)} for the top-wall family
  (the paper's D coefficients times e^{kH}); this is the same solution without e^{kH} entries.
* The z-derivatives in the curl act on the summed coefficients (DP + DCT-I of the correction
  node values), by the Chebyshev derivative recurrence.
"""

import numpy as np

from . import bvp, cheb
from .params import BOTTOM_WALL, FREE, SLIT
from .transfer import interpolate, interpolate_curl, spread, spread_curl


def wavenumbers(p):
    """k_x, k_y on the full FFT grid (shape (ny, nx)) and the Nyquist mask (Sec. III.A; k = 2 pi n/L)."""
    nxs = np.fft.fftfreq(p.nx) * p.nx
    nys = np.fft.fftfreq(p.ny) * p.ny
    kx = 2.0 * np.pi * nxs / p.Lx
    ky = 2.0 * np.pi * nys / p.Ly
    KX, KY = np.meshgrid(kx, ky)
    nyq = np.zeros((p.ny, p.nx), dtype=bool)
    if p.nx % 2 == 0:
        nyq[:, p.nx // 2] = True      # fftfreq index nx/2 is n_x = -nx/2
    if p.ny % 2 == 0:
        nyq[p.ny // 2, :] = True
    return KX, KY, nyq


def to_spectral(p, grid):
    """Step 2: (F, nz, ny, nx) real node values -> (F, ny, nx, nz) complex Chebyshev coefficients.
    Forward xy transform sum_x f e^{-i k.x} (unnormalised), then DCT-I in z."""
    fh = np.fft.fft2(grid, axes=(-2, -1))
    C = cheb.dct1_matrix(p.nz)
    return np.einsum("nc,fcyx->fyxn", C, fh)


def to_nodes(p, coef):
    """Step 7: (F, ny, nx, nz) Chebyshev coefficients -> (F, nz, ny, nx) real node values.
    Inverse DCT-I in z, inverse xy transform with 1/(Nx Ny)."""
    Ci = cheb.idct1_matrix(p.nz)
    vals = np.einsum("cn,fyxn->fcyx", Ci, coef)
    out = np.fft.ifft2(vals, axes=(-2, -1))
    imag = np.max(np.abs(out.imag)) if out.size else 0.0
    scale = max(np.max(np.abs(out.real)) if out.size else 0.0, 1e-300)
    assert imag <= 1e-9 * scale + 1e-300, "inverse transform is not real"
    return out.real


def dz(p, a):
    """d/dz of Chebyshev coefficients on [zmin, zmax] (last axis)."""
    return (2.0 / p.H) * cheb.cheb_derivative(a)


def add_torque_curl(p, fcoef, tcoef, kx, ky):
    """f += (1/2) curl t in Fourier-Chebyshev space (Eq. 7, torque route of Sec. III.D).
    fcoef, tcoef: (3, K, N); kx, ky: (K,)."""
    ikx = 1j * kx[:, None]
    iky = 1j * ky[:, None]
    dt = dz(p, tcoef)
    out = fcoef.copy()
    out[0] += 0.5 * (iky * tcoef[2] - dt[1])
    out[1] += 0.5 * (dt[0] - ikx * tcoef[2])
    out[2] += 0.5 * (ikx * tcoef[1] - iky * tcoef[0])
    return out


def dp_solve(p, f, g, hz, kx, ky):
    """Step 3: DP pressure then velocity BVPs for k != 0 (Eqs. 15, 17, 18, 22, 24).
    f, g, hz: (K, N) force coefficients.  Returns pressure and velocity coefficients (K, N)."""
    eta = p.eta
    k = np.hypot(kx, ky)
    ikx = (1j * kx)[:, None]
    iky = (1j * ky)[:, None]
    rp = ikx * f + iky * g + dz(p, hz)
    zero = np.zeros((k.size, 1), dtype=complex)
    pc = bvp.solve(k, p.H, rp[:, None, :], zero, zero, "dtn")[:, 0, :]
    p_top, p_bot = bvp.endpoint_values(pc)
    ru = (ikx * pc - f) / eta
    rv = (iky * pc - g) / eta
    rw = (dz(p, pc) - hz) / eta
    g_top = np.stack([-1j * kx / (2 * k * eta) * p_top,
                      -1j * ky / (2 * k * eta) * p_top,
                      p_top / (2 * eta)], axis=1)
    g_bot = np.stack([1j * kx / (2 * k * eta) * p_bot,
                      1j * ky / (2 * k * eta) * p_bot,
                      p_bot / (2 * eta)], axis=1)
    vel = bvp.solve(k, p.H, np.stack([ru, rv, rw], axis=1), g_top, g_bot, "dtn")
    return pc, vel[:, 0, :], vel[:, 1, :], vel[:, 2, :]


def correction_bw(p, u0, v0, w0, kx, ky):
    """Step 4, bottom wall: Eqs. 41-44 evaluated at the nodes, zeta = z - zmin.
    u0, v0, w0: (K,) wall data (minus the DP velocity at the wall, plus l0 times its z derivative
    for the tangential parts).  With a slip length the solution is correction_bw_slip.
    Returns (3, K, N) node values."""
    if p.slip_bottom:
        return correction_bw_slip(p, u0, v0, w0, kx, ky)
    k = np.hypot(kx, ky)[:, None]
    kxc = kx[:, None]
    kyc = ky[:, None]
    zeta = (cheb.nodes_z(p.nz, p.zmin, p.zmax) - p.zmin)[None, :]
    E = np.exp(-k * zeta)
    u0 = u0[:, None]
    v0 = v0[:, None]
    w0 = w0[:, None]
    common = 1j * k * w0 + kxc * u0 + kyc * v0
    uc = -(kxc / k) * common * zeta * E + u0 * E
    vc = -(kyc / k) * common * zeta * E + v0 * E
    wc = (k * w0 - 1j * kxc * u0 - 1j * kyc * v0) * zeta * E + w0 * E
    return np.stack([uc, vc, wc])


def correction_bw_slip(p, u0, v0, w0, kx, ky, return_coefficients=False):
    """Step 4, bottom wall with slip length l0: the slit construction of Appendix A restricted to
    the family that decays away from the wall (the growing one is excluded by boundedness as
    z -> infinity): unknowns C0, Cx, Cy, Cz of Eqs. A5-A6 from the bottom rows of Eq. A8 (Robin
    rows for u and v, w = w0) and the continuity row at the wall (Eq. A10), dense LU per k."""
    eta, l0 = p.eta, p.slip_bottom
    k = np.hypot(kx, ky)
    K = k.size
    ikx, iky = 1j * kx, 1j * ky
    A = np.zeros((K, 4, 4), dtype=complex)
    # unknown order: C0, Cx, Cy, Cz
    A[:, 0, 0] = ikx * l0 / (2 * eta * k)
    A[:, 0, 1] = 1.0 + k * l0
    A[:, 1, 0] = iky * l0 / (2 * eta * k)
    A[:, 1, 2] = 1.0 + k * l0
    A[:, 2, 3] = 1.0
    A[:, 3, 0] = 1.0 / (2 * eta)
    A[:, 3, 1] = ikx
    A[:, 3, 2] = iky
    A[:, 3, 3] = -k
    rhs = np.stack([u0, v0, w0, np.zeros_like(u0)], axis=1)
    x = np.linalg.solve(A, rhs[:, :, None])[:, :, 0]
    C0, Cx, Cy, Cz = (x[:, i][:, None] for i in range(4))
    zeta = (cheb.nodes_z(p.nz, p.zmin, p.zmax) - p.zmin)[None, :]
    kc = k[:, None]
    Eb = np.exp(-kc * zeta)
    uc = -(C0 * ikx[:, None] / (2 * eta * kc)) * zeta * Eb + Cx * Eb
    vc = -(C0 * iky[:, None] / (2 * eta * kc)) * zeta * Eb + Cy * Eb
    wc = (C0 / (2 * eta)) * zeta * Eb + Cz * Eb
    if return_coefficients:
        return np.stack([uc, vc, wc]), x.T
    return np.stack([uc, vc, wc])


def correction_sc(p, bot, top, kx, ky, return_coefficients=False):
    """Step 4, slit channel: the 8 equations A8 and A10 with slip lengths l0, lH (zero: no-slip),
    in the rescaled basis (top family multiplied by e^{kH}), solved by dense LU per k; then
    Eqs. A5-A6 at the nodes.  bot = (u0, v0, w0), top = (uH, vH, wH), each (K,).  Returns (3, K, N)
    node values."""
    eta = p.eta
    H = p.H
    k = np.hypot(kx, ky)
    K = k.size
    E = np.exp(-k * H)
    ikx = 1j * kx
    iky = 1j * ky
    l0, lH = p.slip_bottom, p.slip_top
    A = np.zeros((K, 8, 8), dtype=complex)
    # unknown order: C0, D0, Cx, Dx, Cy, Dy, Cz, Dz  (D's rescaled by e^{kH})
    # bottom Robin rows (Eq. A8, first line, for u and v) and w = w0
    for row, ik, c, d in ((0, ikx, 2, 3), (1, iky, 4, 5)):
        A[:, row, 0] = ik * l0 / (2 * eta * k)
        A[:, row, 1] = -ik * l0 * E / (2 * eta * k)
        A[:, row, c] = 1.0 + k * l0
        A[:, row, d] = E * (1.0 - k * l0)
    A[:, 2, 6] = 1.0
    A[:, 2, 7] = E
    # top Robin rows (Eq. A8, third line) and w = wH
    for row, ik, c, d in ((3, ikx, 2, 3), (4, iky, 4, 5)):
        A[:, row, 0] = ik * H * E / (2 * eta * k) * (k * lH - lH / H - 1.0)
        A[:, row, 1] = ik * H / (2 * eta * k) * (k * lH + lH / H + 1.0)
        A[:, row, c] = E * (1.0 - k * lH)
        A[:, row, d] = 1.0 + k * lH
    A[:, 5, 0] = H * E / (2 * eta)
    A[:, 5, 1] = H / (2 * eta)
    A[:, 5, 6] = E
    A[:, 5, 7] = 1.0
    A[:, 6, 0] = 1.0 / (2 * eta)
    A[:, 6, 1] = E / (2 * eta)
    A[:, 6, 2] = ikx
    A[:, 6, 3] = ikx * E
    A[:, 6, 4] = iky
    A[:, 6, 5] = iky * E
    A[:, 6, 6] = -k
    A[:, 6, 7] = k * E
    A[:, 7, 0] = E / (2 * eta)
    A[:, 7, 1] = 1.0 / (2 * eta)
    A[:, 7, 2] = ikx * E
    A[:, 7, 3] = ikx
    A[:, 7, 4] = iky * E
    A[:, 7, 5] = iky
    A[:, 7, 6] = -k * E
    A[:, 7, 7] = k
    rhs = np.zeros((K, 8), dtype=complex)
    rhs[:, 0], rhs[:, 1], rhs[:, 2] = bot
    rhs[:, 3], rhs[:, 4], rhs[:, 5] = top
    x = np.linalg.solve(A, rhs[:, :, None])[:, :, 0]
    C0, D0, Cx, Dx, Cy, Dy, Cz, Dz = (x[:, i][:, None] for i in range(8))
    zeta = (cheb.nodes_z(p.nz, p.zmin, p.zmax) - p.zmin)[None, :]
    kc = k[:, None]
    Eb = np.exp(-kc * zeta)
    Et = np.exp(-kc * (H - zeta))
    ikxc = ikx[:, None]
    ikyc = iky[:, None]
    uc = -(C0 * ikxc / (2 * eta * kc)) * zeta * Eb + (D0 * ikxc / (2 * eta * kc)) * zeta * Et + Cx * Eb + Dx * Et
    vc = -(C0 * ikyc / (2 * eta * kc)) * zeta * Eb + (D0 * ikyc / (2 * eta * kc)) * zeta * Et + Cy * Eb + Dy * Et
    wc = (C0 / (2 * eta)) * zeta * Eb + (D0 / (2 * eta)) * zeta * Et + Cz * Eb + Dz * Et
    if return_coefficients:
        return np.stack([uc, vc, wc]), x.T
    return np.stack([uc, vc, wc])


def zero_mode(p, f0, g0):
    """Step 5: k = 0.  w = 0; d^2u/dz^2 = -f/eta with, above one wall, u - l0 du/dz = u^W at zmin
    and du/dz = 0 at zmax (Eqs. 51-52 with the Robin bottom row of Eq. A12), in the slit
    u - l0 du/dz = u^W_0 at zmin and u + lH du/dz = u^W_H at zmax (Eq. A12), and u = 0 in the open
    geometry.  The k = 0 coefficient of a uniform wall velocity is Nx Ny u^W (the forward transform
    is unnormalised).  f0, g0: (N,) coefficients.  Returns (u, v, w) coefficients."""
    N = f0.shape[-1]
    if p.mode == FREE:
        z = np.zeros(N, dtype=complex)
        return z, z.copy(), z.copy()
    bc = "bw0" if p.mode == BOTTOM_WALL else "sc0"
    r = np.stack([-f0 / p.eta, -g0 / p.eta])[None]
    scale = p.nx * p.ny
    g_bot = scale * np.array([p.uw_bottom], dtype=complex)
    g_top = scale * np.array([p.uw_top], dtype=complex) if p.mode == SLIT else np.zeros((1, 2), dtype=complex)
    y = bvp.solve(np.zeros(1), p.H, r, g_top, g_bot, bc, (p.slip_bottom, p.slip_top))[0]
    return y[0], y[1], np.zeros(N, dtype=complex)


def solve_spectral(p, fcoef, tcoef=None, want_curl=False, chunk=4096):
    """Steps 2-6 plus the curl of step 7 on Chebyshev-coefficient spectra.

    fcoef: (3, ny, nx, N) force coefficients; tcoef: same for the torque field or None.
    Returns velocity coefficients (3, ny, nx, N) and, if want_curl, the half-curl
    omega = (1/2) curl u coefficients (3, ny, nx, N)."""
    N = p.nz
    KX, KY, nyq = wavenumbers(p)
    kx_all = KX.ravel()
    ky_all = KY.ravel()
    nyq_all = nyq.ravel()
    f_all = fcoef.reshape(3, -1, N)
    t_all = None if tcoef is None else tcoef.reshape(3, -1, N)
    Kt = kx_all.size
    vel = np.zeros((3, Kt, N), dtype=complex)
    Cd = cheb.dct1_matrix(N)
    for s in range(0, Kt, chunk):
        sl = slice(s, min(s + chunk, Kt))
        kx = kx_all[sl]
        ky = ky_all[sl]
        fb = f_all[:, sl, :]
        if t_all is not None:
            fb = add_torque_curl(p, fb, t_all[:, sl, :], kx, ky)
        k = np.hypot(kx, ky)
        act = (k > 0) & ~nyq_all[sl]
        if np.any(act):
            idx = np.nonzero(act)[0]
            _, u, v, w = dp_solve(p, fb[0, idx], fb[1, idx], fb[2, idx], kx[idx], ky[idx])
            if p.mode != FREE:
                # wall data (Eq. A3): minus the DP velocity at the wall, and for the tangential
                # parts plus l0 (bottom) or minus lH (top) times its z derivative there
                sign = (-1.0) ** np.arange(N)
                ub, vb, wb = (np.stack([u, v, w]) * sign).sum(axis=-1)
                dub, dvb = (dz(p, np.stack([u, v])) * sign).sum(axis=-1)
                l0, lH = p.slip_bottom, p.slip_top
                bot = (-ub + l0 * dub, -vb + l0 * dvb, -wb)
                if p.mode == BOTTOM_WALL:
                    corr = correction_bw(p, *bot, kx[idx], ky[idx])
                else:
                    ut, vt, wt = np.stack([u, v, w]).sum(axis=-1)
                    dut, dvt = dz(p, np.stack([u, v])).sum(axis=-1)
                    top = (-ut - lH * dut, -vt - lH * dvt, -wt)
                    corr = correction_sc(p, bot, top, kx[idx], ky[idx])
                corr_coef = np.einsum("nc,fkc->fkn", Cd, corr)
                u = u + corr_coef[0]
                v = v + corr_coef[1]
                w = w + corr_coef[2]
            vel[0, sl][idx] = u
            vel[1, sl][idx] = v
            vel[2, sl][idx] = w
        z0 = np.nonzero((k == 0) & ~nyq_all[sl])[0]
        for i in z0:
            u, v, w = zero_mode(p, fb[0, i], fb[1, i])
            vel[0, s + i] = u
            vel[1, s + i] = v
            vel[2, s + i] = w
    omega = None
    if want_curl:
        ikx = (1j * kx_all)[:, None]
        iky = (1j * ky_all)[:, None]
        d = dz(p, vel)
        omega = np.stack([0.5 * (iky * vel[2] - d[1]),
                          0.5 * (d[0] - ikx * vel[2]),
                          0.5 * (ikx * vel[1] - iky * vel[0])])
        omega = omega.reshape(3, p.ny, p.nx, N)
    return vel.reshape(3, p.ny, p.nx, N), omega


def wrap_positions(p, pos):
    """x, y taken modulo the periods; z unchanged."""
    pos = np.array(pos, dtype=float, copy=True)
    pos[:, 0] = np.mod(pos[:, 0], p.Lx)
    pos[:, 1] = np.mod(pos[:, 1], p.Ly)
    return pos


TORQUE_ROUTES = ("spectral_curl", "kernel_derivative")


def mobility(p, pos, F, T=None, return_grids=False, torque_route="spectral_curl"):
    """The mobility product [U; Omega] = M [F; T] of Eq. 58 by steps 1-8 of Sec. III.D.

    torque_route selects one of the two ways Sec. III.D gives for torques: 'spectral_curl' spreads
    tau Delta^W_D and takes the half-curl of the torque field and of the velocity in
    Fourier-Chebyshev space; 'kernel_derivative' spreads (1/2) grad Delta^W_D x tau with the force
    density and interpolates Omega with the envelope gradient, so only the three velocity fields are
    transformed.  pos, F, T: (N, 3).  Returns U (N, 3) and Omega (N, 3) (None when T is None)."""
    if torque_route not in TORQUE_ROUTES:
        raise ValueError(f"unknown torque route {torque_route!r}")
    pos = wrap_positions(p, pos)
    fgrid = spread(p, pos, F, "M")
    derivative = T is not None and torque_route == "kernel_derivative"
    if derivative:
        fgrid = fgrid + spread_curl(p, pos, T)
    fcoef = to_spectral(p, fgrid[None] if fgrid.ndim == 3 else fgrid)
    tcoef = None
    if T is not None and not derivative:
        tgrid = spread(p, pos, T, "D")
        tcoef = to_spectral(p, tgrid)
    vcoef, ocoef = solve_spectral(p, fcoef, tcoef, want_curl=T is not None and not derivative)
    ugrid = to_nodes(p, vcoef)
    U = interpolate(p, pos, ugrid, "M")
    Om = None
    if derivative:
        Om = interpolate_curl(p, pos, ugrid)
    elif T is not None:
        ogrid = to_nodes(p, ocoef)
        Om = interpolate(p, pos, ogrid, "D")
    if return_grids:
        return U, Om, {"f": fgrid, "u": ugrid}
    return U, Om
