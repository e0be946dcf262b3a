"""Pins for the oracle's per-wavenumber BVPs (Eqs. 15-24, 51-52, A12) and wall corrections
(Eqs. 41-44, A4-A10): manufactured solutions, closed forms, and domain-extension invariance
of the Dirichlet-to-Neumann rows."""

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb
from scipy import special

from oracle import bvp, cheb, stokes
from oracle.params import Params

Z0, Z1 = 0.0, 8.0


def _coef(fun, nz, z0=Z0, z1=Z1):
    return cheb.dct1_matrix(nz) @ fun(cheb.nodes_z(nz, z0, z1))


def _vals(coef, nz):
    return cheb.idct1_matrix(nz) @ coef


@pytest.mark.parametrize("bc", ["dtn", "bw0", "sc0"])
@pytest.mark.parametrize("k", [0.0, 0.35, 2.0, 7.5])
def test_manufactured_smooth_solution(bc, k):
    if bc == "dtn" and k == 0.0:
        pytest.skip("the DtN rows are only used for k > 0")
    nz = 49
    H = Z1 - Z0
    om, b, ph = 0.9, -0.15, 0.3
    y = lambda z: np.exp(b * z) * np.sin(om * z + ph)
    yp = lambda z: np.exp(b * z) * (b * np.sin(om * z + ph) + om * np.cos(om * z + ph))
    ypp = lambda z: np.exp(b * z) * ((b * b - om * om) * np.sin(om * z + ph) + 2 * b * om * np.cos(om * z + ph))
    r = _coef(lambda z: ypp(z) - k * k * y(z), nz)
    if bc == "dtn":
        gt, gb = yp(Z1) + k * y(Z1), yp(Z0) - k * y(Z0)
    elif bc == "bw0":
        gt, gb = yp(Z1), y(Z0)
    else:
        gt, gb = y(Z1), y(Z0)
    sol = bvp.solve(np.array([k]), H, r[None, None, :].astype(complex),
                    np.array([[gt]], dtype=complex), np.array([[gb]], dtype=complex), bc)[0, 0]
    err = np.max(np.abs(_vals(sol, nz) - y(cheb.nodes_z(nz, Z0, Z1))))
    assert err < 1e-11


@pytest.mark.parametrize("bc", ["bw0", "sc0"])
def test_zero_mode_polynomial_exact(bc):
    # u'' = -f/eta with constant f: exact quadratic solution (Eqs. 51-52; Eq. A12 with zero slip).
    nz, eta, f = 17, 1.3, 2.0
    H = Z1 - Z0
    if bc == "bw0":
        exact = lambda z: -f / (2 * eta) * z * z + f / eta * Z1 * z    # u(0)=0, u'(H)=0
    else:
        exact = lambda z: -f / (2 * eta) * z * (z - Z1)                # u(0)=u(H)=0
    r = np.zeros(nz, dtype=complex)
    r[0] = -f / eta
    sol = bvp.solve(np.zeros(1), H, r[None, None], np.zeros((1, 1)), np.zeros((1, 1)), bc)[0, 0]
    assert np.max(np.abs(_vals(sol, nz) - exact(cheb.nodes_z(nz, Z0, Z1)))) < 1e-12


def _gauss_conv(z, c, sig, k):
    """I(z) = int exp(-k|z-z'|) exp(-(z'-c)^2/sig^2) dz' and dI/dz, in closed form (erfc/erfcx)."""
    t = z - c
    a = 0.5 * k * sig
    xp, xm = a - t / sig, a + t / sig
    pre = 0.5 * np.sqrt(np.pi) * sig

    def piece(x, sgn):
        out = np.empty_like(x)
        neg = x < 0
        out[~neg] = np.exp(-(t[~neg] / sig) ** 2) * special.erfcx(x[~neg])
        out[neg] = np.exp(a * a - sgn * k * t[neg]) * special.erfc(x[neg])
        return pre * out

    Ip = piece(xp, +1.0)   # from below: int_{-inf}^{z} e^{-k(z-z')} g
    Im = piece(xm, -1.0)   # from above
    return Ip + Im, -k * Ip + k * Im


@pytest.mark.parametrize("k", [0.4, 1.7, 6.0])
def test_dtn_pressure_against_free_space_green_function(k):
    # Eq. 15 on the whole line with a source compactly supported in (zmin, zmax); the exact
    # solution is the convolution with -exp(-k|z|)/(2k).  The DtN rows of Eq. 17 must reproduce it
    # on [zmin, zmax].
    nz, c, sig = 129, 4.0, 0.6
    A, Bz = 0.7 - 0.2j, -0.4 + 1.1j                # S = A g + Bz g'
    g = lambda z: np.exp(-((z - c) / sig) ** 2)
    gp = lambda z: -2 * (z - c) / sig**2 * g(z)
    r = _coef(lambda z: A * g(z) + Bz * gp(z), nz)
    sol = bvp.solve(np.array([k]), Z1 - Z0, r[None, None], np.zeros((1, 1)), np.zeros((1, 1)), "dtn")[0, 0]
    zn = cheb.nodes_z(nz, Z0, Z1)
    I, dI = _gauss_conv(zn, c, sig, k)
    exact = -(A * I + Bz * dI) / (2 * k)
    assert np.max(np.abs(_vals(sol, nz) - exact)) < 1e-11 * np.max(np.abs(exact))


@pytest.mark.parametrize("kx,ky", [(0.9, 0.0), (0.6, -1.3), (3.0, 2.5)])
def test_dp_solution_invariant_under_domain_extension(kx, ky):
    # The DP problem lives on the whole line (Sec. III.A); the DtN rows (Eqs. 17, 22, 24) make
    # the solution on [zmin, zmax] independent of where the computational boundaries are put,
    # as long as the source vanishes outside.  A wrong DtN constant breaks this.
    eta = 0.8
    c, sig = 4.0, 0.6
    amps = np.array([0.3 + 0.5j, -0.7 + 0.1j, 0.2 - 0.9j])

    def run(z0, z1, nz):
        p = Params(Lx=1.0, Ly=1.0, zmin=z0, zmax=z1, mode="free", nx=2, ny=2, nz=nz, m_M=4,
                   beta_M=7.0, eta=eta)
        zn = cheb.nodes_z(nz, z0, z1)
        src = np.exp(-((zn - c) / sig) ** 2)
        C = cheb.dct1_matrix(nz)
        f, g, h = (C @ (a * src) for a in amps)
        pc, u, v, w = stokes.dp_solve(p, f[None], g[None], h[None], np.array([kx]), np.array([ky]))
        return [coef[0] for coef in (pc, u, v, w)]

    small = run(0.0, 8.0, 129)
    big = run(-1.5, 10.0, 161)
    zq = cheb.nodes_z(129, 0.0, 8.0)
    for a_s, a_b in zip(small, big):
        vs = _vals(a_s, 129)
        vb = npcheb.chebval(2 * (zq + 1.5) / 11.5 - 1, a_b)
        assert np.max(np.abs(vs - vb)) < 1e-10 * np.max(np.abs(vs))


def _gauss_derivs(z, c, sig):
    """Gaussian exp(-((z-c)/sig)^2) and its first four derivatives (Hermite form)."""
    x = (z - c) / sig
    g = np.exp(-x * x)
    h = [np.ones_like(x), 2 * x, 4 * x * x - 2, 8 * x**3 - 12 * x, 16 * x**4 - 48 * x * x + 12]
    return [(-1) ** n * h[n] * g / sig**n for n in range(5)]


@pytest.mark.parametrize("kx,ky", [(0.8, 0.3), (-2.2, 1.1), (5.0, -4.0)])
def test_manufactured_dp_stokes_mode(kx, ky):
    # P1: choose pressure and a divergence-free velocity that vanish at both ends, form the force
    # from Eq. 18 and check that the pressure and velocity BVPs return them.
    nz, eta = 129, 1.4
    k2 = kx * kx + ky * ky
    zn = cheb.nodes_z(nz, Z0, Z1)
    B = _gauss_derivs(zn, 3.6, 0.55)
    G = _gauss_derivs(zn, 4.3, 0.5)
    P = _gauss_derivs(zn, 4.0, 0.6)
    cB, cG, cP = 0.8 - 0.3j, 0.4 + 0.6j, -1.2 + 0.2j
    u = [1j * kx * cB * B[n + 1] / k2 + ky * cG * G[n] for n in range(3)]
    v = [1j * ky * cB * B[n + 1] / k2 - kx * cG * G[n] for n in range(3)]
    w = [cB * B[n] for n in range(3)]
    pr = [cP * P[n] for n in range(2)]
    assert np.max(np.abs(1j * kx * u[0] + 1j * ky * v[0] + w[1])) < 1e-12
    f = -eta * (u[2] - k2 * u[0]) + 1j * kx * pr[0]
    g = -eta * (v[2] - k2 * v[0]) + 1j * ky * pr[0]
    h = -eta * (w[2] - k2 * w[0]) + pr[1]
    C = cheb.dct1_matrix(nz)
    p = Params(Lx=1.0, Ly=1.0, zmin=Z0, zmax=Z1, mode="free", nx=2, ny=2, nz=nz, m_M=4, beta_M=7.0, eta=eta)
    out = stokes.dp_solve(p, (C @ f)[None], (C @ g)[None], (C @ h)[None], np.array([kx]), np.array([ky]))
    for coef, exact in zip(out, (pr[0], u[0], v[0], w[0])):
        assert np.max(np.abs(_vals(coef[0], nz) - exact)) < 1e-9 * np.max(np.abs(exact))


def _check_homogeneous_stokes(p, nodes, kx, ky, pres):
    """Correction fields must be divergence free and satisfy eta(D^2-k^2)u = i k p (Eqs. 25-26)."""
    C = cheb.dct1_matrix(p.nz)
    k2 = kx * kx + ky * ky
    u, v, w = (C @ nodes[i] for i in range(3))
    pc = C @ pres
    d = lambda a: stokes.dz(p, a)
    div = 1j * kx * u + 1j * ky * v + d(w)
    mx = p.eta * (d(d(u)) - k2 * u) - 1j * kx * pc
    mz = p.eta * (d(d(w)) - k2 * w) - d(pc)
    scale = np.max(np.abs(nodes))
    return [np.max(np.abs(x)) / scale for x in (div, mx, mz)]


@pytest.mark.parametrize("kx,ky", [(0.5, 0.2), (1.5, -2.0)])
def test_bw_correction_is_homogeneous_stokes_with_wall_data(kx, ky):
    p = Params(Lx=1.0, Ly=1.0, zmin=0.0, zmax=8.0, mode="bottom_wall", nx=2, ny=2, nz=65, m_M=4,
               beta_M=7.0, eta=0.7)
    u0, v0, w0 = 0.3 - 0.2j, -0.5 + 0.4j, 0.25 + 0.1j
    corr = stokes.correction_bw(p, np.array([u0]), np.array([v0]), np.array([w0]), np.array([kx]),
                                np.array([ky]))[:, 0, :]
    assert np.allclose(corr[:, -1], [u0, v0, w0], atol=1e-15)          # node c = nz-1 is the wall
    k = np.hypot(kx, ky)
    zeta = cheb.nodes_z(65, 0.0, 8.0)
    pres = 2 * p.eta * (k * w0 - 1j * kx * u0 - 1j * ky * v0) * np.exp(-k * zeta)   # Eq. 41
    errs = _check_homogeneous_stokes(p, corr, kx, ky, pres)
    assert max(errs) < 1e-8


@pytest.mark.parametrize("kx,ky,H", [(0.4, 0.3, 20.0), (1.2, -0.7, 6.0), (0.05, 0.02, 3.0)])
def test_slit_correction_satisfies_walls_and_stokes(kx, ky, H):
    p = Params(Lx=1.0, Ly=1.0, zmin=0.0, zmax=H, mode="slit", nx=2, ny=2, nz=65, m_M=4, beta_M=7.0,
               eta=1.1)
    bot = (np.array([0.3 - 0.2j]), np.array([-0.5 + 0.4j]), np.array([0.25 + 0.1j]))
    top = (np.array([-0.1 + 0.6j]), np.array([0.2j]), np.array([0.7 - 0.3j]))
    corr, coefs = stokes.correction_sc(p, bot, top, np.array([kx]), np.array([ky]), return_coefficients=True)
    corr = corr[:, 0, :]
    assert np.allclose(corr[:, -1], [b[0] for b in bot], atol=1e-13)
    assert np.allclose(corr[:, 0], [t[0] for t in top], atol=1e-13)
    C0, D0 = coefs[0][0], coefs[1][0]
    k = np.hypot(kx, ky)
    zeta = cheb.nodes_z(65, 0.0, H)
    pres = C0 * np.exp(-k * zeta) + D0 * np.exp(-k * (H - zeta))     # Eq. A4, rescaled
    errs = _check_homogeneous_stokes(p, corr, kx, ky, pres)
    assert max(errs) < 1e-7


def test_slit_correction_tends_to_bottom_wall_for_wide_channel():
    kx, ky = 1.3, 0.9
    H = 60.0
    ps = Params(Lx=1.0, Ly=1.0, zmin=0.0, zmax=H, mode="slit", nx=2, ny=2, nz=65, m_M=4, beta_M=7.0)
    pb = Params(Lx=1.0, Ly=1.0, zmin=0.0, zmax=H, mode="bottom_wall", nx=2, ny=2, nz=65, m_M=4, beta_M=7.0)
    bot = (np.array([0.3 - 0.2j]), np.array([-0.5 + 0.4j]), np.array([0.25 + 0.1j]))
    zero = (np.zeros(1, complex),) * 3
    sc = stokes.correction_sc(ps, bot, zero, np.array([kx]), np.array([ky]))
    bw = stokes.correction_bw(pb, *bot, np.array([kx]), np.array([ky]))
    assert np.max(np.abs(sc - bw)) < 1e-13
