"""Pins for partial-slip walls and uniform wall velocities in the oracle (Appendix A, Eqs. A1-A12).

* The k = 0 mode: a uniform body force gives the closed-form quadratic profile of the Robin
  problem; uniform wall velocities give the closed-form Couette (slit) and plug (bottom wall)
  profiles, which every particle then follows.
* k != 0: the solved slit coefficients satisfy the Robin rows, the w rows and continuity at both
  walls, checked by differentiating the correction profile numerically; the total velocity (DP +
  correction, from its Chebyshev coefficients) satisfies the wall conditions at every wavenumber;
  the bottom-wall slip solution reduces to the closed form (Eqs. 41-44) as l0 -> 0.
* The mobility is continuous as the slip lengths go to zero, a slit with slip tends to the bottom
  wall with the same slip as H grows, and making the bottom wall shear-free (l0 -> infinity) changes
  the self mobility by the difference of the leading image corrections of a free surface and of a
  no-slip wall: (3/8 + 9/16)(a/z) parallel, (9/8 - 3/4)(a/z) normal.
* Symmetric positive-definite grand mobility with slip.
"""

import numpy as np
import pytest

from oracle import Params, bvp, cheb, mobility, table1, table2
from oracle import stokes


def _slit(l0, lH, nz=33, **kw):
    _, bm, bd = table1(5)
    return Params(Lx=24.0, Ly=24.0, zmin=0.0, zmax=10.0, mode="slit", nx=36, ny=36, nz=nz, m_M=5, beta_M=5 * bm,
                  m_D=5, beta_D=5 * bd, eta=0.9, slip_bottom=l0, slip_top=lH, **kw)


@pytest.mark.parametrize("l0,lH", [(0.0, 0.0), (0.7, 0.0), (0.3, 2.5)])
def test_zero_mode_quadratic_profile(l0, lH):
    H, N, f, eta = 10.0, 17, 1.3, 0.9
    r = np.zeros((1, 1, N), dtype=complex)
    r[0, 0, 0] = -f / eta
    zero = np.zeros((1, 1), dtype=complex)
    y = bvp.solve(np.zeros(1), H, r, zero, zero, "sc0", (l0, lH))[0, 0]
    zeta = cheb.nodes_z(N, 0.0, H)
    a = H * (H + 2 * lH) / (H + l0 + lH)
    want = f / (2 * eta) * (-zeta**2 + a * zeta + l0 * a)
    got = cheb.idct1_matrix(N) @ y
    assert np.allclose(got.real, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))
    # bottom wall: Robin row at zmin, zero stress at the top
    y = bvp.solve(np.zeros(1), H, r, zero, zero, "bw0", (l0, 0.0))[0, 0]
    want = f / (2 * eta) * (-zeta**2 + 2 * H * zeta + 2 * H * l0)
    assert np.allclose((cheb.idct1_matrix(N) @ y).real, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))


@pytest.mark.parametrize("l0,lH", [(0.0, 0.0), (0.6, 1.7)])
def test_wall_velocities_drive_couette_flow(l0, lH):
    U0, UH = np.array([0.4, -0.2]), np.array([-1.1, 0.5])
    p = _slit(l0, lH, uw_bottom=tuple(U0), uw_top=tuple(UH))
    pos = np.array([[5.1, 7.3, 3.0], [12.2, 4.4, 6.5], [20.0, 17.0, 5.0]])
    U, W = mobility(p, pos, np.zeros((3, 3)), np.zeros((3, 3)))
    c1 = (UH - U0) / (p.H + l0 + lH)
    c0 = U0 + l0 * c1
    want = c0[None, :] + c1[None, :] * pos[:, 2:3]
    # the monopole kernel's discrete mass differs from 1 by about e^{-beta_M} (beta_M = 6.5 here)
    assert np.allclose(U[:, :2], want, rtol=0, atol=3e-3 * np.max(np.abs(want)))
    assert np.allclose(U[:, 2], 0.0, atol=1e-12)
    # uniform shear: angular velocity (1/2) curl u = (1/2)(-du_y/dz, du_x/dz, 0)
    assert np.allclose(W[:, 0], -0.5 * c1[1], atol=2e-5) and np.allclose(W[:, 1], 0.5 * c1[0], atol=2e-5)


def test_bottom_wall_velocity_is_a_plug_flow():
    _, bm = table2(5)
    p = Params(Lx=24.0, Ly=24.0, zmin=0.0, zmax=10.0, mode="bottom_wall", nx=36, ny=36, nz=33, m_M=5,
               beta_M=5 * bm, slip_bottom=0.8, uw_bottom=(0.3, -0.6))
    pos = np.array([[5.1, 7.3, 2.0], [12.2, 4.4, 5.5]])
    U, _ = mobility(p, pos, np.zeros((2, 3)))
    assert np.allclose(U, [[0.3, -0.6, 0.0]] * 2, rtol=0, atol=3e-3)


def _profile(x, kx, ky, eta, z, H):
    """Velocity of Eqs. A5-A6 (unscaled basis; D's given rescaled by e^{kH}) at heights z."""
    C0, D0, Cx, Dx, Cy, Dy, Cz, Dz = x
    k = np.hypot(kx, ky)
    Eb, Et = np.exp(-k * z), np.exp(-k * (H - z))
    u = -(C0 * 1j * kx / (2 * eta * k)) * z * Eb + (D0 * 1j * kx / (2 * eta * k)) * z * Et + Cx * Eb + Dx * Et
    v = -(C0 * 1j * ky / (2 * eta * k)) * z * Eb + (D0 * 1j * ky / (2 * eta * k)) * z * Et + Cy * Eb + Dy * Et
    w = (C0 / (2 * eta)) * z * Eb + (D0 / (2 * eta)) * z * Et + Cz * Eb + Dz * Et
    return u, v, w


@pytest.mark.parametrize("l0,lH", [(0.0, 0.0), (0.9, 0.0), (0.4, 3.0)])
def test_slit_coefficients_satisfy_robin_rows_and_continuity(l0, lH):
    p = _slit(l0, lH)
    rng = np.random.default_rng(5)
    kx = np.array([0.3, -1.2, 2.0])
    ky = np.array([0.5, 0.1, -0.7])
    bot = tuple(rng.standard_normal(3) + 1j * rng.standard_normal(3) for _ in range(3))
    top = tuple(rng.standard_normal(3) + 1j * rng.standard_normal(3) for _ in range(3))
    _, X = stokes.correction_sc(p, bot, top, kx, ky, return_coefficients=True)
    H, eta, d = p.H, p.eta, 1e-6
    for i in range(3):
        x = X[:, i]
        prof = lambda z: _profile(x, kx[i], ky[i], eta, z, H)
        dprof = lambda z: [(a - b) / (2 * d) for a, b in zip(prof(z + d), prof(z - d))]
        u0, v0, w0 = prof(0.0)
        du0, dv0, dw0 = dprof(0.0)
        uH, vH, wH = prof(H)
        duH, dvH, dwH = dprof(H)
        scale = max(abs(c) for c in (*bot, *top) for c in c)
        tol = 1e-7 * scale
        assert abs(u0 - l0 * du0 - bot[0][i]) < tol and abs(v0 - l0 * dv0 - bot[1][i]) < tol
        assert abs(w0 - bot[2][i]) < tol
        assert abs(uH + lH * duH - top[0][i]) < tol and abs(vH + lH * dvH - top[1][i]) < tol
        assert abs(wH - top[2][i]) < tol
        for ww, uu, vv in ((dw0, u0, v0), (dwH, uH, vH)):
            assert abs(1j * kx[i] * uu + 1j * ky[i] * vv + ww) < 1e-6 * scale


@pytest.mark.parametrize("mode,l0,lH", [("slit", 0.9, 0.0), ("slit", 0.4, 3.0), ("bottom_wall", 0.7, 0.0)])
def test_total_velocity_satisfies_the_wall_conditions(mode, l0, lH):
    # DP + correction (step 6) for smooth random force spectra: at every k != 0 the tangential
    # velocity obeys u - l0 du/dz = 0 at zmin (and u + lH du/dz = 0 at zmax in the slit), w = 0
    # there, evaluated from the Chebyshev coefficients
    _, bm = table2(5)
    p = Params(Lx=24.0, Ly=24.0, zmin=0.0, zmax=10.0, mode=mode, nx=8, ny=8, nz=65, m_M=5, beta_M=5 * bm,
               eta=0.9, slip_bottom=l0, slip_top=lH)
    rng = np.random.default_rng(8)
    N = p.nz
    decay = np.exp(-np.arange(N) / 4.0)
    f = (rng.standard_normal((3, 8, 8, N)) + 1j * rng.standard_normal((3, 8, 8, N))) * decay
    vel, _ = stokes.solve_spectral(p, f)
    KX, KY, nyq = stokes.wavenumbers(p)
    live = (np.hypot(KX, KY) > 0) & ~nyq
    sign = (-1.0) ** np.arange(N)
    d = stokes.dz(p, vel)
    bot, dbot = (vel * sign).sum(-1), (d * sign).sum(-1)
    top, dtop = vel.sum(-1), d.sum(-1)
    scale = np.max(np.abs(vel[:, live]))
    assert np.max(np.abs((bot[:2] - l0 * dbot[:2])[:, live])) < 1e-8 * scale
    assert np.max(np.abs(bot[2][live])) < 1e-8 * scale
    if mode == "slit":
        assert np.max(np.abs((top[:2] + lH * dtop[:2])[:, live])) < 1e-8 * scale
        assert np.max(np.abs(top[2][live])) < 1e-8 * scale


def test_bottom_wall_slip_solution_tends_to_the_closed_form():
    _, bm = table2(5)
    base = dict(Lx=24.0, Ly=24.0, zmin=0.0, zmax=10.0, mode="bottom_wall", nx=36, ny=36, nz=33, m_M=5, beta_M=5 * bm)
    rng = np.random.default_rng(6)
    kx = np.array([0.3, -1.2, 2.0])
    ky = np.array([0.5, 0.1, -0.7])
    d = [rng.standard_normal(3) + 1j * rng.standard_normal(3) for _ in range(3)]
    closed = stokes.correction_bw(Params(**base), *d, kx, ky)
    lu = stokes.correction_bw_slip(Params(**base, slip_bottom=1e-13), *d, kx, ky)
    assert np.allclose(lu, closed, rtol=0, atol=1e-10 * np.max(np.abs(closed)))


def test_mobility_continuous_as_slip_vanishes():
    pos = np.array([[5.1, 7.3, 2.2], [12.2, 4.4, 6.5]])
    rng = np.random.default_rng(7)
    F, T = rng.standard_normal((2, 3)), rng.standard_normal((2, 3))
    U0, W0 = mobility(_slit(0.0, 0.0), pos, F, T)
    U1, W1 = mobility(_slit(1e-9, 1e-9), pos, F, T)
    assert np.max(np.abs(U1 - U0)) < 1e-7 * np.max(np.abs(U0))
    assert np.max(np.abs(W1 - W0)) < 1e-7 * np.max(np.abs(W0))
    U2, _ = mobility(_slit(0.5, 0.5), pos, F, T)
    assert np.max(np.abs(U2 - U0)) > 1e-3 * np.max(np.abs(U0))  # slip changes the answer


@pytest.mark.slow
def test_slit_with_slip_tends_to_the_bottom_wall_with_slip():
    _, bm = table2(5)
    pos = np.array([[6.1, 5.2, 2.0]])
    F = np.array([[1.0, 0.3, -0.5]])
    common = dict(Lx=16.0, Ly=16.0, zmin=0.0, nx=24, ny=24, m_M=5, beta_M=5 * bm, slip_bottom=0.8)
    Ub, _ = mobility(Params(**common, zmax=8.0, mode="bottom_wall", nz=33), pos, F)
    # the difference is the k = 0 mean flow of the unit net force, which falls as 1/H
    d = []
    for zmax, nz in ((40.0, 97), (80.0, 129)):
        Us, _ = mobility(Params(**common, zmax=zmax, mode="slit", nz=nz, slip_top=0.4), pos, F)
        d.append(np.max(np.abs(Us - Ub)) / np.max(np.abs(Ub)))
    assert d[0] < 2e-2 and 0.4 * d[0] < d[1] < 0.6 * d[0]


@pytest.mark.slow
@pytest.mark.parametrize("zr", [4.0, 6.0])
def test_perfect_slip_wall_matches_free_surface_images(zr):
    # Leading image corrections for a sphere near a plane: no-slip 1 - (9/16) a/z parallel and
    # 1 - (9/8) a/z normal; shear-free 1 + (3/8) a/z and 1 - (3/4) a/z; the next terms are
    # O((a/z)^3).  The bottom wall is made shear-free with l0 -> infinity; a tall slit keeps the k = 0
    # problem well posed (above one shear-free wall with an open top it has no steady solution) and
    # the difference slip - no-slip removes the distant top wall to leading order.
    rh_h, bm = table2(6)
    base = dict(Lx=96.0, Ly=96.0, zmin=0.0, zmax=48.0, mode="slit", nx=96, ny=96, nz=97, m_M=6,
                beta_M=6 * bm)
    Rh = rh_h * 1.0
    pos = np.array([[48.3, 48.7, zr * Rh]])
    mu = {}
    for l0 in (0.0, 1e9):
        p = Params(**base, slip_bottom=l0)
        Ux, _ = mobility(p, pos, np.array([[1.0, 0, 0]]))
        Uz, _ = mobility(p, pos, np.array([[0, 0, 1.0]]))
        mu[l0] = (6 * np.pi * p.eta * Rh * Ux[0, 0], 6 * np.pi * p.eta * Rh * Uz[0, 2])
    x = 1.0 / zr
    d_par = mu[1e9][0] - mu[0.0][0]
    d_perp = mu[1e9][1] - mu[0.0][1]
    assert d_par == pytest.approx((3 / 8 + 9 / 16) * x, abs=x**3 + 3e-3)
    assert d_perp == pytest.approx((9 / 8 - 3 / 4) * x, abs=x**3 + 3e-3)


@pytest.mark.slow
def test_grand_mobility_with_slip_symmetric_positive_definite():
    p = Params(Lx=20.0, Ly=20.0, zmin=0.0, zmax=10.0, mode="slit", nx=40, ny=40, nz=65, m_M=6,
               beta_M=6 * table1(6)[1], m_D=6, beta_D=6 * table1(6)[2], slip_bottom=0.7, slip_top=2.0)
    pos = np.array([[4.1, 5.3, 2.6], [7.2, 4.4, 3.9]])
    n = 2
    M = np.zeros((6 * n, 6 * n))
    for col in range(6 * n):
        e = np.zeros(6 * n)
        e[col] = 1.0
        U, W = mobility(p, pos, e[: 3 * n].reshape(n, 3), e[3 * n:].reshape(n, 3))
        M[:, col] = np.concatenate([U.ravel(), W.ravel()])
    assert np.linalg.norm(M - M.T) / np.linalg.norm(M) < 2e-4
    assert np.min(np.linalg.eigvalsh(0.5 * (M + M.T))) > 0.0


def test_slip_rejected_where_there_is_no_wall():
    _, bm = table2(5)
    with pytest.raises(ValueError):
        Params(Lx=24.0, Ly=24.0, zmin=0.0, zmax=10.0, mode="bottom_wall", nx=36, ny=36, nz=33, m_M=5,
               beta_M=5 * bm, slip_top=1.0)
    with pytest.raises(ValueError):
        Params(Lx=24.0, Ly=24.0, zmin=0.0, zmax=10.0, mode="free", nx=36, ny=36, nz=33, m_M=5, beta_M=5 * bm,
               uw_bottom=(1.0, 0.0))
    with pytest.raises(ValueError):
        _slit(-0.1, 0.0)
