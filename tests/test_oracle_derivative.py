"""Pins for the oracle's second torque route (ES-kernel derivatives; Sec. III.D, the paragraph after
the algorithm and its footnotes).

* The derivative kernel and the imaged z factor against central differences of the kernel itself.
* The truncation point against a brute-force search for the smallest |phi'| near the edge.
* A particle on a wall is immobile: every component of the gradient vanishes there (the reason the
  paper gives for the sign of the image in the z derivative).
* Curl spreading and curl interpolation are adjoint under the quadrature inner product.
* Invariances of the full product: xy translation by cells and periods, x mirror, slit midplane
  reflection.
* Both torque routes approximate the same continuum operator: their difference falls quickly when
  the grid is refined at a fixed physical kernel.  Rotation near a wall matches the classical
  leading wall corrections, and the grand mobility is symmetric and positive definite.
"""

import numpy as np
import pytest

from oracle import Params, cheb, mobility, table1
from oracle.kernel import (es, es_derivative, es_derivative_cutoff, es_normalization, z_envelope,
                           z_envelope_derivative)
from oracle.transfer import interpolate_curl, spread_curl

ROUTE = "kernel_derivative"


def _small(mode, nz=25):
    _, bm, bd = table1(5)
    return Params(Lx=24.0, Ly=24.0, zmin=0.0, zmax=10.0, mode=mode, nx=36, ny=36, nz=nz, m_M=5,
                  beta_M=5 * bm, m_D=5, beta_D=5 * bd, eta=0.9)


def _particles(p, n, seed, zlo, zhi):
    rng = np.random.default_rng(seed)
    pos = np.stack([rng.uniform(0, p.Lx, n), rng.uniform(0, p.Ly, n), rng.uniform(zlo, zhi, n)], 1)
    return pos, rng.standard_normal((n, 3)), rng.standard_normal((n, 3))


@pytest.mark.parametrize("alpha,beta", [(5 / 3, 11.16), (5 / 3, 6.525), (2.0, 13.296)])
def test_derivative_matches_central_differences(alpha, beta):
    Z = es_normalization(alpha, beta)
    cut = es_derivative_cutoff(alpha, beta)
    t = np.linspace(-0.999 * cut, 0.999 * cut, 801)
    eps = 1e-6 * alpha
    fd = (es(t + eps, alpha, beta, Z) - es(t - eps, alpha, beta, Z)) / (2 * eps)
    d = es_derivative(t, alpha, beta, Z, cut)
    assert np.max(np.abs(d - fd)) < 1e-6 * np.max(np.abs(d))
    # zero beyond the truncation point, odd inside
    assert np.all(es_derivative(np.array([1.0001 * cut, -1.0001 * cut, alpha]), alpha, beta, Z, cut) == 0.0)
    assert np.allclose(es_derivative(-t, alpha, beta, Z, cut), -d, rtol=0, atol=1e-15)


@pytest.mark.parametrize("mode,zp", [("bottom_wall", 0.7), ("slit", 0.4), ("slit", 9.2), ("free", 5.0)])
def test_z_derivative_with_images_matches_central_differences(mode, zp):
    alpha, beta = 5 / 3, 11.16
    Z = es_normalization(alpha, beta)
    cut = es_derivative_cutoff(alpha, beta)
    # node heights where no term sits on its truncation point, inside [0, 10]
    zc = np.linspace(0.0, 10.0, 4001)
    terms = [zc - zp]
    if mode in ("bottom_wall", "slit"):
        terms.append(zc + zp)
    if mode == "slit":
        terms.append(zc - (20.0 - zp))
    keep = np.all([np.abs(np.abs(tt) - cut) > 1e-3 for tt in terms], axis=0)
    keep &= np.all([np.abs(np.abs(tt) - alpha) > 1e-3 for tt in terms], axis=0)
    zc = zc[keep]
    eps = 1e-7
    fd = (z_envelope(zc + eps, zp, alpha, beta, mode, 0.0, 10.0, Z)
          - z_envelope(zc - eps, zp, alpha, beta, mode, 0.0, 10.0, Z)) / (2 * eps)
    d = z_envelope_derivative(zc, zp, alpha, beta, mode, 0.0, 10.0, Z, cut)
    # away from the truncation band the derivative is the exact one of the imaged envelope
    band = np.any([(np.abs(tt[keep]) > cut) & (np.abs(tt[keep]) <= alpha) for tt in terms], axis=0)
    assert np.max(np.abs(d[~band] - fd[~band])) < 1e-6 * np.max(np.abs(d))
    assert np.all(d[band & np.all([np.abs(tt[keep]) > cut for tt in terms], axis=0)] == 0.0)


@pytest.mark.parametrize("alpha,beta", [(5 / 3, 11.16), (1.5, 10.2), (1.0, 4.0)])
def test_cutoff_is_the_smallest_derivative_before_the_edge(alpha, beta):
    # |phi'| by central differences of phi on a dense grid, minimised between its maximum and the
    # edge, where it blows up
    Z = es_normalization(alpha, beta)
    t = np.linspace(0.5 * alpha, alpha * (1 - 1e-9), 400001)
    eps = 1e-9 * alpha
    mag = np.abs(es(t + eps, alpha, beta, Z) - es(t - eps, alpha, beta, Z)) / (2 * eps)
    peak = np.argmax(mag[: len(t) // 2])
    i = peak + np.argmin(mag[peak:])
    assert es_derivative_cutoff(alpha, beta) == pytest.approx(t[i], abs=4 * (t[1] - t[0]))


def test_cutoff_needs_an_interior_minimum():
    with pytest.raises(ValueError):
        es_derivative_cutoff(1.0, 2.5)  # beta <= 3 sqrt(3) / 2: |phi'| grows up to the edge


@pytest.mark.parametrize("mode", ["bottom_wall", "slit"])
def test_particle_on_wall_is_immobile(mode):
    p = _small(mode)
    pos, F, T = _particles(p, 2, 14, 2.0, 7.0)
    pos[0, 2] = 0.0
    U, W = mobility(p, pos, F, T, torque_route=ROUTE)
    assert np.all(U[0] == 0.0) and np.all(W[0] == 0.0)
    U1, W1 = mobility(p, pos[1:], F[1:], T[1:], torque_route=ROUTE)
    assert np.allclose(U[1], U1[0], atol=1e-14) and np.allclose(W[1], W1[0], atol=1e-14)


@pytest.mark.parametrize("mode", ["bottom_wall", "slit", "free"])
def test_curl_spreading_and_interpolation_are_adjoint(mode):
    p = _small(mode)
    pos, _, T = _particles(p, 5, 17, 1.8 if mode == "free" else 0.3, 7.5)
    rng = np.random.default_rng(19)
    u = rng.standard_normal((3, p.nz, p.ny, p.nx))
    lhs = np.sum(interpolate_curl(p, pos, u) * T)
    wz = cheb.clenshaw_curtis_weights(p.nz, p.H)
    rhs = p.h * p.h * np.sum(spread_curl(p, pos, T) * u * wz[None, :, None, None])
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_uniform_rotation_field_gives_its_angular_velocity():
    # u = Omega0 x (x - c) is interpolated exactly enough by the gradient kernel: Omega_j = Omega0
    # for a particle far from walls (integration by parts of Eq. 11 with the unit envelope).
    p = Params(Lx=24.0, Ly=24.0, zmin=0.0, zmax=10.0, mode="free", nx=72, ny=72, nz=65, m_M=10,
               beta_M=10 * table1(5)[1], m_D=10, beta_D=5 * table1(5)[2])
    om0 = np.array([0.3, -0.7, 0.5])
    c = np.array([12.1, 11.7, 5.0])
    zn = cheb.nodes_z(p.nz, p.zmin, p.zmax)
    X, Y, Zg = np.meshgrid(np.arange(p.nx) * p.h, np.arange(p.ny) * p.h, zn, indexing="ij")
    r = np.stack([X - c[0], Y - c[1], Zg - c[2]])
    u = np.cross(om0[:, None, None, None], r, axis=0)           # (3, nx, ny, nz)
    u = np.transpose(u, (0, 3, 2, 1))                           # (3, nz, ny, nx)
    pos = np.array([[12.4, 11.2, 5.3], [11.9, 12.6, 4.6]])
    W = interpolate_curl(p, pos, u)
    assert np.max(np.abs(W - om0)) < 2e-3 * np.max(np.abs(om0))


@pytest.mark.parametrize("mode", ["bottom_wall", "slit", "free"])
def test_translation_by_cells_and_periods(mode):
    p = _small(mode)
    pos, F, T = _particles(p, 4, 11, 2.0, 7.5)
    U, W = mobility(p, pos, F, T, torque_route=ROUTE)
    for shift in ([3 * p.h, -5 * p.h, 0.0], [p.Lx, -2 * p.Ly, 0.0]):
        U2, W2 = mobility(p, pos + np.array(shift), F, T, torque_route=ROUTE)
        assert np.max(np.abs(U2 - U)) < 1e-12 * np.max(np.abs(U))
        assert np.max(np.abs(W2 - W)) < 1e-12 * np.max(np.abs(W))


@pytest.mark.parametrize("mode", ["bottom_wall", "free"])
def test_x_mirror(mode):
    p = _small(mode)
    pos, F, T = _particles(p, 3, 16, 2.0, 7.5)
    U, W = mobility(p, pos, F, T, torque_route=ROUTE)
    ref = np.array([-1.0, 1.0, 1.0])
    pref = np.array([1.0, -1.0, -1.0])
    pos2 = pos.copy()
    pos2[:, 0] = -pos[:, 0]
    U2, W2 = mobility(p, pos2, F * ref, T * pref, torque_route=ROUTE)
    assert np.max(np.abs(U2 - U * ref)) < 1e-12 * np.max(np.abs(U))
    assert np.max(np.abs(W2 - W * pref)) < 1e-12 * np.max(np.abs(W))


def test_slit_midplane_reflection():
    p = _small("slit")
    pos, F, T = _particles(p, 3, 15, 0.5, 9.5)
    U, W = mobility(p, pos, F, T, torque_route=ROUTE)
    ref = np.array([1.0, 1.0, -1.0])
    pref = np.array([-1.0, -1.0, 1.0])
    pos2 = pos.copy()
    pos2[:, 2] = p.zmin + p.zmax - pos[:, 2]
    U2, W2 = mobility(p, pos2, F * ref, T * pref, torque_route=ROUTE)
    assert np.max(np.abs(U2 - U * ref)) < 1e-12 * np.max(np.abs(U))
    assert np.max(np.abs(W2 - W * pref)) < 1e-12 * np.max(np.abs(W))


@pytest.mark.slow
def test_routes_converge_together_under_refinement():
    # Same physical kernels (alpha = 5/3, Table I shapes for m = 5) sampled with h = 2/3 and 1/3:
    # the two routes differ by the sampling error of the kernel, which falls fast with h.
    _, bm, bd = table1(5)
    rng = np.random.default_rng(3)
    pos = np.stack([rng.uniform(0, 24, 3), rng.uniform(0, 24, 3), rng.uniform(2.5, 7.0, 3)], 1)
    F = np.zeros((3, 3))
    T = rng.standard_normal((3, 3))
    dW, dU = [], []
    for nx, m, nz in ((36, 5, 65), (72, 10, 65)):
        p = Params(Lx=24.0, Ly=24.0, zmin=0.0, zmax=10.0, mode="bottom_wall", nx=nx, ny=nx, nz=nz, m_M=m,
                   beta_M=5 * bm, m_D=m, beta_D=5 * bd, eta=0.9)
        U1, W1 = mobility(p, pos, F, T)
        U2, W2 = mobility(p, pos, F, T, torque_route=ROUTE)
        dW.append(np.linalg.norm(W1 - W2) / np.linalg.norm(W1))
        dU.append(np.linalg.norm(U1 - U2) / np.linalg.norm(U1))
    assert dW[0] < 3e-2 and dW[1] < 2e-4 and dW[1] < dW[0] / 50
    assert dU[0] < 3e-2 and dU[1] < dU[0] / 3


@pytest.mark.slow
@pytest.mark.parametrize("zr", [2.0, 4.0])
def test_self_rotation_vs_wall_asymptotics(zr):
    # Leading wall corrections to the rotational mobility: 1 - (5/16)(a/z)^3 about an axis parallel
    # to the wall, 1 - (1/8)(a/z)^3 about the normal (the same bar as the spectral-curl route).
    rh_h, bm, bd = table1(6)
    p = Params(Lx=160.0, Ly=160.0, zmin=0.0, zmax=16.0, mode="bottom_wall", nx=160, ny=160, nz=33,
               m_M=6, beta_M=6 * bm, m_D=6, beta_D=6 * bd)
    Rh = rh_h * p.h
    pos = np.array([[80.3, 80.7, zr * Rh]])
    zero = np.zeros((1, 3))
    _, Wx = mobility(p, pos, zero, np.array([[1.0, 0, 0]]), torque_route=ROUTE)
    _, Wz = mobility(p, pos, zero, np.array([[0, 0, 1.0]]), torque_route=ROUTE)
    norm = 8 * np.pi * p.eta * Rh**3
    assert norm * Wx[0, 0] == pytest.approx(1 - 5 / 16 / zr**3, rel=1e-2)
    assert norm * Wz[0, 2] == pytest.approx(1 - 1 / 8 / zr**3, rel=1e-2)


@pytest.mark.slow
@pytest.mark.parametrize("mode", ["bottom_wall", "slit"])
def test_grand_mobility_symmetric_positive_definite(mode):
    p = Params(Lx=20.0, Ly=20.0, zmin=0.0, zmax=10.0, mode=mode, nx=40, ny=40, nz=65, m_M=6,
               beta_M=6 * table1(6)[1], m_D=6, beta_D=6 * table1(6)[2])
    pos = np.array([[4.1, 5.3, 2.6], [7.2, 4.4, 3.9]])
    n = pos.shape[0]
    M = np.zeros((6 * n, 6 * n))
    for col in range(6 * n):
        e = np.zeros(6 * n)
        e[col] = 1.0
        U, W = mobility(p, pos, e[: 3 * n].reshape(n, 3), e[3 * n:].reshape(n, 3), torque_route=ROUTE)
        M[:, col] = np.concatenate([U.ravel(), W.ravel()])
    assert np.linalg.norm(M - M.T) / np.linalg.norm(M) < 2e-4
    assert np.min(np.linalg.eigvalsh(0.5 * (M + M.T))) > 0.0
