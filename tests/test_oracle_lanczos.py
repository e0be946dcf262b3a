"""Pins for the oracle's Krylov square root (Sec. IV.C, Lanczos for g = M^{1/2} W).

* T^{1/2} e_1 from the eigendecomposition equals scipy's Schur-based sqrtm of T.
* Run to the full dimension, the process returns A^{1/2} w exactly (scipy sqrtm) for a random SPD
  matrix, and sqrt(lambda) w for a diagonal one.
* The reported eps_n equal ||g_n - g_{n-1}|| / ||g_{n-1}|| of the explicit iterates.
* With the oracle's own mobility product as the operator (three particles above a wall, forces
  only), the result matches the square root of the assembled matrix to its symmetry error.
"""

import numpy as np
import pytest
import scipy.linalg

from oracle import Params, mobility, table2
from oracle.lanczos import lanczos_sqrt, sqrt_tridiagonal_e1


def _spd(n, seed, cond=50.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1.0, cond, n)
    return (Q * lam) @ Q.T


def test_tridiagonal_square_root_matches_schur_sqrtm():
    rng = np.random.default_rng(1)
    a = rng.uniform(2.0, 3.0, 9)
    b = rng.uniform(-0.8, 0.8, 8)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    want = np.real(scipy.linalg.sqrtm(T))[:, 0]
    assert np.allclose(sqrt_tridiagonal_e1(a, b), want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [7, 25])
def test_full_dimension_gives_the_exact_square_root(n):
    A = _spd(n, n)
    w = np.random.default_rng(n + 1).standard_normal(n)
    g, eps, it = lanczos_sqrt(lambda x: A @ x, w, tol=0.0, max_iter=n)
    want = np.real(scipy.linalg.sqrtm(A)) @ w
    assert it == n
    assert np.linalg.norm(g - want) <= 1e-10 * np.linalg.norm(want)


def test_diagonal_operator():
    lam = np.array([0.5, 1.0, 2.0, 4.0, 9.0])
    w = np.array([1.0, -2.0, 0.5, 3.0, -1.0])
    g, _, _ = lanczos_sqrt(lambda x: lam * x, w, tol=0.0, max_iter=5)
    assert np.allclose(g, np.sqrt(lam) * w, rtol=0, atol=1e-12)


def test_eps_history_is_the_relative_change_of_the_iterates():
    A = _spd(30, 3, cond=200.0)
    w = np.random.default_rng(4).standard_normal(30)
    gs = [lanczos_sqrt(lambda x: A @ x, w, tol=0.0, max_iter=k)[0] for k in range(1, 8)]
    _, eps, _ = lanczos_sqrt(lambda x: A @ x, w, tol=0.0, max_iter=7)
    explicit = [np.linalg.norm(gs[k] - gs[k - 1]) / np.linalg.norm(gs[k - 1]) for k in range(1, 7)]
    assert np.allclose(eps, explicit, rtol=1e-9, atol=0)
    # the stopping rule: the first n with eps_n <= tol
    tol = explicit[3] * 1.0001
    _, eps2, it = lanczos_sqrt(lambda x: A @ x, w, tol=tol, max_iter=30)
    assert it == 5 and eps2[-1] <= tol


def test_zero_vector():
    g, eps, it = lanczos_sqrt(lambda x: 2 * x, np.zeros(4))
    assert it == 0 and not np.any(g)


@pytest.mark.slow
def test_with_the_oracle_mobility():
    _, bm = table2(4)
    p = Params(Lx=16.0, Ly=16.0, zmin=0.0, zmax=8.0, mode="bottom_wall", nx=24, ny=24, nz=33, m_M=4,
               beta_M=4 * bm)
    pos = np.array([[3.1, 4.2, 1.9], [6.4, 5.0, 2.7], [9.9, 11.3, 1.6]])
    n = len(pos)

    def matvec(x):
        return mobility(p, pos, x.reshape(n, 3))[0].ravel()

    M = np.column_stack([matvec(e) for e in np.eye(3 * n)])
    Ms = 0.5 * (M + M.T)
    asym = np.linalg.norm(M - M.T) / np.linalg.norm(M)
    w = np.random.default_rng(9).standard_normal(3 * n)
    g, _, _ = lanczos_sqrt(matvec, w, tol=0.0, max_iter=3 * n)
    want = np.real(scipy.linalg.sqrtm(Ms)) @ w
    assert np.linalg.norm(g - want) <= 10 * asym * np.linalg.norm(want) + 1e-12
