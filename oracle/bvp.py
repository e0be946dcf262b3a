"""Per-wavenumber Chebyshev boundary-value problems (test infrastructure only).

Every BVP of the method has the form  (d^2/dz^2 - k^2) y(z) = r(z)  on [zmin, zmax] with two
boundary rows (Eqs. 15/17 for the pressure, 18/22/24 for the velocity, 51/52 and A12 for the
zero mode).  The paper defers the discretisation to Greengard's spectral-integration method
(step 3 of Sec. III.D) without printing it; the reading used here is:

* s = 2(z - zmin)/H - 1, so d/dz = (2/H) d/ds.
* Unknowns: the N Chebyshev coefficients c of y_ss plus two constants a0, a1, with
  y = trunc_N(B(B c)) + a0 T_0 + a1 T_1, B the exact Chebyshev antiderivative
  (cheb.cheb_antiderivative) applied twice and trunc_N keeping coefficients 0..N-1.
* N equation rows: (2/H)^2 c_n - k^2 y_n = r_n, n = 0..N-1, r the Chebyshev coefficients of
  the right-hand side.
* Two boundary rows on the truncated y, using T_n(+-1) = (+-1)^n and T_n'(+-1) = (+-1)^(n+1) n^2:
  - 'dtn'  : (2/H) y_s(+1) + k y(+1) = g_top,  (2/H) y_s(-1) - k y(-1) = g_bot
             (the Dirichlet-to-Neumann rows of Eqs. 17, 22, 24);
  - 'bw0'  : y(-1) - l0 (2/H) y_s(-1) = g_bot, (2/H) y_s(+1) = g_top   (Eq. 52, zero mode above
             one wall; the Robin bottom row with slip length l0 follows Eq. A12);
  - 'sc0'  : y(-1) - l0 (2/H) y_s(-1) = g_bot, y(+1) + lH (2/H) y_s(+1) = g_top   (Eq. A12).
  slip = (l0, lH), zero by default (no-slip walls).

The oracle assembles the full dense (N+2) x (N+2) real matrix and solves it by LU
(numpy.linalg.solve); the matrix is real because it depends on k only through k and k^2.
"""

import numpy as np

from .cheb import cheb_antiderivative


def antiderivative_matrix(n_in):
    """Matrix of the antiderivative B acting on n_in coefficients, shape (n_in+1, n_in)."""
    return cheb_antiderivative(np.eye(n_in)).T


def y_map(N):
    """Y: unknowns [c_0..c_{N-1}, a0, a1] -> coefficients y_0..y_{N-1} (truncated), (N, N+2)."""
    B1 = antiderivative_matrix(N)          # (N+1, N)
    B2 = antiderivative_matrix(N + 1)      # (N+2, N+1)
    Y = np.zeros((N, N + 2))
    Y[:, :N] = (B2 @ B1)[:N, :]
    Y[0, N] = 1.0
    Y[1, N + 1] = 1.0
    return Y


def _endpoint_rows(N):
    n = np.arange(N, dtype=float)
    val_top = np.ones(N)
    val_bot = (-1.0) ** n
    der_top = n * n
    der_bot = (-1.0) ** (n + 1) * n * n
    return val_top, val_bot, der_top, der_bot


def assemble(k, N, H, bc, slip=(0.0, 0.0)):
    """Dense BVP matrices for an array of wavenumber magnitudes k (shape (K,)): (K, N+2, N+2)."""
    k = np.atleast_1d(np.asarray(k, dtype=float))
    Y = y_map(N)
    s = 2.0 / H
    E0 = np.zeros((N, N + 2))
    E0[:, :N] = s * s * np.eye(N)
    A = np.empty((k.size, N + 2, N + 2))
    A[:, :N, :] = E0[None] - (k * k)[:, None, None] * Y[None]
    vt, vb, dt, db = _endpoint_rows(N)
    if bc == "dtn":
        A[:, N, :] = s * (dt @ Y)[None] + k[:, None] * (vt @ Y)[None]
        A[:, N + 1, :] = s * (db @ Y)[None] - k[:, None] * (vb @ Y)[None]
    elif bc == "bw0":
        A[:, N, :] = s * (dt @ Y)[None]
        A[:, N + 1, :] = ((vb - slip[0] * s * db) @ Y)[None]
    elif bc == "sc0":
        A[:, N, :] = ((vt + slip[1] * s * dt) @ Y)[None]
        A[:, N + 1, :] = ((vb - slip[0] * s * db) @ Y)[None]
    else:
        raise ValueError(bc)
    return A, Y


def solve(k, H, r, g_top, g_bot, bc, slip=(0.0, 0.0)):
    """Solve (D^2 - k^2) y = r with the boundary rows `bc` for many wavenumbers at once.

    k: (K,) magnitudes; r: (K, R, N) complex Chebyshev coefficients of R right-hand sides;
    g_top, g_bot: (K, R) complex boundary data.  Returns y coefficients (K, R, N) complex.
    """
    r = np.asarray(r, dtype=complex)
    K, R, N = r.shape
    A, Y = assemble(k, N, H, bc, slip)
    rhs = np.zeros((K, N + 2, 2 * R))
    rhs[:, :N, :R] = np.transpose(r.real, (0, 2, 1))
    rhs[:, :N, R:] = np.transpose(r.imag, (0, 2, 1))
    rhs[:, N, :R] = np.real(g_top)
    rhs[:, N, R:] = np.imag(g_top)
    rhs[:, N + 1, :R] = np.real(g_bot)
    rhs[:, N + 1, R:] = np.imag(g_bot)
    sol = np.linalg.solve(A, rhs)                      # (K, N+2, 2R)
    y = np.einsum("nm,kmr->krn", Y, sol)               # (K, 2R, N)
    return y[:, :R, :] + 1j * y[:, R:, :]


def endpoint_values(y):
    """(y(z_top), y(z_bottom)) of Chebyshev series y along the last axis: sum_n y_n (+-1)^n."""
    N = y.shape[-1]
    sign = (-1.0) ** np.arange(N)
    return y.sum(axis=-1), (y * sign).sum(axis=-1)
