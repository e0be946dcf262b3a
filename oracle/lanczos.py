"""Krylov square root of the mobility for Brownian increments (test infrastructure only).

Sec. IV.C: Brownian dynamics needs g = M^{1/2} W with W a vector of i.i.d. standard normal numbers;
the paper estimates it with the Lanczos process in the Krylov subspace of M and measures
convergence by eps_n = ||g_n - g_{n-1}|| / ||g_{n-1}||.

Steps (the Lanczos process for a function of a symmetric operator applied to a vector):
  beta_0 = ||W||, v_1 = W / beta_0;
  for j = 1, 2, ...:
      w = M v_j, orthogonalised against v_1..v_j (two classical Gram-Schmidt passes; the
      coefficient on v_j is alpha_j), beta_j = ||w||, v_{j+1} = w / beta_j;
      T_j = tridiag(beta_1..beta_{j-1}; alpha_1..alpha_j; beta_1..beta_{j-1});
      g_j = beta_0 V_j T_j^{1/2} e_1, with T_j^{1/2} from the eigendecomposition of T_j.
Readings where the paper is silent:
* Full re-orthogonalisation (two passes) keeps V_j orthonormal, so ||g_j - g_{j-1}|| and
  ||g_{j-1}|| are computed from the coefficient vectors y_j = T_j^{1/2} e_1.
* Eigenvalues of T_j below zero (a mobility that is singular, e.g. with a particle on a wall, or
  slightly non-symmetric at coarse Nz) take a zero square root.
* The process stops when eps_j <= tol (j >= 2), when beta_j vanishes (an invariant subspace: the
  result is then exact), or after max_iter steps.
"""

import numpy as np


def sqrt_tridiagonal_e1(alpha, beta):
    """T^{1/2} e_1 for the symmetric tridiagonal T with diagonal alpha and off-diagonal beta."""
    j = len(alpha)
    T = np.diag(np.asarray(alpha, dtype=float))
    if j > 1:
        T += np.diag(np.asarray(beta[: j - 1], dtype=float), 1) + np.diag(np.asarray(beta[: j - 1], dtype=float), -1)
    lam, Q = np.linalg.eigh(T)
    return Q @ (np.sqrt(np.maximum(lam, 0.0)) * Q[0, :])


def lanczos_sqrt(matvec, w, tol=1e-3, max_iter=50):
    """g ~ M^{1/2} w by Lanczos with full re-orthogonalisation.

    matvec: x -> M x on 1-D float arrays; w: 1-D array.  Returns (g, eps, iters) with eps the list
    of eps_n for n = 2..iters (the convergence history of Sec. IV.C)."""
    w = np.asarray(w, dtype=float)
    beta0 = np.linalg.norm(w)
    if beta0 == 0.0:
        return np.zeros_like(w), [], 0
    V = [w / beta0]
    alpha, beta, eps = [], [], []
    y_prev = None
    for j in range(1, max_iter + 1):
        r = matvec(V[-1])
        Vm = np.array(V)
        c1 = Vm @ r
        r = r - Vm.T @ c1
        c2 = Vm @ r
        r = r - Vm.T @ c2
        alpha.append(c1[-1] + c2[-1])
        b = np.linalg.norm(r)
        y = sqrt_tridiagonal_e1(alpha, beta)
        if y_prev is not None:
            d = y.copy()
            d[: len(y_prev)] -= y_prev
            eps.append(np.linalg.norm(d) / np.linalg.norm(y_prev))
        y_prev = y
        done = (eps and eps[-1] <= tol) or b == 0.0 or j == max_iter
        if done:
            g = beta0 * (np.array(V).T @ y)
            return g, eps, j
        beta.append(b)
        V.append(r / b)
    raise AssertionError("unreachable")


__all__ = ["lanczos_sqrt", "sqrt_tridiagonal_e1"]
