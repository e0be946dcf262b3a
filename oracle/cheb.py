"""Chebyshev machinery in z (test infrastructure only).

Grid (Sec. III.D): "type-2" Chebyshev nodes including both endpoints, read as the extrema
(Gauss-Lobatto) nodes s_c = cos(pi*c/(Nz-1)), c = 0..Nz-1, mapped to
z_c = zmin + (H/2)(1 + s_c).  Node c = 0 is the top (zmax), c = Nz-1 the bottom (zmin).
This is the node set on which a 2Nz-2 point FFT computes Chebyshev coefficients
(footnote to Sec. III.D).
"""

import numpy as np


def nodes_s(nz):
    """Extrema Chebyshev nodes s_c = cos(pi c/(nz-1)) on [-1, 1] (Sec. III.D)."""
    c = np.arange(nz)
    return np.cos(np.pi * c / (nz - 1))


def nodes_z(nz, zmin, zmax):
    """Chebyshev nodes mapped to [zmin, zmax] (Sec. III.D)."""
    return zmin + 0.5 * (zmax - zmin) * (1.0 + nodes_s(nz))


def dct1_matrix(nz):
    """Forward DCT-I as a matrix: node values -> Chebyshev coefficients (step 2, Sec. III.D).

    a_n = (2/(N-1)) * sum''_c g_c cos(pi n c/(N-1)), where sum'' halves the c = 0 and
    c = N-1 terms, and a_0, a_{N-1} are halved afterwards.  This is the interpolating
    Chebyshev series through the node values.
    """
    n1 = nz - 1
    c = np.arange(nz)
    C = np.cos(np.pi * np.outer(c, c) / n1) * (2.0 / n1)
    C[:, 0] *= 0.5
    C[:, -1] *= 0.5
    C[0, :] *= 0.5
    C[-1, :] *= 0.5
    return C


def idct1_matrix(nz):
    """Inverse DCT-I: Chebyshev coefficients -> node values, g_c = sum_n a_n T_n(s_c) (step 7)."""
    n1 = nz - 1
    c = np.arange(nz)
    return np.cos(np.pi * np.outer(c, c) / n1)


def dct1_via_fft(g):
    """Chebyshev coefficients by the FFT of the even extension of length 2N-2 (Sec. III.D
    footnote).  Used only to cross-check dct1_matrix.  g has the node axis last."""
    g = np.asarray(g)
    n1 = g.shape[-1] - 1
    ext = np.concatenate([g, g[..., -2:0:-1]], axis=-1)
    G = np.fft.fft(ext, axis=-1)[..., : n1 + 1] / n1
    G[..., 0] *= 0.5
    G[..., -1] *= 0.5
    return G.real if np.isrealobj(g) else G


def clenshaw_curtis_weights(nz, H):
    """Quadrature weights w_c on the nodes: integral of the interpolating Chebyshev series.

    int_{-1}^{1} T_n ds = 2/(1-n^2) for even n and 0 for odd n, so w = C^T I with C the
    forward DCT-I matrix; scaled by H/2 for [zmin, zmax] (step 8 of Sec. III.D: trapezoid rule in xy,
    Chebyshev quadrature in z).
    """
    integ = np.zeros(nz)
    n_even = np.arange(0, nz, 2).astype(float)
    integ[0::2] = 2.0 / (1.0 - n_even**2)
    return 0.5 * H * (dct1_matrix(nz).T @ integ)


def cheb_derivative(a, axis=-1):
    """d/ds of a Chebyshev series by the standard recurrence (step 2, Sec. III.D).

    b_{N-1} = 0, b_{N-2} = 2(N-1) a_{N-1}, b_{n-1} = b_{n+1} + 2 n a_n, then b_0 <- b_0/2.
    """
    a = np.moveaxis(np.asarray(a), axis, -1)
    N = a.shape[-1]
    b = np.zeros_like(a)
    if N >= 2:
        b[..., N - 2] = 2 * (N - 1) * a[..., N - 1]
    for n in range(N - 2, 0, -1):
        b[..., n - 1] = (b[..., n + 1] if n + 1 < N else 0) + 2 * n * a[..., n]
    b[..., 0] *= 0.5
    return np.moveaxis(b, -1, axis)


def cheb_antiderivative(c):
    """Exact antiderivative B of a Chebyshev series with zero constant term.

    (Bc)_n = (gamma_{n-1} c_{n-1} - c_{n+1}) / (2n) for n >= 1, gamma_0 = 2, gamma_{n>0} = 1,
    c_n = 0 beyond the input length, (Bc)_0 = 0.  Output length = input length + 1.
    This is the integration operator of Greengard's spectral-integration BVP method on which
    the paper's BVP solver is based (Sec. III.D, step 3).
    """
    c = np.asarray(c)
    N = c.shape[-1]
    out = np.zeros(c.shape[:-1] + (N + 1,), dtype=c.dtype)
    for n in range(1, N + 1):
        lo = c[..., n - 1] * (2.0 if n - 1 == 0 else 1.0)
        hi = c[..., n + 1] if n + 1 < N else 0.0
        out[..., n] = (lo - hi) / (2.0 * n)
    return out
