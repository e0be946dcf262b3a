"""Pins for the oracle's Chebyshev machinery (Sec. III.D) against closed forms and library
routines that are independent of it."""

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

from oracle import cheb


@pytest.mark.parametrize("nz", [5, 17, 33, 65, 97])
def test_dct_matrix_equals_even_extension_fft(nz):
    # Sec. III.D footnote: Chebyshev coefficients from a 2Nz-2 point FFT of the even extension.
    rng = np.random.default_rng(1)
    g = rng.standard_normal((4, nz)) + 1j * rng.standard_normal((4, nz))
    a_mat = g @ cheb.dct1_matrix(nz).T
    a_fft = cheb.dct1_via_fft(g)
    assert np.max(np.abs(a_mat - a_fft)) < 1e-13 * np.max(np.abs(g)) * nz


@pytest.mark.parametrize("nz", [9, 65])
def test_dct_recovers_chebyshev_polynomials(nz):
    s = cheb.nodes_s(nz)
    for n in range(nz):
        samples = npcheb.chebval(s, np.eye(nz)[n])          # T_n at the nodes (library)
        a = cheb.dct1_matrix(nz) @ samples
        assert np.max(np.abs(a - np.eye(nz)[n])) < 1e-13


@pytest.mark.parametrize("nz", [9, 65])
def test_inverse_dct_round_trip(nz):
    rng = np.random.default_rng(2)
    a = rng.standard_normal(nz)
    g = cheb.idct1_matrix(nz) @ a
    assert np.allclose(g, npcheb.chebval(cheb.nodes_s(nz), a), atol=1e-13)
    assert np.allclose(cheb.dct1_matrix(nz) @ g, a, atol=1e-13)


def test_nodes_order_and_endpoints():
    z = cheb.nodes_z(65, 0.0, 8.0)
    assert z[0] == pytest.approx(8.0) and z[-1] == pytest.approx(0.0, abs=1e-15)
    assert np.all(np.diff(z) < 0)


def _clencurt_closed_form(n):
    # Explicit Clenshaw-Curtis weights on the n+1 extrema nodes (Waldvogel's formula as given in
    # Trefethen, Spectral Methods in MATLAB, ch. 12); an independent restatement.
    theta = np.pi * np.arange(n + 1) / n
    w = np.zeros(n + 1)
    v = np.ones(n - 1)
    ii = np.arange(1, n)
    if n % 2 == 0:
        w[0] = w[n] = 1.0 / (n * n - 1)
        for k in range(1, n // 2):
            v -= 2.0 * np.cos(2 * k * theta[ii]) / (4 * k * k - 1)
        v -= np.cos(n * theta[ii]) / (n * n - 1)
    else:
        w[0] = w[n] = 1.0 / (n * n)
        for k in range(1, (n - 1) // 2 + 1):
            v -= 2.0 * np.cos(2 * k * theta[ii]) / (4 * k * k - 1)
    w[ii] = 2.0 * v / n
    return w


@pytest.mark.parametrize("nz", [5, 8, 33, 64, 65, 97])
def test_clenshaw_curtis_weights(nz):
    H = 7.5
    w = cheb.clenshaw_curtis_weights(nz, H)
    assert np.allclose(w, 0.5 * H * _clencurt_closed_form(nz - 1), rtol=0, atol=1e-14)
    assert w.sum() == pytest.approx(H, rel=1e-14)
    z = cheb.nodes_z(nz, 1.0, 1.0 + H)
    for d in range(nz):            # exact for polynomials of degree <= nz-1
        exact = ((1.0 + H) ** (d + 1) - 1.0) / (d + 1)
        assert np.dot(w, z**d) == pytest.approx(exact, rel=1e-11)


@pytest.mark.parametrize("N", [3, 8, 33, 65])
def test_derivative_recurrence_matches_library(N):
    rng = np.random.default_rng(3)
    a = rng.standard_normal((5, N))
    ours = cheb.cheb_derivative(a)
    lib = np.stack([np.concatenate([npcheb.chebder(row), [0.0]]) for row in a])
    assert np.max(np.abs(ours - lib)) < 1e-12 * N * N


@pytest.mark.parametrize("N", [2, 8, 33, 65])
def test_antiderivative_matches_library(N):
    rng = np.random.default_rng(4)
    c = rng.standard_normal((3, N))
    ours = cheb.cheb_antiderivative(c)
    for row, o in zip(c, ours):
        lib = npcheb.chebint(row)               # differs only in the constant term
        assert np.allclose(o[1:], lib[1:], atol=1e-14)
        assert o[0] == 0.0
        assert np.allclose(cheb.cheb_derivative(o)[:N], row, atol=1e-12)
