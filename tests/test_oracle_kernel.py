"""Pins for the oracle's ES kernel (Eq. 54) and wall images (Eq. 9)."""

import numpy as np
import pytest
from scipy import integrate

from oracle import kernel
from oracle.params import BOTTOM_WALL, FREE, SLIT


def test_normalization_beta_zero_is_support_length():
    # beta = 0 makes E(t) = 1 on [-alpha, alpha]: Z = 2 alpha exactly.
    assert kernel.es_normalization(1.7, 0.0) == pytest.approx(3.4, rel=1e-14)


@pytest.mark.parametrize("alpha,beta", [(1.5, 10.2), (5 / 3, 6.525), (5 / 3, 11.16), (2.0, 13.296)])
def test_normalization_against_adaptive_quadrature(alpha, beta):
    f = lambda t: np.exp(beta * (np.sqrt(max(0.0, 1 - (t / alpha) ** 2)) - 1.0))
    ref, err = integrate.quad(f, -alpha, alpha, epsabs=1e-14, epsrel=1e-13, limit=400)
    assert kernel.es_normalization(alpha, beta) == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("alpha,beta", [(1.5, 10.2), (5 / 3, 11.16)])
def test_unit_integral_and_support(alpha, beta):
    t = np.linspace(-alpha, alpha, 400001)
    phi = kernel.es(t, alpha, beta)
    assert integrate.trapezoid(phi, t) == pytest.approx(1.0, abs=2e-7)
    assert np.all(kernel.es(np.array([-alpha * 1.0001, alpha * 1.0001, 10.0]), alpha, beta) == 0.0)
    assert kernel.es(np.array([0.0]), alpha, beta)[0] == pytest.approx(1.0 / kernel.es_normalization(alpha, beta))


def test_periodic_offset_minimum_image():
    L = 10.0
    assert kernel.periodic_offset(0.2, 9.9, L) == pytest.approx(0.3)
    assert kernel.periodic_offset(9.9, 0.2, L) == pytest.approx(-0.3)
    assert kernel.periodic_offset(3.0, 3.0, L) == 0.0


def test_wall_image_vanishes_for_particle_on_wall():
    # Eq. 9 with the particle on the wall: the envelope and its negative image cancel exactly.
    zc = np.linspace(0.0, 3.0, 50)
    v = kernel.z_envelope(zc, 0.0, 1.5, 10.2, BOTTOM_WALL, 0.0, 12.0)
    assert np.max(np.abs(v)) < 1e-15
    v = kernel.z_envelope(zc + 17.0, 20.0, 1.5, 10.2, SLIT, 0.0, 20.0)
    assert np.max(np.abs(v)) < 1e-15


def test_image_only_near_wall():
    zc = np.linspace(0.0, 12.0, 200)
    far = kernel.z_envelope(zc, 5.0, 1.5, 10.2, BOTTOM_WALL, 0.0, 12.0)
    free = kernel.z_envelope(zc, 5.0, 1.5, 10.2, FREE, 0.0, 12.0)
    assert np.array_equal(far, free)
    near = kernel.z_envelope(zc, 1.0, 1.5, 10.2, BOTTOM_WALL, 0.0, 12.0)
    free_near = kernel.z_envelope(zc, 1.0, 1.5, 10.2, FREE, 0.0, 12.0)
    img = kernel.es(zc + 1.0, 1.5, 10.2)
    assert np.allclose(near, free_near - img, atol=1e-16)


def test_kernel_tables_match_the_printed_tables():
    """The oracle's Table I/II constants are the paper's printed values (tests/golden fixture)."""
    import os
    from oracle import table1, table2
    path = os.path.join(os.path.dirname(__file__), "golden", "es_kernel_tables.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    assert len(rows) == 5
    for t, m, rh, bm, bd, _, _ in rows:
        m = int(m)
        if t == "I":
            assert table1(m) == (float(rh), float(bm), float(bd))
        else:
            assert table2(m) == (float(rh), float(bm))
