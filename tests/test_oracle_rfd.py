"""Pins for the oracle's random-finite-difference drift (Sec. IV.C footnote).

For one particle above a no-slip wall the divergence of the mobility is d mu_zz / dz in z and zero
in x, y (translation invariance); with W = e_z the RFD is exactly that derivative's central
difference, which must follow the derivative of the Rotne-Prager-Blake normal mobility,
mu_zz = (1 - 9/8 x + 1/2 x^3 - 1/8 x^5) / (6 pi eta a), x = a / z (the paper validates mu_zz
against it for z >~ 2 R_h).  Along a whole-cell translation, under which the discrete mobility is
exactly invariant, the drift vanishes.
"""

import numpy as np
import pytest

from oracle import Params, table2
from oracle.rfd import rfd_drift


def _bw():
    _, bm = table2(6)
    return Params(Lx=160.0, Ly=160.0, zmin=0.0, zmax=16.0, mode="bottom_wall", nx=160, ny=160, nz=33, m_M=6,
                  beta_M=6 * bm)


@pytest.mark.slow
@pytest.mark.parametrize("zr", [2.5, 3.5])
def test_drift_follows_the_wall_mobility_gradient(zr):
    p = _bw()
    a = table2(6)[0] * p.h
    pos = np.array([[80.3, 80.7, zr * a]])
    dU, _ = rfd_drift(p, pos, np.array([[0.0, 0.0, 1.0]]), 1e-3)
    x = 1.0 / zr
    want = (9 / 8 * x**2 - 3 / 2 * x**4 + 5 / 8 * x**6) / (6 * np.pi * p.eta * a * a)
    assert dU[0, 2] == pytest.approx(want, rel=3e-2)
    assert abs(dU[0, 0]) < 1e-12 and abs(dU[0, 1]) < 1e-12


def test_drift_vanishes_along_whole_cell_translations():
    # M is exactly invariant under xy translation by whole cells (Sec. III: periodic grid), so a
    # displacement of every particle by +-1 cell in x gives a zero difference
    _, bm = table2(5)
    p = Params(Lx=24.0, Ly=24.0, zmin=0.0, zmax=10.0, mode="slit", nx=36, ny=36, nz=25, m_M=5, beta_M=5 * bm)
    pos = np.array([[5.1, 7.3, 2.6], [9.2, 6.4, 4.1]])
    W = np.array([[p.h, 0.0, 0.0], [p.h, 0.0, 0.0]])
    dU, _ = rfd_drift(p, pos, W, 2.0)
    assert np.max(np.abs(dU)) < 1e-13
