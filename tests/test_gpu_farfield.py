"""Far-field decay of the pair mobility (Sec. IV.C, Fig. 10) through the C ABI.

Two particles at the same height, a distance d apart along x; a unit force on one, the velocity of
the other in the same direction (nu_par for x, nu_perp for y).  The paper compares with the
asymptotes for d >> R_h: in a slit of width H with the pair at H/2 both tend to 3H / (32 pi eta d^2)
(Liron and Mochon's slit result); above one wall with the pair at height H/2 they tend to
3H^2 / (8 pi eta d^3) and 3H^4 / (64 pi eta d^5) (Blake's image system).  The periodic box is wide
(L = 2048 h) so that the mean flow a net force drives in it (about F H / (4 eta L^2)) and the
periodic images stay below a percent of the values tested.  FP64.
"""

import numpy as np
import pytest

from gpu_helpers import to_dev
from oracle import table2
from paper_2210_01837_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2210_01837_gb300 import build
    build.build()
    binding.load()


def _pair(mode, H, zmax, nz, ds, L=2048.0, n=2048):
    import torch
    _, bm = table2(6)
    params = dict(Lx=L, Ly=L, zmin=0.0, zmax=zmax, mode=mode, nx=n, ny=n, nz=nz, m_M=6, beta_M=6 * bm, eta=1.0)
    plan = binding.Plan.from_params(params, with_torque=False, precision="fp64", max_n=2)
    out = []
    for d in ds:
        pos = np.array([[L / 2, L / 2 + 0.3, H / 2], [L / 2 + d, L / 2 + 0.3, H / 2]])
        nu = []
        for axis in (0, 1):
            F = np.zeros((2, 3))
            F[0, axis] = 1.0
            U, _ = plan.apply(to_dev(pos), to_dev(F), check=True)
            torch.cuda.synchronize()
            nu.append(U.cpu().numpy()[1, axis])
        out.append(nu)
    plan.close()
    return np.array(out)


def _second_moment(m, beta):
    # <t^2> of the ES kernel with support alpha = m h / 2 (h = 1 here)
    from scipy.integrate import quad
    from oracle.kernel import es, es_normalization
    alpha = 0.5 * m
    Z = es_normalization(alpha, beta)
    return quad(lambda t: t * t * es(t, alpha, beta, Z), -alpha, alpha)[0]


def test_slit_pair_mobility_decays_as_liron():
    # Hele-Shaw far field of a force at mid-height: +-3H / (32 pi eta d^2), the sign negative across
    # the force (the backflow the paper notes).  The force is spread, and the velocity averaged, over
    # the kernel, which multiplies the Poiseuille coupling z0 (H - z0) by 1 - <t^2> / (z0 (H - z0))
    # on each side.
    H = 10.0
    ds = np.array([30.0, 45.0, 60.0])
    nu = _pair("slit", H, H, 33, ds)
    m2 = _second_moment(6, 6 * table2(6)[1])
    fac = (1.0 - m2 / (H * H / 4)) ** 2
    asym = fac * 3 * H / (32 * np.pi * ds**2)
    assert np.allclose(nu[:, 0], asym, rtol=1e-2)
    assert np.allclose(nu[:, 1], -asym, rtol=1e-2)


def test_bottom_wall_pair_mobility_decays_as_blake():
    # parallel: 3 H^2 / (8 pi eta d^3) approached as d grows (corrections O(H/d)); normal:
    # 3 H^4 / (64 pi eta d^5), whose d^-5 decay is checked (its prefactor carries the kernel's
    # second moment, (1 + <t^2>/z0^2)^2, and at large d the periodic images)
    H = 5.0  # the pair at height 2.5
    ds = np.array([20.0, 30.0, 45.0, 60.0, 90.0])
    nu = _pair("bottom_wall", H, 12.0, 33, ds)
    ratio = nu[:, 0] / (3 * H**2 / (8 * np.pi * ds**3))
    assert np.all(np.diff(np.abs(ratio - 1.0)) < 0) and abs(ratio[-1] - 1.0) < 1e-2
    slope = np.log(nu[2, 1] / nu[0, 1]) / np.log(ds[2] / ds[0])
    assert nu[0, 1] > 0 and -5.4 < slope < -4.6
