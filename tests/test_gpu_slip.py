"""Parity of partial-slip walls and uniform wall velocities (Appendix A) with the oracle.

Slip changes the wall data (the DP velocity's z derivative at the walls, formed in FP64 in the
solve), the boundary rows of the correction (closed form on the GPU, dense LU in the oracle) and
the k = 0 rows; wall velocities enter the k = 0 rows.  Bars as for no-slip walls: relative L2
<= 1e-9 (FP64) and <= 1e-5 (mixed) per output.
"""

import numpy as np
import pytest

from gpu_helpers import gpu_mobility, oracle_params, rel_l2, small_params
from oracle import mobility
from paper_2210_01837_gb300 import binding
from paper_2210_01837_gb300.workloads import random_particles

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "mixed": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2210_01837_gb300 import build
    build.build()
    binding.load()


# (mode, nx, ny, nz, torque route, wall conditions)
CASES = [
    ("slit", 72, 40, 33, True, dict(slip_bottom=0.7, slip_top=2.0)),
    ("slit", 54, 54, 25, False, dict(slip_bottom=0.0, slip_top=1.3)),
    ("slit", 40, 72, 33, True, dict(slip_bottom=1e6)),  # a shear-free bottom under a no-slip top
    ("bottom_wall", 72, 72, 33, True, dict(slip_bottom=0.9)),
    ("bottom_wall", 45, 35, 17, False, dict(slip_bottom=0.3, uw_bottom=(0.2, -0.4))),
    ("slit", 72, 40, 25, True, dict(uw_bottom=(0.5, 0.1), uw_top=(-0.3, 0.8))),
    ("slit", 54, 40, 25, "kernel_derivative", dict(slip_bottom=0.4, slip_top=0.4, uw_top=(0.6, 0.0))),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("mode,nx,ny,nz,torque,walls", CASES)
def test_parity_against_oracle(mode, nx, ny, nz, torque, walls, precision):
    params = small_params(mode, nx=nx, ny=ny, nz=nz, torque=bool(torque))
    params.update(walls)
    pos, F, T = random_particles(params, 40, seed=nx + 3 * ny + nz, torques=bool(torque))
    route = torque if isinstance(torque, str) else "spectral_curl"
    U_ref, W_ref = mobility(oracle_params(params), pos, F, T, torque_route=route)
    U, W = gpu_mobility(params, pos, F, T, precision, route=route)
    assert rel_l2(U, U_ref) <= TOL[precision]
    if torque:
        assert rel_l2(W, W_ref) <= TOL[precision]


def test_server_keys_plans_by_wall_conditions():
    # the same box served with and without slip: two plans, each result that of its own conditions
    params = small_params("slit", nx=40, ny=40, nz=25, torque=False)
    slip = dict(params, slip_bottom=0.8, slip_top=0.2)
    pos, F, _ = random_particles(params, 30, seed=9, torques=False)
    srv = binding.Server(memory_budget_bytes=8 << 30, slots=2)
    pin = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    tickets = [srv.submit(p, with_torque=False, precision="fp64", max_n=30, pos=pin(pos), F=pin(F))
               for p in (params, slip)]
    for t, p in zip(tickets, (params, slip)):
        r, U, _ = srv.wait(t, timeout_s=300.0)
        assert r.status == binding.DPS_OK
        U_ref, _ = mobility(oracle_params(p), pos, F)
        assert rel_l2(U, U_ref) <= 1e-9
    assert srv.stats()["plans_created"] == 2
    srv.close()
