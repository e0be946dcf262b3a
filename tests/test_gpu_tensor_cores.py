"""The Chebyshev transforms on the tensor cores (tcgen05.mma, tf32 three-product split, mixed
precision: the forward transform, and the backward transform of the spectral-curl torque route)
against the oracle and against the CUDA-core lane kernels they replace.

Cases: every wall mode, forces only and with torques (six-field curl source), 8 to 113 Chebyshev
nodes (8 and 9 in free space: one and two backward K steps per tile, against the backward's two
producer groups that take alternate steps) (accumulator widths 32 to 128 columns per output; beyond 96 nodes the backward transform's
output planes go in two launches), ragged wavenumber tiles (fewer than 64 wavenumbers in the last
tile), plane ranges that end inside a K step of 8 planes, a problem of a single tile, and a plane
range narrow enough that the second backward launch has no planes.  Bars: 1e-5 relative L2 against the oracle (the mixed bar); 3e-6 against the lane
kernel (the same contraction from tf32 operand pairs instead of float products, summed in another
order: 1.3e-6 measured at 97 nodes).
"""

import numpy as np
import pytest

from gpu_helpers import gpu_mobility, oracle_params, rel_l2, small_params
from oracle import mobility
from paper_2210_01837_gb300 import binding
from paper_2210_01837_gb300.workloads import random_particles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2210_01837_gb300 import build
    build.build()
    binding.load()


def _plan(params, torque, tc, monkeypatch):
    monkeypatch.setenv("DPS_CHEB_TC", "3" if tc else "0")
    plan = binding.Plan.from_params(params, with_torque=torque, precision="mixed", max_n=64)
    monkeypatch.delenv("DPS_CHEB_TC")
    # bit 0 forward (nz <= 128), bit 1 backward (spectral-curl torques)
    want = (1 | (2 if torque else 0)) if tc else 0
    assert plan.info().cheb_tensor_cores == want
    return plan


CASES = [
    ("bottom_wall", 72, 40, 65, True),
    ("slit", 54, 40, 97, True),
    ("free", 40, 36, 33, True),
    ("bottom_wall", 45, 35, 17, False),
    ("slit", 72, 72, 33, False),
    ("bottom_wall", 8, 8, 17, True),     # a single 64-wavenumber tile (5 x 8 wavenumbers)
    ("slit", 40, 32, 113, True),         # backward in two launches of up to 64 planes
    ("free", 40, 36, 8, True),           # one backward K step per tile: fewer than the two producer groups
    ("free", 40, 36, 9, True),           # two backward K steps per tile, one per producer group
]


@pytest.mark.parametrize("mode,nx,ny,nz,torque", CASES)
def test_tensor_core_forward_transform(mode, nx, ny, nz, torque, monkeypatch):
    m = 3 if nx <= 8 else 5
    params = small_params(mode, nx=nx, ny=ny, nz=nz, torque=torque, m=m)
    pos, F, T = random_particles(params, 40, seed=nx + ny + nz, torques=torque)
    U_ref, W_ref = mobility(oracle_params(params), pos, F, T)
    got = []
    for tc in (True, False):
        plan = _plan(params, torque, tc, monkeypatch)
        got.append(gpu_mobility(params, pos, F, T, "mixed", plan=plan))
        plan.close()
    (U, W), (U0, W0) = got
    assert rel_l2(U, U_ref) <= 1e-5
    assert rel_l2(U, U0) <= 3e-6
    if torque:
        assert rel_l2(W, W_ref) <= 1e-5
        assert rel_l2(W, W0) <= 3e-6


def test_backward_in_two_launches_with_an_empty_second_part(monkeypatch):
    """97 nodes with every particle in a thin layer near the wall: the occupied planes fit the first
    of the backward transform's two launches, and the second launch has none."""
    params = small_params("bottom_wall", nx=48, ny=40, nz=97, zmax=12.0, torque=True)
    rng = np.random.default_rng(97)
    n = 30
    pos = np.stack([rng.uniform(0, params["Lx"], n), rng.uniform(0, params["Ly"], n), rng.uniform(1.7, 1.8, n)], axis=1)
    F = rng.standard_normal((n, 3))
    T = rng.standard_normal((n, 3))
    U_ref, W_ref = mobility(oracle_params(params), pos, F, T)
    got = []
    for tc in (True, False):
        plan = _plan(params, True, tc, monkeypatch)
        got.append(gpu_mobility(params, pos, F, T, "mixed", plan=plan))
        plan.close()
    (U, W), (U0, W0) = got
    assert rel_l2(U, U_ref) <= 1e-5 and rel_l2(W, W_ref) <= 1e-5
    assert rel_l2(U, U0) <= 3e-6 and rel_l2(W, W0) <= 3e-6


def test_tensor_cores_used_by_default_in_mixed_precision_only():
    params = small_params("bottom_wall", nx=40, ny=40, nz=33, torque=True)
    mixed = binding.Plan.from_params(params, with_torque=True, precision="mixed", max_n=8)
    fp64 = binding.Plan.from_params(params, with_torque=True, precision="fp64", max_n=8)
    assert mixed.info().cheb_tensor_cores == 3 and fp64.info().cheb_tensor_cores == 0
    mixed.close()
    fp64.close()


def test_bounded_wait_reports_timeout_and_the_plan_stays_usable():
    """Failure injection: the forward tensor-core transform withholds its MMA completions, so its
    producers' bounded waits run out (about a second); the kernel records DPS_ERR_TIMEOUT instead
    of hanging, frees its tensor memory, and the next apply of the same plan is correct."""
    from gpu_helpers import to_dev
    params = small_params("bottom_wall", nx=72, ny=40, nz=33, torque=True)
    pos, F, T = random_particles(params, 20, seed=5)
    plan = binding.Plan.from_params(params, with_torque=True, precision="mixed", max_n=len(pos))
    ref = gpu_mobility(params, pos, F, T, "mixed", plan=plan)
    plan.debug_inject(1)
    plan.apply(to_dev(pos), to_dev(F), to_dev(T))
    assert plan.status() == binding.DPS_ERR_TIMEOUT
    got = gpu_mobility(params, pos, F, T, "mixed", plan=plan)
    plan.close()
    assert rel_l2(got[0], ref[0]) <= 1e-6 and rel_l2(got[1], ref[1]) <= 1e-6
