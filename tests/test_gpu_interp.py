"""The interpolation variants (step 8, Eqs. 10-11) against the oracle.

0: a warp per particle gathering from global memory; 1: the tile gather (a block per 32 x 8 tile of
node columns, per-tile partial sums added per particle in a fixed order); 2: the staged gather (a
block per particle bin copies its particles' grid region into shared memory four planes at a time;
mixed precision, m <= 5), with its global-memory path for bins whose region does not fit (forced
here through the test hook, and taken by itself where nx is not a multiple of 4 or the region is
taller than the staged rows).  Each is compared with the oracle's product on boxes with ragged last
tiles in x and y, boxes narrower than one tile (a support's wrapped nodes fall in the same tile),
supports that wrap around the periodic boundary, and a crowded tile (more particles than one
staged batch).  Bars: relative L2 per output <= 1e-9 FP64, <= 1e-5 mixed.
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


CASES = [
    # mode, nx, ny, nz, torque
    ("bottom_wall", 72, 40, 33, True),    # ragged last tile in x (72 = 2 x 32 + 8)
    ("slit", 45, 35, 17, True),           # ragged in x and y (35 = 4 x 8 + 3)
    ("free", 24, 20, 17, False),          # narrower than one tile in x
    ("bottom_wall", 96, 64, 25, False),   # whole tiles
    ("slit", 225, 25, 17, True),          # last tiles one node wide in x (225 = 7 x 32 + 1) and y
]


def _edge_particles(params, n, seed, torque):
    """Random particles, a third of them within a support width of the periodic edges."""
    pos, F, T = random_particles(params, n, seed=seed, torques=torque)
    h = params["Lx"] / params["nx"]
    rng = np.random.default_rng(seed + 1)
    k = n // 3
    pos[:k, 0] = np.mod(params["Lx"] - rng.uniform(0.0, 4 * h, k), params["Lx"])
    pos[k:2 * k, 1] = np.mod(params["Ly"] - rng.uniform(0.0, 4 * h, k), params["Ly"])
    return pos, F, T


def _variants(precision):
    # (variant, force the staged gather's global-memory path)
    return [(0, False), (1, False)] + ([(2, False), (2, True)] if precision == "mixed" else [])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("mode,nx,ny,nz,torque", CASES)
def test_interpolation_variants_match_oracle(mode, nx, ny, nz, torque, precision):
    params = small_params(mode, nx=nx, ny=ny, nz=nz, torque=torque)
    pos, F, T = _edge_particles(params, 36, nx * 7 + ny, torque)
    U_ref, W_ref = mobility(oracle_params(params), pos, F, T)
    got = {}
    for variant, forced in _variants(precision):
        plan = binding.Plan.from_params(params, with_torque=torque, precision=precision, max_n=len(pos))
        plan.set_interp(variant)
        assert plan.info().interp_variant == variant
        if forced:
            plan.debug_inject(2)
        got[(variant, forced)] = gpu_mobility(params, pos, F, T, precision, plan=plan)
        plan.close()
        U, W = got[(variant, forced)]
        assert rel_l2(U, U_ref) <= TOL[precision], f"variant {variant} (global path {forced}): U"
        if torque:
            assert rel_l2(W, W_ref) <= TOL[precision], f"variant {variant} (global path {forced}): Omega"
        # every particle, not only the norm
        assert np.max(np.abs(U - U_ref)) <= 10 * TOL[precision] * np.max(np.abs(U_ref))
    # the variants sum the same products in different orders
    for key, (U, _) in got.items():
        assert rel_l2(U, got[(0, False)][0]) <= TOL[precision], key


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_interpolation_with_a_crowded_tile(precision):
    """200 particles inside one 32 x 8 tile: more candidates than one staged batch of records (tile
    gather) and more particles than one batch of the staged gather's warps (32)."""
    params = small_params("bottom_wall", nx=80, ny=32, nz=17, zmax=6.0, torque=True)
    h = params["Lx"] / params["nx"]
    rng = np.random.default_rng(4243)
    n = 200
    pos = np.stack([rng.uniform(0.0, 32 * h, n), rng.uniform(0.0, 8 * h, n), rng.uniform(0.5, 3.0, n)], axis=1)
    F = rng.standard_normal((n, 3))
    T = rng.standard_normal((n, 3))
    U_ref, W_ref = mobility(oracle_params(params), pos, F, T)
    for variant in (1, 2) if precision == "mixed" else (1,):
        plan = binding.Plan.from_params(params, with_torque=True, precision=precision, max_n=n)
        plan.set_interp(variant)
        U, W = gpu_mobility(params, pos, F, T, precision, plan=plan)
        plan.close()
        assert rel_l2(U, U_ref) <= TOL[precision], variant
        assert rel_l2(W, W_ref) <= TOL[precision], variant


def test_staged_interpolation_forces_only_and_default():
    """The staged gather's three-field form (forces only), and the default variant: the staged
    gather where it applies (mixed precision, m <= 5), else the warp per particle."""
    params = small_params("slit", nx=96, ny=64, nz=33, torque=False)
    pos, F, _ = _edge_particles(params, 50, 5, False)
    U_ref, _ = mobility(oracle_params(params), pos, F, None)
    plan = binding.Plan.from_params(params, with_torque=False, precision="mixed", max_n=len(pos))
    assert plan.info().interp_variant == 2
    U, _ = gpu_mobility(params, pos, F, None, "mixed", plan=plan)
    plan.close()
    assert rel_l2(U, U_ref) <= TOL["mixed"]
    plan = binding.Plan.from_params(params, with_torque=False, precision="fp64", max_n=len(pos))
    assert plan.info().interp_variant == 0
    with pytest.raises(binding.DpsError):
        plan.set_interp(2)
    plan.close()


def test_tile_and_staged_interpolation_are_refused_where_they_do_not_apply():
    params = small_params("bottom_wall", torque=True)
    plan = binding.Plan.from_params(params, with_torque="kernel_derivative", precision="mixed", max_n=8)
    assert plan.info().interp_variant == 0
    for v in (1, 2):
        with pytest.raises(binding.DpsError):
            plan.set_interp(v)
    with pytest.raises(binding.DpsError):
        plan.debug_inject(2)
    plan.close()
    params = small_params("bottom_wall", m=6, torque=True)  # supports of 7 nodes
    plan = binding.Plan.from_params(params, with_torque=True, precision="mixed", max_n=8)
    assert plan.info().interp_variant == 0
    with pytest.raises(binding.DpsError):
        plan.set_interp(2)
    plan.close()


def test_repeat_applies_agree():
    """The tile gather adds a tile's contributions to a particle's shared accumulator with float
    atomics, so repeated applies agree to rounding (the A17 bar, 1e-6 mixed); the warp-per-particle
    and the staged gathers sum in a fixed order and repeat bit for bit."""
    params = small_params("slit", nx=72, ny=40, nz=33, torque=True)
    pos, F, T = _edge_particles(params, 60, 99, True)
    plan = binding.Plan.from_params(params, with_torque=True, precision="mixed", max_n=len(pos))
    plan.set_interp(1)
    a = gpu_mobility(params, pos, F, T, "mixed", plan=plan)
    b = gpu_mobility(params, pos, F, T, "mixed", plan=plan)
    assert rel_l2(a[0], b[0]) <= 1e-6 and rel_l2(a[1], b[1]) <= 1e-6
    for v in (0, 2):
        plan.set_interp(v)
        a = gpu_mobility(params, pos, F, T, "mixed", plan=plan)
        b = gpu_mobility(params, pos, F, T, "mixed", plan=plan)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), v
    plan.close()
