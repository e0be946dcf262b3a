"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same seeded inputs.

FP64 path: relative L2 error <= 1e-9 per output (U and Omega separately).
Mixed path (float transforms, FP64 solves): <= 1e-5.
Grids are chosen to span several 32 x 8 spreading tiles with ragged tails (72, 40, 54 nodes) and
several FFT radices (2, 3); every wall mode is covered with and without torques.
"""

import numpy as np
import pytest

from gpu_helpers import gpu_mobility, oracle_params, read_grid, rel_l2, small_params, to_dev, zrange
from oracle import mobility
from oracle import stokes as ostokes
from oracle import transfer as otransfer
from paper_2210_01837_gb300 import binding
from paper_2210_01837_gb300.workloads import bw_small, random_particles

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "mixed": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2210_01837_gb300 import build
    build.build()
    binding.load()


def test_bw_small_fp64_translation_only():
    # 100 spheres above one wall, 128^2 x 65 grid, m = 6, beta = 10.2, FP64 (forces only)
    params, pos, F, _ = bw_small()
    U_ref, _ = mobility(oracle_params(params), pos, F)
    U, _ = gpu_mobility(params, pos, F, None, "fp64")
    assert rel_l2(U, U_ref) <= 1e-9


CASES = [
    ("bottom_wall", 72, 72, 33, True),
    ("slit", 72, 40, 33, True),
    ("free", 54, 72, 25, True),
    ("bottom_wall", 40, 54, 17, False),
    ("slit", 72, 72, 33, False),
    ("free", 72, 72, 33, False),
    # several spreading tiles in x and y with ragged tails, 7-smooth sizes
    ("slit", 96, 40, 33, True),
    ("bottom_wall", 80, 32, 25, False),
    # odd sizes: radix-5 and radix-7 butterflies, half spectra without a Nyquist column or row
    ("bottom_wall", 45, 35, 17, True),
    ("slit", 63, 50, 25, False),
    ("free", 64, 40, 17, False),  # 64 = 16 * 4: a radix-4 stage
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("mode,nx,ny,nz,torque", CASES)
def test_parity_against_oracle(mode, nx, ny, nz, torque, precision):
    params = small_params(mode, nx=nx, ny=ny, nz=nz, torque=torque)
    pos, F, T = random_particles(params, 40, seed=nx * 1000 + ny + nz, torques=torque)
    U_ref, W_ref = mobility(oracle_params(params), pos, F, T)
    U, W = gpu_mobility(params, pos, F, T, precision)
    assert rel_l2(U, U_ref) <= TOL[precision]
    if torque:
        assert rel_l2(W, W_ref) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spread_stage_matches_oracle(precision):
    params = small_params("slit", nx=72, ny=40, nz=33, torque=True)
    pos, F, T = random_particles(params, 30, seed=5)
    plan = binding.Plan.from_params(params, with_torque=True, precision=precision, max_n=len(pos))
    plan.debug_run(to_dev(pos), to_dev(F), to_dev(T), last_stage=2)
    grid, info = read_grid(plan, params, precision)
    clo, chi = zrange(plan)
    op = oracle_params(params)
    ref = np.concatenate([otransfer.spread(op, pos, F, "M"), otransfer.spread(op, pos, T, "D")])
    occ = np.nonzero(np.any(ref != 0.0, axis=(0, 2, 3)))[0]
    # the device range may include planes on which every envelope vanishes exactly (a wall node
    # where a kernel and its image cancel); it must contain every non-zero plane
    assert clo <= occ.min() and chi >= occ.max()
    assert not np.any(ref[:, :clo]) and not np.any(ref[:, chi + 1:])
    got = grid[:, clo:chi + 1, :, : params["nx"]]
    want = ref[:, clo:chi + 1]
    tol = 1e-13 if precision == "fp64" else 1e-6
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    plan.close()


def test_particle_on_wall_is_immobile_and_empty_apply():
    params = small_params("bottom_wall", torque=True)
    pos, F, T = random_particles(params, 5, seed=3)
    pos[0, 2] = 0.0
    U, W = gpu_mobility(params, pos, F, T, "fp64")
    assert np.all(U[0] == 0.0) and np.all(W[0] == 0.0)
    plan = binding.Plan.from_params(params, with_torque=True, precision="fp64", max_n=5)
    import torch
    e = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    plan.apply(e, e, e, check=True)
    plan.close()


@pytest.mark.parametrize("bad,expect", [("z_out", binding.DPS_ERR_OUT_OF_DOMAIN),
                                        ("open_top", binding.DPS_ERR_OUT_OF_DOMAIN),
                                        ("nan", binding.DPS_ERR_NONFINITE)])
def test_data_errors_reported_by_status(bad, expect):
    params = small_params("bottom_wall", torque=False)
    pos, F, _ = random_particles(params, 6, seed=4, torques=False)
    if bad == "z_out":
        pos[2, 2] = -0.5
    elif bad == "open_top":
        pos[2, 2] = params["zmax"] - 0.1
    else:
        F[1, 0] = np.nan
    plan = binding.Plan.from_params(params, with_torque=False, precision="mixed", max_n=6)
    plan.apply(to_dev(pos), to_dev(F))
    assert plan.status() == expect
    assert plan.status() == binding.DPS_OK     # the status word is cleared by the read
    plan.close()


def test_apply_host_matches_device_apply():
    import torch
    params = small_params("slit", torque=True)
    pos, F, T = random_particles(params, 25, seed=8)
    plan = binding.Plan.from_params(params, with_torque=True, precision="mixed", max_n=32)
    U1, W1 = plan.apply(to_dev(pos), to_dev(F), to_dev(T), check=True)
    torch.cuda.synchronize()
    U2, W2 = plan.apply_host(np.ascontiguousarray(pos), np.ascontiguousarray(F), np.ascontiguousarray(T))
    assert np.allclose(U1.cpu().numpy(), U2, rtol=0, atol=1e-6 * np.abs(U2).max())
    assert np.allclose(W1.cpu().numpy(), W2, rtol=0, atol=1e-6 * np.abs(W2).max())
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_crowded_bin_matches_oracle(precision):
    """200 particles inside one 32 x 8 spreading tile: the spread takes its multi-batch path (more
    candidates than one staged batch of records)."""
    params = small_params("bottom_wall", nx=80, ny=32, nz=17, zmax=6.0, torque=True)
    h = params["Lx"] / params["nx"]
    rng = np.random.default_rng(4242)
    n = 200
    pos = np.stack([rng.uniform(0.0, 32 * h, n), rng.uniform(0.0, 8 * h, n), rng.uniform(0.5, 3.0, n)], axis=1)
    F = rng.standard_normal((n, 3))
    T = rng.standard_normal((n, 3))
    U_ref, W_ref = mobility(oracle_params(params), pos, F, T)
    U, W = gpu_mobility(params, pos, F, T, precision)
    assert rel_l2(U, U_ref) <= TOL[precision]
    assert rel_l2(W, W_ref) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("mode", ["bottom_wall", "slit", "free"])
def test_factorise_as_you_go_solve_matches_oracle(mode, precision, monkeypatch):
    """The FP64 solve without its plan-time factorisation table (the path a plan takes when the
    table does not fit in memory; DPS_SOLVE_TABLE=0 chooses it by hand)."""
    params = small_params(mode, nx=54, ny=40, nz=33, torque=True)
    pos, F, T = random_particles(params, 30, seed=61)
    U_ref, W_ref = mobility(oracle_params(params), pos, F, T)
    monkeypatch.setenv("DPS_SOLVE_TABLE", "0")
    plan = binding.Plan.from_params(params, with_torque=True, precision=precision, max_n=len(pos))
    monkeypatch.delenv("DPS_SOLVE_TABLE")
    U, W = gpu_mobility(params, pos, F, T, precision, plan=plan)
    plan.close()
    assert rel_l2(U, U_ref) <= TOL[precision]
    assert rel_l2(W, W_ref) <= TOL[precision]
