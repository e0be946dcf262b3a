"""Oracle parity on the kernel paths that the 1M-roller workload runs, and properties of the product
at that workload's full size.

The full-size product (3072^2 x 65, N = 2^20) is out of the oracle's reach, so the kernels it uses
are reached here on boxes the oracle finishes in seconds:
* 3072-point rows (a 3072 x 16 box): the x transform takes the register-staged row pass, radices
  16 x 16 x 12, as at full size;
* 3072-point columns (a 16 x 3072 box): the y transform takes the register-staged column pass fed
  by TMA box loads, 4 columns per block, as at full size;
* 65 and 97 Chebyshev nodes with torques in every wall mode: the six-field compact forward
  transform (nz <= 72), its twelve-row split (nz > 96), and the backward transform with the
  correction derivative.
Each case asserts, through dpstokes_plan_info, that the plan chose the variant named above, and
compares U and Omega with the oracle element by element: relative L2 per output and the largest
per-particle error (the norm of the difference of one particle's vector over the RMS norm of the
oracle's vectors), both within the bars of the other parity tests (1e-9 FP64, 1e-5 mixed).

At full size (the 1M-roller workload itself, launch shapes chosen by the autotuner as the bench
does) the tests check what holds at any size: the mixed path against the all-FP64 path (different
FFT variants and transform precision, same discrete operator) within the mixed bar, invariance
under a translation by whole cells, and linearity.
"""

import numpy as np
import pytest

from gpu_helpers import gpu_mobility, oracle_params, rel_l2, small_params, to_dev
from oracle import mobility
from paper_2210_01837_gb300 import binding

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "mixed": 1e-5}
_ORACLE = {}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2210_01837_gb300 import build
    build.build()
    binding.load()


def max_particle_err(got, want):
    """max_i |got_i - want_i| / RMS_i |want_i| over particles i (rows)."""
    d = np.linalg.norm(np.asarray(got) - np.asarray(want), axis=1)
    rms = np.sqrt(np.mean(np.sum(np.asarray(want) ** 2, axis=1)))
    return float(d.max() / max(rms, 1e-300))


def _layer(params, n, seed):
    """Particles of the roller layer's height distribution (|N(1.6, 0.3)| clipped at 1.05) for a
    bottom wall, uniform between the walls for a slit; forces and torques N(0, 1) so that every
    component of the product is exercised."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, params["Lx"], n)
    y = rng.uniform(0.0, params["Ly"], n)
    if params["mode"] == "bottom_wall":
        z = np.maximum(np.abs(rng.normal(1.6, 0.3, n)), 1.05)
    else:
        z = rng.uniform(1.2, params["zmax"] - 1.2, n)
    return np.stack([x, y, z], axis=1), rng.standard_normal((n, 3)), rng.standard_normal((n, 3))


def _case(key, mode, nx, ny, nz, zmax, n, seed):
    if key not in _ORACLE:
        params = small_params(mode, nx=nx, ny=ny, nz=nz, zmax=zmax, torque=True)
        pos, F, T = _layer(params, n, seed)
        U, W = mobility(oracle_params(params), pos, F, T)
        _ORACLE[key] = (params, pos, F, T, U, W)
    return _ORACLE[key]


def _check(params, pos, F, T, U_ref, W_ref, precision, expect=None):
    plan = binding.Plan.from_params(params, with_torque=True, precision=precision, max_n=len(pos))
    info = plan.info()
    if expect is not None:
        for field, value in expect.items():
            assert getattr(info, field) == value, f"{field} = {getattr(info, field)}, expected {value}"
    U, W = gpu_mobility(params, pos, F, T, precision, plan=plan)
    plan.close()
    tol = TOL[precision]
    for name, got, want in (("U", U, U_ref), ("Omega", W, W_ref)):
        e2, em = rel_l2(got, want), max_particle_err(got, want)
        assert e2 <= tol, f"{name}: relative L2 {e2:.3e}"
        assert em <= tol, f"{name}: largest per-particle error {em:.3e}"


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_3072_point_rows_match_oracle(precision):
    params, pos, F, T, U, W = _case("rows", "bottom_wall", 3072, 16, 65, 8.0, 64, 31)
    # mixed: the register-staged row pass (float rows of >= 2048 points, radices 16 16 12)
    _check(params, pos, F, T, U, W, precision, {"fft_register_rows": 1} if precision == "mixed" else None)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_3072_point_columns_match_oracle(precision):
    params, pos, F, T, U, W = _case("cols", "bottom_wall", 16, 3072, 65, 8.0, 64, 32)
    # mixed: the TMA-prefetched register-staged column pass, 4 columns per block
    expect = {"fft_register_cols": 3, "fft_col_width": 4} if precision == "mixed" else None
    _check(params, pos, F, T, U, W, precision, expect)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("mode,nx,ny,nz,zmax", [
    ("bottom_wall", 72, 40, 65, 8.0),   # the 1M-roller z grid: six-field compact forward transform
    ("slit", 72, 40, 65, 12.0),
    ("slit", 72, 40, 97, 20.0),         # the 16k-slit z grid: twelve-row forward split
    ("bottom_wall", 40, 54, 97, 12.0),
    ("free", 54, 40, 65, 20.0),
])
def test_torque_paths_at_65_and_97_nodes(mode, nx, ny, nz, zmax, precision):
    if mode == "free":
        key = f"{mode}-{nx}-{ny}-{nz}"
        if key not in _ORACLE:
            params = small_params(mode, nx=nx, ny=ny, nz=nz, zmax=zmax, torque=True)
            from paper_2210_01837_gb300.workloads import random_particles
            pos, F, T = random_particles(params, 48, seed=nz + nx)
            U, W = mobility(oracle_params(params), pos, F, T)
            _ORACLE[key] = (params, pos, F, T, U, W)
        params, pos, F, T, U, W = _ORACLE[key]
    else:
        params, pos, F, T, U, W = _case(f"{mode}-{nx}-{ny}-{nz}", mode, nx, ny, nz, zmax, 48, nz * 7 + nx)
    _check(params, pos, F, T, U, W, precision)


# ---------------------------------------------------------------------------------------------
# full size: the 1M-roller workload in the bench's launch configuration
# ---------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def full_size():
    import torch
    from paper_2210_01837_gb300.workloads import rollers_1m
    params, pos, F, T = rollers_1m()
    plan = binding.Plan.from_params(params, with_torque=True, precision="mixed", max_n=len(pos))
    d_pos, d_F, d_T = to_dev(pos), to_dev(F), to_dev(T)
    U = torch.empty((len(pos), 3), dtype=torch.float64, device="cuda")
    W = torch.empty_like(U)
    plan.autotune(d_pos, d_F, d_T, U, W)
    yield params, pos, F, T, plan
    plan.close()
    torch.cuda.empty_cache()


def _apply(plan, pos, F, T):
    import torch
    U, W = plan.apply(to_dev(pos), to_dev(F), to_dev(T), check=True)
    torch.cuda.synchronize()
    return U.cpu().numpy(), W.cpu().numpy()


def test_full_size_mixed_matches_fp64(full_size):
    import torch
    params, pos, F, T, plan = full_size
    U, W = _apply(plan, pos, F, T)
    p64 = binding.Plan.from_params(params, with_torque=True, precision="fp64", max_n=len(pos))
    U64, W64 = _apply(p64, pos, F, T)
    p64.close()
    torch.cuda.empty_cache()
    for got, want in ((U, U64), (W, W64)):
        assert rel_l2(got, want) <= TOL["mixed"]
        assert max_particle_err(got, want) <= 10 * TOL["mixed"]


def test_full_size_translation_by_whole_cells(full_size):
    params, pos, F, T, plan = full_size
    U, W = _apply(plan, pos, F, T)
    h = params["Lx"] / params["nx"]
    moved = pos.copy()
    moved[:, 0] = np.mod(moved[:, 0] + 517 * h, params["Lx"])
    moved[:, 1] = np.mod(moved[:, 1] + 1234 * h, params["Ly"])
    U2, W2 = _apply(plan, moved, F, T)
    # the discrete operator is exactly invariant; the float transforms round differently
    assert rel_l2(U2, U) <= TOL["mixed"] and rel_l2(W2, W) <= TOL["mixed"]


def test_full_size_linearity(full_size):
    params, pos, F, T, plan = full_size
    rng = np.random.default_rng(77)
    F2, T2 = rng.standard_normal(F.shape), rng.standard_normal(T.shape)
    a, b = 0.75, -1.5
    U1, W1 = _apply(plan, pos, F, T)
    U2, W2 = _apply(plan, pos, F2, T2)
    U3, W3 = _apply(plan, pos, a * F + b * F2, a * T + b * T2)
    assert rel_l2(U3, a * U1 + b * U2) <= TOL["mixed"]
    assert rel_l2(W3, a * W1 + b * W2) <= TOL["mixed"]
