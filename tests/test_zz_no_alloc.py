"""The allocation-free spreading entry point against the plan-based spreading stage.

dpstokes_spread_noalloc serves callers that cannot call cudaMalloc (a host application whose
memory manager owns all device memory, or a latency-critical loop that cannot take an
allocation's implicit synchronisation): its scratch is a fixed device array inside the library.
This test calls it through the C ABI twice in a row, with different particles, and compares each
result with the spread grid that a plan produces for the same input (dpstokes_debug_run up to the
spreading stage), within the FP64 tolerance of the spreading parity test.  This file is collected
last so that a run stopping at the first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

from gpu_helpers import read_grid, small_params, to_dev, zrange
from paper_2210_01837_gb300 import binding
from paper_2210_01837_gb300.workloads import random_particles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2210_01837_gb300 import build
    build.build()
    binding.load()


def _noalloc(params, pos, F, T, ldx, route):
    import torch
    code = binding.torque_route(route)
    nf = 6 if code == 1 else 3
    out = torch.full((nf, params["nz"], params["ny"], ldx), float("nan"), dtype=torch.float64, device="cuda")
    grid = binding.dps_grid(params["nx"], params["ny"], params["nz"])
    kp = binding.dps_kernel_params(params["m_M"], params["beta_M"], params["m_D"], params["beta_D"], 1.0,
                                   code, binding.PRECISIONS["fp64"], len(pos))
    d_pos, d_F = to_dev(pos), to_dev(F)
    d_T = to_dev(T) if T is not None else None
    st = binding.dpstokes_spread_noalloc(params["Lx"], params["Ly"], params["zmin"], params["zmax"],
                                         binding.MODES[params["mode"]], grid, kp, len(pos), d_pos.data_ptr(),
                                         d_F.data_ptr(), None if d_T is None else d_T.data_ptr(), out.data_ptr(),
                                         ldx, torch.cuda.current_stream().cuda_stream)
    assert st == binding.DPS_OK, binding.dpstokes_error_string(st)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("mode,route", [("slit", "spectral_curl"), ("bottom_wall", "none"),
                                        ("bottom_wall", "kernel_derivative")])
def test_noalloc_spread_matches_plan_spread_twice(mode, route):
    torque = route != "none"
    params = small_params(mode, nx=72, ny=40, nz=33, torque=torque)
    plan = binding.Plan.from_params(params, with_torque=route, precision="fp64", max_n=64)
    ldx = 2 * plan.info().pitch
    for call, seed in enumerate((21, 22)):
        pos, F, T = random_particles(params, 40 + 7 * call, seed=seed, torques=torque)
        plan.debug_run(to_dev(pos), to_dev(F), to_dev(T) if torque else None, last_stage=2)
        ref, _ = read_grid(plan, params, "fp64")
        clo, chi = zrange(plan)
        got = _noalloc(params, pos, F, T, ldx, route)
        assert not np.isnan(got).any()
        nx = params["nx"]
        want = ref[:, clo:chi + 1, :, :nx]
        err = np.max(np.abs(got[:, clo:chi + 1, :, :nx] - want)) / np.max(np.abs(want))
        assert err <= 1e-13, f"call {call}: max relative difference {err:.3e}"
        assert not np.any(got[:, :clo]) and not np.any(got[:, chi + 1:]) and not np.any(got[..., nx:])
    plan.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    params = small_params("slit", nx=72, ny=40, nz=33, torque=True)
    grid = binding.dps_grid(params["nx"], params["ny"], params["nz"])
    kp = binding.dps_kernel_params(params["m_M"], params["beta_M"], params["m_D"], params["beta_D"], 1.0, 1, 0, 1)
    st = binding.dpstokes_spread_noalloc(params["Lx"], params["Ly"], 0.0, params["zmax"], 2, grid, kp, 10 ** 7,
                                         ctypes.c_void_p(16).value, 16, 16, 16, 144, None)
    assert st == binding.DPS_ERR_INVALID_ARG
