"""The allocation-free spreading entry point against the oracle and the plan-based spreading stage.

dpstokes_spread_noalloc serves callers that cannot call cudaMalloc (a host application whose
memory manager owns all device memory, or a latency-critical loop that cannot take an
allocation's implicit synchronisation): its scratch is a fixed device array inside the library.
This test calls it through the C ABI twice in a row, with different particles, and compares each
result with the oracle's spread grid (oracle.transfer) and with the spread grid that a plan
produces for the same input (dpstokes_debug_run up to the spreading stage), within the FP64
tolerance of the spreading parity test.  This file is collected last so that a run stopping at
the first failure has already run every other test.
"""

import numpy as np
import pytest

from gpu_helpers import oracle_params, read_grid, small_params, to_dev, zrange
from oracle import transfer as otransfer
from paper_2210_01837_gb300 import binding
from paper_2210_01837_gb300.workloads import random_particles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2210_01837_gb300 import build
    build.build()
    binding.load()


def _kp(params, code, n):
    return binding.dps_kernel_params(params["m_M"], params["beta_M"], params["m_D"], params["beta_D"], 1.0,
                                     code, binding.PRECISIONS["fp64"], n)


def _noalloc(params, pos, F, T, ldx, route):
    import torch
    code = binding.torque_route(route)
    nf = 6 if code == 1 else 3
    out = torch.full((nf, params["nz"], params["ny"], ldx), float("nan"), dtype=torch.float64, device="cuda")
    grid = binding.dps_grid(params["nx"], params["ny"], params["nz"])
    d_pos, d_F = to_dev(pos), to_dev(F)
    d_T = to_dev(T) if T is not None else None
    st = binding.dpstokes_spread_noalloc(params["Lx"], params["Ly"], params["zmin"], params["zmax"],
                                         binding.MODES[params["mode"]], grid, _kp(params, code, len(pos)), len(pos),
                                         d_pos.data_ptr(), d_F.data_ptr(), None if d_T is None else d_T.data_ptr(),
                                         out.data_ptr(), ldx, torch.cuda.current_stream().cuda_stream)
    assert st == binding.DPS_OK, binding.dpstokes_error_string(st)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _oracle_grid(params, pos, F, T, route):
    op = oracle_params(params)
    if route == "spectral_curl":
        return np.concatenate([otransfer.spread(op, pos, F, "M"), otransfer.spread(op, pos, T, "D")])
    g = otransfer.spread(op, pos, F, "M")
    if route == "kernel_derivative":
        g = g + otransfer.spread_curl(op, pos, T)
    return g


@pytest.mark.parametrize("mode,route", [("slit", "spectral_curl"), ("bottom_wall", "none"),
                                        ("bottom_wall", "kernel_derivative")])
def test_noalloc_spread_matches_oracle_and_plan_spread_twice(mode, route):
    torque = route != "none"
    params = small_params(mode, nx=72, ny=40, nz=33, torque=torque)
    plan = binding.Plan.from_params(params, with_torque=route, precision="fp64", max_n=64)
    ldx = 2 * plan.info().pitch
    nx = params["nx"]
    for call, seed in enumerate((21, 22)):
        pos, F, T = random_particles(params, 40 + 7 * call, seed=seed, torques=torque)
        got = _noalloc(params, pos, F, T, ldx, route)
        assert not np.isnan(got).any()
        assert not np.any(got[..., nx:])
        # the oracle's grid on every plane
        want = _oracle_grid(params, pos, F, T, route)
        err = np.max(np.abs(got[..., :nx] - want)) / np.max(np.abs(want))
        assert err <= 1e-13, f"call {call}: max relative difference from the oracle {err:.3e}"
        # the plan's spreading stage on the same input
        plan.debug_run(to_dev(pos), to_dev(F), to_dev(T) if torque else None, last_stage=2)
        ref, _ = read_grid(plan, params, "fp64")
        clo, chi = zrange(plan)
        err = np.max(np.abs(got[:, clo:chi + 1, :, :nx] - ref[:, clo:chi + 1, :, :nx])) / np.max(np.abs(want))
        assert err <= 1e-13, f"call {call}: max relative difference from the plan's spread {err:.3e}"
        assert not np.any(got[:, :clo]) and not np.any(got[:, chi + 1:])
    plan.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch
    params = small_params("slit", nx=72, ny=40, nz=33, torque=True)
    grid = binding.dps_grid(params["nx"], params["ny"], params["nz"])
    n = 10 ** 7  # records alone need far more than the fixed scratch
    # device buffers of the full sizes the call is told about (no made-up addresses); the call
    # must reject the problem before it enqueues anything
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    pos[:, 2] = 5.0
    F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    T = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    ldx = 144
    out = torch.zeros((6, params["nz"], params["ny"], ldx), dtype=torch.float64, device="cuda")
    st = binding.dpstokes_spread_noalloc(params["Lx"], params["Ly"], 0.0, params["zmax"], 2, grid,
                                         _kp(params, 1, n), n, pos.data_ptr(), F.data_ptr(), T.data_ptr(),
                                         out.data_ptr(), ldx, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == binding.DPS_ERR_INVALID_ARG
    assert not torch.any(out != 0)
