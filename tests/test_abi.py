"""The C ABI library loads on a machine without a GPU, exports every entry point declared in
include/dpstokes.h, and rejects invalid arguments on the host before touching the device."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2210_01837_gb300 import binding, build
    build.build()
    return binding.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "dpstokes.h")).read()
    return sorted(set(re.findall(r"\b(dpstokes_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 9
    for name in names:
        assert hasattr(lib, name), name


def test_no_torch_or_cuda_types_in_header():
    text = open(os.path.join(ROOT, "include", "dpstokes.h")).read()
    assert "torch" not in text and "cudaStream_t " not in text.split("*/")[-1]


def test_error_strings(lib):
    from paper_2210_01837_gb300 import binding
    for code in binding.STATUS:
        s = binding.dpstokes_error_string(code)
        assert isinstance(s, str) and len(s) > 0
    assert binding.dpstokes_error_string(12345) == "unknown status"


def test_struct_layout():
    from paper_2210_01837_gb300 import binding
    assert ctypes.sizeof(binding.dps_grid) == 12
    assert ctypes.sizeof(binding.dps_kernel_params) == 56
    assert binding.dps_kernel_params.max_n.offset == 48


def _create(**over):
    from paper_2210_01837_gb300 import binding
    a = dict(Lx=64.0, Ly=64.0, zmin=0.0, zmax=12.0, mode=1, nx=128, ny=128, nz=65, m_M=6, beta_M=10.2, m_D=0,
             beta_D=0.0, eta=1.0, with_torque=0, precision=0, max_n=100)
    a.update(over)
    grid = binding.dps_grid(a["nx"], a["ny"], a["nz"])
    kp = binding.dps_kernel_params(a["m_M"], a["beta_M"], a["m_D"], a["beta_D"], a["eta"], a["with_torque"],
                                   a["precision"], a["max_n"])
    return binding.dpstokes_plan_create(a["Lx"], a["Ly"], a["zmin"], a["zmax"], a["mode"], grid, kp)


@pytest.mark.parametrize("over", [
    dict(nx=7), dict(nx=11 * 8), dict(nz=4), dict(nz=300), dict(Ly=65.0), dict(zmax=-1.0), dict(mode=3),
    dict(m_M=1), dict(m_M=13), dict(beta_M=0.0), dict(eta=0.0), dict(precision=2), dict(max_n=-1),
    dict(with_torque=1, m_D=0), dict(mode=2, zmax=1.0), dict(Lx=float("nan")),
    dict(with_torque=3, m_D=6, beta_D=13.3), dict(with_torque=-1),
    # the kernel-derivative route needs beta_D > 3 sqrt(3) / 2 (an interior minimum of |phi'|)
    dict(with_torque=2, m_D=6, beta_D=2.5),
])
def test_invalid_plan_arguments_rejected_on_host(lib, over):
    from paper_2210_01837_gb300 import binding
    st, h = _create(**over)
    assert st == binding.DPS_ERR_INVALID_ARG
    assert not h.value


def test_null_plan_rejected(lib):
    from paper_2210_01837_gb300 import binding
    assert binding.dpstokes_apply(None, 0, None, None, None, None, None, None) == binding.DPS_ERR_INVALID_ARG
    assert binding.dpstokes_status(None, None) == binding.DPS_ERR_INVALID_ARG
    st, _ = binding.dpstokes_plan_info(None)
    assert st == binding.DPS_ERR_INVALID_ARG
    assert binding.load().dpstokes_plan_set_fft(None, 1, 1, 2) == binding.DPS_ERR_INVALID_ARG
    assert binding.load().dpstokes_plan_set_pipeline(None, 1, 1) == binding.DPS_ERR_INVALID_ARG
    binding.dpstokes_destroy(None)


def test_struct_layout_matches_the_c_compiler(tmp_path):
    """sizeof/offsetof of every ABI struct from gcc against the ctypes mirrors."""
    from paper_2210_01837_gb300 import binding
    fields = {
        "dps_grid": ["nz"], "dps_kernel_params": ["beta_M", "m_D", "beta_D", "eta", "with_torque", "precision", "max_n"],
        "dps_plan_info": ["nkx", "h", "alpha_D", "launches_per_apply", "nchunks", "fft_col_width", "solve_blocks",
                          "fft_register_cols"],
        "dps_request": ["n", "positions", "torques", "out_angvel", "status"],
        "dps_serve_request": ["wall_mode", "grid", "kp", "n", "positions", "out_angvel", "walls"],
        "dps_wall_params": ["slip_top", "uw_bottom", "uw_top"],
        "dps_serve_result": ["t_submit", "t_done"], "dps_server_stats": ["running", "bytes_resident"],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dpstokes.h"', "int main(void) {"]
    for s, fs in fields.items():
        lines.append(f'  printf("{s} %zu\\n", sizeof({s}));')
        for f in fs:
            lines.append(f'  printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.split() for line in out if line.strip())
    for s, fs in fields.items():
        cls = getattr(binding, s)
        assert int(got[s]) == ctypes.sizeof(cls), s
        for f in fs:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def test_batch_and_server_reject_invalid_arguments_on_host(lib):
    from paper_2210_01837_gb300 import binding
    assert lib.dpstokes_apply_batch(None, -1, None) == binding.DPS_ERR_INVALID_ARG
    assert lib.dpstokes_apply_batch(None, 2, None) == binding.DPS_ERR_INVALID_ARG
    reqs = (binding.dps_request * 1)()  # NULL plan
    assert binding.dpstokes_apply_batch(reqs, None) == binding.DPS_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.dpstokes_server_create(ctypes.byref(h), 0, 4) == binding.DPS_ERR_INVALID_ARG
    assert lib.dpstokes_server_create(ctypes.byref(h), 1 << 30, 0) == binding.DPS_ERR_INVALID_ARG
    assert lib.dpstokes_server_create(None, 1 << 30, 4) == binding.DPS_ERR_INVALID_ARG
    t = ctypes.c_int64()
    assert lib.dpstokes_server_submit(None, None, ctypes.byref(t)) == binding.DPS_ERR_INVALID_ARG
    r = binding.dps_serve_result()
    assert lib.dpstokes_server_wait(None, 0, 0.0, ctypes.byref(r)) == binding.DPS_ERR_INVALID_ARG
    assert lib.dpstokes_server_set_queue_limit(None, 4) == binding.DPS_ERR_INVALID_ARG
    assert lib.dpstokes_debug_inject(None, 1) == binding.DPS_ERR_INVALID_ARG
    assert lib.dpstokes_plan_set_interp(None, 0) == binding.DPS_ERR_INVALID_ARG
    lib.dpstokes_server_destroy(None)


def test_tridiagonal_square_root_on_the_host_matches_the_oracle(lib):
    # the Lanczos sampler's host step (Jacobi eigendecomposition) against the oracle's eigh route
    from oracle.lanczos import sqrt_tridiagonal_e1
    from paper_2210_01837_gb300 import binding
    rng = np.random.default_rng(12)
    for j in (1, 2, 5, 17, 64):
        a = rng.uniform(1.0, 4.0, j)
        b = rng.uniform(-1.0, 1.0, max(j - 1, 0))
        st, y = binding.dpstokes_tridiag_sqrt_e1(a, b)
        assert st == binding.DPS_OK
        assert np.allclose(y, sqrt_tridiagonal_e1(a, b), rtol=0, atol=1e-12)
    # an indefinite T: eigenvalues below zero take a zero root on both sides
    a = np.array([1.0, -2.0, 0.5])
    b = np.array([0.7, 0.3])
    st, y = binding.dpstokes_tridiag_sqrt_e1(a, b)
    assert np.allclose(y, sqrt_tridiagonal_e1(a, b), rtol=0, atol=1e-12)


def test_lanczos_entry_points_reject_invalid_arguments_on_host(lib):
    from paper_2210_01837_gb300 import binding
    st, h = binding.dpstokes_lanczos_create(None, 8)
    assert st == binding.DPS_ERR_INVALID_ARG and not h.value
    st, _, _, _ = binding.dpstokes_lanczos_sample(None, 4, None, None, None, 1e-3, None, 8)
    assert st == binding.DPS_ERR_INVALID_ARG
    assert binding.dpstokes_tridiag_sqrt_e1([], [])[0] == binding.DPS_ERR_INVALID_ARG
    binding.dpstokes_lanczos_destroy(None)


@pytest.mark.parametrize("mode,walls", [
    (0, dict(slip_bottom=0.5)), (0, dict(uw_bottom=(1.0, 0.0))), (1, dict(slip_top=0.5)), (1, dict(uw_top=(0.0, 1.0))),
    (2, dict(slip_bottom=-1.0)), (2, dict(slip_top=float("inf"))), (2, dict(uw_bottom=(float("nan"), 0.0))),
])
def test_invalid_wall_conditions_rejected_on_host(lib, mode, walls):
    from paper_2210_01837_gb300 import binding
    grid = binding.dps_grid(128, 128, 65)
    kp = binding.dps_kernel_params(6, 10.2, 0, 0.0, 1.0, 0, 0, 100)
    wp = binding.wall_params(walls)
    st, h = binding.dpstokes_plan_create_ex(64.0, 64.0, 0.0, 12.0, mode, grid, kp, wp)
    assert st == binding.DPS_ERR_INVALID_ARG and not h.value


def test_rfd_drift_rejects_invalid_arguments_on_host(lib):
    from paper_2210_01837_gb300 import binding
    assert binding.dpstokes_rfd_drift(None, 4, None, None, 1e-3, None, None) == binding.DPS_ERR_INVALID_ARG
