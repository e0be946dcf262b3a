"""The C ABI library loads on a machine without a GPU, exports every entry point declared in
include/dpstokes.h, and rejects invalid arguments on the host before touching the device."""

import ctypes
import os
import re

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
    binding.dpstokes_destroy(None)
