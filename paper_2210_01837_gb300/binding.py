"""Thin ctypes binding of the C ABI in include/dpstokes.h (argument marshalling only).

The module-level functions carry the C names and signatures; ``Plan`` wraps a plan handle for
torch CUDA tensors (device pointers) and numpy arrays (host pointers).  Every computation runs in
libdpstokes.so; when the library is missing this module raises instead of falling back.
"""

import ctypes
import os

import numpy as np

from . import build as _build

MODES = {"free": 0, "bottom_wall": 1, "slit": 2}
PRECISIONS = {"fp64": 0, "mixed": 1}
STATUS = {0: "DPS_OK", -1: "DPS_ERR_INVALID_ARG", -2: "DPS_ERR_OUT_OF_DOMAIN", -3: "DPS_ERR_OOM",
          -4: "DPS_ERR_CUDA", -5: "DPS_ERR_TIMEOUT", -6: "DPS_ERR_NONFINITE"}
DPS_OK, DPS_ERR_INVALID_ARG, DPS_ERR_OUT_OF_DOMAIN, DPS_ERR_OOM = 0, -1, -2, -3
DPS_ERR_CUDA, DPS_ERR_TIMEOUT, DPS_ERR_NONFINITE = -4, -5, -6


class dps_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class dps_kernel_params(ctypes.Structure):
    _fields_ = [("m_M", ctypes.c_int32), ("beta_M", ctypes.c_double), ("m_D", ctypes.c_int32),
                ("beta_D", ctypes.c_double), ("eta", ctypes.c_double), ("with_torque", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_n", ctypes.c_int64)]


class dps_plan_info(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_int64), ("nkx", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("nfields", ctypes.c_int32), ("record_words", ctypes.c_int32), ("h", ctypes.c_double),
                ("alpha_M", ctypes.c_double), ("alpha_D", ctypes.c_double), ("launches_per_apply", ctypes.c_int32),
                ("nchunks", ctypes.c_int32)]


class DpsError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({error_string(status)})")


_LIB = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64


def library_path():
    return _build.LIB


def load(path=None):
    """Load libdpstokes.so (raises OSError/RuntimeError if it is missing or broken)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2210_01837_gb300.build.build()")
    lib = ctypes.CDLL(path)
    sig = {
        "dpstokes_plan_create": (_I32, [ctypes.POINTER(_P), _D, _D, _D, _D, _I32, ctypes.POINTER(dps_grid),
                                        ctypes.POINTER(dps_kernel_params)]),
        "dpstokes_apply": (_I32, [_P, _I64, _P, _P, _P, _P, _P, _P]),
        "dpstokes_apply_host": (_I32, [_P, _I64, _P, _P, _P, _P, _P, _P]),
        "dpstokes_status": (_I32, [_P, _P]),
        "dpstokes_destroy": (None, [_P]),
        "dpstokes_error_string": (ctypes.c_char_p, [_I32]),
        "dpstokes_plan_info": (_I32, [_P, ctypes.POINTER(dps_plan_info)]),
        "dpstokes_enable_timing": (_I32, [_P, _I32]),
        "dpstokes_stage_times": (_I32, [_P, ctypes.POINTER(ctypes.c_double), _I32, ctypes.POINTER(_I32)]),
        "dpstokes_spread_noalloc": (_I32, [_D, _D, _D, _D, _I32, ctypes.POINTER(dps_grid),
                                           ctypes.POINTER(dps_kernel_params), _I64, _P, _P, _P, _P, _I64, _P]),
        "dpstokes_debug_run": (_I32, [_P, _I64, _P, _P, _P, _P, _P, _P, _I32]),
        "dpstokes_debug_copy": (_I32, [_P, _I32, _P, _I64, _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


# ---- C names -------------------------------------------------------------------------------
def dpstokes_error_string(status):
    return load().dpstokes_error_string(int(status)).decode()


error_string = dpstokes_error_string


def dpstokes_plan_create(Lx, Ly, zmin, zmax, wall_mode, grid, kp):
    """Returns (status, handle)."""
    h = _P()
    st = load().dpstokes_plan_create(ctypes.byref(h), Lx, Ly, zmin, zmax, wall_mode, ctypes.byref(grid),
                                     ctypes.byref(kp))
    return st, h


def dpstokes_apply(plan, n, positions, forces, torques, out_vel, out_angvel, stream):
    return load().dpstokes_apply(plan, n, positions, forces, torques, out_vel, out_angvel, stream)


def dpstokes_apply_host(plan, n, positions, forces, torques, out_vel, out_angvel, stream):
    return load().dpstokes_apply_host(plan, n, positions, forces, torques, out_vel, out_angvel, stream)


def dpstokes_status(plan, stream):
    return load().dpstokes_status(plan, stream)


def dpstokes_destroy(plan):
    load().dpstokes_destroy(plan)


def dpstokes_plan_info(plan):
    info = dps_plan_info()
    st = load().dpstokes_plan_info(plan, ctypes.byref(info))
    return st, info


STAGES = ("init", "records", "bins", "spread", "fft_x_fwd", "fft_y_fwd", "cheb_fwd", "solve", "cheb_bwd",
          "fft_y_inv", "fft_x_inv", "interp")


def dpstokes_enable_timing(plan, enable):
    return load().dpstokes_enable_timing(plan, int(enable))


def dpstokes_stage_times(plan):
    """Returns (status, list of per-stage milliseconds of the last timed apply)."""
    buf = (ctypes.c_double * len(STAGES))()
    cnt = _I32(0)
    st = load().dpstokes_stage_times(plan, buf, len(STAGES), ctypes.byref(cnt))
    return st, list(buf)[: cnt.value]


def dpstokes_spread_noalloc(Lx, Ly, zmin, zmax, wall_mode, grid, kp, n, positions, forces, torques, out_grid,
                            ldx, stream):
    """Spreading stage with no device allocation (scratch is a fixed array inside the library)."""
    return load().dpstokes_spread_noalloc(Lx, Ly, zmin, zmax, wall_mode, ctypes.byref(grid), ctypes.byref(kp), n,
                                          positions, forces, torques, out_grid, ldx, stream)


def dpstokes_debug_run(plan, n, positions, forces, torques, out_vel, out_angvel, stream, last_stage):
    return load().dpstokes_debug_run(plan, n, positions, forces, torques, out_vel, out_angvel, stream, last_stage)


def dpstokes_debug_copy(plan, which, dst, dst_bytes, stream):
    return load().dpstokes_debug_copy(plan, which, dst, dst_bytes, stream)


# ---- convenience wrapper --------------------------------------------------------------------
def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.dtype == np.float64 and t.flags.c_contiguous
        return t.ctypes.data
    assert t.dtype.is_floating_point and t.is_contiguous() and t.is_cuda, "expected a contiguous CUDA tensor"
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Plan:
    """A resident problem (box, wall mode, grid, kernels) with its device buffers."""

    def __init__(self, Lx, Ly, zmin, zmax, mode, nx, ny, nz, m_M, beta_M, m_D=0, beta_D=0.0, eta=1.0,
                 with_torque=False, precision="mixed", max_n=1):
        self.with_torque = bool(with_torque)
        self.precision = precision
        self.max_n = int(max_n)
        grid = dps_grid(int(nx), int(ny), int(nz))
        kp = dps_kernel_params(int(m_M), float(beta_M), int(m_D), float(beta_D), float(eta),
                               1 if with_torque else 0, PRECISIONS[precision], int(max_n))
        st, h = dpstokes_plan_create(float(Lx), float(Ly), float(zmin), float(zmax), MODES[mode], grid, kp)
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_plan_create")
        self.handle = h

    @classmethod
    def from_params(cls, params, with_torque, precision, max_n):
        keys = ("Lx", "Ly", "zmin", "zmax", "mode", "nx", "ny", "nz", "m_M", "beta_M", "m_D", "beta_D", "eta")
        return cls(**{k: params[k] for k in keys}, with_torque=with_torque, precision=precision, max_n=max_n)

    def info(self):
        st, info = dpstokes_plan_info(self.handle)
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_plan_info")
        return info

    def apply(self, pos, F, T=None, U=None, W=None, stream=None, check=False):
        """pos, F, T: CUDA float64 tensors [n, 3]; returns (U, W) CUDA tensors (W None without torques)."""
        import torch
        n = pos.shape[0]
        if U is None:
            U = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
        if self.with_torque and W is None:
            W = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
        st = dpstokes_apply(self.handle, n, _ptr(pos), _ptr(F), _ptr(T), _ptr(U), _ptr(W) if self.with_torque else None,
                            _stream(stream))
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_apply")
        if check:
            self.check(stream)
        return U, (W if self.with_torque else None)

    def apply_host(self, pos, F, T=None, U=None, W=None, stream=None):
        """Host (numpy float64, preferably pinned) arrays in and out; synchronises."""
        n = pos.shape[0]
        U = np.empty((n, 3)) if U is None else U
        W = (np.empty((n, 3)) if W is None else W) if self.with_torque else None
        st = dpstokes_apply_host(self.handle, n, _ptr(pos), _ptr(F), _ptr(T), _ptr(U), _ptr(W), _stream(stream))
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_apply_host")
        return U, W

    def status(self, stream=None):
        return dpstokes_status(self.handle, _stream(stream))

    def check(self, stream=None):
        st = self.status(stream)
        if st != DPS_OK:
            raise DpsError(st, "device status")

    def enable_timing(self, enable=True):
        st = dpstokes_enable_timing(self.handle, enable)
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_enable_timing")

    def stage_times(self):
        st, ms = dpstokes_stage_times(self.handle)
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_stage_times")
        return dict(zip(STAGES, ms))

    def debug_run(self, pos, F, T, last_stage, U=None, W=None, stream=None):
        st = dpstokes_debug_run(self.handle, pos.shape[0], _ptr(pos), _ptr(F), _ptr(T), _ptr(U), _ptr(W),
                                _stream(stream), int(last_stage))
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_debug_run")

    def debug_copy(self, which, dst, stream=None):
        st = dpstokes_debug_copy(self.handle, int(which), dst.data_ptr(), dst.numel() * dst.element_size(),
                                 _stream(stream))
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_debug_copy")

    def close(self):
        if getattr(self, "handle", None):
            dpstokes_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
