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
# dps_torque_route; with_torque also takes False (none) and True (the spectral curl)
TORQUE_ROUTES = {"none": 0, "spectral_curl": 1, "kernel_derivative": 2}


def torque_route(with_torque):
    """dps_torque_route code of a with_torque argument: a bool, a route name or the code itself."""
    if isinstance(with_torque, str):
        return TORQUE_ROUTES[with_torque]
    if isinstance(with_torque, bool) or with_torque in (0, 1):
        return 1 if with_torque else 0
    if with_torque == 2:
        return 2
    raise ValueError(f"unknown torque route {with_torque!r}")
STATUS = {0: "DPS_OK", -1: "DPS_ERR_INVALID_ARG", -2: "DPS_ERR_OUT_OF_DOMAIN", -3: "DPS_ERR_OOM",
          -4: "DPS_ERR_CUDA", -5: "DPS_ERR_TIMEOUT", -6: "DPS_ERR_NONFINITE", -7: "DPS_ERR_BUSY"}
DPS_OK, DPS_ERR_INVALID_ARG, DPS_ERR_OUT_OF_DOMAIN, DPS_ERR_OOM = 0, -1, -2, -3
DPS_ERR_CUDA, DPS_ERR_TIMEOUT, DPS_ERR_NONFINITE, DPS_ERR_BUSY = -4, -5, -6, -7


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
                ("nchunks", ctypes.c_int32), ("fft_col_width", ctypes.c_int32), ("solve_blocks", ctypes.c_int32),
                ("fft_register_rows", ctypes.c_int32), ("fft_register_cols", ctypes.c_int32),
                ("interp_variant", ctypes.c_int32), ("cheb_tensor_cores", ctypes.c_int32)]


class dps_request(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("n", ctypes.c_int64), ("positions", ctypes.c_void_p),
                ("forces", ctypes.c_void_p), ("torques", ctypes.c_void_p), ("out_vel", ctypes.c_void_p),
                ("out_angvel", ctypes.c_void_p), ("status", ctypes.c_void_p)]


class dps_wall_params(ctypes.Structure):
    _fields_ = [("slip_bottom", ctypes.c_double), ("slip_top", ctypes.c_double),
                ("uw_bottom", ctypes.c_double * 2), ("uw_top", ctypes.c_double * 2)]


def wall_params(params):
    """dps_wall_params from the optional slip_bottom, slip_top, uw_bottom, uw_top entries of params."""
    ub = params.get("uw_bottom", (0.0, 0.0)) or (0.0, 0.0)
    ut = params.get("uw_top", (0.0, 0.0)) or (0.0, 0.0)
    w = dps_wall_params(float(params.get("slip_bottom", 0.0) or 0.0), float(params.get("slip_top", 0.0) or 0.0))
    w.uw_bottom[0], w.uw_bottom[1] = float(ub[0]), float(ub[1])
    w.uw_top[0], w.uw_top[1] = float(ut[0]), float(ut[1])
    return w


class dps_serve_request(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("zmin", ctypes.c_double),
                ("zmax", ctypes.c_double), ("wall_mode", ctypes.c_int32), ("grid", dps_grid),
                ("kp", dps_kernel_params), ("n", ctypes.c_int64), ("positions", ctypes.c_void_p),
                ("forces", ctypes.c_void_p), ("torques", ctypes.c_void_p), ("out_vel", ctypes.c_void_p),
                ("out_angvel", ctypes.c_void_p), ("walls", dps_wall_params)]


class dps_serve_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class dps_server_stats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("running", ctypes.c_int64), ("plans_resident", ctypes.c_int64),
                ("plans_created", ctypes.c_int64), ("plans_evicted", ctypes.c_int64),
                ("bytes_resident", ctypes.c_int64), ("rejected", ctypes.c_int64)]


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
        "dpstokes_plan_create_ex": (_I32, [ctypes.POINTER(_P), _D, _D, _D, _D, _I32, ctypes.POINTER(dps_grid),
                                           ctypes.POINTER(dps_kernel_params), ctypes.POINTER(dps_wall_params)]),
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
        "dpstokes_plan_set_fft": (_I32, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
        "dpstokes_plan_set_pipeline": (_I32, [_P, ctypes.c_int32, ctypes.c_int32]),
        "dpstokes_plan_set_interp": (_I32, [_P, ctypes.c_int32]),
        "dpstokes_debug_inject": (_I32, [_P, ctypes.c_int32]),
        "dpstokes_plan_autotune": (_I32, [_P, _I64, _P, _P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
        "dpstokes_apply_batch": (_I32, [ctypes.POINTER(dps_request), _I32, _P]),
        "dpstokes_batch_prepare": (_I32, []),
        "dpstokes_server_create": (_I32, [ctypes.POINTER(_P), _I64, _I32]),
        "dpstokes_server_submit": (_I32, [_P, ctypes.POINTER(dps_serve_request), ctypes.POINTER(_I64)]),
        "dpstokes_server_wait": (_I32, [_P, _I64, _D, ctypes.POINTER(dps_serve_result)]),
        "dpstokes_server_stats": (_I32, [_P, ctypes.POINTER(dps_server_stats)]),
        "dpstokes_server_set_queue_limit": (_I32, [_P, _I64]),
        "dpstokes_server_destroy": (None, [_P]),
        "dpstokes_lanczos_create": (_I32, [ctypes.POINTER(_P), _P, _I32]),
        "dpstokes_lanczos_sample": (_I32, [_P, _I64, _P, _P, _P, _D, ctypes.POINTER(_I32), ctypes.POINTER(_D),
                                           ctypes.POINTER(_D), _P]),
        "dpstokes_lanczos_destroy": (None, [_P]),
        "dpstokes_tridiag_sqrt_e1": (_I32, [_I32, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D)]),
        "dpstokes_rfd_drift": (_I32, [_P, _I64, _P, _P, _D, _P, _P]),
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


def dpstokes_plan_create_ex(Lx, Ly, zmin, zmax, wall_mode, grid, kp, wp):
    """Returns (status, handle); wp a dps_wall_params or None."""
    h = _P()
    st = load().dpstokes_plan_create_ex(ctypes.byref(h), Lx, Ly, zmin, zmax, wall_mode, ctypes.byref(grid),
                                        ctypes.byref(kp), None if wp is None else ctypes.byref(wp))
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


def dpstokes_plan_autotune(plan, n, positions, forces, torques, out_vel, out_angvel, stream):
    """Returns (status, best milliseconds)."""
    ms = ctypes.c_double(0.0)
    st = load().dpstokes_plan_autotune(plan, n, positions, forces, torques, out_vel, out_angvel, stream,
                                       ctypes.byref(ms))
    return st, ms.value


def dpstokes_apply_batch(reqs, stream):
    """reqs: a ctypes array of dps_request."""
    return load().dpstokes_apply_batch(reqs, len(reqs), stream)


def dpstokes_batch_prepare():
    return load().dpstokes_batch_prepare()


def dpstokes_server_create(memory_budget_bytes, slots):
    """Returns (status, handle)."""
    h = _P()
    st = load().dpstokes_server_create(ctypes.byref(h), int(memory_budget_bytes), int(slots))
    return st, h


def dpstokes_server_submit(server, req):
    """Returns (status, ticket)."""
    t = _I64(-1)
    st = load().dpstokes_server_submit(server, ctypes.byref(req), ctypes.byref(t))
    return st, t.value


def dpstokes_server_wait(server, ticket, timeout_s):
    """Returns (status, dps_serve_result)."""
    r = dps_serve_result()
    st = load().dpstokes_server_wait(server, int(ticket), float(timeout_s), ctypes.byref(r))
    return st, r


def dpstokes_server_stats(server):
    s = dps_server_stats()
    st = load().dpstokes_server_stats(server, ctypes.byref(s))
    return st, s


def dpstokes_server_set_queue_limit(server, max_queued):
    return load().dpstokes_server_set_queue_limit(server, int(max_queued))


def dpstokes_server_destroy(server):
    load().dpstokes_server_destroy(server)


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
                 with_torque=False, precision="mixed", max_n=1, slip_bottom=0.0, slip_top=0.0,
                 uw_bottom=(0.0, 0.0), uw_top=(0.0, 0.0)):
        self.route = torque_route(with_torque)
        self.with_torque = self.route != 0
        self.precision = precision
        self.max_n = int(max_n)
        grid = dps_grid(int(nx), int(ny), int(nz))
        kp = dps_kernel_params(int(m_M), float(beta_M), int(m_D), float(beta_D), float(eta),
                               self.route, PRECISIONS[precision], int(max_n))
        wp = wall_params(dict(slip_bottom=slip_bottom, slip_top=slip_top, uw_bottom=uw_bottom, uw_top=uw_top))
        st, h = dpstokes_plan_create_ex(float(Lx), float(Ly), float(zmin), float(zmax), MODES[mode], grid, kp, wp)
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_plan_create")
        self.handle = h

    @classmethod
    def from_params(cls, params, with_torque, precision, max_n):
        keys = ("Lx", "Ly", "zmin", "zmax", "mode", "nx", "ny", "nz", "m_M", "beta_M")
        optional = ("m_D", "beta_D", "eta", "slip_bottom", "slip_top", "uw_bottom", "uw_top")
        return cls(**{k: params[k] for k in keys}, **{k: params[k] for k in optional if k in params},
                   with_torque=with_torque, precision=precision, max_n=max_n)

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

    def set_fft(self, row_register, col_register, col_width):
        """Set the xy-FFT variants and column width by hand; raises if the shape does not fit."""
        st = load().dpstokes_plan_set_fft(self.handle, int(row_register), int(col_register), int(col_width))
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_plan_set_fft")

    def debug_inject(self, code):
        st = load().dpstokes_debug_inject(self.handle, int(code))
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_debug_inject")

    def set_interp(self, variant):
        st = load().dpstokes_plan_set_interp(self.handle, int(variant))
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_plan_set_interp")

    def set_pipeline(self, solve_blocks, nchunks):
        """Set the FP64 solve's persistent grid and the column chunks by hand; raises if out of range."""
        st = load().dpstokes_plan_set_pipeline(self.handle, int(solve_blocks), int(nchunks))
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_plan_set_pipeline")

    def autotune(self, pos, F, T=None, U=None, W=None, stream=None):
        """Pick launch shapes by timing applies on these particles; returns the best time in ms."""
        import torch
        n = pos.shape[0]
        U = torch.empty((n, 3), dtype=torch.float64, device=pos.device) if U is None else U
        if self.with_torque and W is None:
            W = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
        st, ms = dpstokes_plan_autotune(self.handle, n, _ptr(pos), _ptr(F), _ptr(T), _ptr(U),
                                        _ptr(W) if self.with_torque else None, _stream(stream))
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_plan_autotune")
        return ms

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


def apply_batch(items, stream=None, status=None):
    """items: list of (Plan, pos, F, T, U, W) with CUDA tensors; status: optional CUDA int32 tensor
    [len(items)] that receives each request's device status."""
    arr = (dps_request * len(items))()
    for i, (plan, pos, F, T, U, W) in enumerate(items):
        arr[i].plan = plan.handle.value if isinstance(plan.handle, ctypes.c_void_p) else plan.handle
        arr[i].n = pos.shape[0]
        arr[i].positions, arr[i].forces, arr[i].torques = _ptr(pos), _ptr(F), _ptr(T)
        arr[i].out_vel, arr[i].out_angvel = _ptr(U), _ptr(W)
        arr[i].status = (status.data_ptr() + 4 * i) if status is not None else None
    st = dpstokes_apply_batch(arr, _stream(stream))
    if st != DPS_OK:
        raise DpsError(st, "dpstokes_apply_batch")


class Server:
    """Request server: host arrays in and out, plans cached under a device-memory budget."""

    def __init__(self, memory_budget_bytes, slots=8, max_queued=0):
        st, h = dpstokes_server_create(memory_budget_bytes, slots)
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_server_create")
        self.handle = h
        self._keep = {}
        if max_queued:
            st = dpstokes_server_set_queue_limit(h, max_queued)
            if st != DPS_OK:
                raise DpsError(st, "dpstokes_server_set_queue_limit")

    def submit(self, params, with_torque, precision, max_n, pos, F, T=None, U=None, W=None):
        """params: dict as in Plan.from_params; pos/F/T host float64 [n, 3] (kept alive until wait).
        Returns a ticket (None when a queue limit refused the request); outputs land in U (and W)."""
        n = pos.shape[0]
        route = torque_route(with_torque)
        U = np.empty((n, 3)) if U is None else U
        W = (np.empty((n, 3)) if W is None else W) if route else None
        r = dps_serve_request()
        r.Lx, r.Ly, r.zmin, r.zmax = (float(params[k]) for k in ("Lx", "Ly", "zmin", "zmax"))
        r.wall_mode = MODES[params["mode"]]
        r.grid = dps_grid(int(params["nx"]), int(params["ny"]), int(params["nz"]))
        r.kp = dps_kernel_params(int(params["m_M"]), float(params["beta_M"]), int(params.get("m_D", 0) or 0),
                                 float(params.get("beta_D", 0.0) or 0.0), float(params.get("eta", 1.0)),
                                 route, PRECISIONS[precision], int(max_n))
        r.n = n
        r.walls = wall_params(params)
        r.positions, r.forces, r.torques = _ptr(pos), _ptr(F), _ptr(T)
        r.out_vel, r.out_angvel = _ptr(U), _ptr(W)
        st, t = dpstokes_server_submit(self.handle, r)
        if st == DPS_ERR_BUSY:
            return None  # queue at its limit: not accepted
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_server_submit")
        self._keep[t] = (pos, F, T, U, W)
        return t

    def wait(self, ticket, timeout_s=600.0):
        """Returns (dps_serve_result, U, W)."""
        st, r = dpstokes_server_wait(self.handle, ticket, timeout_s)
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_server_wait")
        _, _, _, U, W = self._keep.pop(ticket)
        return r, U, W

    def stats(self):
        st, s = dpstokes_server_stats(self.handle)
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_server_stats")
        return {k: getattr(s, k) for k, _ in dps_server_stats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            dpstokes_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- stochastic drift (random finite differences) --------------------------------------------
def dpstokes_rfd_drift(plan, n, positions, W, delta, out, stream):
    return load().dpstokes_rfd_drift(plan, int(n), positions, W, float(delta), out, stream)


def rfd_drift(plan, pos, W, delta, out=None, stream=None):
    """(1/delta)[M(q + delta/2 W) - M(q - delta/2 W)][W; 0] for a Plan; pos, W CUDA float64 [n, 3].
    Returns a CUDA tensor [n, 3] (or [2n, 3] with torques: velocity rows, then angular rows)."""
    import torch
    n = pos.shape[0]
    if out is None:
        out = torch.empty(((2 if plan.with_torque else 1) * n, 3), dtype=torch.float64, device=pos.device)
    st = dpstokes_rfd_drift(plan.handle, n, _ptr(pos), _ptr(W), delta, _ptr(out), _stream(stream))
    if st != DPS_OK:
        raise DpsError(st, "dpstokes_rfd_drift")
    return out


# ---- Brownian increments (Lanczos) -----------------------------------------------------------
def dpstokes_lanczos_create(plan, max_iter):
    h = _P()
    st = load().dpstokes_lanczos_create(ctypes.byref(h), plan, int(max_iter))
    return st, h


def dpstokes_lanczos_sample(lz, n, positions, w, g, tol, stream, max_iter):
    """Returns (status, iterations, last eps, eps history as a list)."""
    it = _I32(0)
    eps = _D(0.0)
    hist = (_D * max(1, int(max_iter)))()
    st = load().dpstokes_lanczos_sample(lz, int(n), positions, w, g, float(tol), ctypes.byref(it), ctypes.byref(eps),
                                        hist, stream)
    return st, it.value, eps.value, [hist[i] for i in range(max(0, it.value - 1))]


def dpstokes_lanczos_destroy(lz):
    load().dpstokes_lanczos_destroy(lz)


def dpstokes_tridiag_sqrt_e1(alpha, beta):
    """y = T^{1/2} e_1 of the symmetric tridiagonal (alpha, beta), computed by the library (host)."""
    j = len(alpha)
    a = (_D * j)(*[float(x) for x in alpha])
    b = (_D * max(1, j - 1))(*[float(x) for x in beta[: j - 1]] if j > 1 else [0.0])
    y = (_D * j)()
    st = load().dpstokes_tridiag_sqrt_e1(j, a, b, y)
    return st, [y[i] for i in range(j)]


class Lanczos:
    """Brownian increments g ~ M^{1/2} w with a plan's mobility product as the operator."""

    def __init__(self, plan, max_iter=32):
        st, h = dpstokes_lanczos_create(plan.handle, max_iter)
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_lanczos_create")
        self.handle = h
        self.plan = plan
        self.max_iter = int(max_iter)

    def sample(self, pos, w, g=None, tol=1e-3, stream=None):
        """pos: CUDA float64 [n, 3]; w: CUDA float64 of 3n (or 6n with torques) values.  Returns
        (g, iterations, eps history)."""
        import torch
        n = pos.shape[0]
        if g is None:
            g = torch.empty_like(w)
        st, it, _, hist = dpstokes_lanczos_sample(self.handle, n, _ptr(pos), _ptr(w), _ptr(g), tol, _stream(stream),
                                                  self.max_iter)
        if st != DPS_OK:
            raise DpsError(st, "dpstokes_lanczos_sample")
        return g, it, hist

    def close(self):
        if self.handle:
            dpstokes_lanczos_destroy(self.handle)
            self.handle = None
