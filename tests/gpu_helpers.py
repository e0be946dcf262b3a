"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI, read the plan's
intermediate buffers, and run the oracle on the same seeded inputs."""

import numpy as np

from oracle import Params, mobility, table1
from oracle import stokes as ostokes
from oracle import transfer as otransfer
from paper_2210_01837_gb300 import binding


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def small_params(mode, nx=72, ny=72, nz=33, L=None, zmax=10.0, m=5, torque=True):
    rh, bm, bd = table1(5)
    h = 2.0 / 3.0 if L is None else L / nx
    return dict(Lx=h * nx, Ly=h * ny, zmin=0.0, zmax=zmax, mode=mode, nx=nx, ny=ny, nz=nz, m_M=m,
                beta_M=m * bm, m_D=m if torque else 0, beta_D=m * bd if torque else 0.0, eta=0.9)


def oracle_params(params):
    return Params(**params)


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def gpu_mobility(params, pos, F, T, precision, plan=None, route="spectral_curl"):
    import torch
    close = plan is None
    if plan is None:
        plan = binding.Plan.from_params(params, with_torque=route if T is not None else False, precision=precision,
                                        max_n=max(1, len(pos)))
    U, W = plan.apply(to_dev(pos), to_dev(F), None if T is None else to_dev(T), check=True)
    torch.cuda.synchronize()
    out = (U.cpu().numpy(), None if W is None else W.cpu().numpy())
    if close:
        plan.close()
    return out


def read_grid(plan, params, precision):
    """The plan's grid/spectrum buffer as a numpy array [fields][nz][ny][2*pitch] (reals)."""
    import torch
    info = plan.info()
    dt = torch.float32 if precision == "mixed" else torch.float64
    buf = torch.empty((info.nfields, params["nz"], params["ny"], 2 * info.pitch), dtype=dt, device="cuda")
    plan.debug_copy(0, buf)
    torch.cuda.synchronize()
    return buf.cpu().numpy().astype(np.float64), info


def zrange(plan):
    import torch
    z = torch.empty(2, dtype=torch.int32, device="cuda")
    plan.debug_copy(2, z)
    torch.cuda.synchronize()
    return tuple(int(v) for v in z.cpu().numpy())
