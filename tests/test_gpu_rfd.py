"""Random-finite-difference drift (Sec. IV.C footnote) through the C ABI against the oracle.

The drift is a difference quotient of two products, so the per-product bars (1e-9 FP64, 1e-5 mixed,
relative) propagate as eps (|M(q+) W| + |M(q-) W|) / delta; the test bounds the difference from the
oracle by exactly that.
"""

import numpy as np
import pytest

from gpu_helpers import oracle_params, small_params, to_dev
from oracle import mobility
from oracle.rfd import rfd_drift
from paper_2210_01837_gb300 import binding
from paper_2210_01837_gb300.workloads import random_particles

pytestmark = pytest.mark.gpu

EPS = {"fp64": 1e-9, "mixed": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2210_01837_gb300 import build
    build.build()
    binding.load()


@pytest.mark.parametrize("precision,delta", [("fp64", 1e-3), ("mixed", 0.1)])
@pytest.mark.parametrize("mode,torque", [("bottom_wall", False), ("slit", True), ("bottom_wall", "kernel_derivative")])
def test_drift_matches_oracle(mode, torque, precision, delta):
    import torch
    params = small_params(mode, nx=54, ny=40, nz=25, torque=bool(torque))
    pos, _, _ = random_particles(params, 30, seed=71, torques=False, margin=0.5)
    W = np.random.default_rng(72).standard_normal(pos.shape)
    route = torque if isinstance(torque, str) else "spectral_curl"
    op = oracle_params(params)
    dU, dW = rfd_drift(op, pos, W, delta, with_torque=bool(torque), torque_route=route)
    plan = binding.Plan.from_params(params, with_torque=torque, precision=precision, max_n=len(pos))
    got = binding.rfd_drift(plan, to_dev(pos), to_dev(W), delta)
    assert plan.status() == binding.DPS_OK
    got = got.cpu().numpy()
    want = np.concatenate([dU, dW]) if torque else dU
    T0 = np.zeros_like(W) if torque else None
    scale = 0.0
    for sgn in (1.0, -1.0):
        U, Om = mobility(op, pos + sgn * 0.5 * delta * W, W, T0, torque_route=route)
        scale += np.linalg.norm(U) + (np.linalg.norm(Om) if torque else 0.0)
    assert np.linalg.norm(got - want) <= EPS[precision] * scale / delta
    plan.close()
