"""Stochastic drift by random finite differences (test infrastructure only).

Sec. IV.C (footnote on Brownian dynamics in confinement): the drift k_B T (d/dq . M) can be had from
two extra mobility solves per step.  Random finite differences: with W a standard normal vector of
the dimension of the configuration q (the particle positions),
    d = (1/delta) [M(q + delta/2 W) - M(q - delta/2 W)] W,
whose average over W is the divergence of M with respect to q, sum_j dM_ij/dq_j, up to O(delta^2).
For spheres the configuration is the positions only, so with torques the vector multiplied is
[W; 0] (no torque part) and the result has a translational and a rotational part.
"""

import numpy as np

from .stokes import mobility


def rfd_drift(p, pos, W, delta, with_torque=False, torque_route="spectral_curl"):
    """(1/delta)[M(q + delta/2 W) - M(q - delta/2 W)] [W; 0].  pos, W: (N, 3).  Returns
    (dU (N, 3), dOmega (N, 3) or None)."""
    pos = np.asarray(pos, dtype=float)
    W = np.asarray(W, dtype=float)
    T = np.zeros_like(W) if with_torque else None
    Up, Wp = mobility(p, pos + 0.5 * delta * W, W, T, torque_route=torque_route)
    Um, Wm = mobility(p, pos - 0.5 * delta * W, W, T, torque_route=torque_route)
    dU = (Up - Um) / delta
    dW = (Wp - Wm) / delta if with_torque else None
    return dU, dW


__all__ = ["rfd_drift"]
