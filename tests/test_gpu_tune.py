"""The autotuner picks valid launch shapes and the product does not depend on them beyond the
summation order (A17 bar for mixed precision, 1e-6 relative L2)."""

import pytest

from paper_2210_01837_gb300 import binding
from paper_2210_01837_gb300.workloads import random_particles

from gpu_helpers import rel_l2, small_params, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,bar", [("mixed", 1e-6), ("fp64", 1e-12)])
def test_autotune_keeps_the_product(precision, bar):
    import torch
    params = small_params("slit", nx=192, ny=160, nz=33, zmax=6.0)
    pos, F, T = random_particles(params, 3000, 77)
    plan = binding.Plan.from_params(params, with_torque=True, precision=precision, max_n=len(pos))
    args = (to_dev(pos), to_dev(F), to_dev(T))
    U0, W0 = plan.apply(*args, check=True)
    U0, W0 = U0.clone(), W0.clone()
    ms = plan.autotune(*args)
    assert ms > 0.0
    info = plan.info()
    assert info.fft_col_width in (1, 2, 4, 8)
    assert info.solve_blocks >= 1
    assert info.nchunks in (1, 2, 4)
    U1, W1 = plan.apply(*args, check=True)
    torch.cuda.synchronize()
    assert rel_l2(U1.cpu().numpy(), U0.cpu().numpy()) <= bar
    assert rel_l2(W1.cpu().numpy(), W0.cpu().numpy()) <= bar
    plan.close()
