"""GB300-native doubly-periodic Force Coupling Method mobility product (Hashemi et al.).

The computation lives in libdpstokes.so (CUDA, sm_103a), reached through the C ABI declared in
include/dpstokes.h; ``binding`` marshals arguments to it.  ``workloads`` holds seeded synthetic
inputs.
"""

from . import build  # noqa: F401

__all__ = ["build", "binding", "workloads"]
