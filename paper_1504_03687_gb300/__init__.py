"""GB300 (sm_103a) regular-force library for NBODY6++GPU-style direct N-body integration.

The regular-force step of Wang et al. (2015): FP64 prediction of all particles,
then for every particle of an active block the acceleration, jerk and potential
from all N particles and the neighbour list inside r_s, computed by hand-written
CUDA kernels behind a C ABI (include/nbgpu.h); around it the irregular force over the
neighbour lists, the adjoint, the batched ensemble form and the block-step sorting list.
This package is the thin Python binding (argument marshalling only).
"""
from .api import (ACIntegrator, Context, ForceResult, NBError, NBOverflow, Scheduler, load_library,  # noqa: F401
                  plan_for)

__all__ = ["ACIntegrator", "Context", "ForceResult", "NBError", "NBOverflow", "Scheduler", "load_library",
           "plan_for"]
