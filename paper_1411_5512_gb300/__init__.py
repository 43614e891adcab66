"""GB300 (sm_103a) library for the ageing simulation of the 3D +-J Edwards-Anderson
model (Manssen & Hartmann, arXiv 1411.5512): bit-packed checkerboard Metropolis
sweeps and on-device ageing observables behind a small C ABI.

Importing the package does not load the CUDA library; ``EAJob`` and the other
entry points load it on first use and raise if it has not been built.
"""
from . import _lib  # noqa: F401


def __getattr__(name):
    if name in ("EAJob", "EABatch", "EAServer", "geometry", "thresholds", "footprint", "use_torch_allocator",
                "use_cuda_allocator"):
        from . import job
        return getattr(job, name)
    raise AttributeError(name)
