"""GB300 (sm_103a) library for the ageing simulation of the 3D +-J Edwards-Anderson
model (Manssen & Hartmann, arXiv 1411.5512): bit-packed checkerboard Metropolis and
heat-bath sweeps and on-device ageing observables behind a small C ABI.  Beside the
binding (``job``): the host analysis of Sec. IV (``analysis``), the reduced p-scan
(``pscan``), placement over ranks (``shard``) and recovery from a rank that stops
(``recovery``).

Importing the package does not load the CUDA library; ``EAJob`` and the other
entry points load it on first use and raise if it has not been built.
"""
from . import _lib  # noqa: F401


def __getattr__(name):
    if name in ("EAJob", "EABatch", "EAServer", "geometry", "thresholds", "footprint",
                "use_torch_allocator", "use_cuda_allocator", "launch_count"):
        from . import job
        return getattr(job, name)
    raise AttributeError(name)
