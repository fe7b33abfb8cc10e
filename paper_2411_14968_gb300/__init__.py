"""GB300 (sm_103a) implementation of the partitioned skyline method of
Ciaccia & Martinenghi, "Optimization Strategies for Parallel Computation of
Skylines" (arXiv 2411.14968).

The method runs in libskyline (CUDA kernels behind the C ABI of
include/skyline.h); ``native`` is its ctypes binding and ``datagen`` the
seeded synthetic workloads.  The library is loaded on first use, not on
import, so that ``datagen`` works on machines without the CUDA toolkit.
"""

__all__ = ["Context", "skyline", "make_params", "SkylineError"]


def __getattr__(name):
    if name in __all__:
        from . import native
        return getattr(native, name)
    raise AttributeError(name)
