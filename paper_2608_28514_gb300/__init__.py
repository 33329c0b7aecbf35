"""GB300-native (sm_103a) batched nested sampler of arXiv 2608.28514.

The sampler runs in the CUDA library ``libns_gb300.so`` behind the C ABI of
``include/ns_gb300.h``; :mod:`._native` is its ctypes binding.  The
workload generators (:mod:`.workloads`) are host-side helpers that describe
the seeded synthetic problems.
"""
from . import workloads  # noqa: F401


def native():
    """The ctypes binding; raises if the CUDA library is not built."""
    from . import _native
    _native.lib()
    return _native
