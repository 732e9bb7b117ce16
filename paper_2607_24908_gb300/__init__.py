"""GB300-native lattice stepper for interacting scalar fields in an expanding
(FLRW) background: hand-written sm_103a CUDA behind a C ABI (include/tl.h),
with this thin ctypes binding on top.

The binding (``paper_2607_24908_gb300.tl``) loads ``libtl.so`` on first use
and raises if it is missing; there is no CPU fallback.
"""
__all__ = ["tl", "workloads"]


def __getattr__(name):
    if name == "tl":
        from . import tl as _tl
        return _tl
    if name == "workloads":
        from . import workloads as _w
        return _w
    raise AttributeError(name)
