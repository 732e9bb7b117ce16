"""GB300-native lattice stepper for interacting scalar fields in an expanding
(FLRW) background: hand-written sm_103a CUDA behind a C ABI (include/tl.h),
with a thin ctypes binding on top (``paper_2607_24908_gb300.tl``).

The binding loads ``libtl.so`` on first use and raises if it is missing;
there is no CPU fallback.
"""
import importlib

__all__ = ["tl", "workloads"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
