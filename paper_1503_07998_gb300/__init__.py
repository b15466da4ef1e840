"""Plane-wise multi-view Richardson-Lucy deconvolution on GB300 (sm_103a).

The compute path is the CUDA library ``_lib/libmvd.so`` behind the C ABI in
``include/mvd.h``; :mod:`.mvd` is its ctypes binding (same function names)
and :mod:`.synth` makes seeded synthetic inputs.  Build the library with
``python -m paper_1503_07998_gb300.build``.
"""

__all__ = ["mvd", "synth", "build"]


def __getattr__(name):
    if name.startswith("mvd_") or name in ("Context", "MvdError", "Info"):
        from . import mvd as _m
        return getattr(_m, name)
    raise AttributeError(name)
