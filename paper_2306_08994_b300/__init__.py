"""Multifrontal direct solver for finite-element matrices on one B300 GPU.

The compute path is libmfsolve.so (hand-written CUDA for sm_103a behind the C
ABI of include/mfsolve.h); this package only binds it.  The binding is loaded
on first use of any name below and raises ImportError if the library has not
been built -- there is no fallback implementation.
"""
_NAMES = {"MF_F32", "MF_F64", "MF_TF32", "MF_TF32_BF16", "Analysis", "Factors", "Mesh", "MFError", "default_options", "lib"}

__all__ = sorted(_NAMES | {"MFSolve"})


def __getattr__(name):
    if name in _NAMES:
        from . import mfsolve
        return getattr(mfsolve, name)
    if name == "MFSolve":
        from .autograd import MFSolve
        return MFSolve
    raise AttributeError(name)
