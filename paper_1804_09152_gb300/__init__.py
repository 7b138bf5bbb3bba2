"""GB300-native layered fields (Zayer et al., arXiv 1804.09152).

The time-iteration runs in the CUDA library ``_build/liblf.so`` behind the C
ABI of ``include/lf.h``; ``paper_1804_09152_gb300.lf`` is its ctypes binding.
``build()`` compiles the library for sm_103a.
"""
from .native import build, LIB

__all__ = ["build", "LIB", "lf"]


def __getattr__(name):
    if name == "lf":
        from . import _lib
        return _lib
    raise AttributeError(name)
