"""GB300-native differentiable state-vector simulator (arXiv 2511.19291 hot path).

The compute path is the CUDA library ``libtqd.so`` (C ABI, ``include/tqd.h``).
This package holds its thin ctypes binding (``sim``), the
``torch.autograd.Function`` on top of it, and the seeded workload builders
(``workloads``).  The library is loaded on first use; if it is missing, every
entry point raises ``TqdLibraryError`` (there is no CPU fallback).
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "sim"]


def __getattr__(name):
    if name == "sim":
        import importlib
        return importlib.import_module(__name__ + ".sim")
    raise AttributeError(name)
