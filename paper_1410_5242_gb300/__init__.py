"""GB300 (sm_103a) implementation of the KPM-DOS hot path of Kreutzer et al.
(IPDPS 2015): the fused augmented sparse-matrix multiple-vector product
behind the C interface of include/kpm.h.

``build`` compiles the CUDA library in-tree; ``kpm`` is the ctypes binding
(importing it raises if the library has not been built); ``model`` holds
the byte and flop counts of the paper's traffic model.
"""
import importlib

__all__ = ["build", "kpm", "model"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
