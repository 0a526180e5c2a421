"""GB300 (sm_103a) implementation of the MLSVD-compressed damped Gauss-Newton
CPD method of F. Bottega Diniz's thesis (arXiv 2110.05997).

The compute path is libcpd.so (CUDA, C ABI in include/cpd.h); ``cpd`` is its
thin ctypes binding and ``build`` compiles it.
"""
from . import cpd  # noqa: F401

__all__ = ["cpd"]
