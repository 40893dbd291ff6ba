"""GB300 (sm_103a) implementation of the Intermediate State Method hot path.

The compute path is libism.so (hand-written CUDA kernels behind the C ABI of include/ism.h);
``abi`` is its ctypes binding.  Nothing here falls back to the CPU.
"""
from .abi import (ISM_FP64, ISM_MIXED, ISM_SCHEME_CHEBYSHEV, ISM_SCHEME_CRANK_NICOLSON, IsmError, Plan,  # noqa: F401
                  Server, footprint, load, pack_hamiltonian)

__all__ = ["Plan", "Server", "IsmError", "load", "pack_hamiltonian", "footprint", "ISM_FP64", "ISM_MIXED",
           "ISM_SCHEME_CHEBYSHEV", "ISM_SCHEME_CRANK_NICOLSON"]
