"""GB300-native (sm_103a) energy-and-force evaluation of an ANI-style neural-network
potential (arXiv 2207.14276, Deep-HP): cell-list neighbour search, atomic
environment vectors (Eqs. 3-5), per-species networks summed to the energy
(Eq. 2) and the analytic backward to forces, as CUDA kernels behind the C ABI
declared in include/nnp.h.  This package is the thin Python binding.
"""
from ._lib import NNPError, LIB_PATH, EXPORTS  # noqa: F401

__all__ = ["Potential", "NNPError", "LIB_PATH", "EXPORTS"]


def __getattr__(name):
    # torch is imported lazily so that the CPU-only tests can inspect the ABI
    if name == "Potential":
        from .potential import Potential
        return Potential
    if name == "NNPFunction":
        from .autograd import NNPFunction
        return NNPFunction
    raise AttributeError(name)
