"""GB300-native PC-LSQR of the Gaia AVU-GSR solver (Cesare et al., 2022).

The computation lives in libgsr.so (hand-written CUDA for sm_103a, C ABI in
include/gsr.h); `Solver` marshals arguments to it.  `gen` builds seeded
synthetic systems of the paper's structure.
"""
from ._lib import GsrError  # noqa: F401


def __getattr__(name):
    if name == "Solver":
        from .solver import Solver
        return Solver
    raise AttributeError(name)
