"""GB300-native (sm_103a) bound-preserving compact-stencil RKDG (cRKDG) library.

Method: Liu, Sun and Zhang, arXiv 2412.16002.  The numerics run in the CUDA
library ``libcrkdg.so`` (C ABI in ``include/crkdg.h``); this package holds its
build script, the ctypes binding (``Solver``) and the seeded input generators.
Importing the package does not load the library; ``Solver`` does, and raises
if it has not been built.
"""
from .build import build  # noqa: F401

__all__ = ["build", "Solver", "TABLEAUX"]


def __getattr__(name):
    if name in ("Solver", "TABLEAUX"):
        from . import solver

        return getattr(solver, name)
    raise AttributeError(name)
