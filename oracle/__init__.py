"""Plain FP64 CPU oracle of the bound-preserving cRKDG method (arXiv 2412.16002).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA product path never imports it and shares no code with it.

The numerics live in ``crkdg_oracle.c`` (plain C, FP64, modal Legendre basis);
this module compiles it with gcc on first use and wraps it with ctypes.
"""
from .oracle import (  # noqa: F401
    Oracle,
    build_oracle,
    gauss_legendre,
    gauss_lobatto,
    legendre,
    dlegendre,
    HEUN3,
    RK4,
    MIDPOINT2,
)
