"""Shared helpers of the GPU parity tests (pairs of CUDA solver and CPU oracle)."""
import numpy as np

from oracle import HEUN3, MIDPOINT2, RK4, Oracle

ORACLE_TABS = {"midpoint2": MIDPOINT2, "heun3": HEUN3, "rk4": RK4}


def pair(dim, nx, ny, k, domain, flux, **kw):
    """(Solver, Oracle) for the same problem."""
    from paper_2412_16002_gb300.solver import Solver

    g = Solver(dim, nx, ny, k, domain, flux, **kw)
    okw = {kk: v for kk, v in kw.items() if kk in ("gamma", "velocity", "bounds", "eps", "bc", "bc_state")}
    o = Oracle(dim, nx, ny, k, domain, flux, **okw)
    return g, o


def pair_from_workload(wl):
    return pair(wl.dim, wl.nx, wl.ny, wl.k, wl.domain, wl.flux, gamma=wl.gamma, velocity=wl.velocity,
                bounds=wl.bounds, eps=wl.eps, bc=wl.bc, bc_state=wl.bc_state)


def rel_linf(a, b, m):
    """max over components of max|a-b| / max|b| (state layout, component axis first)."""
    a = np.asarray(a).reshape(m, -1)
    b = np.asarray(b).reshape(m, -1)
    worst = 0.0
    for c in range(m):
        scale = max(np.abs(b[c]).max(), 1e-300)
        worst = max(worst, np.abs(a[c] - b[c]).max() / scale)
    return worst
