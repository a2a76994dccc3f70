"""Thin Python front end of the ensemble entry points (crkdg_ensemble_* in include/crkdg.h).

An Ensemble advances many independent 2D Euler problems of uneven size (each with
its own mesh, degree, tableau, CFL number and end time) in persistent launches
under one CUDA graph per step.  Argument marshalling only.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from .solver import _is_torch, _Tab


class Ensemble:
    """problems: list of dicts with keys nx, ny, k, domain (x0, x1, y0, y1), bc (4 names),
    tableau (name or (A, b)), cfl, t_end (optional, default: no end)."""

    def __init__(self, problems, gamma=1.4, eps=1e-13, max_halvings=20, indicator="off", tvb_M=10.0):
        self.lib = L.load()
        self.np = len(problems)
        self._tabs = [_Tab(p["tableau"]) for p in problems]
        arr = (L.EnsProblem * self.np)()
        self.shapes = []
        for i, p in enumerate(problems):
            q = arr[i]
            q.mesh.dim, q.mesh.nx, q.mesh.ny = 2, p["nx"], p["ny"]
            q.mesh.x0, q.mesh.x1, q.mesh.y0, q.mesh.y1 = p.get("domain", (0.0, 1.0, 0.0, 1.0))
            for s, name in enumerate(p.get("bc", ("outflow",) * 4)):
                q.mesh.bc[s] = L.BC[name]
            q.k = p["k"]
            q.tableau = C.pointer(self._tabs[i].c)
            q.cfl = p["cfl"]
            q.t_end = p.get("t_end", 1e30)
            n = p["k"] + 1
            self.shapes.append((4, p["ny"], p["nx"], n, n))
        fl = L.Flux(L.FLUX["euler"], gamma, (C.c_double * 2)(0.0, 0.0))
        bd = L.Bounds(0.0, 1.0, eps)
        opt = L.Options()
        self.lib.crkdg_options_default(C.byref(opt))
        opt.max_halvings = max_halvings
        opt.indicator = L.INDICATOR[indicator]
        opt.tvb_M = tvb_M
        self.e = C.c_void_p()
        st = self.lib.crkdg_ensemble_create(self.np, arr, 4, C.byref(fl), C.byref(bd), C.byref(opt), C.byref(self.e))
        if st != L.OK:
            raise L.CrkdgError(st, "crkdg_ensemble_create failed")

    @classmethod
    def from_workloads(cls, workloads, **kw):
        probs = [dict(nx=w.nx, ny=w.ny, k=w.k, domain=w.domain, bc=w.bc, tableau=w.tableau, cfl=w.cfl,
                      t_end=w.t_end) for w in workloads]
        return cls(probs, gamma=workloads[0].gamma, eps=workloads[0].eps, **kw)

    def close(self):
        if getattr(self, "e", None) and self.e.value:
            self.lib.crkdg_ensemble_destroy(self.e)
            self.e = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        L.check_ens(self.lib, self.e, st)

    def state_size(self, i):
        return self.lib.crkdg_ensemble_state_size(self.e, i)

    def set_state(self, i, x):
        """x: numpy array (host) or torch CUDA tensor (device), float64, state layout of problem i."""
        if _is_torch(x):
            assert x.is_cuda and x.element_size() == 8 and x.is_contiguous()
            self._chk(self.lib.crkdg_ensemble_set_state(self.e, i, C.c_void_p(x.data_ptr()), x.numel(), 1))
        else:
            a = np.ascontiguousarray(x, dtype=np.float64)
            self._chk(self.lib.crkdg_ensemble_set_state(self.e, i, C.c_void_p(a.ctypes.data), a.size, 0))

    def get_state(self, i, out=None):
        if out is not None and _is_torch(out):
            self._chk(self.lib.crkdg_ensemble_get_state(self.e, i, C.c_void_p(out.data_ptr()), out.numel(), 1))
            return out
        a = np.empty(self.state_size(i), dtype=np.float64) if out is None else out
        assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == self.state_size(i)
        self._chk(self.lib.crkdg_ensemble_get_state(self.e, i, C.c_void_p(a.ctypes.data), a.size, 0))
        return a.reshape(self.shapes[i])

    def step(self):
        """One step of every running problem; returns how many are still running."""
        active = C.c_int()
        self._chk(self.lib.crkdg_ensemble_step(self.e, C.byref(active)))
        return active.value

    def info(self, i):
        inf = L.EnsInfo()
        self._chk(self.lib.crkdg_ensemble_info(self.e, i, C.byref(inf)))
        return {"t": inf.t, "steps": inf.steps, "restarts": inf.restarts, "done": bool(inf.done),
                "status": inf.status, "dt_taken": inf.last.dt_taken, "last_restarts": inf.last.restarts,
                "troubled": inf.last.troubled, "cells_limited": inf.last.cells_limited}

    def set_mlp(self, params):
        assert _is_torch(params) and params.is_cuda and params.element_size() == 4 and params.numel() == 7105
        self._chk(self.lib.crkdg_ensemble_set_mlp(self.e, C.c_void_p(params.data_ptr())))

    def set_harvest(self, on=True):
        self._chk(self.lib.crkdg_ensemble_set_harvest(self.e, 1 if on else 0))

    def last_features(self, i, out):
        """Problem i's features of the last step ([cells, 44] float32 CUDA tensor `out`)."""
        assert _is_torch(out) and out.is_cuda and out.element_size() == 4 and out.is_contiguous()
        self._chk(self.lib.crkdg_ensemble_last_features(self.e, i, C.c_void_p(out.data_ptr()), 1))
        return out

    def troubled_flags(self, i, out):
        """Problem i's troubled-cell flags of the last step ([cells] int32 CUDA tensor `out`)."""
        assert _is_torch(out) and out.is_cuda and out.element_size() == 4 and out.is_contiguous()
        self._chk(self.lib.crkdg_ensemble_troubled_flags(self.e, i, C.c_void_p(out.data_ptr()), 1))
        return out

    def set_profiling(self, on=True):
        self._chk(self.lib.crkdg_ensemble_set_profiling(self.e, 1 if on else 0))

    def times(self):
        """(milliseconds, steps) of the graph launches timed since profiling was switched on."""
        ms = C.c_double()
        n = C.c_longlong()
        self._chk(self.lib.crkdg_ensemble_times(self.e, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def autotune(self, reps=2):
        """Pick the work-item tile per (degree, size class); returns the 6 chosen tiles."""
        ch = (C.c_int * 6)()
        self._chk(self.lib.crkdg_ensemble_autotune(self.e, reps, ch))
        return list(ch)


def plan(ncells, tiles, cells_per_block):
    """Host-only work-item plan (problem, first block, blocks) of one degree group."""
    lib = L.load()
    n = len(ncells)
    nc = (C.c_longlong * n)(*ncells)
    tl = (C.c_int * n)(*tiles)
    cnt = lib.crkdg_ensemble_plan(n, nc, tl, cells_per_block, None, 0)
    if cnt < 0:
        raise ValueError("bad plan arguments")
    buf = (C.c_int * (3 * max(cnt, 1)))()
    lib.crkdg_ensemble_plan(n, nc, tl, cells_per_block, buf, cnt)
    return np.array(buf[:3 * cnt], dtype=np.int64).reshape(cnt, 3)


def riemann_ensemble_specs(count=64, seed=0, sizes=range(256, 1537, 128), degrees=(2, 3)):
    """Sizes and degrees of the seeded ensemble of four-quadrant Riemann problems: problem i
    has the quadrant states of seed i, a grid drawn uniformly from sizes and a degree drawn
    uniformly from degrees (numpy default_rng(seed))."""
    rng = np.random.default_rng(seed)
    sizes = list(sizes)
    out = []
    for i in range(count):
        n = sizes[int(rng.integers(0, len(sizes)))]
        k = int(degrees[int(rng.integers(0, len(degrees)))])
        out.append((i, n, k))
    return out


def riemann_problem(seed, n, k):
    """Problem dict of a four-quadrant Riemann problem on [0,1]^2 (outflow sides, T = 0.2):
    Q^2 with Heun-3 at CFL 0.178, Q^3 with RK4 at CFL 0.103 (the paper's stage counts and CFL
    numbers).  Its initial state is inputs.riemann_quadrants(seed, n, k).state."""
    cfl = 0.178 if k == 2 else 0.103
    return dict(nx=n, ny=n, k=k, domain=(0.0, 1.0, 0.0, 1.0), bc=("outflow",) * 4,
                tableau="rk4" if k == 3 else "heun3", cfl=cfl, t_end=0.2)


__all__ = ["Ensemble", "plan", "riemann_ensemble_specs", "riemann_problem"]
