"""Thin Python front end of the C ABI: one Solver per crkdg handle.

Only argument marshalling happens here; every step of the method runs in the
CUDA kernels behind libcrkdg.so.  PyTorch supplies device memory (tensors whose
data_ptr() is handed to the library) and streams.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L

# Butcher tableaux of the paper's schemes: eq. (cRKDG2) explicit midpoint,
# eq. (cRKDG3) Heun's third-order method, eq. (cRKDG4) classic RK4.
TABLEAUX = {
    "midpoint2": ([[0.0, 0.0], [0.5, 0.0]], [0.0, 1.0]),
    "heun3": ([[0.0, 0.0, 0.0], [1.0 / 3.0, 0.0, 0.0], [0.0, 2.0 / 3.0, 0.0]], [0.25, 0.0, 0.75]),
    "rk4": ([[0.0, 0.0, 0.0, 0.0], [0.5, 0.0, 0.0, 0.0], [0.0, 0.5, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0]],
            [1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0]),
}


class _Tab:
    def __init__(self, tableau):
        if isinstance(tableau, str):
            tableau = TABLEAUX[tableau]
        A, b = tableau
        self.A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(-1))
        self.b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
        self.s = len(self.b)
        self.c = L.Tableau(self.s, self.A.ctypes.data_as(C.POINTER(C.c_double)),
                           self.b.ctypes.data_as(C.POINTER(C.c_double)))


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _buf(b):
    """(address, bytes, on_device) of a contiguous byte buffer (torch tensor or numpy array)."""
    if _is_torch(b):
        assert b.is_contiguous()
        return b.data_ptr(), b.numel() * b.element_size(), 1 if b.is_cuda else 0
    assert b.flags.c_contiguous
    return b.ctypes.data, b.nbytes, 0


class Solver:
    """A cRKDG problem on the GPU.

    Parameters mirror include/crkdg.h: dim, nx, ny, k, domain (x0,x1[,y0,y1]),
    flux ('advection' | 'burgers' | 'euler'), gamma, velocity, bounds (lo, hi),
    eps, bc (4 side names), bc_state ({side: state}), stream (a torch.cuda.Stream
    or raw handle), max_halvings, precision ('fp64')."""

    def __init__(self, dim, nx, ny, k, domain, flux, gamma=1.4, velocity=(1.0, 0.0), bounds=(0.0, 1.0),
                 eps=1e-13, bc=("periodic",) * 4, bc_state=None, stream=None, max_halvings=20,
                 precision="fp64", indicator="off", tvb_M=10.0, scheme="compact", theta2="ratio",
                 source=None, basis="Q"):
        self.lib = L.load()
        mesh = L.Mesh()
        mesh.dim, mesh.nx, mesh.ny = dim, nx, ny if dim == 2 else 1
        dom = tuple(domain) + (0.0, 1.0)
        mesh.x0, mesh.x1, mesh.y0, mesh.y1 = dom[:4]
        for s in range(4):
            mesh.bc[s] = L.BC[bc[s]]
        for side, v in (bc_state or {}).items():
            for c, val in enumerate(v):
                mesh.bc_state[side][c] = float(val)
        fl = L.Flux(L.FLUX[flux], gamma, (C.c_double * 2)(*velocity))
        bd = L.Bounds(bounds[0], bounds[1], eps)
        opt = L.Options()
        self.lib.crkdg_options_default(C.byref(opt))
        opt.max_halvings = max_halvings
        opt.precision = L.PREC[precision]
        opt.indicator = L.INDICATOR[indicator]
        opt.tvb_M = tvb_M
        opt.scheme = L.SCHEME[scheme]
        opt.theta2 = L.THETA2[theta2]
        opt.source = L.SOURCE[source]
        opt.basis = L.BASIS[basis]
        if stream is not None:
            opt.cuda_stream = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self.m = dim + 2 if flux == "euler" else 1
        self.dim, self.nx, self.ny, self.k, self.n = dim, nx, (ny if dim == 2 else 1), k, k + 1
        self.h = C.c_void_p()
        st = self.lib.crkdg_create(C.byref(mesh), k, self.m, C.byref(fl), C.byref(bd), C.byref(opt), C.byref(self.h))
        if st != L.OK:
            raise L.CrkdgError(st, "crkdg_create failed")
        self.size = self.lib.crkdg_state_size(self.h)
        self._tabs = {}

    @classmethod
    def from_workload(cls, wl, **kw):
        s = cls(wl.dim, wl.nx, wl.ny, wl.k, wl.domain, wl.flux, gamma=wl.gamma, velocity=wl.velocity,
                bounds=wl.bounds, eps=wl.eps, bc=wl.bc, bc_state=wl.bc_state, **kw)
        if getattr(wl, "geo", None) is not None:
            s.set_geometry(wl.geo, wl.geo_states[0], wl.geo_states[1], *wl.shock)
        return s

    def set_geometry(self, geo, state_a=None, state_b=None, shock_x0=0.0, shock_speed=0.0):
        """Non-rectangular domain: one geometry word per cell (numpy uint32, see
        crkdg_set_geometry), the fixed states A and B, and the moving shock line; None removes it."""
        if geo is None:
            self._chk(self.lib.crkdg_set_geometry(self.h, None, None, None, 0.0, 0.0))
            return
        g = np.ascontiguousarray(np.asarray(geo, dtype=np.uint32).reshape(-1))
        if g.size != self.nx * self.ny:
            raise ValueError("set_geometry: one word per cell")
        sa = np.zeros(self.m) if state_a is None else np.ascontiguousarray(state_a, dtype=np.float64)
        sb = np.zeros(self.m) if state_b is None else np.ascontiguousarray(state_b, dtype=np.float64)
        self._chk(self.lib.crkdg_set_geometry(self.h, g.ctypes.data_as(C.POINTER(C.c_uint)),
                                              sa.ctypes.data_as(L._dp), sb.ctypes.data_as(L._dp),
                                              float(shock_x0), float(shock_speed)))

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.crkdg_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        L.check(self.lib, self.h, st)

    def nodal_shape(self):
        return (self.m, self.nx, self.n) if self.dim == 1 else (self.m, self.ny, self.nx, self.n, self.n)

    def _tab(self, tableau):
        key = tableau if isinstance(tableau, str) else id(tableau)
        if key not in self._tabs:
            self._tabs[key] = _Tab(tableau)
        return self._tabs[key]

    # ---- state ---------------------------------------------------------------
    def set_state(self, x):
        """x: numpy array (host), or torch tensor (a CUDA tensor, or a CPU one, e.g. page-locked),
        float64, state layout."""
        if _is_torch(x):
            assert x.dtype.is_floating_point and x.element_size() == 8 and x.is_contiguous()
            self._chk(self.lib.crkdg_set_state(self.h, C.c_void_p(x.data_ptr()), x.numel(), 1 if x.is_cuda else 0))
        else:
            a = np.ascontiguousarray(x, dtype=np.float64)
            self._chk(self.lib.crkdg_set_state(self.h, C.c_void_p(a.ctypes.data), a.size, 0))

    def get_state(self, out=None):
        if out is not None and _is_torch(out):
            assert out.dtype.is_floating_point and out.element_size() == 8 and out.is_contiguous()
            self._chk(self.lib.crkdg_get_state(self.h, C.c_void_p(out.data_ptr()), out.numel(), 1 if out.is_cuda else 0))
            return out
        a = np.empty(self.size, dtype=np.float64) if out is None else out
        self._chk(self.lib.crkdg_get_state(self.h, C.c_void_p(a.ctypes.data), a.size, 0))
        return a.reshape(self.nodal_shape())

    # ---- stepping ------------------------------------------------------------
    def set_time(self, t):
        self._chk(self.lib.crkdg_set_time(self.h, C.c_double(t)))

    def time(self):
        t = C.c_double()
        self._chk(self.lib.crkdg_get_time(self.h, C.byref(t)))
        return t.value

    def max_dt(self, cfl):
        dt = C.c_double()
        self._chk(self.lib.crkdg_max_dt(self.h, cfl, C.byref(dt)))
        return dt.value

    def step(self, dt, tableau="heun3"):
        info = L.StepInfo()
        self._chk(self.lib.crkdg_step(self.h, dt, C.byref(self._tab(tableau).c), C.byref(info)))
        return self._info(info)

    @staticmethod
    def _info(info):
        return {"dt_taken": info.dt_taken, "restarts": info.restarts, "cells_limited": info.cells_limited,
                "theta_min": info.theta_min, "troubled": info.troubled, "mass_drift": info.mass_drift}

    def step_attempt(self, dt, tableau="heun3"):
        """One attempt from u^n (no restart); True if a stage's averages left B."""
        v = C.c_int()
        self._chk(self.lib.crkdg_step_attempt(self.h, dt, C.byref(self._tab(tableau).c), C.byref(v)))
        return bool(v.value)

    def step_accept(self):
        info = L.StepInfo()
        self._chk(self.lib.crkdg_step_accept(self.h, C.byref(info)))
        return self._info(info)

    def set_tensor_cores(self, on):
        self._chk(self.lib.crkdg_set_tensor_cores(self.h, 1 if on else 0))

    # ---- subdomains ----------------------------------------------------------
    def set_subdomain(self, box, global_mesh=None):
        """Owned cells box = (i0, i1, j0, j1) of this mesh; global_mesh: dict(dim, nx, ny,
        domain) of the undecomposed mesh whose cell sizes this window takes."""
        gm = None
        if global_mesh is not None:
            gm = L.Mesh()
            gm.dim, gm.nx, gm.ny = global_mesh["dim"], global_mesh["nx"], global_mesh.get("ny", 1)
            dom = tuple(global_mesh["domain"]) + (0.0, 1.0)
            gm.x0, gm.x1, gm.y0, gm.y1 = dom[:4]
        self._chk(self.lib.crkdg_set_subdomain(self.h, C.byref(gm) if gm is not None else None, *box))

    def cells_bytes(self, cells):
        return int(self.lib.crkdg_cells_bytes(self.h, cells))

    def pack_cells(self, box, buf):
        """Copy the cells of box (i0, i1, j0, j1) of u^n into buf (a uint8 torch tensor on the
        device, or a numpy uint8 array / pinned CPU tensor on the host)."""
        ptr, nbytes, dev = _buf(buf)
        self._chk(self.lib.crkdg_pack_cells(self.h, *box, C.c_void_p(ptr), nbytes, dev))

    def unpack_cells(self, box, buf):
        ptr, nbytes, dev = _buf(buf)
        self._chk(self.lib.crkdg_unpack_cells(self.h, *box, C.c_void_p(ptr), nbytes, dev))

    def advance(self, nsteps, cfl, t_end, tableau="heun3", t=0.0):
        tt = C.c_double(t)
        done = C.c_int()
        rs = C.c_int()
        self._chk(self.lib.crkdg_advance(self.h, nsteps, cfl, t_end, C.byref(self._tab(tableau).c), C.byref(tt),
                                         C.byref(done), C.byref(rs)))
        return tt.value, done.value, rs.value

    def advance_fixed(self, nsteps, dt, t_end, tableau="heun3", t=0.0):
        tt = C.c_double(t)
        done = C.c_int()
        rs = C.c_int()
        self._chk(self.lib.crkdg_advance_fixed(self.h, nsteps, dt, t_end, C.byref(self._tab(tableau).c),
                                               C.byref(tt), C.byref(done), C.byref(rs)))
        return tt.value, done.value, rs.value

    def set_run1d_chunk(self, cells=0):
        """Own cells per block chunk of the 1D device-resident loop (0: automatic)."""
        self._chk(self.lib.crkdg_set_run1d_chunk(self.h, cells))

    # ---- measurement -------------------------------------------------------------
    def set_profiling(self, on=True):
        self._chk(self.lib.crkdg_set_profiling(self.h, 1 if on else 0))

    def kernel_times(self):
        """({'inner','final','run'}: ms, same keys: launches) since profiling was switched on."""
        ms = (C.c_double * 3)()
        n = (C.c_longlong * 3)()
        self._chk(self.lib.crkdg_kernel_times(self.h, ms, n))
        keys = ("inner", "final", "run")
        return dict(zip(keys, ms)), dict(zip(keys, n))

    # ---- verification helpers ---------------------------------------------------
    def apply(self, op, x, out):
        """out = op(x) on device tensors; op in {'G', 'F', 'limit'}."""
        self._chk(self.lib.crkdg_apply_operator(self.h, L.OPS[op], C.c_void_p(x.data_ptr()),
                                                C.c_void_p(out.data_ptr())))
        return out

    def troubled_flags(self):
        f = np.empty(self.nx * self.ny, dtype=np.int32)
        self._chk(self.lib.crkdg_troubled_flags(self.h, C.c_void_p(f.ctypes.data), 0))
        return f

    # ---- learned troubled-cell indicator ---------------------------------------------
    def set_mlp(self, params):
        """Network of the 'mlp' indicator: a CUDA float32 tensor of CRKDG_MLP_NPARAM values."""
        assert _is_torch(params) and params.is_cuda and params.element_size() == 4 and params.numel() == 7105
        self._chk(self.lib.crkdg_set_mlp(self.h, C.c_void_p(params.data_ptr())))

    def set_harvest(self, on=True):
        """Keep each step's indicator features (training data for the network)."""
        self._chk(self.lib.crkdg_set_harvest(self.h, 1 if on else 0))

    def last_features(self, out=None):
        """Features of the last step, [ncell][44] float32 (numpy, or into a CUDA tensor)."""
        if out is not None and _is_torch(out):
            self._chk(self.lib.crkdg_last_features(self.h, C.c_void_p(out.data_ptr()), 1))
            return out
        f = np.empty((self.nx * self.ny, 44), dtype=np.float32)
        self._chk(self.lib.crkdg_last_features(self.h, C.c_void_p(f.ctypes.data), 0))
        return f

    def averages(self):
        a = np.empty(self.nx * self.ny * self.m)
        self._chk(self.lib.crkdg_cell_averages(self.h, C.c_void_p(a.ctypes.data), 0))
        return a.reshape(self.ny, self.nx, self.m) if self.dim == 2 else a.reshape(self.nx, self.m)

    def margins(self):
        m = (C.c_double * 2)()
        self._chk(self.lib.crkdg_bound_margins(self.h, m))
        return np.array([m[0], m[1]])

    def mass(self, comp=0):
        v = C.c_double()
        self._chk(self.lib.crkdg_total_mass(self.h, comp, C.byref(v)))
        return v.value
