"""ctypes wrapper of the C oracle (test infrastructure only; see package docstring)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crkdg_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

FLUX = {"advection": 0, "burgers": 1, "euler": 2}
BC = {"periodic": 0, "outflow": 1, "reflect": 2, "dirichlet": 3, "exact": 4}

# Butcher tableaux of the paper's schemes (A strictly lower, b >= 0).
# eq. (cRKDG2): explicit midpoint;  eq. (cRKDG3): Heun's third order;
# eq. (cRKDG4): classic fourth order.
MIDPOINT2 = (np.array([[0.0, 0.0], [0.5, 0.0]]), np.array([0.0, 1.0]))
HEUN3 = (
    np.array([[0.0, 0.0, 0.0], [1.0 / 3.0, 0.0, 0.0], [0.0, 2.0 / 3.0, 0.0]]),
    np.array([0.25, 0.0, 0.75]),
)
RK4 = (
    np.array(
        [[0.0, 0.0, 0.0, 0.0], [0.5, 0.0, 0.0, 0.0], [0.0, 0.5, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0]]
    ),
    np.array([1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0]),
)


def build_oracle(force: bool = False) -> str:
    """Compile crkdg_oracle.c into liborc.so (plain -O2, portable flags)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "crkdg_oracle.h"))
        ):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(
                ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
            )
            os.replace(tmp, _LIB)
    return _LIB


class _Info(C.Structure):
    _fields_ = [
        ("dt_taken", C.c_double),
        ("restarts", C.c_int),
        ("cells_limited", C.c_longlong),
        ("theta_min", C.c_double),
    ]


_EXACT_FN = C.CFUNCTYPE(None, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double), C.c_void_p)
_dp = C.POINTER(C.c_double)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build_oracle())
    V = C.c_void_p
    lib.orc_gauss_legendre.argtypes = [C.c_int, _dp, _dp]
    lib.orc_gauss_lobatto.argtypes = [C.c_int, _dp, _dp]
    lib.orc_legendre.argtypes = [C.c_int, C.c_double]
    lib.orc_legendre.restype = C.c_double
    lib.orc_dlegendre.argtypes = [C.c_int, C.c_double]
    lib.orc_dlegendre.restype = C.c_double
    lib.orc_create.restype = V
    lib.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int] + [C.c_double] * 4 + [
        C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
        C.POINTER(C.c_int), _dp]
    lib.orc_destroy.argtypes = [V]
    lib.orc_set_exact.argtypes = [V, _EXACT_FN, V]
    lib.orc_set_options.argtypes = [V, C.c_int, C.c_int]
    lib.orc_set_scheme.argtypes = [V, C.c_int]
    lib.orc_set_theta2.argtypes = [V, C.c_int]
    lib.orc_set_source.argtypes = [V, C.c_int]
    lib.orc_set_basis.argtypes = [V, C.c_int]
    lib.orc_set_geometry.argtypes = [V, C.POINTER(C.c_uint), _dp, _dp, C.c_double, C.c_double]
    lib.orc_set_geometry.restype = C.c_int
    lib.orc_is_solid.argtypes = [V, C.c_int]
    lib.orc_is_solid.restype = C.c_int
    lib.orc_scenario1_source.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double)]
    lib.orc_state_size.argtypes = [V]
    lib.orc_state_size.restype = C.c_size_t
    lib.orc_nodal_to_modal.argtypes = [V, _dp, _dp]
    lib.orc_modal_to_nodal.argtypes = [V, _dp, _dp]
    lib.orc_point_state.argtypes = [V, _dp, C.c_int, C.c_double, C.c_double, _dp]
    lib.orc_cell_averages.argtypes = [V, _dp, _dp]
    lib.orc_flux.argtypes = [V, _dp, C.c_int, _dp]
    lib.orc_speed.argtypes = [V, _dp, C.c_int]
    lib.orc_speed.restype = C.c_double
    lib.orc_pressure.argtypes = [V, _dp]
    lib.orc_pressure.restype = C.c_double
    lib.orc_apply.argtypes = [V, C.c_int, _dp, _dp, C.c_double]
    lib.orc_limit.argtypes = [V, _dp, _dp]
    lib.orc_limit.restype = C.c_longlong
    lib.orc_averages_admissible.argtypes = [V, _dp]
    lib.orc_min_margins.argtypes = [V, _dp, _dp]
    lib.orc_set_indicator.argtypes = [V, C.c_int, C.c_double]
    lib.orc_troubled_cells.argtypes = [V, _dp, C.POINTER(C.c_int)]
    lib.orc_troubled_cells.restype = C.c_longlong
    lib.orc_shock_limit.argtypes = [V, _dp, C.POINTER(C.c_int)]
    lib.orc_a0.argtypes = [V, _dp]
    lib.orc_a0.restype = C.c_double
    lib.orc_max_dt.argtypes = [V, _dp, C.c_double]
    lib.orc_max_dt.restype = C.c_double
    lib.orc_step.argtypes = [V, _dp, C.c_double, C.c_int, _dp, _dp, C.c_double, C.POINTER(_Info)]
    lib.orc_step_stages.argtypes = [V, _dp, C.c_double, C.c_int, _dp, _dp, C.c_double, _dp, _dp]
    lib.orc_total_mass.argtypes = [V, _dp, C.c_int]
    lib.orc_total_mass.restype = C.c_double
    lib.orc_l2_error_exact.argtypes = [V, _dp, C.c_double, C.c_int]
    lib.orc_l2_error_exact.restype = C.c_double
    lib.orc_l1_error_exact.argtypes = [V, _dp, C.c_double, C.c_int]
    lib.orc_l1_error_exact.restype = C.c_double
    _lib = lib
    return lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def gauss_legendre(n: int):
    lib = _load()
    x = np.zeros(n)
    w = np.zeros(n)
    lib.orc_gauss_legendre(n, _p(x), _p(w))
    return x, w


def gauss_lobatto(L: int):
    lib = _load()
    x = np.zeros(L)
    w = np.zeros(L)
    lib.orc_gauss_lobatto(L, _p(x), _p(w))
    return x, w


def legendre(i: int, x: float) -> float:
    return _load().orc_legendre(i, x)


def dlegendre(i: int, x: float) -> float:
    return _load().orc_dlegendre(i, x)


class Oracle:
    """One cRKDG problem on a uniform Cartesian mesh, state kept as modal coefficients.

    dim 1 or 2; flux in {'advection','burgers','euler'}; bc: 4 names (left, right,
    bottom, top); bc_state: dict side->state for Dirichlet sides; exact: optional
    python callable (x, y, t) -> state used for 'exact' sides and error norms.
    """

    def __init__(self, dim, nx, ny, k, domain, flux, gamma=1.4, velocity=(1.0, 0.0),
                 bounds=(0.0, 1.0), eps=1e-13, bc=("periodic",) * 4, bc_state=None,
                 exact=None, limiter=True, max_halvings=20, indicator=False, tvb_M=10.0,
                 scheme="compact", theta2="ratio", source=None, basis="Q"):
        lib = _load()
        self.lib = lib
        x0, x1, y0, y1 = (tuple(domain) + (0.0, 1.0))[:4]
        bcs = (C.c_int * 4)(*[BC[b] for b in bc])
        st = np.zeros(16)
        if bc_state:
            for side, v in bc_state.items():
                st[side * 4: side * 4 + len(v)] = v
        self.h = lib.orc_create(dim, nx, ny if dim == 2 else 1, k, x0, x1, y0, y1, FLUX[flux],
                                gamma, velocity[0], velocity[1], bounds[0], bounds[1], eps, bcs,
                                _p(st))
        if not self.h:
            raise ValueError("oracle: unsupported problem")
        self.dim, self.nx, self.ny, self.k = dim, nx, (ny if dim == 2 else 1), k
        self.n = k + 1
        self.m = dim + 2 if flux == "euler" else 1
        self.flux = flux
        self.gamma = gamma
        self.N = lib.orc_state_size(self.h)
        self._exact_py = exact
        self._exact_c = None
        if exact is not None:
            m = self.m

            def cb(x, y, t, u, ctx):
                v = exact(x, y, t)
                for i in range(m):
                    u[i] = float(v[i])

            self._exact_c = _EXACT_FN(cb)
            lib.orc_set_exact(self.h, self._exact_c, None)
        lib.orc_set_options(self.h, 1 if limiter else 0, max_halvings)
        lib.orc_set_indicator(self.h, 1 if indicator else 0, tvb_M)
        lib.orc_set_scheme(self.h, 1 if scheme == "standard" else 0)
        lib.orc_set_theta2(self.h, 1 if theta2 == "exact" else 0)
        lib.orc_set_source(self.h, 1 if source == "scenario1" else 0)
        lib.orc_set_basis(self.h, 1 if basis == "P" else 0)
        self.c = np.zeros(self.N)

    def __del__(self):
        try:
            if self.h:
                self.lib.orc_destroy(self.h)
                self.h = None
        except Exception:
            pass

    # -- state -------------------------------------------------------------
    def nodal_shape(self):
        if self.dim == 1:
            return (self.m, self.nx, self.n)
        return (self.m, self.ny, self.nx, self.n, self.n)

    def to_modal(self, nodal) -> np.ndarray:
        nodal = np.ascontiguousarray(nodal, dtype=np.float64).reshape(-1)
        out = np.zeros(self.N)
        self.lib.orc_nodal_to_modal(self.h, _p(nodal), _p(out))
        return out

    def to_nodal(self, modal=None) -> np.ndarray:
        modal = self.c if modal is None else np.ascontiguousarray(modal)
        out = np.zeros(self.N)
        self.lib.orc_modal_to_nodal(self.h, _p(modal), _p(out))
        return out.reshape(self.nodal_shape())

    def set_state(self, nodal, limit=True):
        self.c = self.to_modal(nodal)
        if limit:
            self.limit()

    def get_state(self) -> np.ndarray:
        return self.to_nodal()

    def set_geometry(self, geo, state_a=None, state_b=None, shock_x0=0.0, shock_speed=0.0):
        """Non-rectangular domain (Examples 4.8, 4.9): per-cell words of boundary kinds and
        the solid bit (see orc_set_geometry); None removes it.  Raises on a bad word."""
        if geo is None:
            self.lib.orc_set_geometry(self.h, None, None, None, 0.0, 0.0)
            self._geo = None
            return
        g = np.ascontiguousarray(np.asarray(geo, dtype=np.uint32).reshape(-1))
        if g.size != self.nx * self.ny:
            raise ValueError("oracle: geometry needs one word per cell")
        sa = np.zeros(4)
        sb = np.zeros(4)
        if state_a is not None:
            sa[: len(state_a)] = state_a
        if state_b is not None:
            sb[: len(state_b)] = state_b
        rc = self.lib.orc_set_geometry(self.h, g.ctypes.data_as(C.POINTER(C.c_uint)), _p(sa), _p(sb),
                                       float(shock_x0), float(shock_speed))
        if rc != 0:
            raise ValueError("oracle: bad geometry word")
        self._geo = g

    def averages(self, modal=None) -> np.ndarray:
        modal = self.c if modal is None else modal
        out = np.zeros(self.nx * self.ny * self.m)
        self.lib.orc_cell_averages(self.h, _p(np.ascontiguousarray(modal)), _p(out))
        return out.reshape(self.ny, self.nx, self.m) if self.dim == 2 else out.reshape(self.nx, self.m)

    def point_state(self, cell, xi, eta=0.0, modal=None):
        modal = self.c if modal is None else modal
        u = np.zeros(self.m)
        self.lib.orc_point_state(self.h, _p(modal), cell, xi, eta, _p(u))
        return u

    # -- operators ---------------------------------------------------------
    def apply(self, op: str, modal=None, t=0.0) -> np.ndarray:
        modal = self.c if modal is None else np.ascontiguousarray(modal)
        out = np.zeros(self.N)
        self.lib.orc_apply(self.h, 0 if op == "G" else 1, _p(modal), _p(out), t)
        return out

    def limit(self, modal=None):
        """Limit in place (self.c by default); returns (#limited cells, theta per cell)."""
        target = self.c if modal is None else modal
        theta = np.zeros(self.nx * self.ny)
        nl = self.lib.orc_limit(self.h, _p(target), _p(theta))
        return nl, theta

    def admissible(self, modal=None) -> bool:
        modal = self.c if modal is None else modal
        return bool(self.lib.orc_averages_admissible(self.h, _p(modal)))

    def min_margins(self, modal=None):
        modal = self.c if modal is None else modal
        out = np.zeros(2)
        self.lib.orc_min_margins(self.h, _p(modal), _p(out))
        return out

    def troubled(self, modal=None):
        """TVB troubled-cell flags of a state (int array per cell)."""
        modal = self.c if modal is None else modal
        flags = np.zeros(self.nx * self.ny, dtype=np.int32)
        self.lib.orc_troubled_cells(self.h, _p(modal), flags.ctypes.data_as(C.POINTER(C.c_int)))
        return flags

    def shock_limit(self, flags, modal=None):
        target = self.c if modal is None else modal
        flags = np.ascontiguousarray(flags, dtype=np.int32)
        self.lib.orc_shock_limit(self.h, _p(target), flags.ctypes.data_as(C.POINTER(C.c_int)))

    def flux_at(self, u, direction=0):
        u = np.ascontiguousarray(u, dtype=np.float64)
        f = np.zeros(self.m)
        self.lib.orc_flux(self.h, _p(u), direction, _p(f))
        return f

    def speed(self, u, direction=0):
        return self.lib.orc_speed(self.h, _p(np.ascontiguousarray(u, dtype=np.float64)), direction)

    def pressure(self, u):
        return self.lib.orc_pressure(self.h, _p(np.ascontiguousarray(u, dtype=np.float64)))

    def a0(self, modal=None):
        modal = self.c if modal is None else modal
        return self.lib.orc_a0(self.h, _p(modal))

    def max_dt(self, cfl):
        return self.lib.orc_max_dt(self.h, _p(self.c), cfl)

    # -- stepping ----------------------------------------------------------
    def step(self, dt, tableau, t=0.0):
        A, b = tableau
        A = np.ascontiguousarray(A, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        info = _Info()
        rc = self.lib.orc_step(self.h, _p(self.c), dt, len(b), _p(A), _p(b), t, C.byref(info))
        return rc, {"dt_taken": info.dt_taken, "restarts": info.restarts,
                    "cells_limited": info.cells_limited, "theta_min": info.theta_min}

    def step_stages(self, dt, tableau, t=0.0, modal=None):
        """Single attempt recording (u^(i), ut^(i)) for i=1..s and the final stage."""
        A, b = tableau
        A = np.ascontiguousarray(A, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        s = len(b)
        modal = self.c if modal is None else modal
        us = np.zeros((s + 1) * self.N)
        uts = np.zeros((s + 1) * self.N)
        rc = self.lib.orc_step_stages(self.h, _p(modal), dt, s, _p(A), _p(b), t, _p(us), _p(uts))
        return rc, us.reshape(s + 1, self.N), uts.reshape(s + 1, self.N)

    def run(self, t_end, cfl, tableau, t=0.0, max_steps=10**9, fixed_dt=None):
        """Advance to t_end with the Sec. 4.1 trial step (or a fixed dt); last step clipped."""
        steps = restarts = 0
        while t < t_end - 1e-14 and steps < max_steps:
            dt = fixed_dt if fixed_dt is not None else self.max_dt(cfl)
            dt = min(dt, t_end - t)
            rc, info = self.step(dt, tableau, t)
            if rc != 0:
                raise RuntimeError("oracle: bounds could not be restored by halving dt")
            t += info["dt_taken"]
            steps += 1
            restarts += info["restarts"]
        return t, steps, restarts

    def total_mass(self, comp=0, modal=None):
        modal = self.c if modal is None else modal
        return self.lib.orc_total_mass(self.h, _p(modal), comp)

    def l2_error(self, t, nq=None):
        return self.lib.orc_l2_error_exact(self.h, _p(self.c), t, nq or self.k + 3)

    def l1_error(self, t, nq=None):
        return self.lib.orc_l1_error_exact(self.h, _p(self.c), t, nq or self.k + 3)
