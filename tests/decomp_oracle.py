"""The CPU oracle behind the stepper interface of the domain decomposition (tests only).

A rank's subdomain drives this stepper exactly as it drives the CUDA solver: set_state,
max_dt, step_attempt / step_accept, set_subdomain and the packed cell copies.  The state is
the oracle's own (modal coefficients, layout [cell][m][modes]); packed cells are those
coefficients, so a halo copy is exact.  Only the owned cells count in the admissibility test
and the trial step: both are taken by a second oracle holding just the owned cells' modal
coefficients (the rate is a per-cell maximum and the test a per-cell predicate, so this is the
oracle's own arithmetic restricted to those cells).
"""
import numpy as np

from oracle import Oracle


class OracleStepper:
    def __init__(self, dim, nx, ny, k, domain, flux, **kw):
        self.kw = dict(kw)
        self.dim, self.nx, self.ny, self.k, self.flux = dim, nx, (ny if dim == 2 else 1), k, flux
        self.domain = tuple(domain)
        self.o = Oracle(dim, nx, ny, k, domain, flux, **kw)
        self.m, self.modes = self.o.m, (k + 1) ** dim
        self.box = (0, nx, 0, self.ny)
        self.sub = self.o
        self.pending = None
        self.t = 0.0

    # cells of the modal state as [ny][nx][m][modes]
    def _cells(self, c):
        return c.reshape(self.ny, self.nx, self.m, self.modes)

    def _owned(self, c):
        i0, i1, j0, j1 = self.box
        return np.ascontiguousarray(self._cells(c)[j0:j1, i0:i1]).reshape(-1)

    def set_subdomain(self, box, global_mesh=None):
        i0, i1, j0, j1 = box
        self.box = (i0, i1, j0, j1)
        w, hgt = i1 - i0, j1 - j0
        hx = (self.domain[1] - self.domain[0]) / self.nx
        if global_mesh is not None:
            # the oracle forms its own cell size: the test meshes have power-of-two cells, for
            # which the window's cell size is the global one exactly
            gd = global_mesh["domain"]
            assert hx == (gd[1] - gd[0]) / global_mesh["nx"], "test meshes need exactly representable cells"
            if self.dim == 2:
                assert (self.domain[3] - self.domain[2]) / self.ny == (gd[3] - gd[2]) / global_mesh["ny"]
        dom = (0.0, w * hx)
        if self.dim == 2:
            hy = (self.domain[3] - self.domain[2]) / self.ny
            dom = dom + (0.0, hgt * hy)
        kw = {kk: v for kk, v in self.kw.items() if kk not in ("bc", "bc_state")}
        self.sub = Oracle(self.dim, w, hgt, self.k, dom, self.flux, bc=("periodic",) * 4, **kw)

    def set_state(self, nodal):
        self.o.set_state(nodal)

    def get_state(self):
        """Modal coefficients as [m][ny][nx][modes] (1D: [m][nx][modes]), the state layout's
        order of the cells."""
        out = np.moveaxis(self._cells(self.o.c), 2, 0).copy()
        return out[:, 0] if self.dim == 1 else out

    def max_dt(self, cfl):
        self.sub.c = self._owned(self.o.c)
        return self.sub.max_dt(cfl)

    def step_attempt(self, dt, tableau):
        A, b = tableau
        s = len(b)
        rc, us, uts = self.o.step_stages(dt, tableau, self.t, modal=self.o.c)
        if rc == 0:
            violated = False
        elif rc <= s:
            # an inner stage failed somewhere in the local mesh; a halo cell's inner stages are
            # those of the cell it copies, so its owner fails as well: the global OR is 1
            violated = True
        else:  # only the final stage failed: count the owned cells alone
            self.sub.c = self._owned(us[s])
            violated = not self.sub.admissible()
        self.pending = None if violated else uts[s].copy()
        self.pending_dt = dt
        return violated

    def step_accept(self):
        assert self.pending is not None
        self.o.c = self.pending
        self.pending = None
        self.t += self.pending_dt
        return {"restarts": 0}

    def cells_bytes(self, cells):
        return cells * self.m * self.modes * 8

    def pack_cells(self, box, buf):
        i0, i1, j0, j1 = box
        blk = self._cells(self.o.c)[j0:j1, i0:i1]
        _bytes_view(buf)[...] = np.ascontiguousarray(blk).reshape(-1).view(np.uint8)

    def unpack_cells(self, box, buf):
        i0, i1, j0, j1 = box
        cells = self._cells(self.o.c)
        blk = _bytes_view(buf).view(np.float64).reshape(j1 - j0, i1 - i0, self.m, self.modes)
        cells[j0:j1, i0:i1] = blk
        self.pending = None


def _bytes_view(buf):
    if type(buf).__module__.startswith("torch"):
        return buf.numpy()
    return buf


def modal_state_layout(o):
    """A global Oracle's modal state as [m][ny][nx][modes] (1D: [m][nx][modes])."""
    out = np.moveaxis(o.c.reshape(o.ny, o.nx, o.m, (o.k + 1) ** o.dim), 2, 0).copy()
    return out[:, 0] if o.dim == 1 else out
