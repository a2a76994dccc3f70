"""Block domain decomposition of one cRKDG mesh over ranks (multi-GPU).

The inner stages of the method are cell-local; only the final stage reads the
neighbouring cells' traces (Sec. 1 and the Compactness remark of Sec. 3.2).  So a
rank that keeps a one-cell halo ring around its block of cells and recomputes the
inner stages on it needs the neighbours' data once per step: one exchange of the
boundary-cell layer of u^n.  Besides that exchange a step takes two reductions:
the minimum of the ranks' trial steps (the maximum wave-speed rate) and the OR of
the ranks' admissibility flags, which decides the Sec. 4.1 restart for all ranks
together.  The owned cells then evolve exactly as in the undecomposed mesh.

Pieces:
  - ``partition`` / ``Layout``: the px x py block split, each rank's owned block,
    halo sides and neighbours (periodic sides wrap).
  - ``Transport``: point-to-point exchange plus the reductions.
    ``TorchTransport`` runs over torch.distributed (gloo with host buffers, NCCL
    with device buffers); ``LocalWorld`` runs ranks as threads of one process.
  - ``DomainSolver``: one rank's subdomain around a stepper with the interface of
    ``solver.Solver`` (set_state, max_dt, step_attempt, step_accept,
    set_subdomain, cells_bytes, pack_cells, unpack_cells).

All arithmetic of the method runs in the stepper (the CUDA library); this module
only moves cells between ranks and takes the two decisions.
"""
from __future__ import annotations

import threading
from dataclasses import dataclass

import numpy as np


def partition(n, parts):
    """Split n cells into `parts` contiguous ranges whose sizes differ by at most one."""
    if not 1 <= parts <= n:
        raise ValueError(f"cannot split {n} cells into {parts} blocks")
    q, r = divmod(n, parts)
    out, start = [], 0
    for p in range(parts):
        stop = start + q + (1 if p < r else 0)
        out.append((start, stop))
        start = stop
    return out


@dataclass
class Layout:
    """Rank `rank` of a px x py block split of an nx x ny mesh (1D: ny = py = 1).

    own: global owned block (gi0, gi1, gj0, gj1); halo: (left, right, bottom, top) in {0, 1},
    1 where the side borders another block or wraps periodically onto one; nbr: the rank across
    each side (None on a physical boundary); local mesh = owned block plus the halo ring."""

    dim: int
    nx: int
    ny: int
    px: int
    py: int
    rank: int
    periodic: tuple

    def __post_init__(self):
        if self.px * self.py < 1 or self.rank >= self.px * self.py:
            raise ValueError("rank outside the process grid")
        self.rx, self.ry = self.rank % self.px, self.rank // self.px
        xs, ys = partition(self.nx, self.px), partition(self.ny, self.py)
        gi0, gi1 = xs[self.rx]
        gj0, gj1 = ys[self.ry]
        self.own = (gi0, gi1, gj0, gj1)
        per_x, per_y = self.periodic

        def across(dx, dy):
            rx, ry = self.rx + dx, self.ry + dy
            if dx and not 0 <= rx < self.px:
                if not per_x or self.px == 1:
                    return None
                rx %= self.px
            if dy and not 0 <= ry < self.py:
                if not per_y or self.py == 1:
                    return None
                ry %= self.py
            if dx and self.px == 1 or dy and self.py == 1:
                return None  # a single block keeps the periodic boundary of the mesh itself
            return ry * self.px + rx

        self.nbr = (across(-1, 0), across(1, 0), across(0, -1), across(0, 1))
        self.halo = tuple(0 if r is None else 1 for r in self.nbr)
        hl, hr, hb, ht = self.halo
        self.nxl = gi1 - gi0 + hl + hr
        self.nyl = gj1 - gj0 + hb + ht if self.dim == 2 else 1
        # owned box in local cell indices
        self.own_local = (hl, hl + gi1 - gi0, hb, hb + gj1 - gj0) if self.dim == 2 else (hl, hl + gi1 - gi0, 0, 1)
        # the global cells the local mesh covers (halo cells wrap across periodic sides)
        self.gx = [(gi0 - hl + i) % self.nx for i in range(self.nxl)]
        self.gy = [(gj0 - hb + j) % self.ny for j in range(self.nyl)] if self.dim == 2 else [0]

    def local_mesh(self, domain, bc):
        """Domain and boundary conditions of the local mesh: sides with a halo take outflow (the
        halo cells' own results are discarded), the others keep the global condition."""
        x0, x1 = domain[0], domain[1]
        hx = (x1 - x0) / self.nx
        gi0, gi1, gj0, gj1 = self.own
        hl, hr, hb, ht = self.halo
        dom = [x0 + (gi0 - hl) * hx, x0 + (gi1 + hr) * hx]
        if self.dim == 2:
            y0, y1 = domain[2], domain[3]
            hy = (y1 - y0) / self.ny
            dom += [y0 + (gj0 - hb) * hy, y0 + (gj1 + ht) * hy]
        sides = []
        for s in range(4):
            if s < 2 * self.dim and self.halo[s]:
                sides.append("outflow")
            else:
                sides.append(bc[s])
        return tuple(dom), tuple(sides)


class Transport:
    """Point-to-point exchange and reductions among the ranks of one decomposition."""

    rank = 0
    size = 1

    def exchange(self, ops):
        """ops: list of (kind, peer, buffer, tag), kind 'send' or 'recv'; every send to a peer
        is matched with that peer's recv of the same tag.  Returns when all are done."""
        raise NotImplementedError

    def min(self, x):
        raise NotImplementedError

    def any(self, flag):
        raise NotImplementedError

    def sum(self, arr):
        raise NotImplementedError

    def gather(self, obj):
        """Rank 0 receives the list of every rank's obj (other ranks: None)."""
        raise NotImplementedError


class TorchTransport(Transport):
    """torch.distributed: gloo with CPU tensors, NCCL with CUDA tensors (the process group is
    initialised by the caller)."""

    def __init__(self, device=None):
        import torch
        import torch.distributed as dist

        self.torch, self.dist = torch, dist
        self.rank, self.size = dist.get_rank(), dist.get_world_size()
        self.device = device if device is not None else torch.device("cpu")

    def exchange(self, ops):
        dist = self.dist
        p2p = []
        for kind, peer, buf, tag in ops:
            fn = dist.isend if kind == "send" else dist.irecv
            p2p.append(dist.P2POp(fn, buf, peer, tag=tag))
        if p2p:
            for req in dist.batch_isend_irecv(p2p):
                req.wait()

    def _reduce(self, value, op, dtype):
        t = self.torch.tensor([value], dtype=dtype, device=self.device)
        self.dist.all_reduce(t, op=op)
        return t.item()

    def min(self, x):
        return float(self._reduce(float(x), self.dist.ReduceOp.MIN, self.torch.float64))

    def any(self, flag):
        return bool(self._reduce(1 if flag else 0, self.dist.ReduceOp.MAX, self.torch.int32))

    def sum(self, arr):
        t = self.torch.tensor(np.asarray(arr, dtype=np.float64), device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return t.cpu().numpy()

    def gather(self, obj):
        out = [None] * self.size if self.rank == 0 else None
        self.dist.gather_object(obj, out, dst=0)
        return out


class LocalWorld:
    """Ranks as threads of one process: a mailbox for the exchange, a barrier for the
    reductions.  ``LocalWorld(n).transport(r)`` is rank r's transport."""

    def __init__(self, size, timeout=60.0):
        self.size = size
        self.timeout = timeout
        self.cv = threading.Condition()
        self.box = {}
        self.barrier = threading.Barrier(size, timeout=timeout)
        self.slots = [None] * size

    def transport(self, rank):
        return _LocalTransport(self, rank)


class _LocalTransport(Transport):
    def __init__(self, world, rank):
        self.w, self.rank, self.size = world, rank, world.size

    def exchange(self, ops):
        w = self.w
        with w.cv:
            for kind, peer, buf, tag in ops:
                if kind == "send":
                    w.box[(self.rank, peer, tag)] = _copy(buf)
            w.cv.notify_all()
        for kind, peer, buf, tag in ops:
            if kind != "recv":
                continue
            key = (peer, self.rank, tag)
            with w.cv:
                if not w.cv.wait_for(lambda: key in w.box, timeout=w.timeout):
                    raise TimeoutError(f"rank {self.rank}: no message {key}")
                data = w.box.pop(key)
            _store(buf, data)

    def _all(self, value):
        w = self.w
        w.slots[self.rank] = value
        w.barrier.wait()
        vals = list(w.slots)
        w.barrier.wait()  # nobody overwrites a slot before everyone has read it
        return vals

    def min(self, x):
        return min(self._all(float(x)))

    def any(self, flag):
        return any(self._all(bool(flag)))

    def sum(self, arr):
        vals = self._all(np.asarray(arr, dtype=np.float64))
        out = np.zeros_like(vals[0])
        for v in vals:  # fixed rank order
            out = out + v
        return out

    def gather(self, obj):
        vals = self._all(obj)
        return vals if self.rank == 0 else None


def _copy(buf):
    if type(buf).__module__.startswith("torch"):
        return buf.detach().clone()
    return np.array(buf, copy=True)


def _store(buf, data):
    if type(buf).__module__.startswith("torch"):
        buf.copy_(data)
    else:
        buf[...] = data


class DomainSolver:
    """One rank's subdomain of a decomposed mesh.

    stepper: a solver.Solver-like object built on the local mesh (``layout.local_mesh``);
    transport: this rank's Transport; domain: the global mesh's domain (the subdomain takes
    its cell sizes from it); device_buffers: exchange through device tensors (NCCL) instead of
    host buffers."""

    # message tags: phase x (0 eastward, 1 westward), phase y (2 northward, 3 southward)
    EAST, WEST, NORTH, SOUTH = 0, 1, 2, 3

    def __init__(self, layout, stepper, transport, domain, device_buffers=False, device=None):
        self.L, self.s, self.t = layout, stepper, transport
        self.device_buffers = device_buffers
        self.device = device
        stepper.set_subdomain(layout.own_local, dict(dim=layout.dim, nx=layout.nx, ny=layout.ny, domain=domain))
        self._plan()

    # ---- exchange plan -------------------------------------------------------
    def _buffer(self, cells):
        nbytes = self.s.cells_bytes(cells)
        if self.device_buffers:
            import torch

            return torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        try:
            import torch

            if torch.cuda.is_available():
                return torch.empty(nbytes, dtype=torch.uint8).pin_memory()
            return torch.empty(nbytes, dtype=torch.uint8)
        except ImportError:  # pragma: no cover - torch is a dependency of the package
            return np.empty(nbytes, dtype=np.uint8)

    def _plan(self):
        """Boxes (local cell indices) of the two phases.  Phase x moves owned columns (owned
        rows only) into the east/west halos; phase y then moves owned rows including the x
        halo cells into the north/south halos, which also fills the corners of the ring."""
        L = self.L
        i0, i1, j0, j1 = L.own_local
        nl, nr, nb, nt = L.nbr
        phases = [[], []]
        # phase x
        if nr is not None:  # eastward: my last owned column -> east neighbour's west halo
            phases[0].append(("send", nr, (i1 - 1, i1, j0, j1), self.EAST))
        if nl is not None:
            phases[0].append(("recv", nl, (0, 1, j0, j1), self.EAST))
        if nl is not None:  # westward: my first owned column -> west neighbour's east halo
            phases[0].append(("send", nl, (i0, i0 + 1, j0, j1), self.WEST))
        if nr is not None:
            phases[0].append(("recv", nr, (L.nxl - 1, L.nxl, j0, j1), self.WEST))
        # phase y (full local width)
        if L.dim == 2:
            if nt is not None:
                phases[1].append(("send", nt, (0, L.nxl, j1 - 1, j1), self.NORTH))
            if nb is not None:
                phases[1].append(("recv", nb, (0, L.nxl, 0, 1), self.NORTH))
            if nb is not None:
                phases[1].append(("send", nb, (0, L.nxl, j0, j0 + 1), self.SOUTH))
            if nt is not None:
                phases[1].append(("recv", nt, (0, L.nxl, L.nyl - 1, L.nyl), self.SOUTH))
        self.phases = []
        for ph in phases:
            ops = []
            for kind, peer, box, tag in ph:
                cells = (box[1] - box[0]) * (box[3] - box[2])
                ops.append((kind, peer, box, tag, self._buffer(cells)))
            self.phases.append(ops)
        self.halo_bytes = sum(self.s.cells_bytes((b[1] - b[0]) * (b[3] - b[2]))
                              for ph in self.phases for k, _, b, _, _ in ph if k == "recv")

    def exchange_halos(self):
        """Refresh the halo ring from the neighbours' owned cells (two phases)."""
        for ops in self.phases:
            for kind, peer, box, tag, buf in ops:
                if kind == "send":
                    self.s.pack_cells(box, buf)
            if self.device_buffers:
                import torch

                torch.cuda.synchronize()  # the packs, issued on the library's stream, are done
            self.t.exchange([(kind, peer, buf, tag) for kind, peer, box, tag, buf in ops])
            if self.device_buffers:
                torch.cuda.synchronize()  # the received bytes are in place before the unpacks
            for kind, peer, box, tag, buf in ops:
                if kind == "recv":
                    self.s.unpack_cells(box, buf)

    # ---- state ----------------------------------------------------------------
    def local_block(self, global_state):
        """This rank's local cells (owned block and halo ring) of a global nodal state."""
        L = self.L
        G = np.asarray(global_state)
        if L.dim == 1:
            return np.ascontiguousarray(G[:, L.gx])
        return np.ascontiguousarray(G[:, L.gy][:, :, L.gx])

    def set_global_state(self, global_state):
        """Every rank passes the same global nodal state; each takes its local cells (the
        limiter is cell-local, so halo cells are limited exactly as their owners)."""
        self.s.set_state(self.local_block(global_state))

    def owned_state(self):
        L = self.L
        U = np.asarray(self.s.get_state())
        i0, i1, j0, j1 = L.own_local
        return U[:, i0:i1] if L.dim == 1 else U[:, j0:j1, i0:i1]

    def gather_state(self):
        """Rank 0: the assembled global nodal state; other ranks: None."""
        parts = self.t.gather((self.L.own, self.owned_state()))
        if parts is None:
            return None
        (gi0, gi1, gj0, gj1), first = parts[0]
        m = first.shape[0]
        tail = first.shape[3:] if self.L.dim == 2 else first.shape[2:]
        shape = (m, self.L.nx) + tail if self.L.dim == 1 else (m, self.L.ny, self.L.nx) + tail
        out = np.empty(shape, dtype=first.dtype)
        for (a0, a1, b0, b1), blk in parts:
            if self.L.dim == 1:
                out[:, a0:a1] = blk
            else:
                out[:, b0:b1, a0:a1] = blk
        return out

    # ---- stepping --------------------------------------------------------------
    def max_dt(self, cfl):
        """The global trial step: min over ranks of the owned cells' trial steps (the maximum
        of the wave-speed rate is exact in any order)."""
        return self.t.min(self.s.max_dt(cfl))

    def step(self, dt, tableau, max_halvings=20):
        """One step of the whole mesh: attempts of size dt, dt/2, ... until no rank's owned
        cells leave B (Sec. 4.1), then every rank accepts and the halos are refreshed."""
        for r in range(max_halvings + 1):
            violated = self.s.step_attempt(dt, tableau)
            if not self.t.any(violated):
                info = self.s.step_accept()
                info["restarts"] = r
                info["dt_taken"] = dt
                self.exchange_halos()
                return info
            dt *= 0.5
        raise RuntimeError("cell averages left the admissible set after max_halvings restarts")
