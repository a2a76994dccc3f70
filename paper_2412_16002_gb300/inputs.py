"""Seeded synthetic inputs for the cRKDG workloads.

This module holds no part of the method's arithmetic: it only places sample
points (Gauss-Legendre nodes from numpy, the same points the nodal state is
defined on) and evaluates initial conditions there.  Both the CUDA path and the
CPU oracle receive the arrays it produces; neither imports the other.

Nodal layout (the C-ABI layout): 1D ``[m][nx][n]``; 2D ``[m][ny][nx][n_y][n_x]``,
values at the tensor Gauss points of each cell, ``n = k + 1``.

Workloads (the paper's analytic initial data; there are no datasets):
  * ``burgers_sine``      u0 = 0.5 + sin(pi x) on [0,2], periodic, bounds [-0.5, 1.5]
  * ``euler_blast_tube``  1D Euler, [0,9], (rho,w,p) = (1,0,0.1(g-1)) for x<3 and
                          (1e-3,0,1e-10(g-1)) for x>3, Dirichlet far states
  * ``sedov``             2D Euler Sedov-type blast on [0,1.1]^2 (Example 4.7 geometry)
  * ``riemann_quadrants`` seeded 2D four-quadrant Riemann problems on [0,1]^2
  * ``random_euler`` / ``random_scalar``  seeded admissible states with
                          zero-mean oscillations for operator and limiter parity
  * ``shock_diffraction`` 2D Euler, Example 4.8: Mach 5.09 shock past a step corner
  * ``double_mach``       2D Euler, Example 4.9: Mach 10 shock at 60 degrees reflecting
                          off a wall and diffracting at its corner
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4


def gauss_nodes(k: int):
    """(k+1) Gauss-Legendre nodes and weights on [-1, 1] (numpy)."""
    return np.polynomial.legendre.leggauss(k + 1)


def node_coords(dim, nx, ny, k, domain):
    """Physical coordinates of every node, in the nodal layout without the component axis."""
    xg, _ = gauss_nodes(k)
    x0, x1 = domain[0], domain[1]
    hx = (x1 - x0) / nx
    cx = x0 + (np.arange(nx) + 0.5) * hx
    if dim == 1:
        return cx[:, None] + 0.5 * hx * xg[None, :]
    y0, y1 = domain[2], domain[3]
    hy = (y1 - y0) / ny
    cy = y0 + (np.arange(ny) + 0.5) * hy
    X = np.broadcast_to(cx[None, :, None, None] + 0.5 * hx * xg[None, None, None, :], (ny, nx, k + 1, k + 1))
    Y = np.broadcast_to(cy[:, None, None, None] + 0.5 * hy * xg[None, None, :, None], (ny, nx, k + 1, k + 1))
    return np.ascontiguousarray(X), np.ascontiguousarray(Y)


def prim_to_cons(rho, w, p, gamma=GAMMA):
    """(rho, velocity tuple, p) -> conservative components (rho, m..., E), eq. (Euler-2)."""
    w = [np.asarray(wi, dtype=np.float64) * np.ones_like(rho) for wi in w]
    kin = 0.5 * rho * sum(wi * wi for wi in w)
    return np.stack([rho] + [rho * wi for wi in w] + [p / (gamma - 1.0) + kin])


@dataclass
class Workload:
    """A problem description shared by the CUDA path and the oracle."""
    name: str
    dim: int
    nx: int
    ny: int
    k: int
    domain: tuple
    flux: str
    bc: tuple
    state: np.ndarray
    gamma: float = GAMMA
    velocity: tuple = (1.0, 0.0)
    bounds: tuple = (0.0, 1.0)
    eps: float = 1e-13
    bc_state: dict = field(default_factory=dict)
    cfl: float = 0.1
    t_end: float = 0.0
    tableau: str = "heun3"
    # non-rectangular domains: one geometry word per cell (GEO_* below) or None, the two
    # fixed states the words refer to, and the moving shock line x_s(t) = shock[0] + shock[1] t
    geo: np.ndarray | None = None
    geo_states: tuple = ()
    shock: tuple = (0.0, 0.0)

    @property
    def m(self):
        return self.dim + 2 if self.flux == "euler" else 1

    @property
    def cells(self):
        return self.nx * self.ny

    @property
    def dofs_per_cell(self):
        return self.m * (self.k + 1) ** self.dim


def burgers_sine(nx=200, k=2, cfl=0.1, t_end=0.3):
    X = node_coords(1, nx, 1, k, (0.0, 2.0))
    u = 0.5 + np.sin(np.pi * X)
    return Workload("burgers_sine", 1, nx, 1, k, (0.0, 2.0), "burgers", ("periodic",) * 4,
                    u[None].copy(), bounds=(-0.5, 1.5), cfl=cfl, t_end=t_end, tableau="heun3")


def euler_blast_tube(nx=4096, k=2, cfl=0.178, t_end=6.0, gamma=GAMMA):
    dom = (0.0, 9.0)
    X = node_coords(1, nx, 1, k, dom)
    left = X < 3.0
    rho = np.where(left, 1.0, 1e-3)
    p = np.where(left, (gamma - 1.0) * 0.1, (gamma - 1.0) * 1e-10)
    U = prim_to_cons(rho, (0.0,), p, gamma)
    sl = prim_to_cons(np.array(1.0), (0.0,), np.array((gamma - 1.0) * 0.1), gamma)
    sr = prim_to_cons(np.array(1e-3), (0.0,), np.array((gamma - 1.0) * 1e-10), gamma)
    return Workload("euler1d_blast_tube", 1, nx, 1, k, dom, "euler",
                    ("dirichlet", "dirichlet", "outflow", "outflow"), np.ascontiguousarray(U),
                    gamma=gamma, eps=1e-13, bc_state={0: sl.tolist(), 1: sr.tolist()}, cfl=cfl,
                    t_end=t_end, tableau="heun3")


def sedov(n=2048, k=3, cfl=0.103, t_end=1.0, gamma=GAMMA, p_ambient=1e-13):
    dom = (0.0, 1.1, 0.0, 1.1)
    dx = 1.1 / n
    U = np.zeros((4, n, n, k + 1, k + 1))
    U[0] = 1.0
    U[3] = p_ambient / (gamma - 1.0)
    U[3, 0, 0] = 0.244816 / (dx * dx)  # the corner cell carries the blast energy
    return Workload("sedov2d", 2, n, n, k, dom, "euler",
                    ("reflect", "outflow", "reflect", "outflow"), np.ascontiguousarray(U),
                    gamma=gamma, eps=1e-13, cfl=cfl, t_end=t_end,
                    tableau="rk4" if k == 3 else "heun3")


def scenario2(n=16, k=2, gamma=GAMMA):
    """Smooth exact Euler solution rho = 0.99 sin(pi(x+y)) + 1, w = (1,1), p = 1 (Example 4.2,
    scenario II) on the periodic square [0,2]^2, where it is periodic."""
    dom = (0.0, 2.0, 0.0, 2.0)
    X, Y = node_coords(2, n, n, k, dom)
    rho = 0.99 * np.sin(np.pi * (X + Y)) + 1.0
    U = prim_to_cons(rho, (1.0, 1.0), np.ones_like(rho), gamma)
    return Workload("euler2d_scenario2", 2, n, n, k, dom, "euler", ("periodic",) * 4, np.ascontiguousarray(U),
                    gamma=gamma, eps=1e-13, cfl=0.1, t_end=0.1024, tableau="rk4" if k == 3 else "heun3")


def sedov_shell(n=2048, k=3, radius=0.3, gamma=GAMMA, p_ambient=1e-13):
    """Sedov-type blast some time after ignition: a dense shell of radius `radius` around the
    corner with hot low-density gas inside and the cold ambient state (p = 1e-13) outside,
    flowing radially; same domain and boundaries as ``sedov``."""
    dom = (0.0, 1.1, 0.0, 1.1)
    X, Y = node_coords(2, n, n, k, dom)
    r = np.sqrt(X * X + Y * Y)
    inside = r < radius
    shell = np.exp(-((r - radius) / (0.03 * radius)) ** 2)
    rho = np.where(inside, 0.2 + 5.0 * shell, 1.0 + 4.0 * shell)
    p = np.where(inside, 0.5 * (1.0 + shell), p_ambient + 0.5 * shell)
    speed = 1.5 * shell * (r / radius)
    rr = np.maximum(r, 1e-12)
    U = prim_to_cons(rho, (speed * X / rr, speed * Y / rr), p, gamma)
    return Workload("sedov2d_shell", 2, n, n, k, dom, "euler", ("reflect", "outflow", "reflect", "outflow"),
                    np.ascontiguousarray(U), gamma=gamma, eps=1e-13, cfl=0.103, t_end=1.0,
                    tableau="rk4" if k == 3 else "heun3")


def riemann_states(seed):
    """Four quadrant states (rho, wx, wy, p): rho~U[0.1,2], p~U[0.01,2], |w|<1 (disc)."""
    rng = np.random.default_rng(seed)
    st = []
    for _ in range(4):
        rho = rng.uniform(0.1, 2.0)
        p = rng.uniform(0.01, 2.0)
        r = math.sqrt(rng.uniform(0.0, 1.0)) * 0.999
        a = rng.uniform(0.0, 2.0 * math.pi)
        st.append((rho, r * math.cos(a), r * math.sin(a), p))
    return st


def riemann_quadrants(seed, n=1024, k=2, cfl=None, t_end=0.2, gamma=GAMMA):
    dom = (0.0, 1.0, 0.0, 1.0)
    X, Y = node_coords(2, n, n, k, dom)
    st = riemann_states(seed)
    q = (X >= 0.5).astype(int) + 2 * (Y >= 0.5).astype(int)  # 0 SW, 1 SE, 2 NW, 3 NE
    rho = np.choose(q, [s[0] for s in st])
    wx = np.choose(q, [s[1] for s in st])
    wy = np.choose(q, [s[2] for s in st])
    p = np.choose(q, [s[3] for s in st])
    U = prim_to_cons(rho, (wx, wy), p, gamma)
    if cfl is None:  # the paper's CFL numbers for 3- and 4-stage schemes
        cfl = 0.178 if k != 3 else 0.103
    return Workload(f"riemann2d_seed{seed}", 2, n, n, k, dom, "euler", ("outflow",) * 4,
                    np.ascontiguousarray(U), gamma=gamma, eps=1e-13, cfl=cfl, t_end=t_end,
                    tableau="rk4" if k == 3 else "heun3")


def riemann_quadrants_device(seed, n, k, device="cuda", gamma=GAMMA):
    """The initial state of riemann_quadrants(seed, n, k) built directly on the device (torch,
    FP64): node coordinates by the same formulas, then each quadrant's conservative state.
    Equal to the host array element for element."""
    import torch

    xg, _ = gauss_nodes(k)
    st = riemann_states(seed)
    cons = prim_to_cons(np.array([s[0] for s in st]), (np.array([s[1] for s in st]), np.array([s[2] for s in st])),
                        np.array([s[3] for s in st]), gamma)  # [4 comps][4 quadrants]
    h = 1.0 / n
    c = 0.0 + (torch.arange(n, device=device, dtype=torch.float64) + 0.5) * h
    off = (0.5 * h) * torch.as_tensor(xg, device=device, dtype=torch.float64)
    X = c[None, :, None, None] + off[None, None, None, :]  # [1, nx, 1, n_x]
    Y = c[:, None, None, None] + off[None, None, :, None]  # [ny, 1, n_y, 1]
    q = (X >= 0.5).to(torch.int64) + 2 * (Y >= 0.5).to(torch.int64)  # [ny, nx, n_y, n_x]
    table = torch.as_tensor(cons, device=device, dtype=torch.float64)  # [4, 4]
    return table[:, q].contiguous()


def _zero_mean(rng, shape_cells, k, dim):
    """Random nodal oscillation with zero cell average under the Gauss weights."""
    _, w = gauss_nodes(k)
    n = k + 1
    r = rng.uniform(-1.0, 1.0, size=shape_cells + (n,) * dim)
    if dim == 1:
        mean = (r * w).sum(-1, keepdims=True) / 2.0
    else:
        mean = (r * w[None, :] * w[:, None]).sum((-1, -2), keepdims=True) / 4.0
    return r - mean


def random_euler(dim, nx, ny, k, seed, osc=0.6, gamma=GAMMA):
    """Smooth admissible Euler field plus zero-mean nodal oscillations.

    With osc near or above 1 some nodes leave the admissible set while every
    cell average stays admissible, which exercises both limiter branches."""
    rng = np.random.default_rng(seed)
    if dim == 1:
        X = node_coords(1, nx, 1, k, (0.0, 1.0))
        cells = (nx,)
        ph = rng.uniform(0, 2 * np.pi, 4)
        rho = 1.0 + 0.5 * np.sin(2 * np.pi * X + ph[0])
        w = (0.5 * np.sin(2 * np.pi * X + ph[1]),)
        p = 1.0 + 0.5 * np.sin(2 * np.pi * X + ph[2])
    else:
        X, Y = node_coords(2, nx, ny, k, (0.0, 1.0, 0.0, 1.0))
        cells = (ny, nx)
        ph = rng.uniform(0, 2 * np.pi, 6)
        rho = 1.0 + 0.5 * np.sin(2 * np.pi * X + ph[0]) * np.cos(2 * np.pi * Y + ph[1])
        w = (0.5 * np.sin(2 * np.pi * Y + ph[2]), 0.5 * np.cos(2 * np.pi * X + ph[3]))
        p = 1.0 + 0.5 * np.sin(2 * np.pi * (X + Y) + ph[4])
    U = prim_to_cons(rho, w, p, gamma)
    m = U.shape[0]
    for c in range(m):
        amp = osc * (np.abs(U[c]).mean() if c in (0, m - 1) else 0.3)
        U[c] = U[c] + amp * _zero_mean(rng, cells, k, dim)
    return np.ascontiguousarray(U)


def random_scalar(dim, nx, ny, k, seed, lo=-0.5, hi=1.5, osc=0.6):
    """Smooth field inside (lo, hi) plus zero-mean oscillations that may cross the bounds."""
    rng = np.random.default_rng(seed)
    mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
    if dim == 1:
        X = node_coords(1, nx, 1, k, (0.0, 1.0))
        u = mid + 0.8 * half * np.sin(2 * np.pi * X + rng.uniform(0, 6.3))
        cells = (nx,)
    else:
        X, Y = node_coords(2, nx, ny, k, (0.0, 1.0, 0.0, 1.0))
        u = mid + 0.8 * half * np.sin(2 * np.pi * X + rng.uniform(0, 6.3)) * np.cos(2 * np.pi * Y)
        cells = (ny, nx)
    u = u + osc * half * _zero_mean(rng, cells, k, dim)
    return np.ascontiguousarray(u[None])


# ----------------------------------------------------------------- non-rectangular domains
# Geometry words (one uint32 per cell of the bounding rectangle): bits 4s..4s+3 hold the
# boundary kind of side s (0 left, 1 right, 2 bottom, 3 top), bit 16 marks a solid cell.
# Kinds: the mesh rule (neighbouring cell or the rectangle side's condition), reflective
# wall, outflow, fixed state A, fixed state B, and the moving planar shock (state A behind
# the line x < x_s(t), state B ahead of it).
GEO_MESH, GEO_WALL, GEO_OUTFLOW, GEO_STATE_A, GEO_STATE_B, GEO_SHOCK = range(6)
GEO_SOLID = 1 << 16


def geo_word(left=GEO_MESH, right=GEO_MESH, bottom=GEO_MESH, top=GEO_MESH, solid=False):
    return (left | right << 4 | bottom << 8 | top << 12) | (GEO_SOLID if solid else 0)


def normal_shock(mach, rho1, p1, gamma=GAMMA):
    """A shock of Mach number `mach` running into gas at rest (rho1, p1): the post-shock
    density, normal velocity and pressure from the normal-shock (Rankine-Hugoniot) relations,
    and the shock speed."""
    c1 = math.sqrt(gamma * p1 / rho1)
    s = mach * c1
    m2 = mach * mach
    rho2 = rho1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (m2 - 1.0))
    u2 = s * (1.0 - rho1 / rho2)
    return rho2, u2, p2, s


def _mark_solid_faces(geo, solid):
    """Put a reflective wall on every side of a fluid cell that faces a solid cell (the
    callers then overwrite the segments that carry other data)."""
    ny, nx = solid.shape
    fluid = ~solid
    w = geo.reshape(ny, nx)
    lft = np.zeros_like(solid)
    lft[:, 1:] = solid[:, :-1]
    rgt = np.zeros_like(solid)
    rgt[:, :-1] = solid[:, 1:]
    bot = np.zeros_like(solid)
    bot[1:, :] = solid[:-1, :]
    top = np.zeros_like(solid)
    top[:-1, :] = solid[1:, :]
    for mask, side in ((lft, 0), (rgt, 1), (bot, 2), (top, 3)):
        sel = mask & fluid
        w[sel] = (w[sel] & ~np.uint32(15 << (4 * side))) | np.uint32(GEO_WALL << (4 * side))
    w[solid] |= np.uint32(GEO_SOLID)


def shock_diffraction(cells_per_unit=64, k=2, cfl=None, t_end=2.3, gamma=GAMMA):
    """Example 4.8: the union of [0,1]x[6,12] and [1,13]x[0,12] on the bounding rectangle
    [0,13]x[0,12] (the solid step [0,1]x[0,6] masked); a right-moving Mach 5.09 shock at
    x = 0.5 running into rho = 1.4, p = 1 at rest; inflow (the post-shock state) on the left,
    outflow on the top, right and bottom, reflective walls y = 6 (x <= 1) and x = 1 (y <= 6).
    Square cells of side 1 / cells_per_unit; solid cells hold the ambient state."""
    nx, ny = 13 * cells_per_unit, 12 * cells_per_unit
    dom = (0.0, 13.0, 0.0, 12.0)
    h = 1.0 / cells_per_unit
    rho2, u2, p2, _ = normal_shock(5.09, 1.4, 1.0, gamma)
    post = prim_to_cons(np.array(rho2), (u2, 0.0), np.array(p2), gamma)
    pre = prim_to_cons(np.array(1.4), (0.0, 0.0), np.array(1.0), gamma)
    xc = (np.arange(nx) + 0.5) * h
    yc = (np.arange(ny) + 0.5) * h
    solid = (yc[:, None] < 6.0) & (xc[None, :] < 1.0)
    geo = np.zeros(ny * nx, dtype=np.uint32)
    _mark_solid_faces(geo, solid)
    X, _ = node_coords(2, nx, ny, k, dom)
    behind = X < 0.5
    U = np.where(behind[None], post.reshape(4, 1, 1, 1, 1), pre.reshape(4, 1, 1, 1, 1))
    U = np.ascontiguousarray(U * np.ones((4, ny, nx, k + 1, k + 1)))
    U[:, solid] = pre.reshape(4, 1, 1, 1)
    if cfl is None:
        cfl = {1: 0.3, 2: 0.178, 3: 0.103}[k]
    return Workload(f"shock_diffraction_q{k}", 2, nx, ny, k, dom, "euler",
                    ("dirichlet", "outflow", "outflow", "outflow"), U, gamma=gamma, eps=1e-13,
                    bc_state={0: post.tolist()}, cfl=cfl, t_end=t_end,
                    tableau={1: "midpoint2", 2: "heun3", 3: "rk4"}[k], geo=geo,
                    geo_states=(post.tolist(), pre.tolist()))


def double_mach(cells_per_unit=360, k=3, cfl=None, t_end=0.2, gamma=GAMMA):
    """Example 4.9: the union of [1,4]x[-1,0] and [0,4]x[0,1] on the bounding rectangle
    [0,4]x[-1,1] (the solid block [0,1]x[-1,0] masked); a Mach 10 shock through (1/6, 0) at
    60 degrees to the x-axis running into rho = 1.4, p = 1 at rest, post-shock state
    rho = 8, w = (4.125 sqrt 3, -4.125), p = 116.5.  Inflow (post-shock) on the left, outflow
    on the right and the bottom, the post-shock state on y = 0 for x < 1/6, reflective walls
    y = 0 (1/6 <= x <= 1) and x = 1 (y <= 0), and on the top side the exact shock motion:
    post-shock where x < 1/6 + (1 + 20 t)/sqrt 3.  Solid cells hold the ambient state.  The
    fixed-state part of the wall is the cells whose centre lies at x < 1/6: exactly [0, 1/6)
    when cells_per_unit is a multiple of 6, as at the paper's 360, 480 and 600."""
    nx, ny = 4 * cells_per_unit, 2 * cells_per_unit
    dom = (0.0, 4.0, -1.0, 1.0)
    h = 1.0 / cells_per_unit
    angle = math.pi / 3.0
    rho2, u2, p2, s = normal_shock(10.0, 1.4, 1.0, gamma)
    wx, wy = u2 * math.sin(angle), -u2 * math.cos(angle)  # along the shock's normal
    post = prim_to_cons(np.array(rho2), (wx, wy), np.array(p2), gamma)
    pre = prim_to_cons(np.array(1.4), (0.0, 0.0), np.array(1.0), gamma)
    xc = (np.arange(nx) + 0.5) * h
    yc = -1.0 + (np.arange(ny) + 0.5) * h
    solid = (yc[:, None] < 0.0) & (xc[None, :] < 1.0)
    geo = np.zeros(ny * nx, dtype=np.uint32)
    _mark_solid_faces(geo, solid)
    w = geo.reshape(ny, nx)
    # y = 0, x < 1/6: the fixed post-shock state on the wall's leading part
    row0 = cells_per_unit  # the first fluid row above y = 0
    lead = xc < 1.0 / 6.0
    w[row0, lead] = (w[row0, lead] & ~np.uint32(15 << 8)) | np.uint32(GEO_STATE_A << 8)
    # the top side follows the shock: it meets y = 1 at x_s(t) = x_s0 + (s / sin 60) t
    x_s0 = 1.0 / 6.0 + 1.0 / math.tan(angle)
    speed = s / math.sin(angle)
    w[ny - 1, :] = (w[ny - 1, :] & ~np.uint32(15 << 12)) | np.uint32(GEO_SHOCK << 12)
    X, Y = node_coords(2, nx, ny, k, dom)
    behind = X < 1.0 / 6.0 + Y / math.tan(angle)
    U = np.where(behind[None], post.reshape(4, 1, 1, 1, 1), pre.reshape(4, 1, 1, 1, 1))
    U = np.ascontiguousarray(U * np.ones((4, ny, nx, k + 1, k + 1)))
    U[:, solid] = pre.reshape(4, 1, 1, 1)
    if cfl is None:
        cfl = {1: 0.3, 2: 0.178, 3: 0.103}[k]
    return Workload(f"double_mach_q{k}", 2, nx, ny, k, dom, "euler",
                    ("dirichlet", "outflow", "outflow", "outflow"), U, gamma=gamma, eps=1e-13,
                    bc_state={0: post.tolist()}, cfl=cfl, t_end=t_end,
                    tableau={1: "midpoint2", 2: "heun3", 3: "rk4"}[k], geo=geo,
                    geo_states=(post.tolist(), pre.tolist()), shock=(x_s0, speed))
